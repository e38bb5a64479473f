// fq_device.cuh -- device helpers of the GB300 FCIQMC kernels.
//
// Everything here is integer or exactly-rounded binary64 arithmetic; kernels
// are compiled with -fmad=false so that no multiply-add is contracted.
#pragma once
#include "fq_internal.h"

namespace fq {

// ---------------------------------------------------------------- bit tricks
__device__ __forceinline__ u64 mask_below(int p) { return p >= 64 ? ~0ULL : ((1ULL << p) - 1ULL); }

// position of the k-th (0-based) set bit of x, by halving with popc
__device__ __forceinline__ int nth_set(u64 x, int k)
{
    int pos = 0;
    int c = __popc((unsigned)x);
    if (k >= c) { k -= c; x >>= 32; pos = 32; }
    unsigned w = (unsigned)x;
    c = __popc(w & 0xffffu);
    if (k >= c) { k -= c; w >>= 16; pos += 16; }
    c = __popc(w & 0xffu);
    if (k >= c) { k -= c; w >>= 8; pos += 8; }
    c = __popc(w & 0xfu);
    if (k >= c) { k -= c; w >>= 4; pos += 4; }
    c = __popc(w & 0x3u);
    if (k >= c) { k -= c; w >>= 2; pos += 2; }
    if (k >= (int)(w & 1u)) pos += 1;
    return pos;
}

// floor(w * m / 2^64): an integer in [0, m)
__device__ __forceinline__ u64 pick(u64 w, u64 m) { return __umul64hi(w, m); }

// x / d for x < 2^32 by the precomputed M = ceil(2^64 / d) (M = 0: d = 1):
// x M / 2^64 = x / d + x e / (d 2^64) with 0 <= e < d, and the second term
// is below 2^-32 < 1/d, so the floor is exact
__device__ __forceinline__ unsigned div_by(unsigned x, u64 M) { return M ? (unsigned)__umul64hi((u64)x, M) : x; }

// number of occupied spin orbitals before canonical position pos, then flip it
__device__ __forceinline__ int flip_parity(u64 &a, u64 &b, int N, int pos)
{
    int c;
    if (pos < N) { c = __popcll(a & mask_below(pos)); a ^= 1ULL << pos; }
    else { c = __popcll(a) + __popcll(b & mask_below(pos - N)); b ^= 1ULL << (pos - N); }
    return c & 1;
}

// ---------------------------------------------------------------- hashing
__device__ __host__ __forceinline__ u64 fmix64(u64 x)
{
    x ^= x >> 33;
    x *= 0xff51afd7ed558ccdULL;
    x ^= x >> 33;
    x *= 0xc4ceb9fe1a85ec53ULL;
    x ^= x >> 33;
    return x;
}
__device__ __host__ __forceinline__ u64 det_hash(u64 a, u64 b) { return fmix64((a * 0x9E3779B97F4A7C15ULL) ^ b); }
__device__ __forceinline__ int bucket_of(u64 h, int bb) { return bb ? (int)(h >> (64 - bb)) : 0; }

// ---------------------------------------------------------------- Philox4x64-10
// Salmon, Moraes, Dror, Shaw, SC'11: ten rounds of two 64x64->128 products.
__device__ __forceinline__ void philox(u64 c0, u64 c1, u64 c2, u64 c3, u64 k0, u64 k1, u64 out[4])
{
    const u64 M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
    const u64 W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
#pragma unroll
    for (int r = 0; r < 10; r++) {
        if (r) { k0 += W0; k1 += W1; }
        const u128 p0 = (u128)M0 * c0, p1 = (u128)M1 * c2;  // one 128-bit product each (fewer
        const u64 hi0 = (u64)(p0 >> 64), lo0 = (u64)p0;        // instructions than separate high and
        const u64 hi1 = (u64)(p1 >> 64), lo1 = (u64)p1;        // low multiplies)
        u64 n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

__device__ __forceinline__ double u53(u64 w) { return (double)(w >> 11) * 0x1p-53; }

// ---------------------------------------------------------------- binary64 by its bits
// Exact integer forms of comparisons and conversions: on GB300 the FP64 pipe
// issues at a small fraction of the integer rate, and these are exact.
constexpr u64 SIGN64 = 0x8000000000000000ULL;
__device__ __forceinline__ u64 dbits(double x) { return (u64)__double_as_longlong(x); }
__device__ __forceinline__ double bitsd(u64 b) { return __longlong_as_double((long long)b); }
__device__ __forceinline__ bool is_zero(double x) { return (dbits(x) << 1) == 0; }
// |x| < y for y positive and finite (false for NaN x)
__device__ __forceinline__ bool abs_lt(double x, double y) { return (dbits(x) & ~SIGN64) < dbits(y); }
__device__ __forceinline__ double with_sign_of(double mag, double s) { return bitsd(dbits(mag) | (dbits(s) & SIGN64)); }
// -x (IEEE negation is a flip of the sign bit) without the binary64 pipe; x if !flip
__device__ __forceinline__ double neg_if(bool flip, double x) { return bitsd(dbits(x) ^ (flip ? SIGN64 : 0ULL)); }

// |x| = M 2^E with M the integer significand
__device__ __forceinline__ void split_abs(double x, u64 &M, int &E)
{
    u64 b = dbits(x);
    int ex = (int)((b >> 52) & 0x7ff);
    M = b & 0xFFFFFFFFFFFFFULL;
    if (ex) { M |= 1ULL << 52; E = ex - 1075; } else E = -1074;
}

// floor(|c| 2^32) for |c| < 2^31
__device__ __forceinline__ u64 fx32(double c)
{
    u64 M;
    int E;
    split_abs(c, M, E);
    int sh = E + 32;
    if (sh >= 0) return M << sh;
    return -sh >= 64 ? 0ULL : (M >> (-sh));
}

// ceil(|c|) for 0 < |c| < 2^31
__device__ __forceinline__ u64 ceil_abs(double c)
{
    u64 M;
    int E;
    split_abs(c, M, E);
    if (E >= 0) return M << E;
    int s = -E;
    return s >= 64 ? 1ULL : ((M + ((1ULL << s) - 1ULL)) >> s);
}

// Eq. (3) decision "u < |v| / c_min" with u = (w >> 11) 2^-53, for 0 < |v| < c_min.
// When c_min = 2^k the quotient is exact and the test is the integer
// comparison (w >> 11) < ceil(|v| 2^(53-k)); otherwise binary64 as written.
__device__ __forceinline__ bool draw_keeps(u64 w, double v, double cmin, int cmin_log2, bool pow2)
{
    if (!pow2) return u53(w) < fabs(v) / cmin;
    u64 M;
    int E;
    split_abs(v, M, E);
    int sh = E + 53 - cmin_log2;
    u64 T;
    if (sh >= 0) T = M << sh;
    else {
        int s = -sh;
        T = s >= 64 ? 1ULL : ((M + ((1ULL << s) - 1ULL)) >> s);
    }
    return (w >> 11) < T;
}

// Eq. (3): |v| >= c_min kept; else sign(v) c_min with probability |v|/c_min, else 0
__device__ __forceinline__ double round_stoch(double v, double cmin, int cmin_log2, bool pow2, u64 w)
{
    if (is_zero(v) || !abs_lt(v, cmin)) return v;
    return draw_keeps(w, v, cmin, cmin_log2, pow2) ? with_sign_of(cmin, v) : 0.0;
}

// ---------------------------------------------------------------- exact sums
// A binary64 x = m 2^e is placed on the fixed grid 2^-F as the integer
// m 2^(e+F).  The host checked that every value summed this way lies on the
// grid and that the sums fit in 126 bits, so the conversion and the integer
// sums are exact and the single rounding happens in fixed_to_double.
__device__ __forceinline__ i128 to_fixed(double x, int F)
{
    u64 bits = (u64)__double_as_longlong(x);
    int ex = (int)((bits >> 52) & 0x7ff);
    u64 m = bits & 0xFFFFFFFFFFFFFULL;
    int e;
    if (ex == 0) { if (m == 0) return 0; e = -1074; } else { m |= 1ULL << 52; e = ex - 1075; }
    int sh = e + F;
    u128 v = sh >= 0 ? ((u128)m << sh) : (sh > -64 ? (u128)(m >> (-sh)) : (u128)0);
    return (bits >> 63) ? -(i128)v : (i128)v;
}

__device__ __forceinline__ i128 fx_load(const ulonglong2 *t, int i)
{
    ulonglong2 v = __ldg(t + i);
    return (i128)(((u128)v.y << 64) | (u128)v.x);
}

// round v 2^-F to the nearest binary64, ties to even (normal range assumed)
__device__ __forceinline__ double fixed_to_double(i128 v, int F)
{
    if (v == 0) return 0.0;
    u64 sign = 0;
    u128 u;
    if (v < 0) { sign = 1ULL << 63; u = (u128)(-v); } else u = (u128)v;
    u64 hi = (u64)(u >> 64), lo = (u64)u;
    int msb = hi ? 127 - __clzll((long long)hi) : 63 - __clzll((long long)lo);
    u64 mant;
    int e2;
    if (msb <= 52) {
        mant = lo << (52 - msb);
        e2 = msb - 52;
    } else {
        int sh = msb - 52;
        u128 q = u >> sh;
        mant = (u64)q;
        u128 rem = u - (q << sh);
        u128 half = (u128)1 << (sh - 1);
        if (rem > half || (rem == half && (mant & 1ULL))) {
            mant++;
            if (mant == (1ULL << 53)) { mant >>= 1; sh++; }
        }
        e2 = sh;
    }
    int E = 52 + e2 - F;
    u64 bits = sign | ((u64)(E + 1023) << 52) | (mant & 0xFFFFFFFFFFFFFULL);
    return __longlong_as_double((long long)bits);
}

__device__ __forceinline__ double u128_to_double(u128 u) { return fixed_to_double((i128)u, 0); }
__device__ __forceinline__ double i128_to_double(i128 v) { return fixed_to_double(v, 0); }


// a global add whose result nobody reads: a reduction, not an atomic that
// returns the old value
__device__ __forceinline__ void red_add(u64 *p, u64 v)
{
    asm volatile("red.relaxed.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// exact per-iteration totals (ACC_* in fq_internal.h): v added as three
// limbs, no add waiting for another's result
__device__ __forceinline__ void limb_add(u64 *acc, i128 v)
{
    const u128 u = (u128)v;
    const u64 mask = (1ULL << LIMB) - 1ULL;
    const u64 l0 = (u64)u & mask, l1 = (u64)(u >> LIMB) & mask, l2 = (u64)(long long)(v >> (2 * LIMB));
    if (l0) red_add(acc, l0);
    if (l1) red_add(acc + 1, l1);
    if (l2) red_add(acc + 2, l2);
}

__device__ __forceinline__ i128 limb_total(const u64 *acc)
{
    const u128 top = (u128)(i128)(long long)acc[2];  // the signed limb, two's complement
    return (i128)((u128)acc[0] + ((u128)acc[1] << LIMB) + (top << (2 * LIMB)));
}

__device__ __forceinline__ i128 shfl_xor_i128(i128 v, int m)
{
    u64 lo = (u64)v, hi = (u64)((u128)v >> 64);
    lo = __shfl_xor_sync(0xffffffffu, lo, m);
    hi = __shfl_xor_sync(0xffffffffu, hi, m);
    return (i128)(((u128)hi << 64) | (u128)lo);
}

// ---------------------------------------------------------------- logarithm
// ln x = k ln2 + 2 atanh(s), x = m 2^k, m in (sqrt(1/2), sqrt(2)],
// s = (m-1)/(m+1); the atanh series is summed in Horner form to z^11, z = s^2.
static __device__ double fq_ln(double x)
{
    if (!(x > 0.0) || isinf(x)) return __longlong_as_double(0x7ff8000000000000LL);
    u64 bits = (u64)__double_as_longlong(x);
    int k;
    if (((bits >> 52) & 0x7ff) == 0) {
        double y = x * 0x1p54;
        bits = (u64)__double_as_longlong(y);
        k = (int)((bits >> 52) & 0x7ff) - 1023 - 54;
    } else {
        k = (int)((bits >> 52) & 0x7ff) - 1023;
    }
    bits = (bits & 0xFFFFFFFFFFFFFULL) | (1023ULL << 52);
    double m = __longlong_as_double((long long)bits);
    if (m > 1.4142135623730951) { m = m * 0.5; k += 1; }
    double s = (m - 1.0) / (m + 1.0);
    double z = s * s;
    double p = 2.0 / 23.0;
    for (int j = 10; j >= 0; j--) p = 2.0 / (double)(2 * j + 1) + z * p;
    double r = s * p;
    const double ln2_hi = 0x1.62e42fefa39efp-1, ln2_lo = 0x1.abc9e3b39803fp-56;
    return (double)k * ln2_hi + ((double)k * ln2_lo + r);
}

// ---------------------------------------------------------------- integrals
__device__ __forceinline__ int pidx(int p, int q) { return p >= q ? p * (p + 1) / 2 + q : q * (q + 1) / 2 + p; }
__device__ __forceinline__ double eri4(const DevInst &I, int p, int q, int r, int s)
{
    return __ldg(I.eri + pidx(pidx(p, q), pidx(r, s)));
}

// single excitation i -> a of spin sp from (pa, pb):
// exact sum of h_ai + sum_{k occ, k != i} (ai|kk) - sum_{k occ same spin, k != i} (ak|ki)
// With the fixed-point table Sfx (entry (a, i, k): (ai|kk) and (ai|kk) - (ak|ki)
// side by side) every occupied k costs one 16-byte load; the loads are issued
// four at a time.  Without it (callers that hold only the integrals) the
// terms are converted on the fly.  Both give the same exact sum.
static __device__ double single_exact(const DevInst &I, u64 pa, u64 pb, int sp, int i, int a)
{
    const int N = I.norb, F = I.F;
    i128 acc = to_fixed(__ldg(I.h + a * N + i), F);
    u64 same = (sp ? pb : pa) & ~(1ULL << i), other = sp ? pa : pb;
    if (I.Sfx) {
        const ulonglong2 *row = I.Sfx + (size_t)(a * N + i) * (size_t)N * 2;
        while (same | other) {
            ulonglong2 v[4];
            for (int r = 0; r < 4; r++) {
                int k = -1, sel = 0;
                if (same) { k = __ffsll((long long)same) - 1; same &= same - 1; sel = 1; }
                else if (other) { k = __ffsll((long long)other) - 1; other &= other - 1; }
                v[r] = k >= 0 ? __ldg(row + 2 * k + sel) : make_ulonglong2(0, 0);
            }
            for (int r = 0; r < 4; r++) acc += (i128)(((u128)v[r].y << 64) | (u128)v[r].x);
        }
        return fixed_to_double(acc, F);
    }
    const int pai = pidx(a, i);
    for (int s = 0; s < 2; s++) {
        u64 x = s ? other : same;
        while (x) {
            int k = __ffsll((long long)x) - 1;
            x &= x - 1;
            acc += to_fixed(__ldg(I.eri + pidx(pai, k * (k + 3) / 2)), F);
            if (s == 0) acc -= to_fixed(__ldg(I.eri + pidx(pidx(a, k), pidx(k, i))), F);
        }
    }
    return fixed_to_double(acc, F);
}

// <D_j|H|D_i>, D_j != D_i (used for E_proj): Slater-Condon rules with the
// same sign convention as the spawning code
static __device__ double hoff_generic(const DevInst &I, u64 ia, u64 ib, u64 ja, u64 jb)
{
    const int N = I.norb;
    u64 ra = ia & ~ja, rb = ib & ~jb, aa = ja & ~ia, ab = jb & ~ib;
    int nr = __popcll(ra) + __popcll(rb);
    if (nr == 0 || nr > 2 || nr != __popcll(aa) + __popcll(ab)) return 0.0;
    if (nr == 1) {
        int sp = ra ? 0 : 1;
        if ((sp == 0 && !aa) || (sp == 1 && !ab)) return 0.0;
        int i = __ffsll((long long)(sp ? rb : ra)) - 1, a = __ffsll((long long)(sp ? ab : aa)) - 1;
        u64 x = sp ? ib : ia;
        u64 between = i < a ? (mask_below(a) & ~mask_below(i + 1)) : (mask_below(i) & ~mask_below(a + 1));
        double v = single_exact(I, ia, ib, sp, i, a);
        return neg_if(__popcll(x & between) & 1, v);
    }
    // canonical positions of the two removed and two added spin orbitals
    int P[2], Q[2], np = 0, nq = 0;
    u64 x;
    x = ra; while (x) { int k = __ffsll((long long)x) - 1; x &= x - 1; P[np++] = k; }
    x = rb; while (x) { int k = __ffsll((long long)x) - 1; x &= x - 1; P[np++] = N + k; }
    x = aa; while (x) { int k = __ffsll((long long)x) - 1; x &= x - 1; Q[nq++] = k; }
    x = ab; while (x) { int k = __ffsll((long long)x) - 1; x &= x - 1; Q[nq++] = N + k; }
    u64 ta = ia, tb = ib;
    int par = flip_parity(ta, tb, N, P[0]);
    par ^= flip_parity(ta, tb, N, P[1]);
    par ^= flip_parity(ta, tb, N, Q[1]);
    par ^= flip_parity(ta, tb, N, Q[0]);
    int si = P[0] >= N, sj = P[1] >= N, sa = Q[0] >= N, sb = Q[1] >= N;
    int oi = P[0] % N, oj = P[1] % N, oa = Q[0] % N, ob = Q[1] % N;
    bool dir = (sa == si) && (sb == sj), exch = (sa == sj) && (sb == si);
    double v;
    if (dir && exch) v = eri4(I, oa, oi, ob, oj) - eri4(I, oa, oj, ob, oi);
    else if (dir) v = eri4(I, oa, oi, ob, oj);
    else if (exch) v = neg_if(true, eri4(I, oa, oj, ob, oi));
    else v = 0.0;
    return neg_if(par, v);
}

// index of a determinant in the sorted key list of D, or -1: through the
// open-addressing set of D keys (one or two probes), or by bisection of the
// sorted keys where the set is not there
__device__ __forceinline__ int d_index_of(const DevInst &I, u64 a, u64 b)
{
    if (I.dhash_idx) {
        const u64 msk = (1ULL << I.dhash_bits) - 1;
        u64 s = det_hash(a, b) & msk;
        for (u64 probe = 0; probe <= msk; probe++) {
            const u64 ka = __ldg(I.dhash_keys + 2 * s), kb = __ldg(I.dhash_keys + 2 * s + 1);
            if (ka == a && kb == b) return __ldg(I.dhash_idx + s);
            if (ka == 0 && kb == 0) return -1;
            s = (s + 1) & msk;
        }
        return -1;
    }
    int lo = 0, hi = I.nd;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        const ulonglong2 k = I.dkey[mid];
        if (k.x == a && k.y == b) return mid;
        if (k.x < a || (k.x == a && k.y < b)) lo = mid + 1; else hi = mid;
    }
    return -1;
}

// orbital of electron e held in register e >> 5 of lane e & 31 (n: electrons,
// the same in every lane; all lanes call this together)
__device__ __forceinline__ int orb_of_electron(const int (&orb)[4], int n, int e)
{
    const int src = e & 31, r = e >> 5;
    int x = __shfl_sync(0xffffffffu, orb[0], src);
    for (int k = 1; k < 4; k++)
        if (n > 32 * k) {
            const int y = __shfl_sync(0xffffffffu, orb[k], src);
            if (r == k) x = y;
        }
    return x;
}

// H_ii - E_ref of D determinants (a[d], b[d]), computed together by one warp:
// the exact sum of h_pp over occupied orbitals and (pp|qq) - delta_spin (pq|qp)
// over occupied pairs, minus the same sum for the reference, rounded once.
// The n + n(n-1)/2 terms are spread evenly over the lanes (term t < n: h_pp
// of electron t; otherwise the pair e1 < e2 with t - n = e2(e2-1)/2 + e1);
// each lane issues the loads of four terms of every determinant before it
// adds any of them.
template <int D>
static __device__ void diag_exact_warp_multi(const DevInst &I, const u64 (&a)[D], const u64 (&b)[D], double (&out)[D])
{
    const int lane = threadIdx.x & 31, N = I.norb, n = I.n, na = I.na;
    // orbital of electron e (alpha electrons first) in register e >> 5 of lane e & 31
    int orb[D][4];
    for (int d = 0; d < D; d++)
        for (int r = 0; r < 4; r++) {
            const int e = lane + 32 * r;
            orb[d][r] = e < n ? (e < na ? nth_set(a[d], e) : nth_set(b[d], e - na)) : 0;
        }
    const int T = n + n * (n - 1) / 2;
    i128 part[D];
    for (int d = 0; d < D; d++) part[d] = 0;
    for (int t0 = 0; t0 < T; t0 += 128) {
        ulonglong2 v[D][4];
#pragma unroll
        for (int r = 0; r < 4; r++) {
            const int t = t0 + 32 * r + lane;
            int e1, e2;
            if (t < n) { e1 = t; e2 = -1; }
            else {
                const int q = t < T ? t - n : 0;
                int c = (int)((1.0f + sqrtf(1.0f + 8.0f * (float)q)) * 0.5f);  // estimate, corrected below
                while (c > 1 && c * (c - 1) / 2 > q) c--;
                while ((c + 1) * c / 2 <= q) c++;
                e2 = c;
                e1 = q - c * (c - 1) / 2;
            }
            const bool same = e2 >= 0 && ((e1 < na) == (e2 < na));
#pragma unroll
            for (int d = 0; d < D; d++) {
                const int p1 = orb_of_electron(orb[d], n, e1);
                const int p2 = orb_of_electron(orb[d], n, e2 < 0 ? 0 : e2);
                v[d][r] = make_ulonglong2(0, 0);
                if (t < T) v[d][r] = __ldg(e2 < 0 ? I.hfx + p1 : (same ? I.JKfx : I.Jfx) + p1 * N + p2);
            }
        }
#pragma unroll
        for (int d = 0; d < D; d++)
#pragma unroll
            for (int r = 0; r < 4; r++) part[d] += (i128)(((u128)v[d][r].y << 64) | (u128)v[d][r].x);
    }
    const i128 xref = (i128)(((u128)I.xref_hi << 64) | (u128)I.xref_lo);
#pragma unroll
    for (int d = 0; d < D; d++) {
        i128 x = part[d];
        for (int m = 16; m >= 1; m >>= 1) x += shfl_xor_i128(x, m);
        out[d] = fixed_to_double(x - xref, I.F);
    }
}

static __device__ double diag_exact_warp(const DevInst &I, u64 a, u64 b)
{
    const u64 aa[1] = {a}, bb[1] = {b};
    double o[1];
    diag_exact_warp_multi<1>(I, aa, bb, o);
    return o[0];
}

// exact H_ii - E_ref of one determinant by one thread (the same sum as the
// warp version, term by term)
static __device__ double diag_exact_thread(const DevInst &I, u64 a, u64 b)
{
    const int N = I.norb;
    i128 x = 0;
    for (int s = 0; s < 2; s++) {
        u64 w = s ? b : a;
        while (w) {
            const int p = __ffsll((long long)w) - 1;
            w &= w - 1;
            x += fx_load(I.hfx, p);
            u64 same = w;  // higher orbitals of the same spin
            while (same) {
                const int q = __ffsll((long long)same) - 1;
                same &= same - 1;
                x += fx_load(I.JKfx, p * N + q);
            }
            if (!s) {
                u64 ob = b;
                while (ob) {
                    const int q = __ffsll((long long)ob) - 1;
                    ob &= ob - 1;
                    x += fx_load(I.Jfx, p * N + q);
                }
            }
        }
    }
    const i128 xref = (i128)(((u128)I.xref_hi << 64) | (u128)I.xref_lo);
    return fixed_to_double(x - xref, I.F);
}

}  // namespace fq
