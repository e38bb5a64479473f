// kernels.cu -- the projector iteration of initiator-FCIQMC on GB300.
//
// One iteration (Eq. (4) of Guther et al. 2020) is a handful of launches over
// the bucketed walker list of every run in the batch:
//   spawning       (a) ceil(|C_i|) attempts per determinant, one Philox block,
//                  one excitation and one Slater-Condon element per attempt;
//                  survivors of the rounding of Eq. (3) are appended to the
//                  spawn bucket of their target.  By default split in two:
//                  k_spawn_draw (per bucket: attempts drawn, classified and
//                  queued in global memory) and k_spawn_eval (one queued
//                  attempt per thread); k_spawn_staged and k_spawn do both
//                  halves inside one per-bucket block (bucket staged by bulk
//                  copies, or loaded plainly).
//   k_spawn_heavy  the same for determinants with more than HEAVY_ATT walkers,
//                  split into fixed-size slices so no block waits on one
//                  heavily populated determinant.
//   annihilation   (b)+(c) per bucket: the bucket's walkers and spawns in
//                  shared memory (k_annihilate_staged: bulk copies one bucket
//                  ahead; k_annihilate: plain loads), equal determinants
//                  grouped in a shared open-addressing table, death and
//                  rounding, the spawns summed exactly, the initiator rule and
//                  rounding, the new bucket written, the new determinants
//                  listed, and N_w, E_num (Eq. (9)) and the counts added to
//                  the run's exact totals by global reductions.
//   k_annihilate_big  the same for buckets too large for shared memory.
//   k_new_diag     exact H_jj of the determinants created in the iteration.
//   k_finalize     per run: read and clear the exact totals, update the
//                  shift, append the statistics row, flip the buffers.
// Options add work to these launches or one more: the semi-stochastic
// projection (semistoch.cu) before annihilation, the trial-estimator probe
// (trial.cu tables) and the adaptive shift's weight sums inside spawning and
// annihilation, and for a replica pair the cross join (replica.cu) before
// k_finalize.
// All of them read the iteration state from device memory, so one iteration
// is captured once as a CUDA graph and replayed.
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "fq_device.cuh"

namespace fq {

__device__ __forceinline__ int find_inst(const int *unit_start, int n_inst, int u)
{
    int lo = 0, hi = n_inst;
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (__ldg(unit_start + mid) <= u) lo = mid; else hi = mid;
    }
    return lo;
}

// D membership (open addressing on the determinant hash; empty slot = (0,0),
// which is never a valid determinant because every run has electrons)
__device__ __forceinline__ bool in_D(const DevInst &I, u64 a, u64 b)
{
    if (I.nd == 0) return false;
    u64 m = (1ULL << I.dhash_bits) - 1;
    u64 s = det_hash(a, b) & m;
    for (int probe = 0; probe < (1 << I.dhash_bits); probe++) {
        u64 ka = __ldg(I.dhash_keys + 2 * s), kb = __ldg(I.dhash_keys + 2 * s + 1);
        if (ka == a && kb == b) return true;
        if (ka == 0 && kb == 0) return false;
        s = (s + 1) & m;
    }
    return false;
}

// ------------------------------------------------------------------ spawning
// One spawning attempt k from parent (pa, pb) draws the Philox block
// (pa, pb, iteration, (k << 8) | spawn).  The block's attempts are first
// drawn and classified (single, double, lattice hop, failed), queued in
// shared memory by class, and then each queue is processed by whole warps, so
// that the long exact sum of a single excitation does not stall warps of
// doubles.  The words each attempt consumes and every decision are the same
// as if the attempts were processed one by one.

// what the spawning code knows about the parent beyond its key: its
// main-list slot, the list parity and the shift at the start of the iteration
struct SpawnCtx {
    unsigned pslot;
    int par;
    double S;
};

// 128-bit add of q to the words p[0] (low), p[1] (high)
__device__ __forceinline__ void atomic_add128(u64 *p, u128 q)
{
    const u64 lo = (u64)q, hi = (u64)(q >> 64);
    const u64 old = atomicAdd((unsigned long long *)p, (unsigned long long)lo);
    atomicAdd((unsigned long long *)(p + 1), (unsigned long long)(hi + (old + lo < old ? 1ULL : 0ULL)));
}

// adaptive shift (Sec. V): the weight |H_ji| / |H_jj - E_ref - S| of a spawn
// from a non-initiator, truncated to 2^-64, into T of the parent, and into A
// as well when the target is occupied at the start of the iteration (the
// initiator rule accepts it); weights of 2^36 or more (|H_jj - E_ref - S| far
// below |H_ji|) and zero denominators are left out
__device__ __noinline__ void adaptive_account(const DevInst &I, u64 ta, u64 tb, double H, int bt, const SpawnCtx &cx)
{
    const unsigned short *kx = I.kidx[cx.par] + (size_t)bt * KIDX;
    unsigned s = (unsigned)det_hash(ta, tb) & (unsigned)(KIDX - 1);
    double hdj = 0.0;
    bool occ = false, found = false;
    for (int probe = 0; probe < KIDX; probe++) {
        const unsigned v = __ldg(kx + s);
        if (!v) break;
        const size_t o = (size_t)bt * CAP_M + (v - 1);
        const ulonglong2 k = I.key[cx.par][o];
        if (k.x == ta && k.y == tb) {
            found = true;
            occ = !is_zero(I.c[cx.par][o]);
            hdj = I.hd[cx.par][o];
            break;
        }
        s = (s + 1) & (unsigned)(KIDX - 1);
    }
    if (!found) hdj = diag_exact_thread(I, ta, tb);
    const double den = bitsd(dbits(hdj - cx.S) & ~SIGN64);
    if (is_zero(den)) return;
    const double w = bitsd(dbits(H) & ~SIGN64) / den;
    u64 M;
    int E;
    split_abs(w, M, E);
    const int sh = E + 64;  // w 2^64 = M 2^sh
    if (sh + 53 > 100) return;  // w >= 2^36
    const u128 q = sh >= 0 ? ((u128)M << sh) : (sh > -64 ? (u128)(M >> (-sh)) : (u128)0);
    u64 *acc = I.facc[cx.par] + (size_t)cx.pslot * 4;
    atomic_add128(acc + 2, q);
    if (occ) atomic_add128(acc, q);
}

// append a surviving spawn (Eq. (3) rounding of the weight ws, D -> D filter) to its bucket
__device__ __forceinline__ void emit_weight(const DevInst &I, u64 ta, u64 tb, double ws, unsigned flags, u64 w3,
                                            double H, const SpawnCtx &cx)
{
    if (abs_lt(ws, I.cmin)) {
        ws = round_stoch(ws, I.cmin, I.cmin_log2, I.cmin_pow2, w3);
        if (is_zero(ws)) return;
    }
    if (!abs_lt(ws, 0x1p31)) { atomicOr(&I.st->err, ERRB_NUMERIC); return; }
    if ((flags & 2u) && in_D(I, ta, tb)) return;  // D -> D is applied exactly
    const int bt = bucket_of(det_hash(ta, tb), I.bb);
    if (I.adaptive && !(flags & 1u)) adaptive_account(I, ta, tb, H, bt, cx);
    const int cap_s = I.cap_s;
    if (flags & 1u) {
        const int s = atomicAdd(I.scnt_i + bt, 1);
        if (s < cap_s) {
            const size_t o = (size_t)bt * cap_s + s;
            I.skey[o] = make_ulonglong2(ta, tb);
            I.sw[o] = ws;
        }
    } else {
        const int s = atomicAdd(I.scnt_n + bt, 1);
        const int slot = cap_s - 1 - s;
        if (slot >= 0) {
            const size_t o = (size_t)bt * cap_s + slot;
            I.skey[o] = make_ulonglong2(ta, tb);
            I.sw[o] = ws;
        }
    }
}

// weight -H tau / p_gen(c) C_i / n_att of a uniformly generated excitation of class c
__device__ __forceinline__ void emit_spawn(const DevInst &I, u64 ta, u64 tb, double H, int cls, double cper,
                                           unsigned flags, u64 w3, const SpawnCtx &cx)
{
    if (is_zero(H)) return;
    emit_weight(I, ta, tb, neg_if(true, H * (I.lam[cls] * cper)), flags, w3, H, cx);
}

// lattice hop (Hubbard): electron e (drawn from w1), neighbour slot w2
__device__ void spawn_hop_e(const DevInst &I, u64 pa, u64 pb, double cper, unsigned flags, int e, u64 w2, u64 w3,
                            const SpawnCtx &cx)
{
    const int sp = e >= I.na;
    u64 x = sp ? pb : pa;
    const int p = nth_set(x, sp ? e - I.na : e);
    const int q = __ldg(I.nbr + 4 * p + (int)pick(w2, (u64)I.z));
    if (q < 0 || ((x >> q) & 1ULL)) return;
    const u64 between = p < q ? (mask_below(q) & ~mask_below(p + 1)) : (mask_below(p) & ~mask_below(q + 1));
    const double H = neg_if(__popcll(x & between) & 1, I.tmt);
    x ^= (1ULL << p) | (1ULL << q);
    emit_spawn(I, sp ? pa : x, sp ? x : pb, H, CLS_HOP, cper, flags, w3, cx);
}

// single excitation (App. A): electron e (drawn from w1), hole of its spin w2
__device__ void spawn_single_e(const DevInst &I, u64 pa, u64 pb, double cper, unsigned flags, int e, u64 w2, u64 w3,
                               const SpawnCtx &cx)
{
    const int sp = e >= I.na;
    u64 x = sp ? pb : pa;
    const int i = nth_set(x, sp ? e - I.na : e);
    const int m = sp ? I.mb : I.ma;
    const int a = nth_set(~x & I.normask, (int)pick(w2, (u64)m));
    const u64 between = i < a ? (mask_below(a) & ~mask_below(i + 1)) : (mask_below(i) & ~mask_below(a + 1));
    const double v = single_exact(I, pa, pb, sp, i, a);
    const double H = neg_if(__popcll(x & between) & 1, v);
    x ^= (1ULL << i) | (1ULL << a);
    emit_spawn(I, sp ? pa : x, sp ? x : pb, H, sp ? CLS_SINGLE_B : CLS_SINGLE_A, cper, flags, w3, cx);
}

// double excitation (App. A): ordered electron pair w1, hole pair w2
__device__ void spawn_double(const DevInst &I, u64 pa, u64 pb, double cper, unsigned flags, unsigned ep, u64 w2, u64 w3,
                       const SpawnCtx &cx)
{
    const int N = I.norb, na = I.na;
    const int e1 = (int)(ep & 0xffu), e2 = (int)(ep >> 8);  // the ordered pair drawn from w1 (classify)
    const int s1 = e1 >= na, s2 = e2 >= na;
    const int o1 = nth_set(s1 ? pb : pa, s1 ? e1 - na : e1);
    const int o2 = nth_set(s2 ? pb : pa, s2 ? e2 - na : e2);
    int P0, P1, Q0, Q1, oi, oj, oa, ob, cls;
    u64 ta, tb;
    if (s1 != s2) {
        oi = s1 ? o2 : o1;
        oj = s1 ? o1 : o2;
        const unsigned y = (unsigned)pick(w2, (u64)(I.ma * I.mb));
        const unsigned ya = div_by(y, I.mg_mb);
        oa = nth_set(~pa & I.normask, (int)ya);
        ob = nth_set(~pb & I.normask, (int)(y - ya * (unsigned)I.mb));
        P0 = oi; P1 = N + oj; Q0 = oa; Q1 = N + ob;
        ta = pa ^ (1ULL << oi) ^ (1ULL << oa);
        tb = pb ^ (1ULL << oj) ^ (1ULL << ob);
        cls = CLS_DOUBLE_AB;
    } else {
        const int m = s1 ? I.mb : I.ma;
        u64 x = s1 ? pb : pa;
        const unsigned y = (unsigned)pick(w2, (u64)(m * (m - 1)));
        const unsigned yh = div_by(y, s1 ? I.mg_mb1 : I.mg_ma1);
        const int h1 = (int)yh, rr = (int)(y - yh * (unsigned)(m - 1));
        const int h2 = rr + (rr >= h1 ? 1 : 0);
        const int q1 = nth_set(~x & I.normask, h1), q2 = nth_set(~x & I.normask, h2);
        oi = min(o1, o2); oj = max(o1, o2); oa = min(q1, q2); ob = max(q1, q2);
        const int off = s1 ? N : 0;
        P0 = off + oi; P1 = off + oj; Q0 = off + oa; Q1 = off + ob;
        x ^= (1ULL << oi) | (1ULL << oj) | (1ULL << oa) | (1ULL << ob);
        ta = s1 ? pa : x;
        tb = s1 ? x : pb;
        cls = s1 ? CLS_DOUBLE_BB : CLS_DOUBLE_AA;
    }
    u64 xa = pa, xb = pb;
    int par = flip_parity(xa, xb, N, P0);
    par ^= flip_parity(xa, xb, N, P1);
    par ^= flip_parity(xa, xb, N, Q1);
    par ^= flip_parity(xa, xb, N, Q0);
    const double v = (cls == CLS_DOUBLE_AB) ? eri4(I, oa, oi, ob, oj) : eri4(I, oa, oi, ob, oj) - eri4(I, oa, oj, ob, oi);
    emit_spawn(I, ta, tb, neg_if(par, v), cls, cper, flags, w3, cx);
}

// heat-bath double (App. A, pre-computed heat-bath sampling): ordered electron
// pair w1 as in the uniform generator, then the alias table of that pair of
// spin orbitals: bin k = floor(w2 K / 2^64), coin = the low 64 bits of w2 K
// (top 53 bits); an occupied hole or an empty table fails the attempt.  With
// p_gen = p_pair |H| / S the weight is -sign(H) lambda_ij C_i / n_att,
// lambda_ij = tau S / p_pair (stored per table).
__device__ void spawn_double_pchb(const DevInst &I, u64 pa, u64 pb, double cper, unsigned flags, unsigned ep, u64 w2,
                                  u64 w3, const SpawnCtx &cx)
{
    const int N = I.norb, na = I.na;
    const int e1 = (int)(ep & 0xffu), e2 = (int)(ep >> 8);  // the ordered pair drawn from w1 (classify)
    const int s1 = e1 >= na, s2 = e2 >= na;
    const int o1 = nth_set(s1 ? pb : pa, s1 ? e1 - na : e1);
    const int o2 = nth_set(s2 ? pb : pa, s2 ? e2 - na : e2);
    int oi, oj, t, K;
    u64 off;
    if (s1 != s2) {
        oi = s1 ? o2 : o1;  // alpha electron
        oj = s1 ? o1 : o2;  // beta electron
        t = oi * N + oj;
        K = N * N;
        off = (u64)t * (u64)K;
    } else {
        oi = min(o1, o2);
        oj = max(o1, o2);
        const int p = oj * (oj - 1) / 2 + oi;
        t = N * N + p;
        K = N * (N - 1) / 2;
        off = I.pchb_ss_base + (u64)p * (u64)K;
    }
    const double2 mt = __ldg(I.pchb_meta + t);
    if (!(dbits(mt.y) != 0)) return;  // S = 0: nothing to propose
    const u64 k = __umul64hi(w2, (u64)K), low = w2 * (u64)K;
    const ulonglong2 e = __ldg(I.pchb_ent + off + k);
    const unsigned hp = ((low >> 11) < e.x) ? (unsigned)(e.y & 0xffffu) : (unsigned)((e.y >> 16) & 0xffffu);
    const int oa = (int)(hp & 0xffu), ob = (int)(hp >> 8);
    int P0, P1, Q0, Q1, cls;
    u64 ta, tb;
    if (s1 != s2) {
        if (((pa >> oa) & 1ULL) || ((pb >> ob) & 1ULL)) return;
        P0 = oi; P1 = N + oj; Q0 = oa; Q1 = N + ob;
        ta = pa ^ (1ULL << oi) ^ (1ULL << oa);
        tb = pb ^ (1ULL << oj) ^ (1ULL << ob);
        cls = CLS_DOUBLE_AB;
    } else {
        u64 x = s1 ? pb : pa;
        if (((x >> oa) & 1ULL) || ((x >> ob) & 1ULL)) return;
        const int sh = s1 ? N : 0;
        P0 = sh + oi; P1 = sh + oj; Q0 = sh + oa; Q1 = sh + ob;
        x ^= (1ULL << oi) | (1ULL << oj) | (1ULL << oa) | (1ULL << ob);
        ta = s1 ? pa : x;
        tb = s1 ? x : pb;
        cls = s1 ? CLS_DOUBLE_BB : CLS_DOUBLE_AA;
    }
    u64 xa = pa, xb = pb;
    int par = flip_parity(xa, xb, N, P0);
    par ^= flip_parity(xa, xb, N, P1);
    par ^= flip_parity(xa, xb, N, Q1);
    par ^= flip_parity(xa, xb, N, Q0);
    const double v = (cls == CLS_DOUBLE_AB) ? eri4(I, oa, oi, ob, oj) : eri4(I, oa, oi, ob, oj) - eri4(I, oa, oj, ob, oi);
    const double H = neg_if(par, v);
    if (is_zero(H)) return;
    const double wv = mt.x * cper;
    emit_weight(I, ta, tb, neg_if(!(dbits(H) & SIGN64), wv), flags, w3, H, cx);
}

// class of one attempt from its first two words, or -1 for a failed attempt;
// *ep = the electron of a single or a hop, or for a double e1 | e2 << 8 (the
// ordered electron pair), all drawn from w1
enum { Q_DOUBLE = 0, Q_SINGLE = 1, Q_HOP = 2, NQ = 3 };
__device__ __forceinline__ int classify(const DevInst &I, u64 pa, u64 pb, u64 w0, u64 w1, unsigned *ep)
{
    if (I.kind == FCIQMC_HUBBARD) {
        *ep = (unsigned)pick(w1, (u64)I.n);  // the electron that hops
        return Q_HOP;
    }
    if ((w0 >> 11) < I.tsingle) {
        const int e = (int)pick(w1, (u64)I.n);
        *ep = (unsigned)e;  // the excited electron
        return (e >= I.na ? I.mb : I.ma) == 0 ? -1 : Q_SINGLE;
    }
    const int n = I.n;
    if (n < 2) return -1;
    const unsigned xe = (unsigned)pick(w1, (u64)(n * (n - 1)));
    const unsigned q1 = div_by(xe, I.mg_n1);
    const int e1 = (int)q1, r = (int)(xe - q1 * (unsigned)(n - 1));
    const int e2 = r + (r >= e1 ? 1 : 0);
    *ep = (unsigned)e1 | ((unsigned)e2 << 8);
    const int s1 = e1 >= I.na, s2 = e2 >= I.na;
    if (s1 != s2) return (I.ma == 0 || I.mb == 0) ? -1 : Q_DOUBLE;
    return (s1 ? I.mb : I.ma) < 2 ? -1 : Q_DOUBLE;
}

// Division of C_i by n_att > 1 (binary64, correctly rounded) occupies the
// binary64 pipe for a whole warp's turn whatever its active lanes, so the
// determinants that need it are listed (one warp-aggregated shared atomic)
// and divided afterwards by full warps.
template <typename SM>
__device__ __forceinline__ void queue_div(SM &S, bool dv, int d, int lane)
{
    const unsigned md = __ballot_sync(0xffffffffu, dv);
    if (!md) return;
    int b0 = 0;
    if (lane == 0) b0 = atomicAdd(&S.ndiv, __popc(md));
    b0 = __shfl_sync(0xffffffffu, b0, 0);
    if (dv) S.divl[b0 + __popc(md & ((1u << lane) - 1u))] = (unsigned short)d;
}

// C / n_att in place for the listed determinants i0, i0 + stride, ...
__device__ __forceinline__ void divide_listed(const unsigned short *divl, int nd, double *c, int i0, int stride)
{
    for (int i = i0; i < nd; i += stride) {
        const int d = divl[i];
        const double x = c[d];
        c[d] = x / (double)ceil_abs(x);
    }
}

constexpr int CHUNK = 1024;  // attempts drawn and queued per round
struct SpawnRec {
    u64 w2, w3;
    unsigned det;
    unsigned ep;  // electron (single, hop) or electron pair (double) drawn from w1 (classify)
};
struct K1Smem {
    static constexpr int chunk = CHUNK;
    ulonglong2 key[CAP_M];
    double cper[CAP_M];
    unsigned off[CAP_M + 1];
    unsigned short att_det[CHUNK];  // parent of attempt a < CHUNK of a bucket, 0xffff: look it up in off[]
    unsigned char fl[CAP_M];
    SpawnRec rec[CHUNK];
    unsigned short divl[CAP_M];  // determinants whose C / n_att (n_att > 1) is still to be divided
    int ndiv;
    int qn[NQ];
    int next;  // evaluation counter of the chunk
    unsigned wsum[K1_THREADS / 32];
    int hdr_err, hdr_par;
    long long hdr_it;
    double hdr_S;
};
static_assert(3 * (sizeof(K1Smem) + 1024) <= 233472, "three spawn blocks per SM (228 KB, 1 KB reserved per block)");

// draw and classify attempts a0 .. a1-1 of a bucket (attempt a of parent
// `det`, slot k) and queue them by class in S.rec: doubles from the front,
// singles and hops from the back (hops only exist without the others), with
// the counts in qn[Q_DOUBLE], qn[Q_SINGLE] (zero on entry); each thread
// draws two attempts per round, so that the two Philox evaluations overlap
template <typename MAP, typename SM>
__device__ __forceinline__ void draw_classify(const DevInst &I, SM &S, long long it, unsigned a0, unsigned a1,
                                              const MAP &map, int *qn)
{
    constexpr int CHUNK = SM::chunk;
    const int t = threadIdx.x, lane = t & 31;
    for (unsigned ab = a0; ab < a1; ab += 2 * K1_THREADS) {
        u64 w[2][4];
        unsigned det[2], ep[2];
        int cls[2];
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const unsigned a = ab + h * K1_THREADS + t;
            cls[h] = -1;
            det[h] = 0;
            ep[h] = 0;
            if (ab + h * K1_THREADS + (unsigned)(t & ~31) < a1) {  // a warp with no attempt left draws nothing
                const unsigned ac = a < a1 ? a : a1 - 1;           // clamped: drawn, then discarded
                u64 k;
                det[h] = map.det_of(ac, k);
                const ulonglong2 kk = map.key(det[h]);
                philox(kk.x, kk.y, (u64)it, (k << 8) | (u64)PURPOSE_SPAWN, I.seed, I.replica, w[h]);
                const int q = classify(I, kk.x, kk.y, w[h][0], w[h][1], &ep[h]);
                cls[h] = a < a1 ? q : -1;
            }
        }
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const bool front = cls[h] == Q_DOUBLE, back = cls[h] == Q_SINGLE || cls[h] == Q_HOP;
            const unsigned mf = __ballot_sync(0xffffffffu, front), mb = __ballot_sync(0xffffffffu, back);
            int bf = 0, bk = 0;
            if (lane == 0) {
                if (mf) bf = atomicAdd(&qn[Q_DOUBLE], __popc(mf));
                if (mb) bk = atomicAdd(&qn[Q_SINGLE], __popc(mb));
            }
            bf = __shfl_sync(0xffffffffu, bf, 0);
            bk = __shfl_sync(0xffffffffu, bk, 0);
            const unsigned below = (1u << lane) - 1u;
            if (front || back) {
                const int slot = front ? bf + __popc(mf & below) : CHUNK - 1 - (bk + __popc(mb & below));
                SpawnRec &r = S.rec[slot];
                r.w2 = w[h][2]; r.w3 = w[h][3]; r.det = det[h]; r.ep = ep[h];
            }
        }
    }
}

// draw and classify the attempts of a bucket chunk by chunk, queue them by
// class, then evaluate them: warps take 32 queued attempts at a time from a
// shared counter, singles (the long exact sums) first, so that no warp idles
// at the chunk's closing barrier while others still hold a long queue
template <typename MAP, typename SM>
__device__ void run_attempts(const DevInst &I, SM &S, long long it, unsigned A, MAP map, int par, double shift)
{
    constexpr int CHUNK = SM::chunk;
    const int t = threadIdx.x, lane = t & 31;
    for (unsigned a0 = 0; a0 < A; a0 += CHUNK) {
        const unsigned a1 = min(A, a0 + CHUNK);
        if (t < NQ) S.qn[t] = 0;
        if (t == 0) S.next = 0;
        __syncthreads();
        draw_classify(I, S, it, a0, a1, map, S.qn);
        __syncthreads();
        const int nd = S.qn[Q_DOUBLE], ns = S.qn[Q_SINGLE], ntot = ns + nd;
        while (true) {
            int g = 0;
            if (lane == 0) g = atomicAdd(&S.next, 32);
            g = __shfl_sync(0xffffffffu, g, 0);
            if (g >= ntot) break;
            const int q = g + lane;
            if (q < ns) {
                const SpawnRec r = S.rec[CHUNK - 1 - q];
                const unsigned d = r.det;
                const ulonglong2 kk = map.key(d);
                const SpawnCtx cx{map.slot(d), par, shift};
                const int e = (int)r.ep;
                if (I.kind == FCIQMC_HUBBARD)
                    spawn_hop_e(I, kk.x, kk.y, map.cper(d), map.flags(d), e, r.w2, r.w3, cx);
                else spawn_single_e(I, kk.x, kk.y, map.cper(d), map.flags(d), e, r.w2, r.w3, cx);
            } else if (q < ntot) {
                const SpawnRec r = S.rec[q - ns];
                const unsigned d = r.det;
                const ulonglong2 kk = map.key(d);
                const SpawnCtx cx{map.slot(d), par, shift};
                if (I.pchb) spawn_double_pchb(I, kk.x, kk.y, map.cper(d), map.flags(d), r.ep, r.w2, r.w3, cx);
                else spawn_double(I, kk.x, kk.y, map.cper(d), map.flags(d), r.ep, r.w2, r.w3, cx);
            }
        }
        __syncthreads();
    }
}

struct BucketMap {
    const K1Smem *S;
    __device__ unsigned det_of(unsigned a, u64 &k) const
    {
        if (a < (unsigned)CHUNK) {
            const unsigned d = S->att_det[a];
            if (d != 0xffffu) {
                k = a - S->off[d];
                return d;
            }
        }
        int lo = 0, hi = CAP_M;  // largest d with off[d] <= a (off[CAP_M] = total > a)
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (S->off[mid] <= a) lo = mid; else hi = mid;
        }
        k = a - S->off[lo];
        return (unsigned)lo;
    }
    __device__ ulonglong2 key(unsigned d) const { return S->key[d]; }
    __device__ double cper(unsigned d) const { return S->cper[d]; }
    __device__ unsigned flags(unsigned d) const { return S->fl[d]; }
    __device__ unsigned slot(unsigned d) const { return base + d; }
    unsigned base;
};

// attempts k0 .. k0+count-1 of one heavy determinant
struct HeavyMap {
    HeavyChunk h;
    __device__ unsigned det_of(unsigned a, u64 &k) const { k = h.k0 + a; return 0; }
    __device__ ulonglong2 key(unsigned) const { return make_ulonglong2(h.a, h.b); }
    __device__ double cper(unsigned) const { return h.cper; }
    __device__ unsigned flags(unsigned) const { return h.flags; }
    __device__ unsigned slot(unsigned) const { return h.slot; }
};

__global__ void __launch_bounds__(K1_THREADS, 3) k_spawn(const DevInst *__restrict__ insts, const int *__restrict__ unit_start,
                                                      int n_inst, int n_units)
{
    extern __shared__ __align__(16) unsigned char k1_raw[];
    K1Smem &S = *reinterpret_cast<K1Smem *>(k1_raw);
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    constexpr int PER = CAP_M / K1_THREADS;
    // the run's state at the start of the iteration, read once per run a
    // block meets (a flag raised by another block during this kernel makes the
    // host repeat the iteration, whose output is then discarded)
    int cur = -1, err = 0, par = 0;
    long long it = 0;
    double shift = 0.0;
    if (t == 0) S.ndiv = 0;  // visible after the first run header's barrier
    for (int u = blockIdx.x; u < n_units; u += gridDim.x) {
        const int ii = find_inst(unit_start, n_inst, u);
        const DevInst &I = insts[ii];
        if (ii != cur) {
            if (t == 0) {
                S.hdr_err = *(volatile int *)&I.st->err;
                S.hdr_par = I.st->parity;
                S.hdr_it = I.st->iter;
                S.hdr_S = I.st->S;
                I.st->err_at_start = S.hdr_err;  // the same value from every block of the run
            }
            __syncthreads();
            err = S.hdr_err;
            par = S.hdr_par;
            it = S.hdr_it;
            shift = S.hdr_S;
            cur = ii;
            __syncthreads();
        }
        if (err) continue;
        const int b = u - I.unit0;
        const int m = I.cnt[par][b];
        const size_t base = (size_t)b * CAP_M;
        // load the bucket: thread t owns determinants PER*t .. PER*t+PER-1
        long long att = 0;
        unsigned mine = 0;
        unsigned nl[PER];
        for (int j = 0; j < PER; j++) {
            const int d = PER * t + j;
            nl[j] = 0;
            bool dv = false;
            if (d < m) {
                const ulonglong2 kk = I.key[par][base + d];
                const double c = I.c[par][base + d];
                const uint8_t f = I.fl[par][base + d];
                unsigned fl = 0;
                double cper = 0.0;
                u64 nat = 0;
                if (!is_zero(c)) {
                    if (!abs_lt(c, 0x1p31)) {
                        atomicOr(&I.st->err, ERRB_NUMERIC);
                    } else {
                        nat = ceil_abs(c);
                        const bool init = (dbits(c) & ~SIGN64) > dbits(I.n_a) || (f & (DFLAG_REF | DFLAG_D));
                        fl = (init ? 1u : 0u) | ((f & DFLAG_D) ? 2u : 0u);
                        cper = c;  // C / n_att: below for n_att > 1 (c / 1 is c)
                        att += (long long)nat;
                        if (nat > HEAVY_ATT) {  // sliced into the heavy queue
                            cper = c / (double)nat;
                            const unsigned nch = (unsigned)((nat + HEAVY_ATT - 1) / HEAVY_ATT);
                            const int q0 = atomicAdd(&I.st->heavy_n, (int)nch);
                            if ((long long)q0 + nch > (long long)I.heavy_cap) atomicOr(&I.st->err, ERRB_HEAVY_CAP);
                            else
                                for (unsigned q = 0; q < nch; q++) {
                                    HeavyChunk h;
                                    h.a = kk.x; h.b = kk.y; h.cper = cper; h.k0 = (u64)q * HEAVY_ATT;
                                    const u64 left = nat - h.k0;
                                    h.count = (unsigned)(left < HEAVY_ATT ? left : HEAVY_ATT);
                                    h.flags = fl;
                                    h.slot = (uint32_t)(base + d);
                                    h.pad = 0;
                                    I.heavy[q0 + q] = h;
                                }
                        } else {
                            nl[j] = (unsigned)nat;
                            dv = nat > 1;
                        }
                    }
                }
                S.key[d] = kk;
                S.cper[d] = cper;
                S.fl[d] = (unsigned char)fl;
                mine += nl[j];
            }
            queue_div(S, dv, d, lane);
        }
        // the parents of the first CHUNK attempts, written below by the
        // determinants with few attempts; the others are found by bisection
        for (int q = t; q < CHUNK; q += K1_THREADS) S.att_det[q] = 0xffffu;
        // exclusive scan of the light attempt counts in determinant order
        unsigned v = mine;
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned y = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += y;
        }
        if (lane == 31) S.wsum[warp] = v;
        __syncthreads();
        if (warp == 0) {
            unsigned x = lane < K1_THREADS / 32 ? S.wsum[lane] : 0u;
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            if (lane < K1_THREADS / 32) S.wsum[lane] = x;
        } else {
            divide_listed(S.divl, S.ndiv, S.cper, t - 32, K1_THREADS - 32);  // warp 0 scans meanwhile
        }
        __syncthreads();
        if (t == 0) S.ndiv = 0;  // read by every thread before the barrier above
        unsigned ex = v - mine + (warp ? S.wsum[warp - 1] : 0u);
        for (int j = 0; j < PER; j++) {
            S.off[PER * t + j] = ex;
            if (nl[j] <= 8u && ex + nl[j] <= (unsigned)CHUNK)
                for (unsigned q = 0; q < nl[j]; q++) S.att_det[ex + q] = (unsigned short)(PER * t + j);
            ex += nl[j];
        }
        if (t == K1_THREADS - 1) S.off[CAP_M] = ex;
        __syncthreads();
        const unsigned total = S.off[CAP_M];
        BucketMap map{&S, (unsigned)base};
        run_attempts(I, S, it, total, map, par, shift);
        // attempts of this bucket (light and heavy) into the run's exact total
        for (int o = 16; o >= 1; o >>= 1) att += __shfl_xor_sync(0xffffffffu, att, o);
        if (lane == 0 && att) red_add(&I.acc[(b % NSHARD) * ACC_STRIDE + ACC_ATT], (u64)att);
    }
}

__global__ void __launch_bounds__(K1_THREADS) k_spawn_heavy(const DevInst *__restrict__ insts, int n_inst)
{
    extern __shared__ __align__(16) unsigned char k1_raw[];
    K1Smem &S = *reinterpret_cast<K1Smem *>(k1_raw);
    for (int ii = 0; ii < n_inst; ii++) {
        const DevInst &I = insts[ii];
        if (threadIdx.x == 0) {
            S.hdr_err = *(volatile int *)&I.st->err;
            S.qn[0] = I.st->heavy_n;
            S.hdr_it = I.st->iter;
            S.hdr_par = I.st->parity;
            S.hdr_S = I.st->S;
        }
        __syncthreads();
        const int err = S.hdr_err, nh = S.qn[0], par = S.hdr_par;
        const long long it = S.hdr_it;
        const double shift = S.hdr_S;
        __syncthreads();
        if (err) continue;
        for (int q = blockIdx.x; q < nh; q += gridDim.x) {
            HeavyMap map{I.heavy[q]};
            run_attempts(I, S, it, map.h.count, map, par, shift);
        }
    }
}

// ------------------------------------------------------------------ annihilation
// Per bucket, one block: the bucket's walkers and spawns are staged (shared
// memory for up to EMAX records, a global scratch slice for larger buckets)
// and every distinct determinant gets one owner record through an
// open-addressing table: walkers are inserted first, then every spawn finds
// its target or inserts itself as the owner of a new determinant.  Accepted
// weights are added to the owner's exact 128-bit accumulator with two 64-bit
// atomics (the low word's carry goes to the high word), so the sum does not
// depend on the order of arrival.
template <typename IDX>
struct Stage {
    ulonglong2 *key;
    double *val;      // C (walkers) or w (spawns); after death C', after annihilation the result
    u64 *acc_lo;
    u64 *acc_hi;
    int *nacc;        // accepted spawns per owner
    int *eflag;       // EF_* bits
    IDX *tab;         // hash table: element index + 1, 0 = empty
    IDX *opos;        // output position of kept owners
};
enum { EF_OWNER = 1, EF_OCC = 2, EF_KEEP = 4, EF_ACC = 8, EF_REF = 16, EF_D = 32, EF_REJ = 64, EF_RREC = 128 };
// EF_REJ: a rejected spawn arrived (owners); EF_RREC: this spawn was rejected;
// EF_ACC: an accepted spawn arrived (owners, three-phase path)

struct K3Shared {
    int wsum[K3_THREADS / 32];
    double red_t[K3_THREADS / 32][2];
    u64 red_u[K3_THREADS / 32][8];
    int n_new, side_n;
    int hdr_err, hdr_par;
    long long hdr_it;
    double hdr_S;
};

struct K3Smem {
    K3Shared sh;
    ulonglong2 key[EMAX];
    double val[EMAX];
    u64 acc_lo[EMAX];
    u64 acc_hi[EMAX];
    int nacc[EMAX];
    int eflag[EMAX];
    unsigned short tab[1 << TABBITS];
    unsigned short opos[EMAX];
};
static_assert(3 * (sizeof(K3Smem) + 1024) <= 233472, "three annihilation blocks per SM");

__device__ __forceinline__ int block_excl_scan(int v, int *wsum, int *total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int x = v;
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int s = lane < K3_THREADS / 32 ? wsum[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < K3_THREADS / 32) wsum[lane] = s;
    }
    __syncthreads();
    int r = x - v + (warp ? wsum[warp - 1] : 0);
    *total = wsum[K3_THREADS / 32 - 1];
    return r;  // wsum is written again only after the caller's next barrier
}

// slot of determinant (a, b) in the trial-estimator table, or -1
__device__ __forceinline__ int trial_find(const DevInst &I, u64 a, u64 b)
{
    const u64 mask = (1ULL << I.trial_bits) - 1;
    u64 s = det_hash(a, b) & mask;
    for (u64 probe = 0; probe <= mask; probe++) {
        if (__ldg(I.trial_state + s) == 0u) return -1;
        if (__ldg(&I.trial_tab[s].a) == a && __ldg(&I.trial_tab[s].b) == b) return (int)s;
        s = (s + 1) & mask;
    }
    return -1;
}

// Death, annihilation and the reductions of one bucket b (steps (b) and (c)
// of Eq. (4)).  All threads of the block call this together.
template <typename IDX>
__device__ void anni_bucket(const DevInst &I, K3Shared &S, Stage<IDX> W, int tabbits, int b, int par, long long it,
                            double shift, int m, int si, int sn)
{
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int E = m + si + sn, cap_s = I.cap_s, TAB = 1 << tabbits;
    const u64 tmask = (u64)(TAB - 1);
    const size_t base = (size_t)b * CAP_M, sbase = (size_t)b * cap_s;
    const ulonglong2 *okey = I.key[par];
    const double *oc = I.c[par], *ohd = I.hd[par];
    const uint8_t *ofl = I.fl[par];

    // 1. stage: walkers [0, m), initiator spawns [m, m+si), other spawns [m+si, E);
    //    four records per thread per round, all loads issued before the stores
    for (int q = t; q < TAB; q += K3_THREADS) W.tab[q] = 0;
    if (t == 0) S.n_new = 0;
    for (int e0 = 0; e0 < E; e0 += 4 * K3_THREADS) {
        ulonglong2 k[4];
        double v[4];
        int f[4];
#pragma unroll
        for (int r = 0; r < 4; r++) {
            const int e = e0 + r * K3_THREADS + t;
            k[r] = make_ulonglong2(0, 0);
            v[r] = 0.0;
            f[r] = 0;
            if (e < m) {
                k[r] = okey[base + e];
                v[r] = oc[base + e];
                const uint8_t fl = ofl[base + e];
                f[r] = EF_OWNER | ((fl & DFLAG_REF) ? EF_REF : 0) | ((fl & DFLAG_D) ? EF_D : 0);
            } else if (e < m + si) {
                k[r] = I.skey[sbase + (e - m)];
                v[r] = I.sw[sbase + (e - m)];
            } else if (e < E) {
                const int slot = cap_s - 1 - (e - m - si);
                k[r] = I.skey[sbase + slot];
                v[r] = I.sw[sbase + slot];
            }
        }
#pragma unroll
        for (int r = 0; r < 4; r++) {
            const int e = e0 + r * K3_THREADS + t;
            if (e < E) {
                W.key[e] = k[r];
                W.val[e] = v[r];
                W.acc_lo[e] = 0;
                W.acc_hi[e] = 0;
                W.nacc[e] = 0;
                W.eflag[e] = f[r] | ((e < m && !is_zero(v[r])) ? EF_OCC : 0);
            }
        }
    }
    __syncthreads();
    // 2. walkers (thread t holds walkers t + r K3_THREADS, r < 4): insert into
    //    the table (keys are distinct); death (b) and Eq. (3), the rounding
    //    draws two at a time
    static_assert(CAP_M <= 4 * K3_THREADS, "walkers per thread");
    double hdr[4];
#pragma unroll
    for (int r = 0; r < 4; r++) {
        const int e = t + r * K3_THREADS;
        hdr[r] = e < m ? ohd[base + e] : 0.0;
    }
#pragma unroll
    for (int r = 0; r < 4; r++) {
        const int e = t + r * K3_THREADS;
        if (e < m) {
            const ulonglong2 k = W.key[e];
            u64 s = det_hash(k.x, k.y) & tmask;
            while (atomicCAS(&W.tab[s], (IDX)0, (IDX)(e + 1)) != (IDX)0) s = (s + 1) & tmask;
        }
    }
#pragma unroll
    for (int r0 = 0; r0 < 4; r0 += 2) {
        double cp[2];
        bool draw[2];
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const int e = t + (r0 + h) * K3_THREADS;
            draw[h] = false;
            cp[h] = 0.0;
            if (e < m) {
                if (W.eflag[e] & EF_D) {
                    const ulonglong2 k = W.key[e];
                    cp[h] = I.dc_new[d_index_of(I, k.x, k.y)];
                } else {
                    // C (1 - tau (H_ii - E_ref - S_i)), then rounding with the death draw;
                    // S_i = f_i S for a non-initiator with the adaptive shift (Sec. V)
                    double Si = shift;
                    const bool init = (dbits(W.val[e]) & ~SIGN64) > dbits(I.n_a) || (W.eflag[e] & EF_REF);
                    if (I.adaptive && !init) {
                        const u64 *acc = I.facc[par] + (base + e) * 4;
                        const u128 A = ((u128)acc[1] << 64) | acc[0], T = ((u128)acc[3] << 64) | acc[2];
                        if (T != 0) Si = (u128_to_double(A) / u128_to_double(T)) * shift;
                    }
                    const double fct = 1.0 - I.tau * (hdr[r0 + h] - Si);
                    cp[h] = W.val[e] * fct;
                    draw[h] = !is_zero(cp[h]) && abs_lt(cp[h], I.cmin);
                }
            }
        }
        if (I.side)  // replica pair: walkers' entries (start amplitude, H_ii - E_ref)
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const int e = t + (r0 + h) * K3_THREADS;
                if (e < m) {
                    SideEnt &se = I.side[(size_t)b * I.side_cap + e];
                    const ulonglong2 k = W.key[e];
                    se.a = k.x; se.b = k.y; se.c0 = W.val[e]; se.hd = hdr[r0 + h]; se.sacc = 0.0; se.srej = 0.0;
                }
            }
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const int e = t + (r0 + h) * K3_THREADS;
            if (draw[h]) {
                const ulonglong2 k = W.key[e];
                u64 w[4];
                philox(k.x, k.y, (u64)it, (u64)PURPOSE_DEATH, I.seed, I.replica, w);
                cp[h] = round_stoch(cp[h], I.cmin, I.cmin_log2, I.cmin_pow2, w[0]);
            }
            if (e < m) W.val[e] = cp[h];
        }
    }
    __syncthreads();
    // 3. spawns: find the target or become the owner of a new determinant;
    //    initiator rule (Sec. I): a non-initiator spawn survives only onto a
    //    determinant occupied at the start of the iteration
    long long rejected = 0;
    i128 ann = 0;
    for (int e = m + t; e < E; e += K3_THREADS) {
        const ulonglong2 k = W.key[e];
        u64 s = det_hash(k.x, k.y) & tmask;
        int target = -1;
        while (true) {
            IDX v = ((volatile IDX *)W.tab)[s];
            if (v == 0) {
                IDX old = atomicCAS(&W.tab[s], (IDX)0, (IDX)(e + 1));
                if (old == 0) { target = e; break; }
                v = old;
            }
            const int tt = (int)v - 1;
            const ulonglong2 kk = W.key[tt];
            if (kk.x == k.x && kk.y == k.y) { target = tt; break; }
            s = (s + 1) & tmask;
        }
        if (target == e) atomicOr(&W.eflag[e], EF_OWNER);
        const bool init = e < m + si;
        const bool accepted = init || (target < m && (W.eflag[target] & EF_OCC));
        if (!accepted) {
            rejected++;
            if (I.side) {
                W.opos[e] = (IDX)target;
                atomicOr(&W.eflag[e], EF_RREC);
                atomicOr(&W.eflag[target], EF_REJ);
            }
            continue;
        }
        const double w = W.val[e];
        const i128 x = to_fixed(w, I.Fw);
        const u64 lo = (u64)x, hi = (u64)((u128)x >> 64);
        const u64 old = atomicAdd((unsigned long long *)&W.acc_lo[target], (unsigned long long)lo);
        atomicAdd((unsigned long long *)&W.acc_hi[target], (unsigned long long)(hi + (old + lo < old ? 1ULL : 0ULL)));
        atomicAdd(&W.nacc[target], 1);
        ann += (i128)fx32(w);
    }
    __syncthreads();
    // replica pair: every owner's entry receives the accepted and the rejected
    // spawn sums (exact, rounded once each); the rejected weights are summed
    // in the accumulators once the accepted sums have been read
    const bool side = I.side != nullptr;
    if (side) {
        if (t == 0) S.side_n = 0;
        __syncthreads();
        for (int e = t; e < E; e += K3_THREADS) {
            const int f = W.eflag[e];
            if (!(f & EF_OWNER)) continue;
            const bool had = W.nacc[e] > 0;
            const double sacc = had ? fixed_to_double((i128)(((u128)W.acc_hi[e] << 64) | (u128)W.acc_lo[e]), I.Fw)
                                    : 0.0;
            const int slot = e < m ? e : m + atomicAdd(&S.side_n, 1);
            SideEnt &se = I.side[(size_t)b * I.side_cap + slot];
            if (e >= m) {
                const ulonglong2 k = W.key[e];
                se.a = k.x; se.b = k.y; se.c0 = 0.0; se.hd = 0.0; se.srej = 0.0;
            }
            se.sacc = sacc;
            W.nacc[e] = (slot << 1) | (had ? 1 : 0);
            W.acc_lo[e] = 0;
            W.acc_hi[e] = 0;
        }
        __syncthreads();
        for (int e = m + t; e < E; e += K3_THREADS) {
            if (!(W.eflag[e] & EF_RREC)) continue;
            const int target = (int)W.opos[e];
            const i128 x = to_fixed(W.val[e], I.Fw);
            const u64 lo = (u64)x, hi = (u64)((u128)x >> 64);
            const u64 old = atomicAdd((unsigned long long *)&W.acc_lo[target], (unsigned long long)lo);
            atomicAdd((unsigned long long *)&W.acc_hi[target], (unsigned long long)(hi + (old + lo < old ? 1ULL : 0ULL)));
        }
        __syncthreads();
        for (int e = t; e < E; e += K3_THREADS) {
            const int f = W.eflag[e];
            if (!(f & EF_OWNER) || !(f & EF_REJ)) continue;
            const i128 X = (i128)(((u128)W.acc_hi[e] << 64) | (u128)W.acc_lo[e]);
            I.side[(size_t)b * I.side_cap + (W.nacc[e] >> 1)].srej = fixed_to_double(X, I.Fw);
        }
        if (t == 0) I.side_cnt[b] = m + S.side_n;
    }
    // 4. owners: sum = C' + exact spawn sum, then Eq. (3) with the annihilation draw
    int nk = 0;
    for (int e = t; e < E; e += K3_THREADS) {
        const int f = W.eflag[e];
        if (!(f & EF_OWNER)) continue;
        const bool present = e < m;
        const double cp = present ? W.val[e] : 0.0;
        double accv = cp;
        if (side ? (W.nacc[e] & 1) : W.nacc[e] > 0) {
            const double sw = side ? I.side[(size_t)b * I.side_cap + (W.nacc[e] >> 1)].sacc
                                   : fixed_to_double((i128)(((u128)W.acc_hi[e] << 64) | (u128)W.acc_lo[e]), I.Fw);
            accv = present ? cp + sw : sw;
            ann += (present ? (i128)fx32(cp) : (i128)0) - (i128)fx32(accv);
            if (!(f & EF_D) && !is_zero(accv) && abs_lt(accv, I.cmin)) {
                const ulonglong2 k = W.key[e];
                u64 w[4];
                philox(k.x, k.y, (u64)it, (u64)PURPOSE_ANNIH, I.seed, I.replica, w);
                accv = round_stoch(accv, I.cmin, I.cmin_log2, I.cmin_pow2, w[0]);
            }
        }
        W.val[e] = accv;
        if (!is_zero(accv) || (f & (EF_REF | EF_D))) {
            W.eflag[e] = f | EF_KEEP;
            nk++;
        }
    }
    // 5. output positions in element order
    int total;
    const int per = (E + K3_THREADS - 1) / K3_THREADS;
    const int e0 = t * per, e1 = min(E, e0 + per);
    int cnt = 0;
    __syncthreads();
    for (int e = e0; e < e1; e++) cnt += (W.eflag[e] & EF_KEEP) ? 1 : 0;
    int o = block_excl_scan(cnt, S.wsum, &total);
    const bool overflow = total > CAP_M;
    if (overflow && t == 0) { atomicOr(&I.st->err, ERRB_MAIN_CAP); atomicMax(&I.st->need_main, total); }
    for (int e = e0; e < e1; e++)
        if (W.eflag[e] & EF_KEEP) W.opos[e] = (IDX)(o++);
    (void)nk;
    __syncthreads();

    // 6. write the new bucket; reductions
    const int np = par ^ 1;
    ulonglong2 *nkey = I.key[np];
    double *nc = I.c[np], *nhd = I.hd[np];
    uint8_t *nfl = I.fl[np];
    u128 nw = 0;
    i128 enm = 0;  // E_num: each term truncated to the grid 2^-Fe (R12), summed exactly
    double tnum = 0.0, tden = 0.0;
    bool bad = false;
    if (!overflow) {
        for (int r = 0; t + r * K3_THREADS < E; r++) {
            const int e = t + r * K3_THREADS;
            const int f = W.eflag[e];
            if (!(f & EF_KEEP)) continue;
            const ulonglong2 k = W.key[e];
            const double c = W.val[e];
            const size_t dst = base + W.opos[e];
            nkey[dst] = k;
            nc[dst] = c;
            nfl[dst] = (uint8_t)(((f & EF_REF) ? DFLAG_REF : 0) | ((f & EF_D) ? DFLAG_D : 0));
            if (e < m) nhd[dst] = ohd[base + e];  // read again: an L2 hit, fewer live registers
            else {
                const int qn = atomicAdd(&S.n_new, 1);
                W.nacc[qn] = e;  // accumulators are free now: reuse as the list of new determinants
            }
            if (!abs_lt(c, 0x1p31)) bad = true;
            else nw += fx32(c);
            if (f & EF_REF) I.st->e_den = c;
            else {
                const int lev = __popcll(k.x ^ I.ref_a) + __popcll(k.y ^ I.ref_b);
                if (lev <= 4 && !is_zero(c)) enm += to_fixed(hoff_generic(I, k.x, k.y, I.ref_a, I.ref_b) * c, I.Fe);
            }
            if (f & EF_D) I.dc_buf[par ^ 1][d_index_of(I, k.x, k.y)] = c;
            if (I.trial_bits && !is_zero(c)) {  // trial-wave-function estimator (Sec. IV)
                const int ts = trial_find(I, k.x, k.y);
                if (ts >= 0) {
                    tnum = tnum + __ldg(&I.trial_tab[ts].w) * c;
                    tden = tden + __ldg(&I.trial_tab[ts].cT) * c;
                }
            }
        }
    }
    if (bad) atomicOr(&I.st->err, ERRB_NUMERIC);
    __syncthreads();
    // adaptive shift: the new list's index (hash -> position + 1) and zeroed
    // weight sums for the next iteration's spawns
    if (I.adaptive && !overflow) {
        for (int q = t; q < KIDX; q += K3_THREADS) W.tab[q] = 0;
        __syncthreads();
        for (int r = 0; t + r * K3_THREADS < E; r++) {
            const int e = t + r * K3_THREADS;
            if (!(W.eflag[e] & EF_KEEP)) continue;
            const ulonglong2 k = W.key[e];
            unsigned sl = (unsigned)det_hash(k.x, k.y) & (unsigned)(KIDX - 1);
            while (atomicCAS(&W.tab[sl], (IDX)0, (IDX)(W.opos[e] + 1)) != (IDX)0) sl = (sl + 1) & (unsigned)(KIDX - 1);
            u64 *acc = I.facc[np] + (base + W.opos[e]) * 4;
            acc[0] = 0; acc[1] = 0; acc[2] = 0; acc[3] = 0;
        }
        __syncthreads();
        for (int q = t; q < KIDX; q += K3_THREADS) I.kidx[np][(size_t)b * KIDX + q] = (unsigned short)W.tab[q];
    }
    // 7. new determinants: their slots go to the run's list; H_jj - E_ref is
    //    computed for all of them at once by k_new_diag, whose warps are not
    //    held back by this block's barriers
    if (!overflow) {  // each warp reserves the entries it writes (q = 32 warp + lane + K3_THREADS k)
        const int nnew = S.n_new;
        int cntw = 0;
        for (int q0 = warp * 32; q0 < nnew; q0 += K3_THREADS) cntw += min(32, nnew - q0);
        int nb0 = 0;
        if (lane == 0 && cntw > 0) nb0 = atomicAdd(&I.st->new_n, cntw);
        nb0 = __shfl_sync(0xffffffffu, nb0, 0);
        for (int q = t, k = 0; q < nnew; q += K3_THREADS, k++)
            I.newdet[nb0 + 32 * k + lane] = (unsigned)(base + W.opos[W.nacc[q]]);
    }
    // 8. bucket reductions (fixed order: lanes by xor tree, warps in index order)
    if (I.trial_bits)  // binary64 adds are slow on this part: only when the estimator is on
        for (int mm = 16; mm >= 1; mm >>= 1) {
            tnum = tnum + __shfl_xor_sync(0xffffffffu, tnum, mm);
            tden = tden + __shfl_xor_sync(0xffffffffu, tden, mm);
        }
    for (int mm = 16; mm >= 1; mm >>= 1) {
        enm += shfl_xor_i128(enm, mm);
        rejected += __shfl_xor_sync(0xffffffffu, rejected, mm);
        ann += shfl_xor_i128(ann, mm);
        nw += (u128)shfl_xor_i128((i128)nw, mm);
    }
    if (lane == 0) {
        S.red_t[warp][0] = tnum;
        S.red_t[warp][1] = tden;
        S.red_u[warp][0] = (u64)nw;
        S.red_u[warp][1] = (u64)(nw >> 64);
        S.red_u[warp][2] = (u64)ann;
        S.red_u[warp][3] = (u64)((u128)ann >> 64);
        S.red_u[warp][4] = (u64)rejected;
        S.red_u[warp][5] = (u64)enm;
        S.red_u[warp][6] = (u64)((u128)enm >> 64);
    }
    __syncthreads();
    if (t == 0) {
        double tn = 0.0, td = 0.0;
        u128 nws = 0;
        i128 anns = 0, ens = 0;
        long long rej = 0;
        for (int k = 0; k < K3_THREADS / 32; k++) {
            if (I.trial_bits) {
                tn = tn + S.red_t[k][0];
                td = td + S.red_t[k][1];
            }
            nws += ((u128)S.red_u[k][1] << 64) | S.red_u[k][0];
            anns += (i128)(((u128)S.red_u[k][3] << 64) | S.red_u[k][2]);
            rej += (long long)S.red_u[k][4];
            ens += (i128)(((u128)S.red_u[k][6] << 64) | S.red_u[k][5]);
        }
        // the bucket's share of the run's exact totals (its line b % NSHARD)
        u64 *acc = I.acc + (b % NSHARD) * ACC_STRIDE;
        limb_add(acc + ACC_NW, (i128)nws);
        limb_add(acc + ACC_ANN, anns);
        limb_add(acc + ACC_ENUM, ens);
        red_add(&acc[ACC_NDET], (u64)total);
        if (rej) red_add(&acc[ACC_REJ], (u64)rej);
        red_add(&acc[ACC_SPAWNS], (u64)(si + sn));
        if (I.trial_bits) {
            Partial &P = I.part[b];
            P.t_num = tn;
            P.t_den = td;
        }
        if (!overflow) I.cnt[np][b] = total;
        I.scnt_i[b] = 0;
        I.scnt_n[b] = 0;
    }
    // no closing barrier: what thread 0 still reads (the warp sums) is written
    // again only after the next bucket's barriers
}

// The same steps for a run without replica side lists or adaptive shift, in
// three block phases per bucket: (A) walkers inserted into the table, death
// and Eq. (3); (B) every spawn finds its target or becomes the owner of a new
// determinant, initiator rule, exact accumulation; (C) owners finalised
// (Eq. (3) with the annihilation draw), each kept one written straight to the
// new bucket at a position taken from a shared counter (the order inside a
// bucket affects no result), the new determinants listed, the bucket's totals
// reduced, and the table cleared for the next bucket.  Writes beyond the
// bucket's capacity are skipped: the overflow flag makes the host repeat the
// iteration after growth.
//
// Where the records come from is a policy: LoadStage reads them from global
// memory in phase A into the block's shared arrays; BulkStage finds them
// already in shared memory, placed there by bulk copies issued while the
// previous bucket was processed.
struct Work3 {       // per-record working arrays shared by both policies
    u64 *acc_lo, *acc_hi;
    int *eflag;
    unsigned short *tab;
};

struct LoadStage {
    ulonglong2 *key;  // [EMAX]: walkers, then spawns
    double *val;      // [EMAX]: C' after death (walkers), w (spawns)
    int m, si, sn, cap_s;
    size_t base, sbase;
    const DevInst *I;
    int par;
    __device__ void walker(int e, ulonglong2 &k, double &c, double &hd, uint8_t &f) const
    {
        k = I->key[par][base + e];
        c = I->c[par][base + e];
        hd = I->hd[par][base + e];
        f = I->fl[par][base + e];
    }
    __device__ void put_walker(int e, ulonglong2 k) const { key[e] = k; }
    __device__ void stage_spawns(int t) const  // spawns: initiator [m, m+si), the others [m+si, E)
    {
        for (int e = m + t; e < m + si + sn; e += K3_THREADS) {
            const int q = e - m;
            const size_t o = sbase + (q < si ? q : cap_s - 1 - (q - si));
            key[e] = I->skey[o];
            val[e] = I->sw[o];
        }
    }
    __device__ ulonglong2 k(int e) const { return key[e]; }
    __device__ double v(int e) const { return val[e]; }
    __device__ void set_v(int e, double x) const { val[e] = x; }
    __device__ double hd_out(int e) const { return I->hd[par][base + e]; }  // read again: an L2 hit
};

// one bucket's raw records in shared memory, filled by bulk copies
template <int SCAP>
struct AStage {
    ulonglong2 wkey[CAP_M];
    ulonglong2 skey[SCAP];      // initiator spawns [0, si), the others [si, si + sn)
    double wc[CAP_M];           // C; after death C'
    double whd[CAP_M];
    double sw[SCAP + 2];        // initiator weights [0, si), the others from swo (16-byte aligned copies)
    uint8_t wfl[CAP_M];
};

template <int SCAP>
struct BulkStage {
    AStage<SCAP> *st;
    int m, si, swo;
    __device__ void walker(int e, ulonglong2 &k, double &c, double &hd, uint8_t &f) const
    {
        k = st->wkey[e];
        c = st->wc[e];
        hd = st->whd[e];
        f = st->wfl[e];
    }
    __device__ void put_walker(int, ulonglong2) const {}
    __device__ void stage_spawns(int) const {}
    __device__ ulonglong2 k(int e) const { return e < m ? st->wkey[e] : st->skey[e - m]; }
    __device__ double v(int e) const
    {
        if (e < m) return st->wc[e];
        const int q = e - m;
        return q < si ? st->sw[q] : st->sw[swo + (q - si)];
    }
    __device__ void set_v(int e, double x) const { st->wc[e] = x; }  // walkers only
    __device__ double hd_out(int e) const { return st->whd[e]; }
};

// A thread's share of a run's exact integer totals over the buckets its
// block meets in one annihilation launch (integer sums: any order gives the
// same total), added to the run's accumulators once, when the block leaves
// the run
struct AnniTotals {
    u128 nw = 0;            // N_w * 2^32
    i128 ann = 0;           // annihilated walkers * 2^32
    i128 enm = 0;           // E_num * 2^Fe (terms truncated to the grid)
    long long rej = 0;      // rejected non-initiator spawns
    long long ndet = 0;     // determinants kept (thread 0)
    long long spawns = 0;   // spawns received (thread 0)
};

// every thread of the block: the totals into the run's accumulators (line
// blockIdx.x % NSHARD), then zero
__device__ void anni_flush(const DevInst &I, AnniTotals &T)
{
    const int lane = threadIdx.x & 31;
    for (int mm = 16; mm >= 1; mm >>= 1) {
        T.rej += __shfl_xor_sync(0xffffffffu, T.rej, mm);
        T.ann += shfl_xor_i128(T.ann, mm);
        T.nw += (u128)shfl_xor_i128((i128)T.nw, mm);
        T.enm += shfl_xor_i128(T.enm, mm);
    }
    u64 *acc = I.acc + (blockIdx.x % NSHARD) * ACC_STRIDE;
    if (lane == 0) {
        limb_add(acc + ACC_NW, (i128)T.nw);
        limb_add(acc + ACC_ANN, T.ann);
        limb_add(acc + ACC_ENUM, T.enm);
        if (T.rej) red_add(&acc[ACC_REJ], (u64)T.rej);
    }
    if (threadIdx.x == 0) {
        if (T.ndet) red_add(&acc[ACC_NDET], (u64)T.ndet);
        if (T.spawns) red_add(&acc[ACC_SPAWNS], (u64)T.spawns);
    }
    T = AnniTotals{};
}

template <typename SRC>
__device__ void anni_bucket_3p(const DevInst &I, K3Shared &S, const Work3 &W, const SRC &R, int b, int par,
                               long long it, double shift, int m, int si, int sn, AnniTotals &T)
{
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int E = m + si + sn;
    constexpr u64 tmask = (u64)((1 << TABBITS) - 1);
    const size_t base = (size_t)b * CAP_M;
    const unsigned below = (1u << lane) - 1u;

    // A. walkers, two per thread at a time: loads issued first, then
    //    insertion and death (b) with Eq. (3)
    static_assert(CAP_M <= 4 * K3_THREADS, "walkers per thread");
#pragma unroll
    for (int r0 = 0; r0 < 4; r0 += 2) {
        ulonglong2 k[2];
        double c[2], hd[2];
        int f[2];
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const int e = t + (r0 + h) * K3_THREADS;
            k[h] = make_ulonglong2(0, 0);
            c[h] = 0.0;
            hd[h] = 0.0;
            f[h] = 0;
            if (e < m) {
                uint8_t fl;
                R.walker(e, k[h], c[h], hd[h], fl);
                f[h] = EF_OWNER | ((fl & DFLAG_REF) ? EF_REF : 0) | ((fl & DFLAG_D) ? EF_D : 0);
            }
        }
        double cp[2];
        bool draw[2];
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const int e = t + (r0 + h) * K3_THREADS;
            draw[h] = false;
            cp[h] = 0.0;
            if (e < m) {
                R.put_walker(e, k[h]);
                W.acc_lo[e] = 0;
                W.acc_hi[e] = 0;
                W.eflag[e] = f[h] | (!is_zero(c[h]) ? EF_OCC : 0);
                u64 sl = det_hash(k[h].x, k[h].y) & tmask;
                while (atomicCAS(&W.tab[sl], (unsigned short)0, (unsigned short)(e + 1)) != 0) sl = (sl + 1) & tmask;
                if (f[h] & EF_D) cp[h] = I.dc_new[d_index_of(I, k[h].x, k[h].y)];
                else {
                    cp[h] = c[h] * (1.0 - I.tau * (hd[h] - shift));
                    draw[h] = !is_zero(cp[h]) && abs_lt(cp[h], I.cmin);
                }
            }
        }
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const int e = t + (r0 + h) * K3_THREADS;
            if (draw[h]) {
                u64 w[4];
                philox(k[h].x, k[h].y, (u64)it, (u64)PURPOSE_DEATH, I.seed, I.replica, w);
                cp[h] = round_stoch(cp[h], I.cmin, I.cmin_log2, I.cmin_pow2, w[0]);
            }
            if (e < m) R.set_v(e, cp[h]);
        }
    }
    R.stage_spawns(t);
    for (int e = m + t; e < E; e += K3_THREADS) {
        W.acc_lo[e] = 0;
        W.acc_hi[e] = 0;
        W.eflag[e] = 0;
    }
    __syncthreads();

    // B. spawns: find the target or become the owner of a new determinant;
    //    initiator rule (Sec. I): a non-initiator spawn survives only onto a
    //    determinant occupied at the start of the iteration
    long long rejected = 0;
    i128 ann = 0;
    for (int e = m + t; e < E; e += K3_THREADS) {
        const ulonglong2 k = R.k(e);
        u64 sl = det_hash(k.x, k.y) & tmask;
        int target = -1;
        while (true) {
            unsigned short v = ((volatile unsigned short *)W.tab)[sl];
            if (v == 0) {
                const unsigned short old = atomicCAS(&W.tab[sl], (unsigned short)0, (unsigned short)(e + 1));
                if (old == 0) { target = e; break; }
                v = old;
            }
            const int tt = (int)v - 1;
            const ulonglong2 kk = R.k(tt);
            if (kk.x == k.x && kk.y == k.y) { target = tt; break; }
            sl = (sl + 1) & tmask;
        }
        if (target == e) atomicOr(&W.eflag[e], EF_OWNER);  // EF_ACC may be arriving from another spawn
        const bool accepted = (e < m + si) || (target < m && (W.eflag[target] & EF_OCC));
        if (!accepted) { rejected++; continue; }
        const double w = R.v(e);
        const i128 x = to_fixed(w, I.Fw);
        const u64 lo = (u64)x, hi = (u64)((u128)x >> 64);
        const u64 old = atomicAdd((unsigned long long *)&W.acc_lo[target], (unsigned long long)lo);
        atomicAdd((unsigned long long *)&W.acc_hi[target], (unsigned long long)(hi + (old + lo < old ? 1ULL : 0ULL)));
        atomicOr(&W.eflag[target], EF_ACC);
        ann += (i128)fx32(w);
    }
    __syncthreads();

    // C. owners: sum = C' + exact spawn sum, Eq. (3) with the annihilation
    //    draw; kept determinants written to the new bucket
    const int np = par ^ 1;
    ulonglong2 *nkey = I.key[np];
    double *nc = I.c[np], *nhd = I.hd[np];
    uint8_t *nfl = I.fl[np];
    u128 nw = 0;
    double tnum = 0.0, tden = 0.0;
    bool bad = false;
    for (int e0 = 0; e0 < E; e0 += K3_THREADS) {
        const int e = e0 + t;
        int f = 0;
        double accv = 0.0;
        bool keep = false;
        if (e < E) {
            f = W.eflag[e];
            if (f & EF_OWNER) {
                const bool present = e < m;
                const double cp = present ? R.v(e) : 0.0;
                accv = cp;
                if (f & EF_ACC) {
                    const double sw = fixed_to_double((i128)(((u128)W.acc_hi[e] << 64) | (u128)W.acc_lo[e]), I.Fw);
                    accv = present ? cp + sw : sw;
                    ann += (present ? (i128)fx32(cp) : (i128)0) - (i128)fx32(accv);
                    if (!(f & EF_D) && !is_zero(accv) && abs_lt(accv, I.cmin)) {
                        const ulonglong2 k = R.k(e);
                        u64 w[4];
                        philox(k.x, k.y, (u64)it, (u64)PURPOSE_ANNIH, I.seed, I.replica, w);
                        accv = round_stoch(accv, I.cmin, I.cmin_log2, I.cmin_pow2, w[0]);
                    }
                }
                keep = !is_zero(accv) || (f & (EF_REF | EF_D));
            }
        }
        // positions in the new bucket from a shared counter, one atomic per warp
        const unsigned mk = __ballot_sync(0xffffffffu, keep);
        int pb = 0;
        if (lane == 0 && mk) pb = atomicAdd(&S.n_new, __popc(mk));
        pb = __shfl_sync(0xffffffffu, pb, 0);
        const int pos = pb + __popc(mk & below);
        const bool write = keep && pos < CAP_M;
        // the slots of new determinants go to the run's list (H_jj by k_new_diag)
        const unsigned mn = __ballot_sync(0xffffffffu, write && e >= m);
        int qb = 0;
        if (lane == 0 && mn) qb = atomicAdd(&I.st->new_n, __popc(mn));
        qb = __shfl_sync(0xffffffffu, qb, 0);
        if (write) {
            const ulonglong2 k = R.k(e);
            const size_t dst = base + pos;
            nkey[dst] = k;
            nc[dst] = accv;
            nfl[dst] = (uint8_t)(((f & EF_REF) ? DFLAG_REF : 0) | ((f & EF_D) ? DFLAG_D : 0));
            if (e < m) nhd[dst] = R.hd_out(e);
            else I.newdet[qb + __popc(mn & below)] = (unsigned)dst;
            if (!abs_lt(accv, 0x1p31)) bad = true;
            else nw += fx32(accv);
            if (f & EF_REF) I.st->e_den = accv;
            else {
                const int lev = __popcll(k.x ^ I.ref_a) + __popcll(k.y ^ I.ref_b);
                if (lev <= 4 && !is_zero(accv))  // E_num term on the grid 2^-Fe (R12)
                    T.enm += to_fixed(hoff_generic(I, k.x, k.y, I.ref_a, I.ref_b) * accv, I.Fe);
            }
            if (f & EF_D) I.dc_buf[np][d_index_of(I, k.x, k.y)] = accv;
            if (I.trial_bits && !is_zero(accv)) {  // trial-wave-function estimator (Sec. IV)
                const int ts = trial_find(I, k.x, k.y);
                if (ts >= 0) {
                    tnum = tnum + __ldg(&I.trial_tab[ts].w) * accv;
                    tden = tden + __ldg(&I.trial_tab[ts].cT) * accv;
                }
            }
        }
    }
    // the table is read no more in this bucket: clear it for the next one
    {
        uint4 *tz = reinterpret_cast<uint4 *>(W.tab);
        for (int q = t; q < (int)((sizeof(unsigned short) << TABBITS) / sizeof(uint4)); q += K3_THREADS)
            tz[q] = make_uint4(0, 0, 0, 0);
    }
    if (bad) atomicOr(&I.st->err, ERRB_NUMERIC);
    // bucket reductions (fixed order: lanes by xor tree, warps in index order)
    // the integer totals (E_num's truncated terms among them) stay in the
    // thread and are added to the run's accumulators when the block leaves
    // the run; the trial sums are binary64, summed per bucket in a fixed order
    // (lanes by xor tree, warps in index order)
    T.rej += rejected;
    T.ann += ann;
    T.nw += nw;
    if (I.trial_bits)
        for (int mm = 16; mm >= 1; mm >>= 1) {
            tnum = tnum + __shfl_xor_sync(0xffffffffu, tnum, mm);
            tden = tden + __shfl_xor_sync(0xffffffffu, tden, mm);
        }
    if (lane == 0) {
        S.red_t[warp][0] = tnum;
        S.red_t[warp][1] = tden;
    }
    __syncthreads();
    if (t == 0) {
        const int total = S.n_new;
        S.n_new = 0;  // next used after two more barriers
        double tn = 0.0, td = 0.0;
        if (I.trial_bits)
            for (int k = 0; k < K3_THREADS / 32; k++) {
                tn = tn + S.red_t[k][0];
                td = td + S.red_t[k][1];
            }
        if (total > CAP_M) { atomicOr(&I.st->err, ERRB_MAIN_CAP); atomicMax(&I.st->need_main, total); }
        T.ndet += total;
        T.spawns += si + sn;
        if (I.trial_bits) {
            Partial &P = I.part[b];
            P.t_num = tn;
            P.t_den = td;
        }
        if (total <= CAP_M) I.cnt[np][b] = total;
        I.scnt_i[b] = 0;
        I.scnt_n[b] = 0;
    }
}

// ------------------------------------------------------------------ staged annihilation
// Bulk copies (cp.async.bulk, global -> this CTA's shared memory; source in
// this GPU's own memory, no multicast), completion counted in bytes on an
// mbarrier.  Addresses and sizes are multiples of 16 bytes.
__device__ __forceinline__ unsigned smem_addr(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(u64 *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(u64 *bar, unsigned bytes)
{
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, u64 *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}
// one bounded probe of the barrier's phase (the hardware may suspend the thread a while)
__device__ __forceinline__ bool mbar_test(u64 *bar, unsigned parity)
{
    unsigned ok;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok)
                 : "r"(smem_addr(bar)), "r"(parity)
                 : "memory");
    return ok != 0;
}
constexpr long long MBAR_POLLS = 1LL << 24;  // bound on the polls of one wait
__device__ __forceinline__ bool mbar_wait(u64 *bar, unsigned parity)
{
    for (long long k = 0; k < MBAR_POLLS; k++)
        if (mbar_test(bar, parity)) return true;
    return false;
}

template <int SCAP>
struct K4Smem {
    K3Shared sh;
    u64 bar[2];
    int binfo[2][8];  // per stage: bucket (-1: nothing staged), m, si, sn, swo, run, parity, error
    long long bit[2];
    double bS[2];
    AStage<SCAP> st[2];
    u64 acc_lo[CAP_M + SCAP], acc_hi[CAP_M + SCAP];
    int eflag[CAP_M + SCAP];
    unsigned short tab[1 << TABBITS];
};
static_assert(2 * (sizeof(K4Smem<STAGED_SCAP>) + 1024) <= 233472, "two staged annihilation blocks per SM");

// What thread 0 knows of a unit before its copies go out: the run's state
// (read once per run the block meets) and the bucket's counts, loaded one
// bucket ahead of their use so that their latency is hidden
struct StageMeta {
    int u, ii, b, m, si, sn, par, err;
    long long it;
    double S;
};

__device__ __forceinline__ void meta_load(const DevInst *__restrict__ insts, const int *__restrict__ unit_start,
                                          int n_inst, int u, StageMeta &M)
{
    M.u = u;
    if (u < 0) return;
    const int ii = find_inst(unit_start, n_inst, u);
    const DevInst &I = insts[ii];
    if (ii != M.ii) {
        M.ii = ii;
        M.err = *(volatile int *)&I.st->err;
        M.par = I.st->parity;
        M.it = I.st->iter;
        M.S = I.st->S;
    }
    M.b = u - I.unit0;
    M.m = I.cnt[M.par][M.b];
    M.si = I.scnt_i[M.b];
    M.sn = I.scnt_n[M.b];
}

// thread 0: the checks of k_annihilate on unit M.u, then the bulk copies of
// its bucket into stage q (completion on bar[q]); the stage's info tells the
// block whether and what to process
template <int SCAP>
__device__ void stage_issue(const DevInst *__restrict__ insts, const StageMeta &M, K4Smem<SCAP> &Sm, int q)
{
    int *bi = Sm.binfo[q];
    bi[0] = -1;
    if (M.u < 0 || M.err) return;
    const DevInst &I = insts[M.ii];
    const int par = M.par, b = M.b, m = M.m, si = M.si, sn = M.sn, cap_s = I.cap_s;
    if (si + sn > cap_s) {
        atomicOr(&I.st->err, ERRB_SPAWN_CAP);
        atomicMax(&I.st->need_spawn, si + sn);
        atomicAdd(&I.st->n_spawn_over, 1);
        return;
    }
    if (m + si + sn > EMAX) {  // too large for shared memory: deferred to k_annihilate_big
        I.big_list[atomicAdd(&I.st->big_n, 1)] = b;
        return;
    }
    if (si + sn > SCAP) {
        // more spawns than the stage holds, but within the working arrays: the
        // block loads this bucket itself (no copies; the phase completes at once)
        bi[1] = m; bi[2] = si; bi[3] = sn; bi[4] = 0; bi[5] = M.ii; bi[6] = par; bi[7] = 1;
        Sm.bit[q] = M.it;
        Sm.bS[q] = M.S;
        bi[0] = b;
        asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_addr(&Sm.bar[q]))
                     : "memory");
        return;
    }
    AStage<SCAP> &st = Sm.st[q];
    const size_t base = (size_t)b * CAP_M, sbase = (size_t)b * cap_s;
    // 16-byte multiples: C and H_ii rounded up to an even count, flags to 16
    // (all within the bucket's CAP_M slots); the non-initiator weights start
    // at an even slot (one slot early when cap_s - sn is odd)
    const unsigned m2 = (unsigned)((m + 1) & ~1), m16 = (unsigned)((m + 15) & ~15);
    const unsigned si2 = (unsigned)((si + 1) & ~1);
    const int n0 = cap_s - sn, n0e = n0 & ~1;
    const unsigned nw_cnt = (unsigned)(cap_s - n0e);
    const unsigned bytes = (m ? (unsigned)m * 16u + m2 * 8u * 2u + m16 : 0u) + (unsigned)(si + sn) * 16u +
                           (si ? si2 * 8u : 0u) + (sn ? nw_cnt * 8u : 0u);
    bi[1] = m; bi[2] = si; bi[3] = sn; bi[4] = (int)si2 + (n0 - n0e); bi[5] = M.ii; bi[6] = par; bi[7] = 0;
    Sm.bit[q] = M.it;
    Sm.bS[q] = M.S;
    bi[0] = b;
    if (bytes == 0) {  // an empty bucket: complete the phase without copies
        asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_addr(&Sm.bar[q]))
                     : "memory");
        return;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // earlier generic accesses of the stage first
    mbar_expect_tx(&Sm.bar[q], bytes);
    if (m) {
        bulk_g2s(st.wkey, I.key[par] + base, (unsigned)m * 16u, &Sm.bar[q]);
        bulk_g2s(st.wc, I.c[par] + base, m2 * 8u, &Sm.bar[q]);
        bulk_g2s(st.whd, I.hd[par] + base, m2 * 8u, &Sm.bar[q]);
        bulk_g2s(st.wfl, I.fl[par] + base, m16, &Sm.bar[q]);
    }
    if (si) {
        bulk_g2s(st.skey, I.skey + sbase, (unsigned)si * 16u, &Sm.bar[q]);
        bulk_g2s(st.sw, I.sw + sbase, si2 * 8u, &Sm.bar[q]);
    }
    if (sn) {
        bulk_g2s(st.skey + si, I.skey + sbase + n0, (unsigned)sn * 16u, &Sm.bar[q]);
        bulk_g2s(st.sw + si2, I.sw + sbase + n0e, nw_cnt * 8u, &Sm.bar[q]);
    }
}

// The three-phase annihilation with every bucket's records brought into
// shared memory by bulk copies one bucket ahead: while a block works on one
// bucket, the next one's keys, amplitudes, H_ii, flags and spawns are in
// flight.  For runs without replica side lists or adaptive shift whose spawn
// capacity fits the stage (the host picks this kernel then).
__global__ void __launch_bounds__(K3_THREADS, 2) k_annihilate_staged(const DevInst *__restrict__ insts,
                                                                     const int *__restrict__ unit_start, int n_inst,
                                                                     int n_units)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    K4Smem<STAGED_SCAP> &Sm = *reinterpret_cast<K4Smem<STAGED_SCAP> *>(smem_raw);
    K3Shared &S = Sm.sh;
    const int t = threadIdx.x;
    {
        uint4 *tz = reinterpret_cast<uint4 *>(Sm.tab);
        for (int q = t; q < (int)(sizeof(Sm.tab) / sizeof(uint4)); q += K3_THREADS) tz[q] = make_uint4(0, 0, 0, 0);
    }
    // the last thread (the least loaded in the phases of a bucket) issues the
    // copies and keeps the counts of the bucket whose copies go out next
    constexpr int ISSUER = K3_THREADS - 1;
    StageMeta nxt;
    nxt.ii = -1;
    if (t == ISSUER) {
        S.n_new = 0;
        mbar_init(&Sm.bar[0], 1);
        mbar_init(&Sm.bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        StageMeta first;
        first.ii = -1;
        meta_load(insts, unit_start, n_inst, (int)blockIdx.x < n_units ? (int)blockIdx.x : -1, first);
        stage_issue(insts, first, Sm, 0);
        nxt.ii = first.ii;
        nxt.err = first.err; nxt.par = first.par; nxt.it = first.it; nxt.S = first.S;
        const int un = (int)blockIdx.x + (int)gridDim.x;
        meta_load(insts, unit_start, n_inst, un < n_units ? un : -1, nxt);
    }
    __syncthreads();
    unsigned phase[2] = {0u, 0u};
    const Work3 W3{Sm.acc_lo, Sm.acc_hi, Sm.eflag, Sm.tab};
    AnniTotals T;
    int q = 0, cur = -1;
    for (int u = blockIdx.x; u < n_units; u += gridDim.x, q ^= 1) {
        // the next bucket's copies go out while this one is processed; its
        // stage was last read before the previous bucket's closing barrier
        auto issue_next = [&]() {
            stage_issue(insts, nxt, Sm, q ^ 1);
            const int un = u + 2 * (int)gridDim.x;
            meta_load(insts, unit_start, n_inst, un < n_units ? un : -1, nxt);
        };
        const int b = Sm.binfo[q][0];
        if (b < 0) {
            if (t == ISSUER) issue_next();
            __syncthreads();  // binfo[q ^ 1] is written before anyone reads it
            continue;
        }
        const bool ok = mbar_wait(&Sm.bar[q], phase[q]);
        const int ii = Sm.binfo[q][5];
        const DevInst &I = insts[ii];
        if (__syncthreads_or(!ok)) {
            // the copies did not land within the bound: report, wait once
            // more (bounded) for them, stop (stage q ^ 1 holds none: its
            // last copies were waited for one bucket ago)
            if (t == 0) atomicOr(&I.st->err, ERRB_TIMEOUT);
            mbar_wait(&Sm.bar[q], phase[q]);
            return;
        }
        if (t == ISSUER) issue_next();
        phase[q] ^= 1u;
        if (ii != cur) {  // a new run: the previous run's totals are complete
            if (cur >= 0) anni_flush(insts[cur], T);
            cur = ii;
        }
        const int m = Sm.binfo[q][1], si = Sm.binfo[q][2], sn = Sm.binfo[q][3], swo = Sm.binfo[q][4];
        const int par = Sm.binfo[q][6];
        if (Sm.binfo[q][7]) {
            // loaded by the block: the stage's contiguous key arrays (walkers,
            // then spawns: CAP_M + SCAP = EMAX entries) and amplitude arrays
            // (2 CAP_M >= EMAX) serve as the records of LoadStage
            static_assert(CAP_M + STAGED_SCAP >= EMAX && 2 * CAP_M >= EMAX, "stage arrays hold EMAX records");
            static_assert(offsetof(AStage<STAGED_SCAP>, skey) == offsetof(AStage<STAGED_SCAP>, wkey) +
                                                                     sizeof(ulonglong2) * CAP_M &&
                              offsetof(AStage<STAGED_SCAP>, whd) == offsetof(AStage<STAGED_SCAP>, wc) +
                                                                    sizeof(double) * CAP_M,
                          "walker and spawn key arrays, and amplitude and H_ii arrays, adjacent");
            AStage<STAGED_SCAP> &st = Sm.st[q];
            const LoadStage R{st.wkey, st.wc, m, si, sn, I.cap_s, (size_t)b * CAP_M, (size_t)b * I.cap_s, &I, par};
            anni_bucket_3p(I, S, W3, R, b, par, Sm.bit[q], Sm.bS[q], m, si, sn, T);
            continue;
        }
        const BulkStage<STAGED_SCAP> R{&Sm.st[q], m, si, swo};
        anni_bucket_3p(I, S, W3, R, b, par, Sm.bit[q], Sm.bS[q], m, si, sn, T);
    }
    if (cur >= 0) anni_flush(insts[cur], T);
}

// ------------------------------------------------------------------ staged spawning
// The spawning kernel with every bucket's keys, amplitudes and flags brought
// into shared memory by bulk copies one bucket ahead (the bucket's count one
// bucket earlier still), as in the staged annihilation; C_i / n_att is
// written over the staged amplitude.  Chunks of 512 attempts keep three
// blocks per SM.
constexpr int CHUNK_S = 512;
struct K6Smem {
    static constexpr int chunk = CHUNK_S;
    ulonglong2 skey[2][CAP_M];
    double sc[2][CAP_M];            // C as copied; C / n_att once the bucket is loaded
    unsigned char sfl[2][CAP_M];
    unsigned off[CAP_M + 1];
    unsigned short att_det[CHUNK_S];
    unsigned char fl[CAP_M];        // initiator | in-D bits of the current bucket
    SpawnRec rec[CHUNK_S];
    unsigned short divl[CAP_M];     // determinants whose C / n_att (n_att > 1) is still to be divided
    int ndiv;
    int qn[NQ];
    int next;
    unsigned wsum[K1_THREADS / 32];
    u64 bar[2];
    int binfo[2][4];                // per stage: bucket (-1: nothing staged), m, run, parity
    long long bit[2];
    double bS[2];
};
static_assert(3 * (sizeof(K6Smem) + 1024) <= 233472, "three staged spawning blocks per SM");

struct StagedBucketMap {
    const K6Smem *S;
    int q;
    __device__ unsigned det_of(unsigned a, u64 &k) const
    {
        if (a < (unsigned)CHUNK_S) {
            const unsigned d = S->att_det[a];
            if (d != 0xffffu) {
                k = a - S->off[d];
                return d;
            }
        }
        int lo = 0, hi = CAP_M;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (S->off[mid] <= a) lo = mid; else hi = mid;
        }
        k = a - S->off[lo];
        return (unsigned)lo;
    }
    __device__ ulonglong2 key(unsigned d) const { return S->skey[q][d]; }
    __device__ double cper(unsigned d) const { return S->sc[q][d]; }
    __device__ unsigned flags(unsigned d) const { return S->fl[d]; }
    __device__ unsigned slot(unsigned d) const { return base + d; }
    unsigned base;
};

struct SpawnMeta {
    int u, ii, b, m, par, err;
    long long it;
    double S;
};

// thread 0: the run's state (once per run the block meets) and the bucket's count
__device__ __forceinline__ void spawn_meta_load(const DevInst *__restrict__ insts, const int *__restrict__ unit_start,
                                                int n_inst, int u, SpawnMeta &M)
{
    M.u = u;
    if (u < 0) return;
    const int ii = find_inst(unit_start, n_inst, u);
    const DevInst &I = insts[ii];
    if (ii != M.ii) {
        M.ii = ii;
        M.err = *(volatile int *)&I.st->err;
        M.par = I.st->parity;
        M.it = I.st->iter;
        M.S = I.st->S;
        I.st->err_at_start = M.err;  // the state seen when this run's spawning began
    }
    M.b = u - I.unit0;
    M.m = I.cnt[M.par][M.b];
}

// thread 0: the bulk copies of unit M.u's bucket into stage q
__device__ void spawn_stage_issue(const DevInst *__restrict__ insts, const SpawnMeta &M, K6Smem &S, int q)
{
    int *bi = S.binfo[q];
    bi[0] = -1;
    if (M.u < 0 || M.err) return;
    const DevInst &I = insts[M.ii];
    const int m = M.m, par = M.par;
    const size_t base = (size_t)M.b * CAP_M;
    const unsigned m2 = (unsigned)((m + 1) & ~1), m16 = (unsigned)((m + 15) & ~15);
    const unsigned bytes = m ? (unsigned)m * 16u + m2 * 8u + m16 : 0u;
    bi[1] = m; bi[2] = M.ii; bi[3] = par;
    S.bit[q] = M.it;
    S.bS[q] = M.S;
    bi[0] = M.b;
    if (bytes == 0) {
        asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_addr(&S.bar[q]))
                     : "memory");
        return;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_expect_tx(&S.bar[q], bytes);
    bulk_g2s(S.skey[q], I.key[par] + base, (unsigned)m * 16u, &S.bar[q]);
    bulk_g2s(S.sc[q], I.c[par] + base, m2 * 8u, &S.bar[q]);
    bulk_g2s(S.sfl[q], I.fl[par] + base, m16, &S.bar[q]);
}

__global__ void __launch_bounds__(K1_THREADS, 3) k_spawn_staged(const DevInst *__restrict__ insts,
                                                             const int *__restrict__ unit_start, int n_inst,
                                                             int n_units)
{
    extern __shared__ __align__(128) unsigned char k6_raw[];
    K6Smem &S = *reinterpret_cast<K6Smem *>(k6_raw);
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    constexpr int PER = CAP_M / K1_THREADS;
    SpawnMeta nxt;
    nxt.ii = -1;
    if (t == 0) {
        S.ndiv = 0;
        mbar_init(&S.bar[0], 1);
        mbar_init(&S.bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        SpawnMeta first;
        first.ii = -1;
        spawn_meta_load(insts, unit_start, n_inst, (int)blockIdx.x < n_units ? (int)blockIdx.x : -1, first);
        spawn_stage_issue(insts, first, S, 0);
        nxt.ii = first.ii;
        nxt.err = first.err; nxt.par = first.par; nxt.it = first.it; nxt.S = first.S;
        const int un = (int)blockIdx.x + (int)gridDim.x;
        spawn_meta_load(insts, unit_start, n_inst, un < n_units ? un : -1, nxt);
    }
    __syncthreads();
    unsigned phase[2] = {0u, 0u};
    int q = 0;
    for (int u = blockIdx.x; u < n_units; u += gridDim.x, q ^= 1) {
        if (t == 0) {
            spawn_stage_issue(insts, nxt, S, q ^ 1);
            const int un = u + 2 * (int)gridDim.x;
            spawn_meta_load(insts, unit_start, n_inst, un < n_units ? un : -1, nxt);
        }
        const int b = S.binfo[q][0];
        if (b < 0) {
            __syncthreads();  // binfo[q ^ 1] is written before anyone reads it
            continue;
        }
        const bool ok = mbar_wait(&S.bar[q], phase[q]);
        const int m = S.binfo[q][1], ii = S.binfo[q][2], par = S.binfo[q][3];
        const long long it = S.bit[q];
        const double shift = S.bS[q];
        const DevInst &I = insts[ii];
        if (__syncthreads_or(!ok)) {  // the copies did not land within the bound
            if (t == 0) atomicOr(&I.st->err, ERRB_TIMEOUT);
            mbar_wait(&S.bar[q], phase[q]);
            if (S.binfo[q ^ 1][0] >= 0) mbar_wait(&S.bar[q ^ 1], phase[q ^ 1]);
            return;
        }
        phase[q] ^= 1u;
        const size_t base = (size_t)b * CAP_M;
        // the bucket from the stage: thread t owns determinants PER*t .. PER*t+PER-1
        long long att = 0;
        unsigned mine = 0;
        unsigned nl[PER];
        for (int j = 0; j < PER; j++) {
            const int d = PER * t + j;
            nl[j] = 0;
            bool dv = false;
            if (d < m) {
                const double c = S.sc[q][d];
                const uint8_t f = S.sfl[q][d];
                unsigned fl = 0;
                double cper = 0.0;
                u64 nat = 0;
                if (!is_zero(c)) {
                    if (!abs_lt(c, 0x1p31)) {
                        atomicOr(&I.st->err, ERRB_NUMERIC);
                    } else {
                        nat = ceil_abs(c);
                        const bool init = (dbits(c) & ~SIGN64) > dbits(I.n_a) || (f & (DFLAG_REF | DFLAG_D));
                        fl = (init ? 1u : 0u) | ((f & DFLAG_D) ? 2u : 0u);
                        cper = c;  // C / n_att: below for n_att > 1 (c / 1 is c)
                        att += (long long)nat;
                        if (nat > HEAVY_ATT) {  // sliced into the heavy queue
                            cper = c / (double)nat;
                            const ulonglong2 kk = S.skey[q][d];
                            const unsigned nch = (unsigned)((nat + HEAVY_ATT - 1) / HEAVY_ATT);
                            const int q0 = atomicAdd(&I.st->heavy_n, (int)nch);
                            if ((long long)q0 + nch > (long long)I.heavy_cap) atomicOr(&I.st->err, ERRB_HEAVY_CAP);
                            else
                                for (unsigned h = 0; h < nch; h++) {
                                    HeavyChunk hc;
                                    hc.a = kk.x; hc.b = kk.y; hc.cper = cper; hc.k0 = (u64)h * HEAVY_ATT;
                                    const u64 left = nat - hc.k0;
                                    hc.count = (unsigned)(left < HEAVY_ATT ? left : HEAVY_ATT);
                                    hc.flags = fl;
                                    hc.slot = (uint32_t)(base + d);
                                    hc.pad = 0;
                                    I.heavy[q0 + h] = hc;
                                }
                        } else {
                            nl[j] = (unsigned)nat;
                            dv = nat > 1;
                        }
                    }
                }
                S.sc[q][d] = cper;
                S.fl[d] = (unsigned char)fl;
                mine += nl[j];
            }
            queue_div(S, dv, d, lane);
        }
        for (int a = t; a < CHUNK_S; a += K1_THREADS) S.att_det[a] = 0xffffu;
        // exclusive scan of the light attempt counts in determinant order
        unsigned v = mine;
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned y = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += y;
        }
        if (lane == 31) S.wsum[warp] = v;
        __syncthreads();
        if (warp == 0) {
            unsigned x = lane < K1_THREADS / 32 ? S.wsum[lane] : 0u;
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            if (lane < K1_THREADS / 32) S.wsum[lane] = x;
        } else {
            divide_listed(S.divl, S.ndiv, S.sc[q], t - 32, K1_THREADS - 32);  // warp 0 scans meanwhile
        }
        __syncthreads();
        if (t == 0) S.ndiv = 0;  // read by every thread before the barrier above
        unsigned ex = v - mine + (warp ? S.wsum[warp - 1] : 0u);
        for (int j = 0; j < PER; j++) {
            S.off[PER * t + j] = ex;
            if (nl[j] <= 8u && ex + nl[j] <= (unsigned)CHUNK_S)
                for (unsigned a = 0; a < nl[j]; a++) S.att_det[ex + a] = (unsigned short)(PER * t + j);
            ex += nl[j];
        }
        if (t == K1_THREADS - 1) S.off[CAP_M] = ex;
        __syncthreads();
        const unsigned total = S.off[CAP_M];
        StagedBucketMap map{&S, q, (unsigned)base};
        run_attempts(I, S, it, total, map, par, shift);
        for (int o = 16; o >= 1; o >>= 1) att += __shfl_xor_sync(0xffffffffu, att, o);
        if (lane == 0 && att) red_add(&I.acc[(b % NSHARD) * ACC_STRIDE + ACC_ATT], (u64)att);
    }
}

// ------------------------------------------------------------------ split spawning: the draw
// The first half of split spawning: the staged bucket (bulk copies one bucket
// ahead, as above), n_att and C_i / n_att per determinant, then the attempts
// drawn, classified and written to the run's attempt queues for
// k_spawn_eval.  The block that draws bucket b of a run owns segment
// b mod (grid size) of both of the run's queues (every bucket of the run it
// meets has the same residue), so its fill is a count every thread of the
// block keeps alike and no global atomic is needed; a run needs
// min(grid size, buckets) segments.  With double-buffered stage, flags and
// class counters a bucket
// takes three block barriers (one more per extra chunk of attempts):
//   A  the bucket is in shared memory, n_att counted per warp
//   B  the block scan of the attempt offsets and the divisions are done
//   C  the chunk's attempts are drawn and queued in shared memory
// after which the chunk's records go out while the next bucket starts.
struct K7Smem {
    static constexpr int chunk = CHUNK_S;
    ulonglong2 skey[2][CAP_M];
    double sc[2][CAP_M];            // C as copied; C / n_att once the bucket is loaded
    unsigned char sfl[2][CAP_M];
    unsigned char fl[2][CAP_M];     // initiator | in-D bits, per stage
    unsigned off[CAP_M];
    unsigned short att_det[CHUNK_S];
    unsigned short divl[CAP_M];
    SpawnRec rec[CHUNK_S];
    int ndiv;
    int qn[2][NQ];                  // class counts, by chunk parity
    unsigned wsum[K1_THREADS / 32];
    u64 bar[2];
    int binfo[2][4];
    long long bit[2];
    double bS[2];
};
static_assert(3 * (sizeof(K7Smem) + 1024) <= 233472, "three draw blocks per SM");

// Thread t of the draw block owns slots t, t + 256, t + 512, t + 768 of the
// bucket (consecutive threads on consecutive slots: the per-determinant work
// is spread over the block and the shared-memory accesses are conflict-free);
// attempt offsets run over the owner-major order v = 4 t + j, j the slot's
// round, so off[] is indexed by v and slot(v) = (v >> 2) + (v & 3) 256.
__device__ __forceinline__ unsigned draw_slot(unsigned v) { return (v >> 2) + (v & 3u) * K1_THREADS; }
__device__ __forceinline__ unsigned draw_order(unsigned d) { return (d % K1_THREADS) * 4u + d / K1_THREADS; }
static_assert(CAP_M == 4 * K1_THREADS, "four slots per draw thread");

struct DrawBucketMap {
    const K7Smem *S;
    int q;
    unsigned base;
    __device__ unsigned det_of(unsigned a, u64 &k) const
    {
        if (a < (unsigned)CHUNK_S) {
            const unsigned d = S->att_det[a];
            if (d != 0xffffu) {
                k = a - S->off[draw_order(d)];
                return d;
            }
        }
        int lo = 0, hi = CAP_M;  // largest v with off[v] <= a (slots past the count hold the total)
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (S->off[mid] <= a) lo = mid; else hi = mid;
        }
        k = a - S->off[lo];
        return draw_slot((unsigned)lo);
    }
    __device__ ulonglong2 key(unsigned d) const { return S->skey[q][d]; }
    __device__ double cper(unsigned d) const { return S->sc[q][d]; }
    __device__ unsigned flags(unsigned d) const { return S->fl[q][d]; }
    __device__ unsigned slot(unsigned d) const { return base + d; }
};

// thread 0: the bulk copies of unit M.u's bucket into stage q of the draw kernel
__device__ void draw_stage_issue(const DevInst *__restrict__ insts, const SpawnMeta &M, K7Smem &S, int q)
{
    int *bi = S.binfo[q];
    bi[0] = -1;
    if (M.u < 0 || M.err) return;
    const DevInst &I = insts[M.ii];
    const int m = M.m, par = M.par;
    const size_t base = (size_t)M.b * CAP_M;
    const unsigned m2 = (unsigned)((m + 1) & ~1), m16 = (unsigned)((m + 15) & ~15);
    const unsigned bytes = m ? (unsigned)m * 16u + m2 * 8u + m16 : 0u;
    bi[1] = m; bi[2] = M.ii; bi[3] = par;
    S.bit[q] = M.it;
    S.bS[q] = M.S;
    bi[0] = M.b;
    if (bytes == 0) {
        asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_addr(&S.bar[q]))
                     : "memory");
        return;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_expect_tx(&S.bar[q], bytes);
    bulk_g2s(S.skey[q], I.key[par] + base, (unsigned)m * 16u, &S.bar[q]);
    bulk_g2s(S.sc[q], I.c[par] + base, m2 * 8u, &S.bar[q]);
    bulk_g2s(S.sfl[q], I.fl[par] + base, m16, &S.bar[q]);
}

// thread 0: the queue fill of this block's segment of a run
__device__ __forceinline__ void draw_flush(const DevInst &I, int seg, long long q0, long long q1)
{
    I.qcnt[seg] = (int)min(q0, 0x7fffffffLL);
    I.qcnt[I.qnseg + seg] = (int)min(q1, 0x7fffffffLL);
}

__global__ void __launch_bounds__(K1_THREADS, 3) k_spawn_draw(const DevInst *__restrict__ insts,
                                                              const int *__restrict__ unit_start, int n_inst,
                                                              int n_units)
{
    extern __shared__ __align__(128) unsigned char k7_raw[];
    K7Smem &S = *reinterpret_cast<K7Smem *>(k7_raw);
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    constexpr int PER = CAP_M / K1_THREADS;
    // the last thread (its determinants are the last slots of a bucket, mostly
    // empty) issues the copies and keeps the meta data of the next bucket
    constexpr int ISSUER = K1_THREADS - 1;
    SpawnMeta nxt;
    nxt.ii = -1;
    if (t == ISSUER) {
        S.ndiv = 0;
        for (int k = 0; k < 2 * NQ; k++) S.qn[k / NQ][k % NQ] = 0;
        mbar_init(&S.bar[0], 1);
        mbar_init(&S.bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        SpawnMeta first;
        first.ii = -1;
        spawn_meta_load(insts, unit_start, n_inst, (int)blockIdx.x < n_units ? (int)blockIdx.x : -1, first);
        draw_stage_issue(insts, first, S, 0);
        nxt.ii = first.ii;
        nxt.err = first.err; nxt.par = first.par; nxt.it = first.it; nxt.S = first.S;
        const int un = (int)blockIdx.x + (int)gridDim.x;
        spawn_meta_load(insts, unit_start, n_inst, un < n_units ? un : -1, nxt);
    }
    __syncthreads();
    unsigned phase[2] = {0u, 0u};
    int q = 0, cp = 0;             // stage, chunk parity
    int cur = -1, seg = 0;         // the run whose segment (seg) fill is held in qf0, qf1
    long long qf0 = 0, qf1 = 0;    // entries this block queued for run `cur` (singles, doubles)
    for (int u = blockIdx.x; u < n_units; u += gridDim.x, q ^= 1) {
        const int b = S.binfo[q][0];
        bool ok = true;
        int m = 0, ii = 0;
        if (b >= 0) {
            ok = mbar_wait(&S.bar[q], phase[q]);
            m = S.binfo[q][1];
            ii = S.binfo[q][2];
        }
        const DevInst &I = insts[ii];
        // A: the bucket from the stage; thread t owns slots t + 256 j (draw_slot)
        long long att = 0;
        unsigned mine = 0;
        unsigned nl[PER];
        for (int j = 0; j < PER; j++) {
            const int d = t + j * K1_THREADS;
            nl[j] = 0;
            bool dv = false;
            if (d < m && ok) {
                const double c = S.sc[q][d];
                const uint8_t f = S.sfl[q][d];
                unsigned fl = 0;
                double cper = 0.0;
                u64 nat = 0;
                if (!is_zero(c)) {
                    if (!abs_lt(c, 0x1p31)) {
                        atomicOr(&I.st->err, ERRB_NUMERIC);
                    } else {
                        nat = ceil_abs(c);
                        const bool init = (dbits(c) & ~SIGN64) > dbits(I.n_a) || (f & (DFLAG_REF | DFLAG_D));
                        fl = (init ? 1u : 0u) | ((f & DFLAG_D) ? 2u : 0u);
                        cper = c;  // C / n_att: after A for n_att > 1 (c / 1 is c)
                        att += (long long)nat;
                        if (nat > HEAVY_ATT) {  // sliced into the heavy queue
                            cper = c / (double)nat;
                            const ulonglong2 kk = S.skey[q][d];
                            const unsigned nch = (unsigned)((nat + HEAVY_ATT - 1) / HEAVY_ATT);
                            const int q0 = atomicAdd(&I.st->heavy_n, (int)nch);
                            if ((long long)q0 + nch > (long long)I.heavy_cap) atomicOr(&I.st->err, ERRB_HEAVY_CAP);
                            else
                                for (unsigned h = 0; h < nch; h++) {
                                    HeavyChunk hc;
                                    hc.a = kk.x; hc.b = kk.y; hc.cper = cper; hc.k0 = (u64)h * HEAVY_ATT;
                                    const u64 left = nat - hc.k0;
                                    hc.count = (unsigned)(left < HEAVY_ATT ? left : HEAVY_ATT);
                                    hc.flags = fl;
                                    hc.slot = (uint32_t)((size_t)b * CAP_M + d);
                                    hc.pad = 0;
                                    I.heavy[q0 + h] = hc;
                                }
                        } else {
                            nl[j] = (unsigned)nat;
                            dv = nat > 1;
                        }
                    }
                }
                S.sc[q][d] = cper;
                S.fl[q][d] = (unsigned char)fl;
                mine += nl[j];
            }
            queue_div(S, dv, d, lane);
        }
        for (int a = t; a < CHUNK_S; a += K1_THREADS) S.att_det[a] = 0xffffu;
        unsigned v = mine;  // inclusive warp scan of the light attempt counts in owner-major order
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned y = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += y;
        }
        if (lane == 31) S.wsum[warp] = v;
        if (__syncthreads_or(!ok)) {  // A; the copies did not land within the bound
            if (t == 0) atomicOr(&I.st->err, ERRB_TIMEOUT);
            mbar_wait(&S.bar[q], phase[q]);
            return;
        }
        if (t == ISSUER) {  // every thread is past the last reads of stage q ^ 1 (bucket u - grid)
            draw_stage_issue(insts, nxt, S, q ^ 1);
            const int un = u + 2 * (int)gridDim.x;
            spawn_meta_load(insts, unit_start, n_inst, un < n_units ? un : -1, nxt);
        }
        if (b < 0) {
            __syncthreads();  // stage q ^ 1's info is written before anyone reads it
            continue;
        }
        phase[q] ^= 1u;
        if (ii != cur) {  // a new run: the previous run's segment fill is final
            if (t == 0 && cur >= 0) draw_flush(insts[cur], seg, qf0, qf1);
            cur = ii;
            seg = b % (int)gridDim.x;
            qf0 = qf1 = 0;
        }
        const long long it = S.bit[q];
        // B: attempt offsets (each warp sums the warp totals before its own), parents of the first
        // CHUNK_S attempts, and C / n_att of the listed determinants
        unsigned ex = v - mine, total = 0;
        for (int w = 0; w < K1_THREADS / 32; w++) {
            const unsigned x = S.wsum[w];
            ex += w < warp ? x : 0u;
            total += x;
        }
        for (int j = 0; j < PER; j++) {
            S.off[PER * t + j] = ex;
            if (nl[j] <= 8u && ex + nl[j] <= (unsigned)CHUNK_S)
                for (unsigned a = 0; a < nl[j]; a++) S.att_det[ex + a] = (unsigned short)(t + j * K1_THREADS);
            ex += nl[j];
        }
        divide_listed(S.divl, S.ndiv, S.sc[q], t, K1_THREADS);
        __syncthreads();  // B
        if (t == 0) S.ndiv = 0;
        const DrawBucketMap map{&S, q, (unsigned)((size_t)b * CAP_M)};
        for (unsigned a0 = 0; a0 < total; a0 += CHUNK_S) {
            if (a0) __syncthreads();  // the previous chunk's records are out before rec[] is reused
            draw_classify(I, S, it, a0, min(total, a0 + CHUNK_S), map, S.qn[cp]);
            __syncthreads();  // C
            const int nd = S.qn[cp][Q_DOUBLE], ns = S.qn[cp][Q_SINGLE], ntot = ns + nd;
            if (t < NQ) S.qn[cp ^ 1][t] = 0;  // every thread read the other counts before C
            cp ^= 1;
            const long long b0 = qf0, b1 = qf1;
            qf0 += ns;
            qf1 += nd;
            bool over = false;
            for (int r = t; r < ntot; r += K1_THREADS) {
                const bool single = r < ns;
                const SpawnRec rr = single ? S.rec[CHUNK_S - 1 - r] : S.rec[r - ns];
                const int c = single ? 0 : 1;
                const long long idx = single ? b0 + r : b1 + (r - ns);
                if (idx >= I.qcap[c]) { over = true; continue; }
                const unsigned d = rr.det;
                const ulonglong2 kk = map.key(d);
                QRec o;
                o.ka = kk.x; o.kb = kk.y; o.cper = map.cper(d); o.w2 = rr.w2; o.w3 = rr.w3;
                o.slot = map.slot(d);
                o.info = (rr.ep & 0xffffu) | (map.flags(d) << 16);
                I.qrec[c][(size_t)seg * I.qcap[c] + idx] = o;
            }
            if (over) atomicOr(&I.st->err, ERRB_QUEUE_CAP);
            if (t == 0) {
                if (qf0 > I.qcap[0]) atomicMax(&I.st->need_queue[0], (int)min(qf0, 0x7fffffffLL));
                if (qf1 > I.qcap[1]) atomicMax(&I.st->need_queue[1], (int)min(qf1, 0x7fffffffLL));
            }
        }
        for (int o = 16; o >= 1; o >>= 1) att += __shfl_xor_sync(0xffffffffu, att, o);
        if (lane == 0 && att) red_add(&I.acc[(b % NSHARD) * ACC_STRIDE + ACC_ATT], (u64)att);
    }
    if (t == 0 && cur >= 0) draw_flush(insts[cur], seg, qf0, qf1);
}

// The evaluation of the queued attempts of every run: one attempt per
// thread, doubles first, then singles and hops, with no block barrier; the
// parent's key, C_i / n_att, flags and slot travel in the record.
__global__ void __launch_bounds__(256) k_spawn_eval(const DevInst *__restrict__ insts, int n_inst)
{
    __shared__ long long s_off[2][NSEG_MAX + 1];
    __shared__ int s_err, s_par;
    __shared__ double s_S;
    const long long gt = (long long)blockIdx.x * blockDim.x + threadIdx.x, gs = (long long)gridDim.x * blockDim.x;
    for (int ii = 0; ii < n_inst; ii++) {
        const DevInst &I = insts[ii];
        const int ns = I.qnseg;
        if (threadIdx.x < 32) {  // warp 0: the segment offsets of both classes by a warp scan
            const int lane = threadIdx.x;
            if (lane == 0) {
                s_err = I.st->err_at_start;  // the state this run's spawning began with
                s_par = I.st->parity;
                s_S = I.st->S;
            }
            const int per = (ns + 31) / 32;  // segments lane*per .. lane*per+per-1
            for (int c = 0; c < 2; c++) {
                long long mine = 0;
                for (int r = 0; r < per; r++) {
                    const int g = lane * per + r;
                    if (g < ns) mine += min((long long)I.qcnt[c * ns + g], I.qcap[c]);
                }
                long long inc = mine;
                for (int o = 1; o < 32; o <<= 1) {
                    const long long y = __shfl_up_sync(0xffffffffu, inc, o);
                    if (lane >= o) inc += y;
                }
                long long ex = inc - mine;
                for (int r = 0; r < per; r++) {
                    const int g = lane * per + r;
                    if (g < ns) {
                        s_off[c][g] = ex;
                        ex += min((long long)I.qcnt[c * ns + g], I.qcap[c]);
                    }
                }
                if (lane == 31) s_off[c][ns] = inc;
            }
        }
        __syncthreads();
        const int err = s_err, par = s_par;
        const double shift = s_S;
        const long long nd = s_off[1][ns], ntot = nd + s_off[0][ns];
        if (!err)
            for (long long i = gt; i < ntot; i += gs) {
                const int c = i < nd ? 1 : 0;
                const long long j = c ? i : i - nd;
                int lo = 0, hi = ns;  // the segment holding entry j: the last g with s_off[c][g] <= j
                while (hi - lo > 1) {
                    const int mid = (lo + hi) >> 1;
                    if (s_off[c][mid] <= j) lo = mid; else hi = mid;
                }
                const QRec r = I.qrec[c][(size_t)lo * I.qcap[c] + (j - s_off[c][lo])];
                const SpawnCtx cx{r.slot, par, shift};
                const unsigned flags = r.info >> 16, sel = r.info & 0xffffu;
                if (c == 1) {
                    if (I.pchb) spawn_double_pchb(I, r.ka, r.kb, r.cper, flags, sel, r.w2, r.w3, cx);
                    else spawn_double(I, r.ka, r.kb, r.cper, flags, sel, r.w2, r.w3, cx);
                } else if (I.kind == FCIQMC_HUBBARD) spawn_hop_e(I, r.ka, r.kb, r.cper, flags, (int)sel, r.w2, r.w3, cx);
                else spawn_single_e(I, r.ka, r.kb, r.cper, flags, (int)sel, r.w2, r.w3, cx);
            }
        __syncthreads();
    }
}

// GENERAL: the batch holds a run with replica side lists or adaptive shift,
// whose buckets take the general path (anni_bucket); the others the
// three-phase one.  Without it the kernel holds the three-phase path alone.
template <bool GENERAL>
__global__ void __launch_bounds__(K3_THREADS, 3) k_annihilate(const DevInst *__restrict__ insts,
                                                              const int *__restrict__ unit_start, int n_inst, int n_units)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    K3Smem &Sm = *reinterpret_cast<K3Smem *>(smem_raw);
    K3Shared &S = Sm.sh;
    Stage<unsigned short> W{Sm.key, Sm.val, Sm.acc_lo, Sm.acc_hi, Sm.nacc, Sm.eflag, Sm.tab, Sm.opos};
    const int t = threadIdx.x;
    // the three-phase path expects a cleared table and output counter; the
    // general path (replica side lists, adaptive shift) leaves both used
    bool clean = false;
    // the run's state at the start of the iteration, read once per run a
    // block meets
    int cur = -1, err = 0, par = 0;
    long long it = 0;
    double shift = 0.0;
    AnniTotals T;
    for (int u = blockIdx.x; u < n_units; u += gridDim.x) {
        const int ii = find_inst(unit_start, n_inst, u);
        const DevInst &I = insts[ii];
        if (ii != cur) {
            if (cur >= 0) anni_flush(insts[cur], T);  // the previous run's totals are complete
            if (t == 0) {
                S.hdr_err = *(volatile int *)&I.st->err;
                S.hdr_par = I.st->parity;
                S.hdr_it = I.st->iter;
                S.hdr_S = I.st->S;
            }
            __syncthreads();
            err = S.hdr_err;
            par = S.hdr_par;
            it = S.hdr_it;
            shift = S.hdr_S;
            cur = ii;
            __syncthreads();
        }
        if (err) continue;
        const int b = u - I.unit0;
        const int m = I.cnt[par][b], si = I.scnt_i[b], sn = I.scnt_n[b];
        if (si + sn > I.cap_s) {
            if (t == 0) {
                atomicOr(&I.st->err, ERRB_SPAWN_CAP);
                atomicMax(&I.st->need_spawn, si + sn);
                atomicAdd(&I.st->n_spawn_over, 1);
            }
            continue;
        }
        if (m + si + sn > EMAX) {  // too large for shared memory: deferred to k_annihilate_big
            if (t == 0) I.big_list[atomicAdd(&I.st->big_n, 1)] = b;
            continue;
        }
        if (GENERAL && (I.side || I.adaptive)) {
            anni_bucket<unsigned short>(I, S, W, TABBITS, b, par, it, shift, m, si, sn);
            clean = false;
            continue;
        }
        if (!clean) {
            uint4 *tz = reinterpret_cast<uint4 *>(Sm.tab);
            for (int q = t; q < (int)(sizeof(Sm.tab) / sizeof(uint4)); q += K3_THREADS) tz[q] = make_uint4(0, 0, 0, 0);
            if (t == 0) S.n_new = 0;
            __syncthreads();
            clean = true;
        }
        const LoadStage R{Sm.key, Sm.val, m, si, sn, I.cap_s, (size_t)b * CAP_M, (size_t)b * I.cap_s, &I, par};
        const Work3 W3{Sm.acc_lo, Sm.acc_hi, Sm.eflag, Sm.tab};
        anni_bucket_3p(I, S, W3, R, b, par, it, shift, m, si, sn, T);
    }
    if (cur >= 0) anni_flush(insts[cur], T);
}

__global__ void __launch_bounds__(K3_THREADS) k_annihilate_big(const DevInst *__restrict__ insts, int n_inst)
{
    __shared__ K3Shared S;
    const int t = threadIdx.x;
    for (int ii = 0; ii < n_inst; ii++) {
        const DevInst &I = insts[ii];
        if (t == 0) {
            S.hdr_err = *(volatile int *)&I.st->err;
            S.hdr_par = I.st->parity;
            S.hdr_it = I.st->iter;
            S.hdr_S = I.st->S;
            S.n_new = I.st->big_n;
        }
        __syncthreads();
        const int err = S.hdr_err, par = S.hdr_par, nbig = S.n_new;
        const long long it = S.hdr_it;
        const double shift = S.hdr_S;
        __syncthreads();
        if (err || nbig == 0) continue;
        if (!I.big_scratch) {  // no scratch yet: report, the host allocates it and repeats the iteration
            if (t == 0) atomicOr(&I.st->err, ERRB_SPAWN_CAP);
            continue;
        }
        // this block's scratch slice
        const int Ecap = CAP_M + I.cap_s, tabbits = I.big_tabbits;
        unsigned char *p = I.big_scratch + (size_t)blockIdx.x * I.big_stride;
        Stage<unsigned> W;
        W.key = (ulonglong2 *)p; p += (size_t)Ecap * sizeof(ulonglong2);
        W.val = (double *)p; p += (size_t)Ecap * sizeof(double);
        W.acc_lo = (u64 *)p; p += (size_t)Ecap * 8;
        W.acc_hi = (u64 *)p; p += (size_t)Ecap * 8;
        W.nacc = (int *)p; p += (size_t)Ecap * 4;
        W.eflag = (int *)p; p += (size_t)Ecap * 4;
        W.opos = (unsigned *)p; p += (size_t)Ecap * 4;
        W.tab = (unsigned *)p;
        for (int q = blockIdx.x; q < nbig; q += gridDim.x) {
            const int b = I.big_list[q];
            const int m = I.cnt[par][b], si = I.scnt_i[b], sn = I.scnt_n[b];
            anni_bucket<unsigned>(I, S, W, tabbits, b, par, it, shift, m, si, sn);
        }
    }
}

// ------------------------------------------------------------------ finalize
__global__ void __launch_bounds__(K5_THREADS) k_finalize(const DevInst *__restrict__ insts, int n_inst)
{
    const DevInst &I = insts[blockIdx.x];
    IterState *st = I.st;
    __shared__ int s_err;
    __shared__ double s_r[K5_THREADS];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int nbk = 1 << I.bb;
    const bool pair = I.partner > (int)blockIdx.x;  // the first replica reports the cross estimators
    const bool trial = I.trial_bits != 0;
    const bool tree = trial || pair;  // binary64 estimator sums need the whole block; otherwise warp 0 alone
    if (!tree && warp != 0) return;
    int e = 0;
    if (t == 0) {
        e = *(volatile int *)&st->err;
        // a replica commits its iteration only together with its partner: not
        // if the partner skipped it (a flag was up when its spawning began) or
        // failed in it
        const IterState *pst = I.partner >= 0 ? insts[I.partner].st : nullptr;
        if (!e && pst && (*(volatile const int *)&pst->err_at_start ||
                          (*(volatile const int *)&pst->err & ERRB_STAGE))) {
            st->err = ERRB_PARTNER;
            e = ERRB_PARTNER;
        }
    }
    if (tree) {
        if (t == 0) s_err = e;
        __syncthreads();
        e = s_err;
    } else {
        e = __shfl_sync(0xffffffffu, e, 0);
    }
    if (e) return;
    // Binary64 sums of the estimators that have them (trial numerator and
    // denominator; replica-pair terms), per tile of K5_THREADS buckets: one
    // value per thread into shared memory and a halving tree, so that every
    // binary64 add is a full-warp instruction (a partly active warp costs as
    // much on this part's slow binary64 pipe); tile sums added in tile order.
    constexpr int NF = 6;  // words 0 .. 5 of a partial
    double dsum[NF];
#pragma unroll
    for (int f = 0; f < NF; f++) dsum[f] = 0.0;
    if (tree)
        for (int tile0 = 0; tile0 < nbk; tile0 += K5_THREADS) {
#pragma unroll
            for (int f = 0; f < NF; f++) {
                if (f < 2 ? !trial : !pair) continue;
                const int u = tile0 + t;
                s_r[t] = u < nbk ? reinterpret_cast<const double *>(I.part + u)[f] : 0.0;
                __syncthreads();
                for (int h = K5_THREADS / 2; h >= 32; h >>= 1) {
                    if (t < h) s_r[t] = s_r[t] + s_r[t + h];
                    __syncthreads();
                }
                if (warp == 0) {
                    double v = s_r[lane];
                    for (int mm = 16; mm >= 1; mm >>= 1) v = v + __shfl_xor_sync(0xffffffffu, v, mm);
                    if (lane == 0) dsum[f] = dsum[f] + v;
                }
                __syncthreads();
            }
        }
    if (warp != 0) return;
    // the shift state, loaded now so that its latency overlaps the totals'
    const long long it = st->iter, cnt0 = st->cnt, shift_start0 = st->shift_start, stop_iter = st->stop_iter;
    const long long semi_built = st->semi_built, trial_built = st->trial_built;
    const int vary0 = st->vary, par0 = st->parity;
    const double S0 = st->S, e_den = st->e_den;
    const u64 nwl_lo0 = st->nwl_lo, nwl_hi0 = st->nwl_hi;
    // the exact totals the buckets added up: lane k sums word k of the NSHARD
    // lines (each limb's total stays below 2^64) and clears it
    u64 v = 0;
    if (lane < NACC) {
        u64 x[NSHARD];
#pragma unroll
        for (int j = 0; j < NSHARD; j++) x[j] = I.acc[j * ACC_STRIDE + lane];
#pragma unroll
        for (int j = 0; j < NSHARD; j++) {
            I.acc[j * ACC_STRIDE + lane] = 0;
            v += x[j];
        }
    }
    u64 w[NACC];
#pragma unroll
    for (int k = 0; k < NACC; k++) w[k] = __shfl_sync(0xffffffffu, v, k);
    if (I.qcnt)  // the attempt queues of split spawning start empty
        for (int g = lane; g < 2 * I.qnseg; g += 32) I.qcnt[g] = 0;
    if (lane != 0) return;
    const u128 W = (u128)limb_total(w + ACC_NW);
    const i128 A = limb_total(w + ACC_ANN), EN = limb_total(w + ACC_ENUM);
    const long long nd = (long long)w[ACC_NDET], rj = (long long)w[ACC_REJ], sps = (long long)w[ACC_SPAWNS],
                    at = (long long)w[ACC_ATT];
    const double e_num = fixed_to_double(EN, I.Fe);
    const double t_num = trial ? dsum[0] : 0.0, t_den = trial ? dsum[1] : 0.0;
    const double x_ov = pair ? dsum[2] : 0.0, x_hd = pair ? dsum[3] : 0.0, x_cr = pair ? dsum[4] : 0.0;
    const double x_pt = pair ? dsum[5] : 0.0;
    const double nwd = u128_to_double(W) * 0x1p-32;
    // shift update (Booth, Thom, Alavi 2009)
    int vary = vary0;
    long long cnt = cnt0, shift_start = shift_start0;
    double S = S0;
    u64 nwl_lo = nwl_lo0, nwl_hi = nwl_hi0;
    if (!vary) {
        if (nwd >= I.target) {
            vary = 1;
            shift_start = it;
            nwl_lo = (u64)W; nwl_hi = (u64)(W >> 64);
            cnt = 0;
        }
    } else if (++cnt == I.A) {
        const u128 L = ((u128)nwl_hi << 64) | nwl_lo;
        const double ratio = nwd / (u128_to_double(L) * 0x1p-32);
        S = S - I.cz * fq_ln(ratio);
        nwl_lo = (u64)W; nwl_hi = (u64)(W >> 64);
        cnt = 0;
    }
    int flags = 0;
    if (!(S == S) || !(nwd == nwd)) flags |= ERRB_NUMERIC;
    fciqmc_iter_stats &R = I.ring[it & (long long)(I.ring_cap - 1)];  // ring_cap is a power of two
    R.iteration = it; R.nw = nwd; R.shift = S; R.e_num = e_num; R.e_den = e_den;
    R.ndet = nd; R.attempts = at; R.spawns = sps; R.rejected = rj;
    R.annihilated = i128_to_double(A) * 0x1p-32; R.vary = vary; R.pad0 = 0;
    R.trial_num = t_num; R.trial_den = t_den;
    R.x_overlap = x_ov;
    R.x_var_num = pair ? x_hd - x_cr / (2.0 * I.tau) : 0.0;
    R.x_pt2 = pair ? x_pt / (I.tau * I.tau) : 0.0;
    st->vary = vary; st->shift_start = shift_start; st->cnt = cnt; st->S = S;
    st->nwl_lo = nwl_lo; st->nwl_hi = nwl_hi;
    st->iter = it + 1;
    st->parity = par0 ^ 1;
    st->heavy_n = 0;
    st->big_n = 0;
    st->new_n = 0;
    if (I.semi_size > 0 && !semi_built && vary && it + 1 == shift_start + I.semi_start) flags |= ERRB_PAUSE_SEMI;
    if (I.trial_size > 0 && !trial_built && vary && it + 1 == shift_start + I.trial_start) flags |= ERRB_PAUSE_TRIAL;
    if (it + 1 >= stop_iter) flags |= ERRB_STOP;
    if (flags) st->err |= flags;
}

// ------------------------------------------------------------------ growth and import
// per-bucket list index of list `par` (adaptive shift), and zeroed weight sums
__global__ void k_build_kidx(const DevInst *__restrict__ Ip, int par, int nb)
{
    __shared__ unsigned short tab[KIDX];
    const DevInst &I = *Ip;
    for (int b = blockIdx.x; b < nb; b += gridDim.x) {
        for (int q = threadIdx.x; q < KIDX; q += blockDim.x) tab[q] = 0;
        __syncthreads();
        const int m = min(I.cnt[par][b], CAP_M);
        for (int e = threadIdx.x; e < m; e += blockDim.x) {
            const ulonglong2 k = I.key[par][(size_t)b * CAP_M + e];
            unsigned sl = (unsigned)det_hash(k.x, k.y) & (unsigned)(KIDX - 1);
            while (atomicCAS(&tab[sl], (unsigned short)0, (unsigned short)(e + 1)) != 0) sl = (sl + 1) & (unsigned)(KIDX - 1);
            u64 *acc = I.facc[par] + ((size_t)b * CAP_M + e) * 4;
            acc[0] = 0; acc[1] = 0; acc[2] = 0; acc[3] = 0;
        }
        __syncthreads();
        for (int q = threadIdx.x; q < KIDX; q += blockDim.x) I.kidx[par][(size_t)b * KIDX + q] = tab[q];
        __syncthreads();
    }
}

// split every bucket of src (bb bits) into two buckets of dst (bb+1 bits)
__global__ void k_rebucket(const DevInst *__restrict__ src, const DevInst *__restrict__ dst, int nb_src, int par)
{
    for (int b = blockIdx.x; b < nb_src; b += gridDim.x) {
        const int m = src->cnt[par][b];
        for (int e = threadIdx.x; e < m; e += blockDim.x) {
            size_t o = (size_t)b * CAP_M + e;
            ulonglong2 k = src->key[par][o];
            int nbk = bucket_of(det_hash(k.x, k.y), dst->bb);
            int slot = atomicAdd(dst->cnt[par] + nbk, 1);
            if (slot >= CAP_M) { atomicOr(&dst->st->err, ERRB_MAIN_CAP); continue; }
            size_t d = (size_t)nbk * CAP_M + slot;
            dst->key[par][d] = k;
            dst->c[par][d] = src->c[par][o];
            dst->hd[par][d] = src->hd[par][o];
            dst->fl[par][d] = src->fl[par][o];
        }
    }
}

// H_ii - E_ref and reference flags for every determinant of buffer par
__global__ void k_diag(const DevInst *__restrict__ I, int par, int nb)
{
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    for (int b = gw; b < nb; b += nw) {
        const int m = I->cnt[par][b];
        for (int e = 0; e < m; e++) {
            size_t o = (size_t)b * CAP_M + e;
            ulonglong2 k = I->key[par][o];
            double hdv = diag_exact_warp(*I, k.x, k.y);
            if (lane == 0) {
                I->hd[par][o] = hdv;
                uint8_t f = I->fl[par][o] & DFLAG_D;
                if (k.x == I->ref_a && k.y == I->ref_b) f |= DFLAG_REF;
                I->fl[par][o] = f;
            }
        }
    }
}

// ------------------------------------------------------------------ time-step bound
// sum_j |<D_j|H|D_ref>| over every single and double excitation of the
// reference; fixed grid, fixed per-thread order and fixed reduction tree, so
// the result is deterministic.
constexpr int REFSUM_BLOCKS = 64;
__global__ void __launch_bounds__(256) k_ref_abs_sum(const DevInst *__restrict__ Ip, double *partial)
{
    const DevInst &I = *Ip;
    const u64 ra = I.ref_a, rb = I.ref_b, va = ~ra & I.normask, vb = ~rb & I.normask;
    const long long na = I.na, nb = I.nb, ma = I.ma, mb = I.mb;
    const long long s1 = na * ma, s2 = nb * mb, s3 = na * nb * ma * mb, s4 = na * na * ma * ma, s5 = nb * nb * mb * mb;
    const long long total = s1 + s2 + s3 + s4 + s5;
    double acc = 0.0;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        long long q = idx;
        u64 ta = ra, tb = rb;
        if (q < s1) {
            ta ^= (1ULL << nth_set(ra, (int)(q / ma))) | (1ULL << nth_set(va, (int)(q % ma)));
        } else if ((q -= s1) < s2) {
            tb ^= (1ULL << nth_set(rb, (int)(q / mb))) | (1ULL << nth_set(vb, (int)(q % mb)));
        } else if ((q -= s2) < s3) {
            const int b = (int)(q % mb); q /= mb;
            const int a = (int)(q % ma); q /= ma;
            const int j = (int)(q % nb), i = (int)(q / nb);
            ta ^= (1ULL << nth_set(ra, i)) | (1ULL << nth_set(va, a));
            tb ^= (1ULL << nth_set(rb, j)) | (1ULL << nth_set(vb, b));
        } else if ((q -= s3) < s4) {
            const int b = (int)(q % ma); q /= ma;
            const int a = (int)(q % ma); q /= ma;
            const int j = (int)(q % na), i = (int)(q / na);
            if (!(i < j && a < b)) continue;
            ta ^= (1ULL << nth_set(ra, i)) | (1ULL << nth_set(ra, j)) | (1ULL << nth_set(va, a)) | (1ULL << nth_set(va, b));
        } else {
            q -= s4;
            const int b = (int)(q % mb); q /= mb;
            const int a = (int)(q % mb); q /= mb;
            const int j = (int)(q % nb), i = (int)(q / nb);
            if (!(i < j && a < b)) continue;
            tb ^= (1ULL << nth_set(rb, i)) | (1ULL << nth_set(rb, j)) | (1ULL << nth_set(vb, a)) | (1ULL << nth_set(vb, b));
        }
        acc = acc + fabs(hoff_generic(I, ra, rb, ta, tb));
    }
    __shared__ double sm[8];
    for (int m = 16; m >= 1; m >>= 1) acc = acc + __shfl_xor_sync(0xffffffffu, acc, m);
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int k = 0; k < 8; k++) s = s + sm[k];
        partial[blockIdx.x] = s;
    }
}

cudaError_t ref_abs_sum(const DevInst *dinst, double *dpartial, double *out, cudaStream_t s)
{
    k_ref_abs_sum<<<REFSUM_BLOCKS, 256, 0, s>>>(dinst, dpartial);
    double hp[REFSUM_BLOCKS];
    cudaError_t e = cudaMemcpyAsync(hp, dpartial, sizeof(hp), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    double acc = 0.0;
    for (int k = 0; k < REFSUM_BLOCKS; k++) acc = acc + hp[k];
    *out = acc;
    return cudaSuccess;
}

// ------------------------------------------------------------------ launchers
static int g_num_sms = 0;
static int num_sms()
{
    if (!g_num_sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
        if (g_num_sms <= 0) g_num_sms = 1;
    }
    return g_num_sms;
}

void launch_build_kidx(const DevInst *dinst, int parity, int nb, cudaStream_t s)
{
    int grid = nb < num_sms() * 8 ? nb : num_sms() * 8;
    k_build_kidx<<<grid, 256, 0, s>>>(dinst, parity, nb);
}

// launch geometry, chosen by fciqmc_autotune (grid blocks per SM; beyond the
// resident count, here 3 per SM for the spawning and annihilation kernels, the
// hardware hands the next block to whichever slot frees first, which evens out
// buckets of unequal size)
// g_spawn_bps = 0 and g_anni_bps = 0 select the staged kernels (one resident
// wave, bulk copies one bucket ahead) wherever the batch fits them, and
// g_spawn_bps = 1 the staged draw with the flat evaluation (split spawning);
// otherwise the plain-load kernels with that many blocks per SM
static int g_spawn_bps = 1, g_heavy_bps = 2, g_anni_bps = 0;
static int g_geometry_gen = 0;  // changes with every set_launch_geometry
int launch_geometry_generation() { return g_geometry_gen; }
void set_launch_geometry(int spawn_bps, int heavy_bps, int anni_bps)
{
    g_geometry_gen++;
    g_spawn_bps = spawn_bps;
    g_heavy_bps = heavy_bps;
    g_anni_bps = anni_bps;
}
void get_launch_geometry(int *spawn_bps, int *heavy_bps, int *anni_bps)
{
    *spawn_bps = g_spawn_bps;
    *heavy_bps = g_heavy_bps;
    *anni_bps = g_anni_bps;
}

// the staged spawning kernel (g_spawn_bps = 0: one resident wave of three
// blocks per SM) where every run's list arrays are 16-byte aligned; else the
// plain-load kernel with g_spawn_bps blocks per SM
void launch_spawn(const DevInst *dinst, const int *unit_start, int n_inst, int n_units, bool staged, bool split,
                  cudaStream_t s)
{
    if (staged && (g_spawn_bps == 0 || g_spawn_bps == 1)) {
        int grid = n_units < num_sms() * 3 ? n_units : num_sms() * 3;
        if (grid < 1) grid = 1;
        if (split && g_spawn_bps == 1)  // grid <= draw_segments(): at most one queue segment per block and run
            k_spawn_draw<<<grid, K1_THREADS, sizeof(K7Smem), s>>>(dinst, unit_start, n_inst, n_units);
        else k_spawn_staged<<<grid, K1_THREADS, sizeof(K6Smem), s>>>(dinst, unit_start, n_inst, n_units);
        return;
    }
    const int bps = g_spawn_bps > 0 ? g_spawn_bps : 8;
    int grid = n_units < num_sms() * bps ? n_units : num_sms() * bps;
    if (grid < 1) grid = 1;
    k_spawn<<<grid, K1_THREADS, sizeof(K1Smem), s>>>(dinst, unit_start, n_inst, n_units);
}

// split spawning (queues in global memory, flat evaluation): geometry 1
bool spawn_split_selected() { return g_spawn_bps == 1 && draw_segments() <= NSEG_MAX; }
int draw_segments() { return num_sms() * 3; }

void launch_spawn_eval(const DevInst *dinst, int n_inst, cudaStream_t s)
{
    k_spawn_eval<<<num_sms() * 4, 256, 0, s>>>(dinst, n_inst);  // one resident wave (64 registers)
}

bool staged_spawn_fits(const DevInst &I)
{
    auto al = [](const void *p) { return ((uintptr_t)p & 15u) == 0; };
    for (int k = 0; k < 2; k++)
        if (!al(I.key[k]) || !al(I.c[k]) || !al(I.fl[k])) return false;
    return true;
}

void launch_spawn_heavy(const DevInst *dinst, int n_inst, cudaStream_t s)
{
    k_spawn_heavy<<<num_sms() * g_heavy_bps, K1_THREADS, sizeof(K1Smem), s>>>(dinst, n_inst);
}

cudaError_t init_kernels()
{
    cudaError_t e = cudaFuncSetAttribute(k_annihilate<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sizeof(K3Smem));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_annihilate<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(K3Smem));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_annihilate_staged, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sizeof(K4Smem<STAGED_SCAP>));
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_spawn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(K1Smem));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_spawn_staged, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(K6Smem));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_spawn_draw, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(K7Smem));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_spawn_heavy, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(K1Smem));
    return e;
}

size_t annihilate_smem_bytes() { return sizeof(K3Smem); }

// Whether a run's buckets can go through the staged kernel: every array a
// bulk copy reads on a 16-byte boundary (a caller-supplied allocator may
// return less aligned memory) and an even spawn capacity; buckets whose
// spawns exceed the stage are deferred to the large-bucket kernel
bool staged_annihilation_fits(const DevInst &I)
{
    auto al = [](const void *p) { return ((uintptr_t)p & 15u) == 0; };
    if (I.side || I.adaptive || (I.cap_s & 1)) return false;
    for (int k = 0; k < 2; k++)
        if (!al(I.key[k]) || !al(I.c[k]) || !al(I.hd[k]) || !al(I.fl[k])) return false;
    return al(I.skey) && al(I.sw);
}

// general: some run of the batch has replica side lists or adaptive shift;
// staged: every run fits the staged kernel (bulk copies one bucket ahead),
// launched as one resident wave of blocks (two per SM)
cudaError_t launch_annihilate(const DevInst *dinst, const int *unit_start, int n_inst, int n_units, bool general,
                              bool staged, cudaStream_t s)
{
    if (staged && !general && g_anni_bps == 0) {
        int grid = n_units < num_sms() * 2 ? n_units : num_sms() * 2;
        if (grid < 1) grid = 1;
        k_annihilate_staged<<<grid, K3_THREADS, sizeof(K4Smem<STAGED_SCAP>), s>>>(dinst, unit_start, n_inst, n_units);
        return cudaGetLastError();
    }
    const size_t smem = sizeof(K3Smem);
    const int bps = g_anni_bps > 0 ? g_anni_bps : 9;
    int grid = n_units < num_sms() * bps ? n_units : num_sms() * bps;
    if (grid < 1) grid = 1;
    if (general) k_annihilate<true><<<grid, K3_THREADS, smem, s>>>(dinst, unit_start, n_inst, n_units);
    else k_annihilate<false><<<grid, K3_THREADS, smem, s>>>(dinst, unit_start, n_inst, n_units);
    return cudaGetLastError();
}

void launch_annihilate_big(const DevInst *dinst, int n_inst, cudaStream_t s)
{
    k_annihilate_big<<<BIG_BLOCKS, K3_THREADS, 0, s>>>(dinst, n_inst);
}

void launch_finalize(const DevInst *dinst, int n_inst, cudaStream_t s)
{
    k_finalize<<<n_inst, K5_THREADS, 0, s>>>(dinst, n_inst);
}

// H_jj - E_ref of the determinants created in this iteration (new list,
// parity ^ 1), four per warp with eight lanes each.  The terms (h_pp of
// electron e1, or the pair e1 < e2) are listed once per block in shared
// memory, and each warp keeps the occupied orbitals of its four determinants
// there, so a term costs two shared loads and one table load; each lane group
// sums its terms exactly and reduces over its eight lanes.
constexpr int ND_PAIRS = 2080;  // n (n + 1) / 2 terms for up to 64 electrons

// H_ii - E_ref of the determinants at the slots list[0 .. nn) of list `np`
// (whole block; every thread calls it)
__device__ void diag_list(const DevInst &I, const unsigned *__restrict__ list, int nn, int np,
                          unsigned short *s_term, unsigned char (*s_orb)[4][64])
{
    const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    const int gw = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5), nwarp = (int)((gridDim.x * blockDim.x) >> 5);
    const ulonglong2 *nkey = I.key[np];
    double *nhd = I.hd[np];
    const int n = I.n, na = I.na, N = I.norb, T = n + n * (n - 1) / 2;
    if (n > 64) {  // beyond the table: the generic warp sum
        for (int q = 2 * gw; q < nn; q += 2 * nwarp) {
            const unsigned d0 = list[q], d1 = q + 1 < nn ? list[q + 1] : d0;
            const ulonglong2 k0 = nkey[d0], k1 = nkey[d1];
            const u64 ka[2] = {k0.x, k1.x}, kb[2] = {k0.y, k1.y};
            double hdv[2];
            diag_exact_warp_multi<2>(I, ka, kb, hdv);
            if (lane == 0) {
                nhd[d0] = hdv[0];
                if (q + 1 < nn) nhd[d1] = hdv[1];
            }
        }
        return;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < T; t += blockDim.x) {
        if (t < n) { s_term[t] = (unsigned short)(t | (255 << 8)); continue; }
        const int q = t - n;
        int c = 1;
        while ((c + 1) * c / 2 <= q) c++;
        s_term[t] = (unsigned short)((q - c * (c - 1) / 2) | (c << 8));
    }
    __syncthreads();
    // four determinants per warp, eight lanes each: lane group g takes
    // determinant q + g (a short last round repeats determinant q and
    // stores nothing for it), its lanes the terms sl, sl + 8, ...
    const int g = lane >> 3, sl = lane & 7;
    const i128 xref = (i128)(((u128)I.xref_hi << 64) | (u128)I.xref_lo);
    for (int q = 4 * gw; q < nn; q += 4 * nwarp) {
        const unsigned d = list[q + g < nn ? q + g : q];
        const ulonglong2 key = nkey[d];
        for (int e = sl; e < n; e += 8)
            s_orb[wl][g][e] = (unsigned char)(e < na ? nth_set(key.x, e) : nth_set(key.y, e - na));
        __syncwarp();
        i128 part = 0;
        for (int t0 = sl; t0 < T; t0 += 32) {
            ulonglong2 v[4];
#pragma unroll
            for (int r = 0; r < 4; r++) {
                const int t = t0 + 8 * r;
                v[r] = make_ulonglong2(0, 0);
                if (t < T) {
                    const unsigned tm = s_term[t];
                    const int e1 = (int)(tm & 0xffu), e2 = (int)(tm >> 8);
                    const int p1 = s_orb[wl][g][e1];
                    if (e2 == 255) v[r] = __ldg(I.hfx + p1);
                    else v[r] = __ldg((((e1 < na) == (e2 < na)) ? I.JKfx : I.Jfx) + p1 * N + s_orb[wl][g][e2]);
                }
            }
#pragma unroll
            for (int r = 0; r < 4; r++) part += (i128)(((u128)v[r].y << 64) | (u128)v[r].x);
        }
        for (int m = 4; m >= 1; m >>= 1) part += shfl_xor_i128(part, m);
        if (sl == 0 && q + g < nn) nhd[d] = fixed_to_double(part - xref, I.F);
        __syncwarp();
    }
}

__global__ void __launch_bounds__(256) k_new_diag(const DevInst *__restrict__ insts, int n_inst)
{
    __shared__ unsigned short s_term[ND_PAIRS];   // e1 | e2 << 8, e2 = 255 for h_pp
    __shared__ unsigned char s_orb[8][4][64];
    for (int ii = 0; ii < n_inst; ii++) {
        const DevInst &I = insts[ii];
        if (*(volatile int *)&I.st->err) continue;
        diag_list(I, I.newdet, I.st->new_n, I.st->parity ^ 1, s_term, s_orb);
    }
}

// H_ii - E_ref of every determinant of list `par`, given by its slots (import)
__global__ void __launch_bounds__(256) k_diag_list(const DevInst *__restrict__ I, int par, const unsigned *list, int nn)
{
    __shared__ unsigned short s_term[ND_PAIRS];
    __shared__ unsigned char s_orb[8][4][64];
    diag_list(*I, list, nn, par, s_term, s_orb);
}

void launch_diag_list(const DevInst *dinst, int par, const unsigned *list, int nn, cudaStream_t s)
{
    if (nn > 0) k_diag_list<<<num_sms() * 3, 256, 0, s>>>(dinst, par, list, nn);
}

void launch_new_diag(const DevInst *dinst, int n_inst, cudaStream_t s)
{
    // one resident wave (3 blocks per SM at 80 registers): fewer blocks repeat the term-table set-up
    k_new_diag<<<num_sms() * 3, 256, 0, s>>>(dinst, n_inst);
}

void launch_rebucket(const DevInst *src, const DevInst *dst, int nb_src, int parity, cudaStream_t s)
{
    int grid = nb_src < num_sms() * 8 ? nb_src : num_sms() * 8;
    k_rebucket<<<grid, 256, 0, s>>>(src, dst, nb_src, parity);
}

void launch_diag(const DevInst *dinst, int parity, int nb, cudaStream_t s)
{
    int warps = nb;
    int blocks = (warps * 32 + 255) / 256;
    if (blocks > num_sms() * 16) blocks = num_sms() * 16;
    if (blocks < 1) blocks = 1;
    k_diag<<<blocks, 256, 0, s>>>(dinst, parity, nb);
}

u64 det_hash_host(u64 a, u64 b) { return det_hash(a, b); }

}  // namespace fq
