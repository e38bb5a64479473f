/*
 * fciqmc_oracle.c -- CPU oracle for the initiator-FCIQMC projector iteration.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is a plain, slow, single-threaded
 * restatement of the method of Guther et al., "NECI: N-Electron Configuration
 * Interaction with an emphasis on state-of-the-art stochastic methods"
 * (J. Chem. Phys. 153, 034107 (2020), arXiv:2006.14956).  It is used only by
 * tests/, by __graft_entry__.smoke() and by the cpu_baseline leg of bench.py.
 * The GPU library never links, loads or calls it, and it shares no code with
 * the GPU library.
 *
 * Build: gcc -O2 -std=gnu11 -ffp-contract=off -fno-fast-math -shared -fPIC
 * (-ffp-contract=off is essential: every floating-point expression below is
 * evaluated as written, one IEEE-754 binary64 operation at a time, with no
 * fused multiply-add.)
 *
 * What is computed, in the paper's order (Sec. I, Eq. (4)):
 *   (a) spawn:  sum_{j != i} -dtau H_ji C_i |D_j>, sampled with one excitation
 *       per attempt, p_s = dtau |H_ij| / p_gen(j|i) (Sec. II, Eq. (5));
 *   (b) death:  (1 - dtau (H_ii - S)) C_i, then stochastic rounding (Eq. (3));
 *   (c) annihilation: all spawned contributions to a determinant are summed
 *       into it, with the initiator rule (Sec. I) applied to spawns onto
 *       unoccupied determinants, then stochastic rounding;
 *   plus the shift update (Eq. (2), S(tau) "updated to match the ground
 *   state energy"), the reference projected energy (Sec. IV, Eq. (9)), and
 *   semi-stochastic projection (Sec. III, Eqs. (7)-(8)).
 *
 * Readings adopted where the paper is silent (each listed in the design notes):
 *   R1  determinant = (alpha word, beta word); canonical operator order is
 *       alpha_0 < ... < alpha_{N-1} < beta_0 < ... < beta_{N-1}.
 *   R2  integrals are chemist (pq|rs), packed with 8-fold symmetry (FCIDUMP).
 *   R3  random numbers: Philox4x64-10 (Salmon et al., SC'11), key = (seed, 0),
 *       counter = (alpha, beta, iteration, (slot << 8) | purpose).
 *   R4  every multi-term sum in a matrix element (H_ii, single-excitation H_ij)
 *       and the sum of the spawns onto one determinant is the exact sum of its
 *       binary64 terms, rounded once to nearest-even ("fsum").
 *   R5  spawn weight w = -(H_ji * (lambda_c * (C_i / n_att))) with
 *       lambda_c = dtau / p_gen(c); n_att = ceil(|C_i|).
 *   R6  N_w = 2^-32 * sum floor(|C_i| 2^32) (exact integer sum).
 *   R7  shift: S <- S - (zeta / (A dtau)) ln(N_w(t) / N_w(t - A)) every A
 *       iterations once N_w first reaches the target (Booth, Thom and Alavi,
 *       J. Chem. Phys. 131, 054106 (2009), cited by the paper); ln is the
 *       argument-reduction + atanh-series recipe in orc_ln below.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

typedef unsigned __int128 u128;
typedef __int128 i128;

/* ------------------------------------------------------------------ */
/* Philox4x64-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: */
/* as easy as 1, 2, 3", SC'11): ten rounds of two 64x64->128 products. */
/* ------------------------------------------------------------------ */
#define PHILOX_M0 0xD2E7470EE14C6C93ULL
#define PHILOX_M1 0xCA5A826395121157ULL
#define PHILOX_W0 0x9E3779B97F4A7C15ULL /* golden ratio */
#define PHILOX_W1 0xBB67AE8584CAA73BULL /* sqrt(3) - 1 */

void orc_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4])
{
    uint64_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint64_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; r++) {
        if (r > 0) { k0 += PHILOX_W0; k1 += PHILOX_W1; }
        u128 p0 = (u128)PHILOX_M0 * c0;
        u128 p1 = (u128)PHILOX_M1 * c2;
        uint64_t hi0 = (uint64_t)(p0 >> 64), lo0 = (uint64_t)p0;
        uint64_t hi1 = (uint64_t)(p1 >> 64), lo1 = (uint64_t)p1;
        uint64_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

enum { PURPOSE_SPAWN = 1, PURPOSE_DEATH = 2, PURPOSE_ANNIH = 3 };

/* one Philox block; the key's second word is the replica index (0 for a
 * single run), so that replicas draw independent streams */
static void draw(uint64_t seed, uint64_t replica, uint64_t a, uint64_t b, int64_t iter, uint64_t slot,
                 int purpose, uint64_t w[4])
{
    uint64_t ctr[4] = { a, b, (uint64_t)iter, (slot << 8) | (uint64_t)purpose };
    uint64_t key[2] = { seed, replica };
    orc_philox4x64_10(ctr, key, w);
}

/* uniform double in [0,1) from the top 53 bits of a word */
static double u53(uint64_t w) { return (double)(w >> 11) * 0x1p-53; }
/* integer in [0, m): floor(w * m / 2^64) */
static uint64_t pick(uint64_t w, uint64_t m) { return (uint64_t)(((u128)w * m) >> 64); }

/* ------------------------------------------------------------------ */
/* Exact summation (reading R4): a fixed-point accumulator spanning the  */
/* whole binary64 range (Kulisch).  Digits are 32-bit, kept in int64    */
/* so that carries can be deferred.  value = sum l[k] 2^(32k - 1088).   */
/* ------------------------------------------------------------------ */
#define XL 70
typedef struct { int64_t l[XL]; int bad; } xacc;

static void xacc_zero(xacc *x) { memset(x, 0, sizeof *x); }

static void xacc_add(xacc *x, double v, int negate)
{
    uint64_t bits;
    memcpy(&bits, &v, 8);
    int ex = (int)((bits >> 52) & 0x7ff);
    if (ex == 0x7ff) { x->bad = 1; return; }
    uint64_t m = bits & ((1ULL << 52) - 1);
    int e;
    if (ex == 0) e = -1074; else { m |= 1ULL << 52; e = ex - 1075; }
    if (m == 0) return;
    int neg = (int)(bits >> 63) ^ (negate ? 1 : 0);
    int pos = e + 1088;
    int k = pos / 32, s = pos % 32;
    u128 t = (u128)m << s;
    int64_t d0 = (int64_t)(uint32_t)t, d1 = (int64_t)(uint32_t)(t >> 32), d2 = (int64_t)(uint32_t)(t >> 64);
    if (neg) { x->l[k] -= d0; x->l[k + 1] -= d1; x->l[k + 2] -= d2; }
    else     { x->l[k] += d0; x->l[k + 1] += d1; x->l[k + 2] += d2; }
}

static void xacc_merge(xacc *x, const xacc *y, int negate)
{
    for (int k = 0; k < XL; k++) x->l[k] += negate ? -y->l[k] : y->l[k];
    x->bad |= y->bad;
}

/* round the exact value to the nearest binary64, ties to even */
static double xacc_round(const xacc *x)
{
    if (x->bad) return NAN;
    uint32_t d[XL];
    int64_t carry = 0;
    for (int k = 0; k < XL; k++) {
        int64_t t = x->l[k] + carry;
        d[k] = (uint32_t)t;
        carry = t >> 32; /* arithmetic: floor division */
    }
    int neg = carry < 0;
    if (neg) { /* two's complement negation of the digit string */
        uint64_t c = 1;
        for (int k = 0; k < XL; k++) {
            uint64_t t = (uint64_t)(uint32_t)~d[k] + c;
            d[k] = (uint32_t)t;
            c = t >> 32;
        }
    }
    int top = XL - 1;
    while (top >= 0 && d[top] == 0) top--;
    if (top < 0) return 0.0;
    int msb = 32 * top + (31 - __builtin_clz(d[top]));
    int lsb = msb - 52;
    if (lsb < 14) lsb = 14; /* bit 14 has weight 2^-1074 */
#define GETBIT(i) ((d[(i) >> 5] >> ((i) & 31)) & 1u)
    uint64_t mant = 0;
    for (int i = msb; i >= lsb; i--) mant = (mant << 1) | GETBIT(i);
    int rb = 0, sticky = 0;
    if (lsb - 1 >= 0) rb = (int)GETBIT(lsb - 1);
    for (int i = lsb - 2; i >= 0 && !sticky; i--) sticky = (int)GETBIT(i);
#undef GETBIT
    if (rb && (sticky || (mant & 1))) mant++;
    double r = ldexp((double)mant, lsb - 1088);
    return neg ? -r : r;
}

double orc_fsum(const double *v, int64_t n)
{
    xacc x;
    xacc_zero(&x);
    for (int64_t i = 0; i < n; i++) xacc_add(&x, v[i], 0);
    return xacc_round(&x);
}

/* ------------------------------------------------------------------ */
/* Natural logarithm for the shift update (reading R7): write x = m 2^k  */
/* with m in (sqrt(1/2), sqrt(2)], then ln x = k ln2 + 2 atanh(s),       */
/* s = (m-1)/(m+1), with the atanh series summed to z^11 (z = s^2).     */
/* ------------------------------------------------------------------ */
double orc_ln(double x)
{
    if (!(x > 0.0) || isinf(x)) return NAN;
    uint64_t bits;
    memcpy(&bits, &x, 8);
    int k;
    if (((bits >> 52) & 0x7ff) == 0) { /* subnormal: scale into range first */
        double y = x * 0x1p54;
        memcpy(&bits, &y, 8);
        k = (int)((bits >> 52) & 0x7ff) - 1023 - 54;
    } else {
        k = (int)((bits >> 52) & 0x7ff) - 1023;
    }
    bits = (bits & ((1ULL << 52) - 1)) | (1023ULL << 52);
    double m;
    memcpy(&m, &bits, 8);
    if (m > 1.4142135623730951) { m = m * 0.5; k += 1; }
    double s = (m - 1.0) / (m + 1.0);
    double z = s * s;
    double p = 2.0 / 23.0;
    for (int j = 10; j >= 0; j--) p = 2.0 / (double)(2 * j + 1) + z * p;
    double r = s * p;
    const double ln2_hi = 0x1.62e42fefa39efp-1, ln2_lo = 0x1.abc9e3b39803fp-56;
    return (double)k * ln2_hi + ((double)k * ln2_lo + r);
}

/* ------------------------------------------------------------------ */
/* System: integrals and reference determinant                          */
/* ------------------------------------------------------------------ */
typedef struct {
    int norb, na, nb, kind; /* kind 0: ab initio, 1: Hubbard */
    double ecore;
    double *h;   /* norb x norb, row-major */
    double *eri; /* packed 8-fold */
    int lx, ly, z; /* Hubbard lattice; z neighbour slots per site */
    double t, U;
    int *nbr; /* nbr[site * 4 + k], -1 when absent */
    uint64_t ref_a, ref_b;
    xacc xref; /* exact diagonal sum X(D_ref) */
    double eref;
    int Fe;    /* grid 2^-Fe of the E_num terms (reading R12) */
} orc_sys;

void orc_sys_free(orc_sys *s);
static int64_t pairidx(int64_t i, int64_t j) { return i >= j ? i * (i + 1) / 2 + j : j * (j + 1) / 2 + i; }

static double eri(const orc_sys *s, int p, int q, int r, int t)
{
    return s->eri[pairidx(pairidx(p, q), pairidx(r, t))];
}

static uint64_t lowmask(int p) { return p >= 64 ? ~0ULL : ((1ULL << p) - 1); }
static int popc(uint64_t x) { return __builtin_popcountll(x); }

/* exact diagonal sum X(D) = sum_occ h_pp + sum_{pairs} [(pp|qq) - delta_spin (pq|qp)] */
static void xdiag(const orc_sys *s, uint64_t a, uint64_t b, xacc *x)
{
    int occ[128], spin[128], n = 0;
    for (int p = 0; p < s->norb; p++) if ((a >> p) & 1) { occ[n] = p; spin[n] = 0; n++; }
    for (int p = 0; p < s->norb; p++) if ((b >> p) & 1) { occ[n] = p; spin[n] = 1; n++; }
    xacc_zero(x);
    for (int i = 0; i < n; i++) xacc_add(x, s->h[occ[i] * s->norb + occ[i]], 0);
    for (int i = 0; i < n; i++)
        for (int j = i + 1; j < n; j++) {
            xacc_add(x, eri(s, occ[i], occ[i], occ[j], occ[j]), 0);
            if (spin[i] == spin[j]) xacc_add(x, eri(s, occ[i], occ[j], occ[j], occ[i]), 1);
        }
}

/* H_ii - E_ref, rounded once from the exact difference (reading R4) */
double orc_hdiag_rel(const orc_sys *s, uint64_t a, uint64_t b)
{
    xacc x;
    xdiag(s, a, b, &x);
    xacc_merge(&x, &s->xref, 1);
    return xacc_round(&x);
}

double orc_eref(const orc_sys *s) { return s->eref; }

/* occupation test / operator application on the canonical ordering */
static int occupied(uint64_t a, uint64_t b, int norb, int pos)
{
    return pos < norb ? (int)((a >> pos) & 1) : (int)((b >> (pos - norb)) & 1);
}
static int n_before(uint64_t a, uint64_t b, int norb, int pos)
{
    return pos < norb ? popc(a & lowmask(pos)) : popc(a) + popc(b & lowmask(pos - norb));
}
static void flip(uint64_t *a, uint64_t *b, int norb, int pos)
{
    if (pos < norb) *a ^= 1ULL << pos; else *b ^= 1ULL << (pos - norb);
}
/* apply a_pos (create=0) or a+_pos (create=1); returns sign (+1/-1) or 0 */
static int apply_op(uint64_t *a, uint64_t *b, int norb, int pos, int create)
{
    int o = occupied(*a, *b, norb, pos);
    if (create == o) return 0;
    int sg = (n_before(*a, *b, norb, pos) & 1) ? -1 : 1;
    flip(a, b, norb, pos);
    return sg;
}

/* <D_j|H|D_i> for D_j != D_i (Slater-Condon rules) */
double orc_hoff(const orc_sys *s, uint64_t ia, uint64_t ib, uint64_t ja, uint64_t jb)
{
    int N = s->norb;
    uint64_t da = ia ^ ja, db = ib ^ jb;
    int nd = popc(da) + popc(db);
    if (nd == 0 || nd > 4) return 0.0;
    if (popc(ia) != popc(ja) || popc(ib) != popc(jb)) return 0.0;
    int rem[2], add[2], nr = 0, nadd = 0;
    for (int pos = 0; pos < 2 * N; pos++) {
        int oi = occupied(ia, ib, N, pos), oj = occupied(ja, jb, N, pos);
        if (oi && !oj) rem[nr++] = pos;
        if (!oi && oj) add[nadd++] = pos;
    }
    if (nr == 1) {
        int i = rem[0], a = add[0];
        uint64_t xa = ia, xb = ib;
        int g = apply_op(&xa, &xb, N, i, 0);
        g *= apply_op(&xa, &xb, N, a, 1);
        int sp = i >= N, oi = i % N, oa = a % N;
        xacc x;
        xacc_zero(&x);
        xacc_add(&x, s->h[oa * N + oi], 0);
        for (int k = 0; k < 2 * N; k++) {
            if (k == i || !occupied(ia, ib, N, k)) continue;
            int ok = k % N;
            xacc_add(&x, eri(s, oa, oi, ok, ok), 0);
            if ((k >= N) == sp) xacc_add(&x, eri(s, oa, ok, ok, oi), 1);
        }
        double v = xacc_round(&x);
        return g < 0 ? -v : v;
    }
    /* double: i < j removed, a < b added; gamma from a+_a a+_b a_j a_i |D_i> */
    int i = rem[0], j = rem[1], a = add[0], b = add[1];
    uint64_t xa = ia, xb = ib;
    int g = apply_op(&xa, &xb, N, i, 0);
    g *= apply_op(&xa, &xb, N, j, 0);
    g *= apply_op(&xa, &xb, N, b, 1);
    g *= apply_op(&xa, &xb, N, a, 1);
    int si = i >= N, sj = j >= N, sa = a >= N, sb = b >= N;
    int oi = i % N, oj = j % N, oa = a % N, ob = b % N;
    /* <ab|ij> = (ai|bj) d(sa,si) d(sb,sj);  <ab|ji> = (aj|bi) d(sa,sj) d(sb,si) */
    int dir = (sa == si) && (sb == sj), exch = (sa == sj) && (sb == si);
    double v;
    if (dir && exch) v = eri(s, oa, oi, ob, oj) - eri(s, oa, oj, ob, oi);
    else if (dir) v = eri(s, oa, oi, ob, oj);
    else if (exch) v = -eri(s, oa, oj, ob, oi);
    else v = 0.0;
    return g < 0 ? -v : v;
}

/* E_num of Eq. (9) (reading R12): each term H_ref,j C_j is the binary64
 * product truncated toward zero to a multiple of 2^-Fe; the truncated terms
 * are summed exactly and the sum is rounded once.  Fe = min(64, 60 - m - L),
 * m = floor(log2 max |integral|) over h, (pq|rs) and E_core (Fe = 64 when all
 * vanish), L = ceil(log2(2n + 1)): |H_ref,j| < (2n + 1) 2^(m + 1), |C_j| <
 * 2^31 and at most 2^34 terms keep the sum below 2^126 grid steps. */
static int enum_grid(const orc_sys *s)
{
    int64_t nh = (int64_t)s->norb * s->norb, np = (int64_t)s->norb * (s->norb + 1) / 2, ne = np * (np + 1) / 2;
    int any = 0, m = 0;
    for (int64_t i = 0; i < nh + ne + 1; i++) {
        double x = i < nh ? s->h[i] : (i < nh + ne ? s->eri[i - nh] : s->ecore);
        if (x == 0.0) continue;
        int e;
        frexp(fabs(x), &e); /* |x| in [2^(e-1), 2^e) */
        if (!any || e - 1 > m) m = e - 1;
        any = 1;
    }
    if (!any) return 64;
    int n = s->na + s->nb, L = 0;
    while ((1LL << L) < 2LL * n + 1) L++;
    int fe = 60 - m - L;
    return fe > 64 ? 64 : fe;
}

static double trunc_grid(double p, int F)
{
    /* exact: p 2^F stays far below 2^1023, its integer part has at most 53
     * significant bits, and a nonzero result is at least 2^-F >= 2^-64 */
    return ldexp(trunc(ldexp(p, F)), -F);
}

static int sys_finish(orc_sys *s)
{
    if (popc(s->ref_a) != s->na || popc(s->ref_b) != s->nb) return -1;
    if (s->norb < 64 && ((s->ref_a | s->ref_b) >> s->norb) != 0) return -1;
    s->Fe = enum_grid(s);
    xdiag(s, s->ref_a, s->ref_b, &s->xref);
    xacc x = s->xref;
    xacc_add(&x, s->ecore, 0);
    s->eref = xacc_round(&x);
    return 0;
}

/* Integral grid (reading): the GPU library sums integrals exactly in 128-bit
 * fixed point, which caps the span between the largest integral and the
 * finest bit it must represent.  Where the integrals' finest bit lies beyond
 * that span, every h_pq, (pq|rs) and E_core is replaced by its nearest
 * multiple of 2^-G (ties to even), with
 *   G = 125 - m - 2 - max(ceil(log2(n^2 + 2n + 4)), ceil(log2(N^2)) + 2),
 * m = floor(log2 max |integral|), n electrons, N orbitals; otherwise the
 * integrals are used as given.  Returns nonzero when no such grid exists. */
static int lowest_bit(double x)  /* exponent of the lowest set bit of x != 0 */
{
    int e;
    double m = frexp(fabs(x), &e); /* |x| = m 2^e, m in [0.5, 1) */
    uint64_t q = (uint64_t)ldexp(m, 53);  /* exact: 53-bit integer */
    int z = 0;
    while (!(q & 1)) { q >>= 1; z++; }
    return e - 53 + z;
}

static int integral_grid(orc_sys *s, int64_t ne)
{
    int64_t nh = (int64_t)s->norb * s->norb;
    int any = 0, lo = 0, hi = 0;
    for (int64_t i = 0; i < nh + ne + 1; i++) {
        double x = i < nh ? s->h[i] : (i < nh + ne ? s->eri[i - nh] : s->ecore);
        if (x == 0.0) continue;
        if (!isfinite(x)) return 1;
        int e;
        frexp(fabs(x), &e);
        int l = lowest_bit(x);
        if (!any || l < lo) lo = l;
        if (!any || e - 1 > hi) hi = e - 1;
        any = 1;
    }
    if (!any) return 0;
    int n = s->na + s->nb, tb = 0, kb = 0;
    while ((1LL << tb) < (long long)n * n + 2 * n + 4) tb++;
    while ((1LL << kb) < (long long)s->norb * s->norb) kb++;
    int G = 125 - hi - 2 - (tb > kb + 2 ? tb : kb + 2);
    if (-lo <= G) return 0;
    if (G < 0) return 1;
    for (int64_t i = 0; i < nh; i++) s->h[i] = ldexp(nearbyint(ldexp(s->h[i], G)), -G);
    for (int64_t i = 0; i < ne; i++) s->eri[i] = ldexp(nearbyint(ldexp(s->eri[i], G)), -G);
    s->ecore = ldexp(nearbyint(ldexp(s->ecore, G)), -G);
    return 0;
}

orc_sys *orc_sys_abinitio(int norb, int na, int nb, double ecore, const double *h,
                          const double *eri_packed, const uint64_t *ref)
{
    if (norb < 1 || norb > 64 || na < 0 || nb < 0 || na > norb || nb > norb) return NULL;
    orc_sys *s = calloc(1, sizeof *s);
    s->norb = norb; s->na = na; s->nb = nb; s->kind = 0; s->ecore = ecore;
    int64_t np = (int64_t)norb * (norb + 1) / 2, ne = np * (np + 1) / 2;
    s->h = malloc(sizeof(double) * norb * norb);
    s->eri = malloc(sizeof(double) * ne);
    memcpy(s->h, h, sizeof(double) * norb * norb);
    memcpy(s->eri, eri_packed, sizeof(double) * ne);
    if (integral_grid(s, ne)) { orc_sys_free(s); return NULL; }
    if (ref) { s->ref_a = ref[0]; s->ref_b = ref[1]; }
    else { s->ref_a = lowmask(na); s->ref_b = lowmask(nb); } /* aufbau */
    if (sys_finish(s)) { orc_sys_free(s); return NULL; }
    return s;
}

/* Hubbard model: h_pq = -t for lattice neighbours, (pp|pp) = U.
 * Sites are numbered x + lx*y; neighbour slots in the order -x, +x, -y, +y. */
orc_sys *orc_sys_hubbard(int lx, int ly, int px, int py, double t, double U, int na, int nb,
                         const uint64_t *ref)
{
    int ns = lx * ly;
    if (ns < 1 || ns > 64 || (px && lx < 3 && lx > 1) || (py && ly < 3 && ly > 1)) return NULL;
    orc_sys *s = calloc(1, sizeof *s);
    s->norb = ns; s->na = na; s->nb = nb; s->kind = 1; s->lx = lx; s->ly = ly; s->t = t; s->U = U;
    s->z = ly > 1 ? 4 : 2;
    s->nbr = malloc(sizeof(int) * 4 * ns);
    for (int y = 0; y < ly; y++)
        for (int x = 0; x < lx; x++) {
            int p = x + lx * y, *nb4 = s->nbr + 4 * p;
            nb4[0] = x > 0 ? p - 1 : (px && lx > 1 ? p + lx - 1 : -1);
            nb4[1] = x < lx - 1 ? p + 1 : (px && lx > 1 ? p - (lx - 1) : -1);
            nb4[2] = y > 0 ? p - lx : (py && ly > 1 ? p + lx * (ly - 1) : -1);
            nb4[3] = y < ly - 1 ? p + lx : (py && ly > 1 ? p - lx * (ly - 1) : -1);
        }
    int64_t np = (int64_t)ns * (ns + 1) / 2, ne = np * (np + 1) / 2;
    s->h = calloc((size_t)ns * ns, sizeof(double));
    s->eri = calloc((size_t)ne, sizeof(double));
    for (int p = 0; p < ns; p++)
        for (int k = 0; k < s->z; k++) {
            int q = s->nbr[4 * p + k];
            if (q >= 0) s->h[p * ns + q] = -t;
        }
    for (int p = 0; p < ns; p++) s->eri[pairidx(pairidx(p, p), pairidx(p, p))] = U;
    if (ref) { s->ref_a = ref[0]; s->ref_b = ref[1]; }
    else { /* Neel: alpha on (x+y) even, beta on (x+y) odd */
        for (int y = 0; y < ly; y++)
            for (int x = 0; x < lx; x++) {
                if (((x + y) & 1) == 0) s->ref_a |= 1ULL << (x + lx * y);
                else s->ref_b |= 1ULL << (x + lx * y);
            }
    }
    if (sys_finish(s)) { orc_sys_free(s); return NULL; }
    return s;
}

void orc_sys_free(orc_sys *s)
{
    if (!s) return;
    free(s->h); free(s->eri); free(s->nbr); free(s);
}

void orc_sys_ref(const orc_sys *s, uint64_t out[2]) { out[0] = s->ref_a; out[1] = s->ref_b; }

/* dense H - E_ref over a given list of determinants (for exact diagonalisation) */
void orc_build_hamiltonian(const orc_sys *s, int64_t n, const uint64_t *da, const uint64_t *db, double *H)
{
    for (int64_t i = 0; i < n; i++)
        for (int64_t j = 0; j < n; j++)
            H[i * n + j] = (i == j) ? orc_hdiag_rel(s, da[i], db[i]) : orc_hoff(s, da[j], db[j], da[i], db[i]);
}

/* ------------------------------------------------------------------ */
/* Excitation generation (Sec. II; App. A, "Uniform excitation          */
/* generation" with spin conditioning; lattice hops for Hubbard).       */
/* ------------------------------------------------------------------ */
enum { CLS_SINGLE_A = 0, CLS_SINGLE_B, CLS_DOUBLE_AB, CLS_DOUBLE_AA, CLS_DOUBLE_BB, CLS_HOP, NCLS };

/* generation probability of one outcome of class c */
double orc_pgen(const orc_sys *s, double p_single, int c)
{
    int n = s->na + s->nb, N = s->norb;
    int64_t ma = N - s->na, mb = N - s->nb;
    int64_t nn = (int64_t)n * (n - 1);
    switch (c) {
    case CLS_SINGLE_A: return p_single / ((double)n * (double)ma);
    case CLS_SINGLE_B: return p_single / ((double)n * (double)mb);
    case CLS_DOUBLE_AB: return ((1.0 - p_single) * 2.0) / ((double)nn * (double)(ma * mb));
    case CLS_DOUBLE_AA: return ((1.0 - p_single) * 4.0) / ((double)nn * (double)(ma * (ma - 1)));
    case CLS_DOUBLE_BB: return ((1.0 - p_single) * 4.0) / ((double)nn * (double)(mb * (mb - 1)));
    case CLS_HOP: return 1.0 / ((double)n * (double)s->z);
    }
    return 0.0;
}

/* orbital of electron e (alpha electrons first, each spin ascending) */
static int electron_orb(uint64_t a, uint64_t b, int na, int e, int *spin)
{
    uint64_t w = e < na ? a : b;
    int k = e < na ? e : e - na;
    *spin = e < na ? 0 : 1;
    for (int p = 0; p < 64; p++)
        if ((w >> p) & 1) { if (k == 0) return p; k--; }
    return -1;
}
/* k-th empty orbital of a spin word */
static int kth_empty(uint64_t w, int norb, int k)
{
    for (int p = 0; p < norb; p++)
        if (!((w >> p) & 1)) { if (k == 0) return p; k--; }
    return -1;
}

/* One generation from D = (a,b) with the four words of its draw.
 * Returns the class, or -1 for a failed attempt; target in (*ta, *tb). */
int orc_generate(const orc_sys *s, double p_single, uint64_t a, uint64_t b, const uint64_t w[4],
                 uint64_t *ta, uint64_t *tb)
{
    int N = s->norb, n = s->na + s->nb;
    *ta = a; *tb = b;
    if (n == 0) return -1;
    if (s->kind == 1) {
        int sp, e = (int)pick(w[1], (uint64_t)n);
        int p = electron_orb(a, b, s->na, e, &sp);
        int q = s->nbr[4 * p + (int)pick(w[2], (uint64_t)s->z)];
        if (q < 0) return -1;
        uint64_t *x = sp ? tb : ta;
        if ((*x >> q) & 1) return -1;
        *x ^= (1ULL << p) | (1ULL << q);
        return CLS_HOP;
    }
    int ma = N - s->na, mb = N - s->nb;
    if (u53(w[0]) < p_single) {
        int sp, e = (int)pick(w[1], (uint64_t)n);
        int i = electron_orb(a, b, s->na, e, &sp);
        int m = sp ? mb : ma;
        if (m == 0) return -1;
        uint64_t *x = sp ? tb : ta;
        int h = kth_empty(*x, N, (int)pick(w[2], (uint64_t)m));
        *x ^= (1ULL << i) | (1ULL << h);
        return sp ? CLS_SINGLE_B : CLS_SINGLE_A;
    }
    if (n < 2) return -1;
    uint64_t xe = pick(w[1], (uint64_t)n * (uint64_t)(n - 1));
    int e1 = (int)(xe / (uint64_t)(n - 1)), r = (int)(xe % (uint64_t)(n - 1));
    int e2 = r + (r >= e1 ? 1 : 0);
    int s1, s2;
    int o1 = electron_orb(a, b, s->na, e1, &s1), o2 = electron_orb(a, b, s->na, e2, &s2);
    if (s1 != s2) {
        if (ma == 0 || mb == 0) return -1;
        int oa = s1 == 0 ? o1 : o2, ob = s1 == 0 ? o2 : o1;
        uint64_t y = pick(w[2], (uint64_t)ma * (uint64_t)mb);
        int ha = kth_empty(a, N, (int)(y / (uint64_t)mb)), hb = kth_empty(b, N, (int)(y % (uint64_t)mb));
        *ta ^= (1ULL << oa) | (1ULL << ha);
        *tb ^= (1ULL << ob) | (1ULL << hb);
        return CLS_DOUBLE_AB;
    }
    int m = s1 ? mb : ma;
    if (m < 2) return -1;
    uint64_t *x = s1 ? tb : ta;
    uint64_t y = pick(w[2], (uint64_t)m * (uint64_t)(m - 1));
    int h1 = (int)(y / (uint64_t)(m - 1)), rr = (int)(y % (uint64_t)(m - 1));
    int h2 = rr + (rr >= h1 ? 1 : 0);
    int pa = kth_empty(*x, N, h1), pb = kth_empty(*x, N, h2);
    *x ^= (1ULL << o1) | (1ULL << o2) | (1ULL << pa) | (1ULL << pb);
    return s1 ? CLS_DOUBLE_BB : CLS_DOUBLE_AA;
}

/* ------------------------------------------------------------------ */
/* FCIQMC run                                                           */
/* ------------------------------------------------------------------ */
typedef struct {
    double tau, shift_damping, target_walkers, initial_walkers, initial_shift;
    double initiator_threshold, c_min, p_single;
    int64_t shift_interval;
    uint64_t seed;
    int64_t semistoch_size, semistoch_start;
    int64_t generator; /* 0: uniform doubles, 1: pre-computed heat-bath doubles (App. A) */
    int64_t trial_size, trial_start; /* trial space T of the E_Trial estimator (Sec. IV) */
    int64_t replica;                 /* replica index: second word of the Philox key */
    int64_t adaptive_shift;          /* 1: local shift f_i S for non-initiators (Sec. V, adaptive shift) */
} orc_params;

typedef struct { uint64_t a, b; double c, hd; int flags; } odet; /* flags: 1 ref, 2 in D */
typedef struct { uint64_t a, b; double w; int init; int64_t parent; } ospawn;

typedef struct {
    int64_t iter;
    double nw, S, e_num, e_den;
    int64_t ndet, attempts, spawns, rejected;
    double annihilated;
    int vary;
    double t_num, t_den; /* E_Trial: <Psi^T|H - E_ref|Psi>, <Psi^T|Psi> after the iteration */
    /* replica pair (Sec. V, VI), filled in the first replica's row:
     * <Psi^1|Psi^2>, the variational numerator and the PT2 numerator */
    double x_overlap, x_var_num, x_pt2;
} orc_stat;

/* Pre-computed heat-bath tables (App. A, "Pre-computed heat-bath sampling",
 * Eq. (hbs)): for every pair of occupied spatial orbitals one distribution
 * over hole pairs with p(ab|ij) = |H_ij^ab| / sum_a'b' |H_ij^a'b'|, sampled by
 * Walker's alias method.  Reading: the tables carry explicit spins -- one per
 * ordered pair (i alpha, j beta) over (a alpha, b beta), H = (ai|bj), and one
 * per same-spin pair i < j over a < b, H = (ai|bj) - (aj|bi) -- which makes
 * the paper's exchange/no-exchange split of the spatial tables unnecessary.
 * H_ij^ab is the element of a double excitation, so an entry whose hole is
 * one of the two electrons' own spin orbitals (a = i or b = j for opposite
 * spins; a or b in {i, j} for equal spins) has weight 0. */
typedef struct {
    int K;        /* entries */
    double S;     /* exact sum of |H| over the entries, rounded once */
    double lam;   /* (tau * S) / p_pair: |H| / p_gen, the same for every entry */
    double *prob; /* alias thresholds in [0, 1] */
    int *alias;
    int *ea, *eb; /* the hole pair of each entry */
    double *val;  /* H_ij^ab of each entry (without the determinant's sign) */
} opchb;

typedef struct {
    orc_sys *s;
    orc_params p;
    double lam[NCLS];
    opchb *pchb_ab; /* [i * N + j], i alpha, j beta */
    opchb *pchb_ss; /* [i * N + j], i < j, same spin */
    int pchb_n;     /* N of the tables (kept: the system may be released first) */
    odet *L;
    int64_t n, cap;
    int64_t iter;
    double S;
    int vary;
    int64_t shift_start, cnt;
    u128 nw_last;
    /* semi-stochastic space: D sorted by key; CSR over D indices */
    int64_t nd;
    uint64_t *Da, *Db;
    int64_t *rowptr, *col;
    double *val;
    orc_stat *st;
    int64_t nst, stcap;
    int err;
    /* trial space T (sorted keys), its H^T ground state (cT, E^T relative to
     * E_ref), and W_j = sum_{i in T} <D_j|H - E_ref|D_i> cT_i over T and the
     * space C connected to it (sorted keys) */
    int64_t nt, nwt;
    uint64_t *Ta, *Tb, *Wa, *Wb;
    double *cT, *W, ET;
    /* the last iteration's start list and spawns, kept for a replica pair */
    int keep_last;
    odet *L0;
    int64_t n0;
    ospawn *sp0;
    int64_t ns0;
    double *f0; /* the last iteration's f_i per start-list entry (adaptive shift) */
} orc_run;

static int cmp_key(uint64_t a1, uint64_t b1, uint64_t a2, uint64_t b2)
{
    if (a1 != a2) return a1 < a2 ? -1 : 1;
    if (b1 != b2) return b1 < b2 ? -1 : 1;
    return 0;
}
static int cmp_odet(const void *x, const void *y)
{
    const odet *p = x, *q = y;
    return cmp_key(p->a, p->b, q->a, q->b);
}
static int cmp_ospawn(const void *x, const void *y)
{
    const ospawn *p = x, *q = y;
    return cmp_key(p->a, p->b, q->a, q->b);
}

static int64_t find_det(const odet *L, int64_t n, uint64_t a, uint64_t b)
{
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t mid = (lo + hi) / 2;
        int c = cmp_key(L[mid].a, L[mid].b, a, b);
        if (c == 0) return mid;
        if (c < 0) lo = mid + 1; else hi = mid;
    }
    return -1;
}
static int64_t find_D(const orc_run *r, uint64_t a, uint64_t b)
{
    int64_t lo = 0, hi = r->nd;
    while (lo < hi) {
        int64_t mid = (lo + hi) / 2;
        int c = cmp_key(r->Da[mid], r->Db[mid], a, b);
        if (c == 0) return mid;
        if (c < 0) lo = mid + 1; else hi = mid;
    }
    return -1;
}

/* floor(|c| 2^32) as an integer (reading R6) */
static u128 fx32(double c) { return (u128)(uint64_t)floor(fabs(c) * 4294967296.0); }

/* Walker's alias method, Vose's construction in a fixed order:
 * q_k = (|H_k| / S) * K; indices with q < 1 go on the stack "small", the rest
 * on "large" (both filled by ascending k, popped from the top); while both are
 * non-empty: s = pop(small), l = pop(large), prob[s] = q_s, alias[s] = l,
 * q_l = (q_l + q_s) - 1, and l is pushed on small if q_l < 1, else on large;
 * whatever remains gets prob = 1 (alias = itself). */
static void alias_build(int K, const double *absv, double S, double *prob, int *alias)
{
    double *q = malloc(sizeof(double) * K);
    int *sm = malloc(sizeof(int) * K), *lg = malloc(sizeof(int) * K);
    int ns = 0, nl = 0;
    for (int k = 0; k < K; k++) {
        q[k] = (absv[k] / S) * (double)K;
        if (q[k] < 1.0) sm[ns++] = k; else lg[nl++] = k;
        alias[k] = k;
        prob[k] = 1.0;
    }
    while (ns > 0 && nl > 0) {
        int a = sm[--ns], l = lg[--nl];
        prob[a] = q[a];
        alias[a] = l;
        q[l] = (q[l] + q[a]) - 1.0;
        if (q[l] < 1.0) sm[ns++] = l; else lg[nl++] = l;
    }
    free(q); free(sm); free(lg);
}

static void pchb_fill(opchb *t, int K, const int *ea, const int *eb, const double *val, double tau, double ppair)
{
    xacc x;
    xacc_zero(&x);
    double *absv = malloc(sizeof(double) * (K ? K : 1));
    for (int k = 0; k < K; k++) { absv[k] = fabs(val[k]); xacc_add(&x, absv[k], 0); }
    t->K = K;
    t->S = xacc_round(&x);
    t->lam = (tau * t->S) / ppair;
    t->prob = malloc(sizeof(double) * (K ? K : 1));
    t->alias = malloc(sizeof(int) * (K ? K : 1));
    t->ea = malloc(sizeof(int) * (K ? K : 1));
    t->eb = malloc(sizeof(int) * (K ? K : 1));
    t->val = malloc(sizeof(double) * (K ? K : 1));
    memcpy(t->ea, ea, sizeof(int) * K);
    memcpy(t->eb, eb, sizeof(int) * K);
    memcpy(t->val, val, sizeof(double) * K);
    if (t->S > 0.0) alias_build(K, absv, t->S, t->prob, t->alias);
    free(absv);
}

static void pchb_build(orc_run *r)
{
    const orc_sys *s = r->s;
    const int N = s->norb, n = s->na + s->nb;
    const double ppair = ((1.0 - r->p.p_single) * 2.0) / ((double)n * (double)(n - 1));
    r->pchb_ab = calloc((size_t)N * N, sizeof(opchb));
    r->pchb_ss = calloc((size_t)N * N, sizeof(opchb));
    r->pchb_n = N;
    int *ea = malloc(sizeof(int) * N * N), *eb = malloc(sizeof(int) * N * N);
    double *val = malloc(sizeof(double) * N * N);
    for (int i = 0; i < N; i++)
        for (int j = 0; j < N; j++) {
            int K = 0;
            for (int a = 0; a < N; a++)
                for (int b = 0; b < N; b++) {
                    ea[K] = a; eb[K] = b;
                    val[K] = (a == i || b == j) ? 0.0 : eri(s, a, i, b, j);
                    K++;
                }
            pchb_fill(&r->pchb_ab[i * N + j], K, ea, eb, val, r->p.tau, ppair);
            if (i < j) {
                K = 0;
                for (int b = 1; b < N; b++)
                    for (int a = 0; a < b; a++) {
                        ea[K] = a; eb[K] = b;
                        val[K] = (a == i || a == j || b == i || b == j) ? 0.0
                                                                         : eri(s, a, i, b, j) - eri(s, a, j, b, i);
                        K++;
                    }
                pchb_fill(&r->pchb_ss[i * N + j], K, ea, eb, val, r->p.tau, ppair);
            }
        }
    free(ea); free(eb); free(val);
}

static void pchb_free(orc_run *r)
{
    if (!r->pchb_ab) return;
    int N = r->pchb_n;
    for (int k = 0; k < 2 * N * N; k++) {
        opchb *t = k < N * N ? &r->pchb_ab[k] : &r->pchb_ss[k - N * N];
        free(t->prob); free(t->alias); free(t->ea); free(t->eb); free(t->val);
    }
    free(r->pchb_ab); free(r->pchb_ss);
}

/* One heat-bath double from D with the words of its draw (w0 has already
 * chosen a double): ordered electron pair from w1 as in the uniform generator;
 * bin k = floor(w2 K / 2^64), coin u = ((w2 K mod 2^64) >> 11) 2^-53, entry k
 * if u < prob[k], else alias[k]; failed if the table is empty (S = 0) or a hole
 * is occupied.  Returns the class and, through *lam and *hval, |H|/p_gen and the
 * entry's matrix element. */
static int pchb_double(const orc_run *r, uint64_t a, uint64_t b, const uint64_t w[4], uint64_t *ta, uint64_t *tb,
                       double *lam, double *hval)
{
    const orc_sys *s = r->s;
    int N = s->norb, n = s->na + s->nb;
    *ta = a; *tb = b;
    if (n < 2) return -1;
    uint64_t xe = pick(w[1], (uint64_t)n * (uint64_t)(n - 1));
    int e1 = (int)(xe / (uint64_t)(n - 1)), rr = (int)(xe % (uint64_t)(n - 1));
    int e2 = rr + (rr >= e1 ? 1 : 0);
    int s1, s2;
    int o1 = electron_orb(a, b, s->na, e1, &s1), o2 = electron_orb(a, b, s->na, e2, &s2);
    const opchb *t;
    int cls;
    if (s1 != s2) {
        int oa = s1 == 0 ? o1 : o2, ob = s1 == 0 ? o2 : o1;
        t = &r->pchb_ab[oa * N + ob];
        cls = CLS_DOUBLE_AB;
    } else {
        int lo = o1 < o2 ? o1 : o2, hi = o1 < o2 ? o2 : o1;
        t = &r->pchb_ss[lo * N + hi];
        cls = s1 ? CLS_DOUBLE_BB : CLS_DOUBLE_AA;
    }
    if (!(t->S > 0.0)) return -1;
    u128 prod = (u128)w[2] * (uint64_t)t->K;
    int k = (int)(prod >> 64);
    double u = u53((uint64_t)prod);
    if (!(u < t->prob[k])) k = t->alias[k];
    int ha = t->ea[k], hb = t->eb[k];
    if (s1 != s2) {
        int oa = s1 == 0 ? o1 : o2, ob = s1 == 0 ? o2 : o1;
        if (((a >> ha) & 1) || ((b >> hb) & 1)) return -1;
        *ta = a ^ (1ULL << oa) ^ (1ULL << ha);
        *tb = b ^ (1ULL << ob) ^ (1ULL << hb);
    } else {
        uint64_t *x = s1 ? tb : ta;
        uint64_t occ = s1 ? b : a;
        if (((occ >> ha) & 1) || ((occ >> hb) & 1)) return -1;
        *x ^= (1ULL << o1) | (1ULL << o2) | (1ULL << ha) | (1ULL << hb);
    }
    *lam = t->lam;
    *hval = t->val[k];
    return cls;
}

/* heat-bath generation for the tests: class, target, |H|/p_gen */
int orc_generate_pchb(const orc_run *r, uint64_t a, uint64_t b, const uint64_t w[4], uint64_t *ta, uint64_t *tb,
                      double *lam)
{
    double hv;
    if (u53(w[0]) < r->p.p_single) {
        int c = orc_generate(r->s, r->p.p_single, a, b, w, ta, tb);
        *lam = c >= 0 ? r->lam[c] : 0.0;
        return c;
    }
    return pchb_double(r, a, b, w, ta, tb, lam, &hv);
}

/* the table of pair (i, j): K, S, lam and (prob, alias, a, b, value) of each entry */
int orc_pchb_table(const orc_run *r, int same_spin, int i, int j, double *S, double *lam, double *prob, int32_t *alias,
                   int32_t *ea, int32_t *eb, double *val)
{
    int N = r->s->norb;
    const opchb *t = same_spin ? &r->pchb_ss[i * N + j] : &r->pchb_ab[i * N + j];
    if (S) *S = t->S;
    if (lam) *lam = t->lam;
    for (int k = 0; k < t->K; k++) {
        if (prob) prob[k] = t->prob[k];
        if (alias) alias[k] = t->alias[k];
        if (ea) ea[k] = t->ea[k];
        if (eb) eb[k] = t->eb[k];
        if (val) val[k] = t->val[k];
    }
    return t->K;
}

orc_run *orc_create(orc_sys *s, const orc_params *p)
{
    orc_run *r = calloc(1, sizeof *r);
    r->s = s;
    r->p = *p;
    for (int c = 0; c < NCLS; c++) r->lam[c] = p->tau / orc_pgen(s, p->p_single, c);
    r->cap = 1024;
    r->L = malloc(sizeof(odet) * r->cap);
    r->n = 1;
    r->L[0].a = s->ref_a; r->L[0].b = s->ref_b; r->L[0].c = p->initial_walkers;
    r->L[0].hd = 0.0; r->L[0].flags = 1;
    r->S = p->initial_shift;
    if (p->generator == 1 && s->kind == 0) pchb_build(r);
    r->stcap = 1024;
    r->st = malloc(sizeof(orc_stat) * r->stcap);
    return r;
}

void orc_destroy(orc_run *r)
{
    if (!r) return;
    free(r->L); free(r->Da); free(r->Db); free(r->rowptr); free(r->col); free(r->val); free(r->st);
    free(r->Ta); free(r->Tb); free(r->cT); free(r->Wa); free(r->Wb); free(r->W);
    free(r->L0); free(r->sp0); free(r->f0);
    pchb_free(r);
    free(r);
}

/* top-N_D determinants by |C| (ties: ascending key), then H^D in CSR (Sec. III) */
typedef struct { double m; uint64_t a, b; } ocand;
static int cmp_cand(const void *x, const void *y)
{
    const ocand *p = x, *q = y;
    if (p->m != q->m) return p->m > q->m ? -1 : 1;
    return cmp_key(p->a, p->b, q->a, q->b);
}
static void build_D(orc_run *r)
{
    int64_t n = r->n, nd = r->p.semistoch_size < n ? r->p.semistoch_size : n;
    ocand *cd = malloc(sizeof(ocand) * (n ? n : 1));
    for (int64_t i = 0; i < n; i++) { cd[i].m = fabs(r->L[i].c); cd[i].a = r->L[i].a; cd[i].b = r->L[i].b; }
    qsort(cd, n, sizeof(ocand), cmp_cand);
    odet *tmp = malloc(sizeof(odet) * (nd ? nd : 1));
    for (int64_t i = 0; i < nd; i++) { tmp[i].a = cd[i].a; tmp[i].b = cd[i].b; }
    qsort(tmp, nd, sizeof(odet), cmp_odet);
    r->nd = nd;
    r->Da = malloc(sizeof(uint64_t) * (nd ? nd : 1));
    r->Db = malloc(sizeof(uint64_t) * (nd ? nd : 1));
    for (int64_t i = 0; i < nd; i++) { r->Da[i] = tmp[i].a; r->Db[i] = tmp[i].b; }
    r->rowptr = malloc(sizeof(int64_t) * (nd + 1));
    int64_t cap = 16, nnz = 0;
    r->col = malloc(sizeof(int64_t) * cap);
    r->val = malloc(sizeof(double) * cap);
    r->rowptr[0] = 0;
    for (int64_t i = 0; i < nd; i++) {
        for (int64_t j = 0; j < nd; j++) {
            double v;
            if (i == j) v = orc_hdiag_rel(r->s, r->Da[i], r->Db[i]);
            else {
                int lev = popc(r->Da[i] ^ r->Da[j]) + popc(r->Db[i] ^ r->Db[j]);
                if (lev > 4) continue;
                v = orc_hoff(r->s, r->Da[j], r->Db[j], r->Da[i], r->Db[i]); /* <D_i|H|D_j> */
                if (v == 0.0) continue;
            }
            if (nnz == cap) {
                cap *= 2;
                r->col = realloc(r->col, sizeof(int64_t) * cap);
                r->val = realloc(r->val, sizeof(double) * cap);
            }
            r->col[nnz] = j; r->val[nnz] = v; nnz++;
        }
        r->rowptr[i + 1] = nnz;
    }
    for (int64_t i = 0; i < n; i++)
        if (find_D(r, r->L[i].a, r->L[i].b) >= 0) r->L[i].flags |= 2;
    free(cd); free(tmp);
}

/* CSR of H^D - E_ref (rows and columns in ascending key order of D); any
 * output pointer may be NULL */
void orc_semistoch_csr(const orc_run *r, int64_t *rowptr, int64_t *col, double *val, uint64_t *da, uint64_t *db)
{
    for (int64_t k = 0; k < r->nd; k++) {
        if (da) da[k] = r->Da[k];
        if (db) db[k] = r->Db[k];
    }
    if (rowptr) for (int64_t k = 0; k <= r->nd; k++) rowptr[k] = r->rowptr[k];
    int64_t nnz = r->nd ? r->rowptr[r->nd] : 0;
    for (int64_t q = 0; q < nnz; q++) {
        if (col) col[q] = r->col[q];
        if (val) val[q] = r->val[q];
    }
}

static double semi_row_sum(const orc_run *r, const double *cD, int64_t k);

/* y_k of every row for the amplitudes cD (the row sum of the semi-stochastic update) */
void orc_semistoch_rows(const orc_run *r, const double *cD, double *y)
{
    for (int64_t k = 0; k < r->nd; k++) y[k] = semi_row_sum(r, cD, k);
}

int64_t orc_semistoch_info(const orc_run *r, int64_t *nnz)
{
    if (nnz) *nnz = r->nd ? r->rowptr[r->nd] : 0;
    return r->nd;
}

/* ---------------------------------------------------------------- trial wave function
 * E_Trial (Sec. IV): T = the trial_size largest |C| (ties: ascending key) at
 * iteration shift_start + trial_start; Psi^T = the lowest eigenvector of H^T
 * (H projected into T); E_Trial = <Psi^T|H|Psi> / <Psi^T|Psi>, accumulated as
 * the numerator and denominator of every iteration.  W_j = <Psi^T|H - E_ref|D_j>
 * for every D_j in T and in the space C of determinants connected to T. */

/* lowest eigenpair of the symmetric n x n matrix A (row-major, destroyed) by
 * cyclic Jacobi rotations (Jacobi 1846; rotation angle from
 * theta = (A_qq - A_pp) / (2 A_pq), t = sign(theta) / (|theta| + sqrt(theta^2 + 1))),
 * sweeping until the off-diagonal part is below 1e-15 of the matrix norm */
static void jacobi_lowest(int n, double *A, double *E, double *v)
{
    double *V = calloc((size_t)n * n, sizeof(double));
    for (int i = 0; i < n; i++) V[(size_t)i * n + i] = 1.0;
    double norm = 0.0;
    for (size_t k = 0; k < (size_t)n * n; k++) norm += A[k] * A[k];
    for (int sweep = 0; sweep < 100; sweep++) {
        double off = 0.0;
        for (int p = 0; p < n; p++)
            for (int q = p + 1; q < n; q++) off += A[(size_t)p * n + q] * A[(size_t)p * n + q];
        if (!(off > 1e-30 * norm)) break;
        for (int p = 0; p < n; p++)
            for (int q = p + 1; q < n; q++) {
                double apq = A[(size_t)p * n + q];
                if (apq == 0.0) continue;
                double theta = (A[(size_t)q * n + q] - A[(size_t)p * n + p]) / (2.0 * apq);
                double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                double c = 1.0 / sqrt(t * t + 1.0), sn = t * c;
                /* A <- J^T A J with J the rotation in the (p, q) plane */
                for (int k = 0; k < n; k++) {
                    double akp = A[(size_t)k * n + p], akq = A[(size_t)k * n + q];
                    A[(size_t)k * n + p] = c * akp - sn * akq;
                    A[(size_t)k * n + q] = sn * akp + c * akq;
                }
                for (int k = 0; k < n; k++) {
                    double apk = A[(size_t)p * n + k], aqk = A[(size_t)q * n + k];
                    A[(size_t)p * n + k] = c * apk - sn * aqk;
                    A[(size_t)q * n + k] = sn * apk + c * aqk;
                }
                for (int k = 0; k < n; k++) {
                    double vkp = V[(size_t)k * n + p], vkq = V[(size_t)k * n + q];
                    V[(size_t)k * n + p] = c * vkp - sn * vkq;
                    V[(size_t)k * n + q] = sn * vkp + c * vkq;
                }
            }
    }
    int lo = 0;
    for (int i = 1; i < n; i++) if (A[(size_t)i * n + i] < A[(size_t)lo * n + lo]) lo = i;
    *E = A[(size_t)lo * n + lo];
    for (int i = 0; i < n; i++) v[i] = V[(size_t)i * n + lo];
    free(V);
}

int orc_jacobi_lowest(int n, double *A, double *E, double *v) { jacobi_lowest(n, A, E, v); return 0; }

typedef struct { uint64_t a, b; double v; } ocontrib;
static int cmp_contrib(const void *x, const void *y)
{
    const ocontrib *p = x, *q = y;
    return cmp_key(p->a, p->b, q->a, q->b);
}

/* every determinant connected to (a, b) by one application of H: singles of
 * either spin, opposite-spin and same-spin doubles (target list, no values) */
static int64_t connections(const orc_sys *s, uint64_t a, uint64_t b, uint64_t *ta, uint64_t *tb)
{
    const int N = s->norb;
    const uint64_t full = N >= 64 ? ~0ULL : ((1ULL << N) - 1);
    int64_t k = 0;
    for (int sp = 0; sp < 2; sp++) {
        uint64_t w = sp ? b : a, v = ~w & full;
        for (int i = 0; i < N; i++) {
            if (!(w >> i & 1)) continue;
            for (int x = 0; x < N; x++) {
                if (!(v >> x & 1)) continue;
                uint64_t y = w ^ (1ULL << i) ^ (1ULL << x);
                ta[k] = sp ? a : y; tb[k] = sp ? y : b; k++;
            }
        }
    }
    uint64_t va = ~a & full, vb = ~b & full;
    for (int i = 0; i < N; i++) {
        if (!(a >> i & 1)) continue;
        for (int j = 0; j < N; j++) {
            if (!(b >> j & 1)) continue;
            for (int x = 0; x < N; x++) {
                if (!(va >> x & 1)) continue;
                for (int y = 0; y < N; y++) {
                    if (!(vb >> y & 1)) continue;
                    ta[k] = a ^ (1ULL << i) ^ (1ULL << x); tb[k] = b ^ (1ULL << j) ^ (1ULL << y); k++;
                }
            }
        }
    }
    for (int sp = 0; sp < 2; sp++) {
        uint64_t w = sp ? b : a, v = ~w & full;
        for (int i = 0; i < N; i++)
            for (int j = i + 1; j < N; j++) {
                if (!(w >> i & 1) || !(w >> j & 1)) continue;
                for (int x = 0; x < N; x++)
                    for (int y = x + 1; y < N; y++) {
                        if (!(v >> x & 1) || !(v >> y & 1)) continue;
                        uint64_t z = w ^ (1ULL << i) ^ (1ULL << j) ^ (1ULL << x) ^ (1ULL << y);
                        ta[k] = sp ? a : z; tb[k] = sp ? z : b; k++;
                    }
            }
    }
    return k;
}

static void build_T(orc_run *r)
{
    const orc_sys *s = r->s;
    int64_t n = r->n, nt = r->p.trial_size < n ? r->p.trial_size : n;
    ocand *cd = malloc(sizeof(ocand) * (n ? n : 1));
    for (int64_t i = 0; i < n; i++) { cd[i].m = fabs(r->L[i].c); cd[i].a = r->L[i].a; cd[i].b = r->L[i].b; }
    qsort(cd, n, sizeof(ocand), cmp_cand);
    odet *tmp = malloc(sizeof(odet) * (nt ? nt : 1));
    for (int64_t i = 0; i < nt; i++) { tmp[i].a = cd[i].a; tmp[i].b = cd[i].b; }
    qsort(tmp, nt, sizeof(odet), cmp_odet);
    r->nt = nt;
    r->Ta = malloc(sizeof(uint64_t) * (nt ? nt : 1));
    r->Tb = malloc(sizeof(uint64_t) * (nt ? nt : 1));
    for (int64_t i = 0; i < nt; i++) { r->Ta[i] = tmp[i].a; r->Tb[i] = tmp[i].b; }
    free(cd); free(tmp);
    /* H^T relative to E_ref, its lowest eigenvector */
    double *A = malloc(sizeof(double) * (size_t)(nt ? nt * nt : 1));
    for (int64_t i = 0; i < nt; i++)
        for (int64_t j = 0; j < nt; j++)
            A[i * nt + j] = i == j ? orc_hdiag_rel(s, r->Ta[i], r->Tb[i])
                                   : orc_hoff(s, r->Ta[j], r->Tb[j], r->Ta[i], r->Tb[i]);
    r->cT = malloc(sizeof(double) * (nt ? nt : 1));
    jacobi_lowest((int)nt, A, &r->ET, r->cT);
    free(A);
    /* W over T and C: contributions <D_j|H - E_ref|D_i> cT_i, summed exactly per j */
    int64_t cap = 1024, nc = 0;
    ocontrib *ct = malloc(sizeof(ocontrib) * cap);
    const int N = s->norb;
    int64_t maxc = (int64_t)N * N * 2 + (int64_t)N * N * N * N * 2 + 16;
    uint64_t *ta = malloc(sizeof(uint64_t) * maxc), *tb = malloc(sizeof(uint64_t) * maxc);
    for (int64_t i = 0; i < nt; i++) {
        int64_t k = connections(s, r->Ta[i], r->Tb[i], ta, tb);
        if (nc + k + 1 > cap) { while (nc + k + 1 > cap) cap *= 2; ct = realloc(ct, sizeof(ocontrib) * cap); }
        ct[nc].a = r->Ta[i]; ct[nc].b = r->Tb[i]; ct[nc].v = orc_hdiag_rel(s, r->Ta[i], r->Tb[i]) * r->cT[i]; nc++;
        for (int64_t q = 0; q < k; q++) {
            double h = orc_hoff(s, r->Ta[i], r->Tb[i], ta[q], tb[q]);
            if (h == 0.0) continue;
            ct[nc].a = ta[q]; ct[nc].b = tb[q]; ct[nc].v = h * r->cT[i]; nc++;
        }
    }
    free(ta); free(tb);
    qsort(ct, nc, sizeof(ocontrib), cmp_contrib);
    r->Wa = malloc(sizeof(uint64_t) * (nc ? nc : 1));
    r->Wb = malloc(sizeof(uint64_t) * (nc ? nc : 1));
    r->W = malloc(sizeof(double) * (nc ? nc : 1));
    int64_t nw = 0;
    for (int64_t q = 0; q < nc;) {
        xacc x;
        xacc_zero(&x);
        int64_t q1 = q;
        while (q1 < nc && ct[q1].a == ct[q].a && ct[q1].b == ct[q].b) { xacc_add(&x, ct[q1].v, 0); q1++; }
        r->Wa[nw] = ct[q].a; r->Wb[nw] = ct[q].b; r->W[nw] = xacc_round(&x); nw++;
        q = q1;
    }
    r->nwt = nw;
    free(ct);
}

static int64_t find_key(const uint64_t *ka, const uint64_t *kb, int64_t n, uint64_t a, uint64_t b)
{
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t mid = (lo + hi) / 2;
        int c = cmp_key(ka[mid], kb[mid], a, b);
        if (c == 0) return mid;
        if (c < 0) lo = mid + 1; else hi = mid;
    }
    return -1;
}

/* trial space: N_T, |T u C|, E^T (relative to E_ref); cT and keys when the arrays are given */
int64_t orc_trial_info(const orc_run *r, int64_t *nw, double *ET, uint64_t *ta, uint64_t *tb, double *cT)
{
    if (nw) *nw = r->nwt;
    if (ET) *ET = r->ET;
    for (int64_t i = 0; i < r->nt; i++) {
        if (ta) ta[i] = r->Ta[i];
        if (tb) tb[i] = r->Tb[i];
        if (cT) cT[i] = r->cT[i];
    }
    return r->nt;
}

static double round_stoch(double v, double cmin, double u)
{
    /* Eq. (3): keep |v| >= C_min; else sign(v) C_min with prob |v|/C_min, else 0 */
    if (v == 0.0 || fabs(v) >= cmin) return v;
    return u < fabs(v) / cmin ? copysign(cmin, v) : 0.0;
}

/* Semi-stochastic row sum (reading R13): y_k = sum_c H^D_kc C_c, where each
 * product is rounded to binary64, then truncated toward zero to a multiple
 * of 2^-64, and the truncated products are summed exactly and rounded once;
 * the new amplitude is C_k - tau (y_k - S C_k), evaluated as written. */
static double trunc_grid64(double p)
{
    /* p 2^64 and its integer part are exact; the result has at most 53
     * significant bits and is 0 or at least 2^-64 in magnitude, so scaling
     * back is exact too */
    return ldexp(trunc(ldexp(p, 64)), -64);
}

static double semi_row_sum(const orc_run *r, const double *cD, int64_t k)
{
    xacc x;
    xacc_zero(&x);
    for (int64_t q = r->rowptr[k]; q < r->rowptr[k + 1]; q++) xacc_add(&x, trunc_grid64(r->val[q] * cD[r->col[q]]), 0);
    return xacc_round(&x);
}

static double semi_update(const orc_run *r, const double *cD, int64_t k)
{
    double y = semi_row_sum(r, cD, k);
    return cD[k] - r->p.tau * (y - r->S * cD[k]);
}

/* one projector iteration; returns 0 or a nonzero error code */
static int one_iteration(orc_run *r)
{
    const orc_sys *s = r->s;
    const orc_params *P = &r->p;
    int64_t it = r->iter;
    double cmin = P->c_min;

    if (P->semistoch_size > 0 && r->nd == 0 && r->vary && it == r->shift_start + P->semistoch_start)
        build_D(r);
    if (P->trial_size > 0 && r->nt == 0 && r->vary && it == r->shift_start + P->trial_start)
        build_T(r);

    if (r->keep_last) {
        free(r->L0);
        r->L0 = malloc(sizeof(odet) * (r->n ? r->n : 1));
        memcpy(r->L0, r->L, sizeof(odet) * r->n);
        r->n0 = r->n;
    }

    /* (a) spawning from the start-of-iteration amplitudes.  Adaptive shift:
     * for a non-initiator D_i, every spawn that survives Eq. (3) adds
     * w_ij = |H_ji| / |H_jj - E_ref - S| (S: the shift at the start of the
     * iteration, the energy estimate of the run), truncated to the grid 2^-64
     * and summed exactly, to T_i, and to A_i as well if the spawn is accepted
     * (its target is occupied at the start of the iteration, the initiator
     * rule); f_i = A_i / T_i (1 without such spawns) scales the shift in the
     * death of D_i. */
    int64_t ns = 0, scap = 1024, attempts = 0;
    ospawn *sp = malloc(sizeof(ospawn) * scap);
    double *fi = malloc(sizeof(double) * (r->n ? r->n : 1));
    int *initf = malloc(sizeof(int) * (r->n ? r->n : 1));
    for (int64_t i = 0; i < r->n; i++) { fi[i] = 1.0; initf[i] = 1; }
    for (int64_t i = 0; i < r->n; i++) {
        odet *d = &r->L[i];
        if (d->c == 0.0) continue;
        double mag = fabs(d->c);
        if (mag >= 0x1p40) { free(sp); free(fi); free(initf); return 3; }
        uint64_t nat = (uint64_t)ceil(mag);
        attempts += (int64_t)nat;
        int init = mag > P->initiator_threshold || (d->flags & 3);
        initf[i] = init;
        u128 accA = 0, accT = 0;
        double cper = d->c / (double)nat;
        for (uint64_t k = 0; k < nat; k++) {
            uint64_t w[4], ta, tb;
            draw(P->seed, (uint64_t)P->replica, d->a, d->b, it, k, PURPOSE_SPAWN, w);
            double ws;
            if (r->pchb_ab && !(u53(w[0]) < P->p_single)) {
                /* heat-bath double: |H| / p_gen = lam for every entry, so the
                 * weight is -(sign(H) * (lam * C_i / n_att)) */
                double lam, hv;
                int cls = pchb_double(r, d->a, d->b, w, &ta, &tb, &lam, &hv);
                if (cls < 0) continue;
                double H = orc_hoff(s, d->a, d->b, ta, tb);
                if (H == 0.0) continue;
                double wv = lam * cper;
                ws = H > 0.0 ? -wv : wv;
            } else {
                int cls = orc_generate(s, P->p_single, d->a, d->b, w, &ta, &tb);
                if (cls < 0) continue;
                double H = orc_hoff(s, d->a, d->b, ta, tb);
                if (H == 0.0) continue;
                ws = -(H * (r->lam[cls] * cper));
            }
            if (fabs(ws) < cmin) {
                ws = round_stoch(ws, cmin, u53(w[3]));
                if (ws == 0.0) continue;
            }
            if ((d->flags & 2) && find_D(r, ta, tb) >= 0) continue; /* D -> D is exact */
            if (P->adaptive_shift && !init) {
                int64_t j = find_det(r->L, r->n, ta, tb);
                int occ = j >= 0 && r->L[j].c != 0.0;
                double hdj = j >= 0 ? r->L[j].hd : orc_hdiag_rel(s, ta, tb);
                double den = fabs(hdj - r->S);
                if (den != 0.0) {
                    double wij = fabs(orc_hoff(s, d->a, d->b, ta, tb)) / den;
                    u128 q = (u128)(wij * 0x1p64); /* floor: w >= 0, exact scaling */
                    accT += q;
                    if (occ) accA += q;
                }
            }
            if (ns == scap) { scap *= 2; sp = realloc(sp, sizeof(ospawn) * scap); }
            sp[ns].a = ta; sp[ns].b = tb; sp[ns].w = ws; sp[ns].init = init; sp[ns].parent = i; ns++;
        }
        if (P->adaptive_shift && !init && accT != 0) fi[i] = (double)accA / (double)accT;
    }
    if (r->keep_last) {
        free(r->f0);
        r->f0 = malloc(sizeof(double) * (r->n ? r->n : 1));
        memcpy(r->f0, fi, sizeof(double) * r->n);
    }

    /* (b) death, in place; deterministic space: exact projection (Sec. III) */
    double *c0 = malloc(sizeof(double) * (r->n ? r->n : 1));
    for (int64_t i = 0; i < r->n; i++) c0[i] = r->L[i].c;
    double *cd_new = NULL;
    if (r->nd) {
        double *cD = malloc(sizeof(double) * r->nd);
        for (int64_t k = 0; k < r->nd; k++) {
            int64_t i = find_det(r->L, r->n, r->Da[k], r->Db[k]);
            cD[k] = i >= 0 ? c0[i] : 0.0;
        }
        cd_new = malloc(sizeof(double) * r->nd);
        for (int64_t k = 0; k < r->nd; k++) cd_new[k] = semi_update(r, cD, k);
        free(cD);
    }
    for (int64_t i = 0; i < r->n; i++) {
        odet *d = &r->L[i];
        if (d->flags & 2) { d->c = cd_new[find_D(r, d->a, d->b)]; continue; }
        double Si = (P->adaptive_shift && !initf[i]) ? fi[i] * r->S : r->S;
        double f = 1.0 - P->tau * (d->hd - Si);
        double cp = d->c * f;
        if (cp != 0.0 && fabs(cp) < cmin) {
            uint64_t w[4];
            draw(P->seed, (uint64_t)P->replica, d->a, d->b, it, 0, PURPOSE_DEATH, w);
            cp = round_stoch(cp, cmin, u53(w[0]));
        }
        d->c = cp;
    }
    free(cd_new);
    free(fi); free(initf);

    /* (c) annihilation with the initiator rule */
    qsort(sp, ns, sizeof(ospawn), cmp_ospawn);
    if (r->keep_last) {
        free(r->sp0);
        r->sp0 = malloc(sizeof(ospawn) * (ns ? ns : 1));
        memcpy(r->sp0, sp, sizeof(ospawn) * ns);
        r->ns0 = ns;
    }
    int64_t outcap = r->n + ns + 1, no = 0, rejected = 0;
    odet *out = malloc(sizeof(odet) * outcap);
    i128 ann = 0;
    int64_t li = 0, si = 0;
    while (li < r->n || si < ns) {
        int c;
        if (li >= r->n) c = 1;
        else if (si >= ns) c = -1;
        else c = cmp_key(r->L[li].a, r->L[li].b, sp[si].a, sp[si].b);
        odet d;
        double cstart = 0.0;
        int present = 0;
        if (c <= 0) { d = r->L[li]; cstart = c0[li]; present = 1; li++; }
        else { d.a = sp[si].a; d.b = sp[si].b; d.c = 0.0; d.hd = 0.0; d.flags = 0; }
        double acc = d.c;
        if (c >= 0) {
            int occ = present && cstart != 0.0;
            xacc x;
            xacc_zero(&x);
            int64_t nacc = 0;
            i128 in = present ? (i128)fx32(d.c) : 0;
            uint64_t ka = d.a, kb = d.b;
            while (si < ns && sp[si].a == ka && sp[si].b == kb) {
                if (sp[si].init || occ) { xacc_add(&x, sp[si].w, 0); in += (i128)fx32(sp[si].w); nacc++; }
                else rejected++;
                si++;
            }
            if (nacc > 0) {
                double sw = xacc_round(&x);
                acc = present ? d.c + sw : sw;
                ann += in - (i128)fx32(acc);
                if (!(d.flags & 2) && acc != 0.0 && fabs(acc) < cmin) {
                    uint64_t w[4];
                    draw(P->seed, (uint64_t)P->replica, d.a, d.b, it, 0, PURPOSE_ANNIH, w);
                    acc = round_stoch(acc, cmin, u53(w[0]));
                }
            }
        }
        d.c = acc;
        if (acc == 0.0 && !(d.flags & 3)) continue;
        if (!present) d.hd = orc_hdiag_rel(s, d.a, d.b);
        out[no++] = d;
    }
    free(sp); free(c0); free(r->L);
    r->L = out; r->n = no; r->cap = outcap;

    /* reductions: N_w (R6), E_num (R12) / E_den (Eq. (9)) */
    u128 W = 0;
    double e_den = 0.0;
    xacc xe;
    xacc_zero(&xe);
    for (int64_t i = 0; i < no; i++) {
        odet *d = &out[i];
        if (fabs(d->c) >= 0x1p31) return 3;
        W += fx32(d->c);
        if (d->flags & 1) { e_den = d->c; continue; }
        int lev = popc(d->a ^ s->ref_a) + popc(d->b ^ s->ref_b);
        if (lev <= 4 && d->c != 0.0)
            xacc_add(&xe, trunc_grid(orc_hoff(s, d->a, d->b, s->ref_a, s->ref_b) * d->c, s->Fe), 0);
    }
    double e_num = xacc_round(&xe);
    double nw = (double)W * 0x1p-32;
    if (!(nw == nw)) return 3;
    /* E_Trial numerator and denominator, in ascending key order */
    double t_num = 0.0, t_den = 0.0;
    if (r->nt > 0)
        for (int64_t i = 0; i < no; i++) {
            if (out[i].c == 0.0) continue;
            int64_t q = find_key(r->Wa, r->Wb, r->nwt, out[i].a, out[i].b);
            if (q >= 0) t_num = t_num + r->W[q] * out[i].c;
            q = find_key(r->Ta, r->Tb, r->nt, out[i].a, out[i].b);
            if (q >= 0) t_den = t_den + r->cT[q] * out[i].c;
        }

    /* shift (reading R7) */
    if (!r->vary) {
        if (nw >= P->target_walkers) { r->vary = 1; r->shift_start = it; r->nw_last = W; r->cnt = 0; }
    } else if (++r->cnt == P->shift_interval) {
        double ratio = nw / ((double)r->nw_last * 0x1p-32);
        double cz = P->shift_damping / ((double)P->shift_interval * P->tau);
        r->S = r->S - cz * orc_ln(ratio);
        r->nw_last = W;
        r->cnt = 0;
    }

    if (r->nst == r->stcap) { r->stcap *= 2; r->st = realloc(r->st, sizeof(orc_stat) * r->stcap); }
    orc_stat *t = &r->st[r->nst++];
    t->iter = it; t->nw = nw; t->S = r->S; t->e_num = e_num; t->e_den = e_den;
    t->ndet = no; t->attempts = attempts; t->spawns = ns; t->rejected = rejected;
    t->annihilated = (double)ann * 0x1p-32; t->vary = r->vary;
    t->t_num = t_num; t->t_den = t_den;
    t->x_overlap = 0.0; t->x_var_num = 0.0; t->x_pt2 = 0.0; /* filled by a replica pair */
    r->iter = it + 1;
    return 0;
}

int orc_step(orc_run *r, int64_t n)
{
    for (int64_t k = 0; k < n; k++) {
        int e = one_iteration(r);
        if (e) { r->err = e; return e; }
    }
    return 0;
}

/* ---------------------------------------------------------------- replicas
 * Two runs of the same system with replica indices 0 and 1 advance together
 * (Sec. V: two independent walker distributions).  After every iteration the
 * first run's row receives, over every determinant j in either start list or
 * spawned onto in either run (C^r_j: amplitude at the start of the iteration;
 * S^r_j = RN(accepted spawns onto j) + RN(rejected spawns onto j), each an
 * exact sum rounded once; R^r_j = RN(rejected spawns onto j), the spawns
 * removed by the initiator rule):
 *   x_overlap = sum_j C^1_j C^2_j                                  <Psi^1|Psi^2>
 *   x_var_num = sum_j (C^1_j (H_jj - E_ref)) C^2_j - (sum_j (C^1_j S^2_j + C^2_j S^1_j)) / (2 tau)
 *               (an unbiased estimate of <Psi^1|H - E_ref|Psi^2>: a spawn
 *               from D_i onto D_j has expectation -tau H_ji C_i)
 *   x_pt2     = (sum over j with R^1_j != 0 and R^2_j != 0 of
 *               (R^1_j R^2_j) / (E_0 - (H_jj - E_ref))) / tau^2      (Sec. VI, Eq. of Delta E_2)
 * with E_0 = (S^1 + S^2) / 2, the replicas' shifts at the start of the
 * iteration (relative to E_ref); a term with E_0 = H_jj - E_ref (possible
 * before the shift has moved, e.g. lattice models with integer diagonals) is
 * undefined and left out; sums in ascending key order. */
typedef struct { uint64_t a, b; double c0, hd, sacc, srej; int has_hd; } oside;

static int cmp_oside(const void *x, const void *y)
{
    const oside *p = x, *q = y;
    return cmp_key(p->a, p->b, q->a, q->b);
}

/* per determinant of one run's last iteration: C at start, H_jj - E_ref if it
 * was occupied, accepted and rejected spawn sums (sorted by key) */
static int64_t side_list(const orc_run *r, oside **out)
{
    int64_t cap = r->n0 + r->ns0 + 1, n = 0;
    oside *v = malloc(sizeof(oside) * cap);
    int64_t li = 0, si = 0;
    while (li < r->n0 || si < r->ns0) {
        int c;
        if (li >= r->n0) c = 1;
        else if (si >= r->ns0) c = -1;
        else c = cmp_key(r->L0[li].a, r->L0[li].b, r->sp0[si].a, r->sp0[si].b);
        oside e;
        memset(&e, 0, sizeof e);
        int occ = 0;
        if (c <= 0) {
            e.a = r->L0[li].a; e.b = r->L0[li].b; e.c0 = r->L0[li].c; e.hd = r->L0[li].hd; e.has_hd = 1;
            occ = e.c0 != 0.0;
            li++;
        } else {
            e.a = r->sp0[si].a; e.b = r->sp0[si].b;
        }
        if (c >= 0) {
            xacc xa, xr;
            xacc_zero(&xa);
            xacc_zero(&xr);
            while (si < r->ns0 && r->sp0[si].a == e.a && r->sp0[si].b == e.b) {
                if (r->sp0[si].init || occ) xacc_add(&xa, r->sp0[si].w, 0);
                else xacc_add(&xr, r->sp0[si].w, 0);
                si++;
            }
            e.sacc = xacc_round(&xa);
            e.srej = xacc_round(&xr);
        }
        v[n++] = e;
    }
    *out = v;
    return n;
}

/* the last iteration (keep_last set): start list, spawns (with parent index
 * into the start list) and the adaptive-shift factors f_i */
void orc_set_keep_last(orc_run *r, int on) { r->keep_last = on; }
int64_t orc_last_iteration(const orc_run *r, int64_t *ns, uint64_t *la, uint64_t *lb, double *lc, double *lhd,
                           double *lf, uint64_t *sa, uint64_t *sb, double *sw, int32_t *sinit, int64_t *spar)
{
    if (ns) *ns = r->ns0;
    for (int64_t i = 0; i < r->n0; i++) {
        if (la) la[i] = r->L0[i].a;
        if (lb) lb[i] = r->L0[i].b;
        if (lc) lc[i] = r->L0[i].c;
        if (lhd) lhd[i] = r->L0[i].hd;
        if (lf) lf[i] = r->f0 ? r->f0[i] : 1.0;
    }
    for (int64_t k = 0; k < r->ns0; k++) {
        if (sa) sa[k] = r->sp0[k].a;
        if (sb) sb[k] = r->sp0[k].b;
        if (sw) sw[k] = r->sp0[k].w;
        if (sinit) sinit[k] = r->sp0[k].init;
        if (spar) spar[k] = r->sp0[k].parent;
    }
    return r->n0;
}

int orc_pair_step(orc_run *r0, orc_run *r1, int64_t n)
{
    r0->keep_last = 1;
    r1->keep_last = 1;
    for (int64_t k = 0; k < n; k++) {
        const double e0 = (r0->S + r1->S) / 2.0;
        int e = one_iteration(r0);
        if (!e) e = one_iteration(r1);
        if (e) { r0->err = r1->err = e; return e; }
        oside *v0, *v1;
        int64_t n0 = side_list(r0, &v0), n1 = side_list(r1, &v1);
        double ov = 0.0, hdg = 0.0, cross = 0.0, pt2 = 0.0;
        int64_t i = 0, j = 0;
        while (i < n0 && j < n1) {
            int c = cmp_key(v0[i].a, v0[i].b, v1[j].a, v1[j].b);
            if (c < 0) { i++; continue; }
            if (c > 0) { j++; continue; }
            const oside *p = &v0[i], *q = &v1[j];
            ov = ov + p->c0 * q->c0;
            if (p->c0 != 0.0 && q->c0 != 0.0) hdg = hdg + (p->c0 * p->hd) * q->c0;
            cross = cross + (p->c0 * (q->sacc + q->srej) + q->c0 * (p->sacc + p->srej));
            if (p->srej != 0.0 && q->srej != 0.0) {
                double hd = p->has_hd ? p->hd : (q->has_hd ? q->hd : orc_hdiag_rel(r0->s, p->a, p->b));
                if (e0 - hd != 0.0) pt2 = pt2 + (p->srej * q->srej) / (e0 - hd); /* undefined term left out */
            }
            i++; j++;
        }
        free(v0); free(v1);
        const double tau = r0->p.tau;
        orc_stat *t = &r0->st[r0->nst - 1];
        t->x_overlap = ov;
        t->x_var_num = hdg - cross / (2.0 * tau);
        t->x_pt2 = pt2 / (tau * tau);
    }
    return 0;
}

int64_t orc_ndet(const orc_run *r) { return r->n; }
int64_t orc_iter(const orc_run *r) { return r->iter; }
double orc_shift(const orc_run *r) { return r->S; }

/* list in ascending key order (the list is kept sorted) */
void orc_export(const orc_run *r, uint64_t *a, uint64_t *b, double *c, double *hd, int32_t *flags)
{
    for (int64_t i = 0; i < r->n; i++) {
        a[i] = r->L[i].a; b[i] = r->L[i].b; c[i] = r->L[i].c; hd[i] = r->L[i].hd; flags[i] = r->L[i].flags;
    }
}

/* shift state: S, vary, shift_start, cnt, nw_last (hi, lo words) */
void orc_export_shift(const orc_run *r, double *S, int64_t st[3], uint64_t nwl[2])
{
    *S = r->S; st[0] = r->vary; st[1] = r->shift_start; st[2] = r->cnt;
    nwl[0] = (uint64_t)(r->nw_last >> 64); nwl[1] = (uint64_t)r->nw_last;
}

/* replace the state (used to time or check iterations from a given point);
 * keys need not be sorted; pinned reference flag is re-derived; D is not imported */
void orc_import(orc_run *r, int64_t n, const uint64_t *a, const uint64_t *b, const double *c,
                int64_t iter, double S, int vary, int64_t shift_start, int64_t cnt, uint64_t nwl_hi, uint64_t nwl_lo)
{
    free(r->L);
    r->cap = n + 1;
    r->L = malloc(sizeof(odet) * r->cap);
    for (int64_t i = 0; i < n; i++) {
        r->L[i].a = a[i]; r->L[i].b = b[i]; r->L[i].c = c[i];
        r->L[i].hd = orc_hdiag_rel(r->s, a[i], b[i]);
        r->L[i].flags = (a[i] == r->s->ref_a && b[i] == r->s->ref_b) ? 1 : 0;
    }
    r->n = n;
    qsort(r->L, n, sizeof(odet), cmp_odet);
    r->iter = iter; r->S = S; r->vary = vary; r->shift_start = shift_start; r->cnt = cnt;
    r->nw_last = ((u128)nwl_hi << 64) | nwl_lo;
}

int64_t orc_nstats(const orc_run *r) { return r->nst; }
void orc_stats(const orc_run *r, int64_t i0, int64_t n, orc_stat *out)
{
    memcpy(out, r->st + i0, sizeof(orc_stat) * n);
}
int orc_stat_size(void) { return (int)sizeof(orc_stat); }
int orc_params_size(void) { return (int)sizeof(orc_params); }

/* E_num, E_den of the current list (Eq. (9)): E_num = sum_{j != ref} H_ref,j C_j
 * as in reading R12 (terms truncated to 2^-Fe, summed exactly, rounded once),
 * E_den = C_ref */
void orc_proj_energy(const orc_run *r, double *num, double *den)
{
    const orc_sys *s = r->s;
    double e_den = 0.0;
    xacc xe;
    xacc_zero(&xe);
    for (int64_t i = 0; i < r->n; i++) {
        const odet *d = &r->L[i];
        if (d->a == s->ref_a && d->b == s->ref_b) { e_den = d->c; continue; }
        int lev = popc(d->a ^ s->ref_a) + popc(d->b ^ s->ref_b);
        if (lev <= 4 && d->c != 0.0)
            xacc_add(&xe, trunc_grid(orc_hoff(s, d->a, d->b, s->ref_a, s->ref_b) * d->c, s->Fe), 0);
    }
    *num = xacc_round(&xe); *den = e_den;
}

int orc_enum_grid(const orc_sys *s) { return s->Fe; }
