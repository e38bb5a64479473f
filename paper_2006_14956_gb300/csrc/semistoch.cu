// semistoch.cu -- deterministic projection inside the space D (Sec. III,
// Eqs. (7)-(8)): selection of the N_D most populated determinants, the sparse
// matrix H^D (relative to E_ref) in CSR, and the per-iteration exact update
// C_D <- C_D - tau (H^D C_D - S C_D), which replaces death for D; stochastic
// spawns D -> D are removed in the spawning kernel.
#include <cuda_runtime.h>

#include "fq_device.cuh"

namespace fq {

// ------------------------------------------------------------------ selection
// 16-bit digit histogram of the bit patterns of |C| (monotone in |C| for
// non-negative binary64) restricted to patterns whose higher digits equal
// `prefix` (the first `shift` bits from the top).
__global__ void k_abs_hist(const DevInst *__restrict__ I, int par, int nb, int shift, u64 prefix, unsigned *hist)
{
    for (int b = blockIdx.x; b < nb; b += gridDim.x) {
        const int m = I->cnt[par][b];
        for (int e = threadIdx.x; e < m; e += blockDim.x) {
            const u64 v = dbits(I->c[par][(size_t)b * CAP_M + e]) & ~SIGN64;
            if (shift > 0 && (v >> (64 - shift)) != prefix) continue;
            atomicAdd(hist + (int)((v >> (48 - shift)) & 0xffffULL), 1u);
        }
    }
}

// every determinant with |C| bits >= thr: keys and |C| bits appended
__global__ void k_abs_collect(const DevInst *__restrict__ I, int par, int nb, u64 thr, ulonglong2 *keys, u64 *mags,
                              int *n, int cap)
{
    for (int b = blockIdx.x; b < nb; b += gridDim.x) {
        const int m = I->cnt[par][b];
        for (int e = threadIdx.x; e < m; e += blockDim.x) {
            const size_t o = (size_t)b * CAP_M + e;
            const u64 v = dbits(I->c[par][o]) & ~SIGN64;
            if (v < thr) continue;
            const int q = atomicAdd(n, 1);
            if (q < cap) { keys[q] = I->key[par][o]; mags[q] = v; }
        }
    }
}

// ------------------------------------------------------------------ H^D
// one warp per row r; columns in ascending D order; pass 0 counts the
// non-zero entries, pass 1 writes them (the diagonal is always stored)
__global__ void k_build_hd(const DevInst *__restrict__ I, int nd, const ulonglong2 *__restrict__ dkey,
                           long long *rowcnt, const long long *__restrict__ rowptr, int *col, double *val, int pass)
{
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nwarp = (gridDim.x * blockDim.x) >> 5;
    for (int r = gw; r < nd; r += nwarp) {
        const ulonglong2 kr = dkey[r];
        long long pos = pass ? rowptr[r] : 0;
        long long cnt = 0;
        const double dg = diag_exact_warp(*I, kr.x, kr.y);
        for (int c0 = 0; c0 < nd; c0 += 32) {
            const int c = c0 + lane;
            double v = 0.0;
            bool nz = false;
            if (c < nd) {
                const ulonglong2 kc = dkey[c];
                if (c == r) { v = dg; nz = true; }
                else if (__popcll(kc.x ^ kr.x) + __popcll(kc.y ^ kr.y) <= 4) {
                    v = hoff_generic(*I, kc.x, kc.y, kr.x, kr.y);  // <D_r|H|D_c>
                    nz = !is_zero(v);
                }
            }
            const unsigned bal = __ballot_sync(0xffffffffu, nz);
            if (pass && nz) {
                const long long q = pos + __popc(bal & ((1u << lane) - 1u));
                col[q] = c;
                val[q] = v;
            }
            pos += __popc(bal);
            cnt += __popc(bal);
        }
        if (!pass && lane == 0) rowcnt[r] = cnt;
    }
}

// flags and the starting amplitudes of D
__global__ void k_mark_d(const DevInst *__restrict__ I, int par, int nb)
{
    for (int b = blockIdx.x; b < nb; b += gridDim.x) {
        const int m = I->cnt[par][b];
        for (int e = threadIdx.x; e < m; e += blockDim.x) {
            const size_t o = (size_t)b * CAP_M + e;
            const ulonglong2 k = I->key[par][o];
            const int d = d_index_of(*I, k.x, k.y);
            if (d >= 0) {
                I->fl[par][o] |= DFLAG_D;
                I->dc_buf[par][d] = I->c[par][o];
            }
        }
    }
}

// ------------------------------------------------------------------ per iteration
// C_D(new) = C_D - tau (y - S C_D) with y_r = sum_c H^D_rc C_D,c: every
// product is rounded to binary64, truncated toward zero to a multiple of
// 2^-64, and the row's truncated products are summed exactly (128-bit fixed
// point on the grid 2^-64) and rounded once.  The sum does not depend on
// the order of its terms, so a warp shares a row: lane k takes the columns
// k, k + 32, ... and the lanes' partial sums are joined by a shuffle tree.
// Products of magnitude 2^48 or more (beyond what 2^14 of them can sum to
// in 127 bits) raise the numeric error.  C_D of the current parity is read;
// the other buffer receives the iteration's result, so a repeated iteration
// starts from unchanged values.
constexpr int SEMI_GRID = 64;
__global__ void __launch_bounds__(256) k_semistoch(const DevInst *__restrict__ insts, int n_inst)
{
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nwarp = (gridDim.x * blockDim.x) >> 5;
    for (int ii = 0; ii < n_inst; ii++) {
        const DevInst &I = insts[ii];
        if (I.nd == 0) continue;
        if (*(volatile int *)&I.st->err) continue;
        const double S = I.st->S;
        const double *cur = I.dc_buf[I.st->parity];
        bool bad = false;
        for (int r = gw; r < I.nd; r += nwarp) {
            const long long q0 = I.drow[r], q1 = I.drow[r + 1];
            i128 acc = 0;
            // four terms per lane in flight: their loads issued before the adds
            long long q = q0 + lane;
            for (; q + 96 < q1; q += 128) {
                double v[4], x[4];
#pragma unroll
                for (int k = 0; k < 4; k++) {
                    v[k] = __ldg(I.dval + q + 32 * k);
                    x[k] = cur[__ldg(I.dcol + q + 32 * k)];
                }
#pragma unroll
                for (int k = 0; k < 4; k++) {
                    const double p = v[k] * x[k];
                    bad |= !abs_lt(p, 0x1p48);
                    acc += to_fixed(p, SEMI_GRID);
                }
            }
            for (; q < q1; q += 32) {
                const double p = __ldg(I.dval + q) * cur[__ldg(I.dcol + q)];
                bad |= !abs_lt(p, 0x1p48);
                acc += to_fixed(p, SEMI_GRID);
            }
            for (int m = 16; m >= 1; m >>= 1) acc += shfl_xor_i128(acc, m);
            if (lane == 0) {
                const double y = fixed_to_double(acc, SEMI_GRID);
                const double c = cur[r];
                I.dc_new[r] = c - I.tau * (y - S * c);
            }
        }
        if (bad) atomicOr(&I.st->err, ERRB_NUMERIC);
    }
}

static int sms()
{
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
}

void launch_semistoch(const DevInst *dinst, int n_inst, int max_nd, cudaStream_t s)
{
    // one warp per row, eight rows per block, at most eight blocks per SM
    int blocks = (max_nd + 7) / 8;
    if (blocks > sms() * 8) blocks = sms() * 8;
    if (blocks < 1) blocks = 1;
    k_semistoch<<<blocks, 256, 0, s>>>(dinst, n_inst);
}

void launch_abs_hist(const DevInst *dinst, int par, int nb, int shift, u64 prefix, unsigned *hist, cudaStream_t s)
{
    k_abs_hist<<<sms() * 8, 256, 0, s>>>(dinst, par, nb, shift, prefix, hist);
}

void launch_abs_collect(const DevInst *dinst, int par, int nb, u64 thr, ulonglong2 *keys, u64 *mags, int *n, int cap,
                        cudaStream_t s)
{
    k_abs_collect<<<sms() * 8, 256, 0, s>>>(dinst, par, nb, thr, keys, mags, n, cap);
}

void launch_build_hd(const DevInst *dinst, int nd, const ulonglong2 *dkey, long long *rowcnt, const long long *rowptr,
                     int *col, double *val, int pass, cudaStream_t s)
{
    int blocks = (nd * 32 + 255) / 256;
    if (blocks > sms() * 16) blocks = sms() * 16;
    if (blocks < 1) blocks = 1;
    k_build_hd<<<blocks, 256, 0, s>>>(dinst, nd, dkey, rowcnt, rowptr, col, val, pass);
}

void launch_mark_d(const DevInst *dinst, int parity, int nb, cudaStream_t s)
{
    k_mark_d<<<sms() * 8, 256, 0, s>>>(dinst, parity, nb);
}

}  // namespace fq
