// replica.cu -- the cross estimators of a replica pair (Sec. V: two
// independent walker distributions of the same system; Sec. VI: the
// Epstein-Nesbet PT2 correction from spawns discarded on both replicas).
//
// Both replicas keep the same bucket layout, so the determinants of bucket b
// of one replica can only meet those of bucket b of the other.  The
// annihilation kernel leaves, per bucket and replica, one entry per
// determinant of the iteration (start amplitude C, H_jj - E_ref when it was
// occupied, accepted and rejected spawn sums); k_replica_cross joins the two
// lists of a bucket through a shared-memory hash table of the first
// replica's entries and reduces, per bucket,
//   sum_j C^1_j C^2_j,  sum_j (C^1_j (H_jj - E_ref)) C^2_j,
//   sum_j (C^1_j S^2_j + C^2_j S^1_j)   (S = accepted + rejected spawns),
//   sum_j R^1_j R^2_j / (E_0 - (H_jj - E_ref))   over j with both rejected sums R nonzero,
// E_0 = the mean of the two shifts at the start of the iteration.  H_jj of
// the last kind (never in either list) is computed here, one warp each.
#include <cuda_runtime.h>

#include "fq_device.cuh"

namespace fq {

constexpr int XC_THREADS = 256;
constexpr int XC_TABBITS = 14;   // hash table of up to 8192 first-replica entries
constexpr int XC_PT2CAP = 1024;  // matched rejected determinants queued for the warps

__global__ void __launch_bounds__(XC_THREADS) k_replica_cross(const DevInst *__restrict__ insts, int n_inst)
{
    extern __shared__ unsigned xtab[];
    __shared__ int s_np;
    __shared__ int s_pair[XC_PT2CAP][2];
    __shared__ double s_red[XC_THREADS / 32][4];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const unsigned mask = (1u << XC_TABBITS) - 1u;
    for (int ii = 0; ii < n_inst; ii++) {
        const DevInst &A = insts[ii];
        if (A.partner <= ii || !A.side) continue;  // the first replica of each pair does the join
        const DevInst &B = insts[A.partner];
        const int errs = *(volatile int *)&A.st->err | *(volatile int *)&B.st->err;
        if ((errs & ERRB_STAGE) || A.st->err_at_start || B.st->err_at_start) continue;  // not committed: repeated
        const double e0 = (A.st->S + B.st->S) * 0.5;
        const int nbk = 1 << A.bb;
        if (A.bb != B.bb) {  // the host keeps the layouts equal; never join unequal ones
            for (int bk = blockIdx.x * blockDim.x + t; bk < nbk; bk += gridDim.x * blockDim.x) {
                Partial &P = A.part[bk];
                P.x_ov = 0.0; P.x_hd = 0.0; P.x_cr = 0.0; P.x_pt2 = 0.0;
            }
            continue;
        }
        for (int bk = blockIdx.x; bk < nbk; bk += gridDim.x) {
            const int n0 = A.side_cnt[bk], n1 = B.side_cnt[bk];
            const SideEnt *S0 = A.side + (size_t)bk * A.side_cap;
            const SideEnt *S1 = B.side + (size_t)bk * B.side_cap;
            const bool use_tab = 2 * n0 <= (int)(mask + 1u);
            if (use_tab) {
                for (int q = t; q <= (int)mask; q += XC_THREADS) xtab[q] = 0u;
                __syncthreads();
                for (int i = t; i < n0; i += XC_THREADS) {
                    unsigned s = (unsigned)det_hash(S0[i].a, S0[i].b) & mask;
                    while (atomicCAS(&xtab[s], 0u, (unsigned)(i + 1)) != 0u) s = (s + 1u) & mask;
                }
            }
            if (t == 0) s_np = 0;
            __syncthreads();
            double ov = 0.0, hdg = 0.0, cr = 0.0, pt2 = 0.0;
            for (int j = t; j < n1; j += XC_THREADS) {
                const SideEnt q = S1[j];
                int i = -1;
                if (use_tab) {
                    unsigned s = (unsigned)det_hash(q.a, q.b) & mask;
                    for (unsigned probe = 0; probe <= mask; probe++) {
                        const unsigned v = xtab[s];
                        if (v == 0u) break;
                        if (S0[v - 1].a == q.a && S0[v - 1].b == q.b) { i = (int)v - 1; break; }
                        s = (s + 1u) & mask;
                    }
                } else {
                    for (int x = 0; x < n0; x++)
                        if (S0[x].a == q.a && S0[x].b == q.b) { i = x; break; }
                }
                if (i < 0) continue;
                const SideEnt p = S0[i];
                ov = ov + p.c0 * q.c0;
                if (!is_zero(p.c0) && !is_zero(q.c0)) hdg = hdg + (p.c0 * p.hd) * q.c0;
                cr = cr + (p.c0 * (q.sacc + q.srej) + q.c0 * (p.sacc + p.srej));
                if (!is_zero(p.srej) && !is_zero(q.srej)) {
                    const int k = atomicAdd(&s_np, 1);
                    if (k < XC_PT2CAP) { s_pair[k][0] = i; s_pair[k][1] = j; }
                    else {
                        const double den = e0 - diag_exact_thread(A, p.a, p.b);
                        if (den != 0.0) pt2 = pt2 + (p.srej * q.srej) / den;  // undefined term left out
                    }
                }
            }
            __syncthreads();
            const int np = min(s_np, XC_PT2CAP);
            for (int k = warp; k < np; k += XC_THREADS / 32) {
                const SideEnt p = S0[s_pair[k][0]], q = S1[s_pair[k][1]];
                const u64 ka[1] = {p.a}, kb[1] = {p.b};
                double hd[1];
                diag_exact_warp_multi<1>(A, ka, kb, hd);
                if (lane == 0 && e0 - hd[0] != 0.0) pt2 = pt2 + (p.srej * q.srej) / (e0 - hd[0]);
            }
            for (int m = 16; m >= 1; m >>= 1) {
                ov = ov + __shfl_xor_sync(0xffffffffu, ov, m);
                hdg = hdg + __shfl_xor_sync(0xffffffffu, hdg, m);
                cr = cr + __shfl_xor_sync(0xffffffffu, cr, m);
                pt2 = pt2 + __shfl_xor_sync(0xffffffffu, pt2, m);
            }
            if (lane == 0) { s_red[warp][0] = ov; s_red[warp][1] = hdg; s_red[warp][2] = cr; s_red[warp][3] = pt2; }
            __syncthreads();
            if (t == 0) {
                double r[4] = {0.0, 0.0, 0.0, 0.0};
                for (int w = 0; w < XC_THREADS / 32; w++)
                    for (int c = 0; c < 4; c++) r[c] = r[c] + s_red[w][c];
                Partial &P = A.part[bk];
                P.x_ov = r[0]; P.x_hd = r[1]; P.x_cr = r[2]; P.x_pt2 = r[3];
            }
            __syncthreads();
        }
    }
}

// shared-memory opt-in of the join kernel (called before any stream capture)
cudaError_t replica_kernel_init()
{
    return cudaFuncSetAttribute(k_replica_cross, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(sizeof(unsigned) << XC_TABBITS));
}

cudaError_t launch_replica_cross(const DevInst *dinst, int n_inst, int max_buckets, cudaStream_t s)
{
    const size_t smem = sizeof(unsigned) << XC_TABBITS;
    int dev = 0, sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sm, cudaDevAttrMultiProcessorCount, dev);
    int blocks = sm * 2;
    if (blocks > max_buckets) blocks = max_buckets;
    if (blocks < 1) blocks = 1;
    k_replica_cross<<<blocks, XC_THREADS, smem, s>>>(dinst, n_inst);
    return cudaGetLastError();
}

}  // namespace fq
