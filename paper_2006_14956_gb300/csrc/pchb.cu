// pchb.cu -- tables of the pre-computed heat-bath excitation generator
// (App. A, pre-computed heat-bath sampling): for each pair of occupied spin
// orbitals (i, j), a distribution over hole pairs (a, b) with
// p(ab|ij) = |H_ij^ab| / sum_a'b' |H_ij^a'b'|, sampled in O(1) by Walker's
// alias method.
//
// Tables carry explicit spins: one per ordered opposite-spin pair (i alpha,
// j beta) over all (a alpha, b beta), with H_ij^ab = (ai|bj), and one per
// same-spin pair i < j over a < b, with H_ij^ab = (ai|bj) - (aj|bi).  Only
// double excitations carry weight: an entry whose hole is one of the two
// electrons' own spin orbitals has |H| = 0.  Entries whose holes are occupied
// in a given determinant stay in the table; such a draw is a failed attempt.
// The tables are built once, on the device, one block per table:
//   1. |H| of every entry and its exact sum S (128-bit fixed point on the
//      integral grid, rounded once);
//   2. q_k = (|H_k| / S) K, then Vose's alias construction in a fixed order:
//      indices with q < 1 on the stack "small", the rest on "large" (both
//      pushed in ascending k, popped from the top); while both are
//      non-empty, s = pop(small), l = pop(large): prob_s = q_s, alias_s = l,
//      q_l <- (q_l + q_s) - 1, and l goes back on small if q_l < 1, else on
//      large; whatever is left keeps prob = 1 and aliases itself;
//   3. each entry stores the threshold T_k = ceil(prob_k 2^53), so that the
//      coin "u < prob_k" on a 53-bit word m (u = m 2^-53) is the integer test
//      m < T_k, and both hole pairs it can return.
// Every step is exactly rounded binary64 or integer arithmetic in a fixed
// order (compiled without multiply-add contraction), so the tables do not
// depend on the launch geometry.
#include <cuda_runtime.h>

#include "fq_device.cuh"

namespace fq {

constexpr int PCHB_THREADS = 256;

// hole pair (a, b) of entry k of a same-spin table: k = b(b-1)/2 + a, a < b
__device__ __forceinline__ void ss_pair(int k, int &a, int &b)
{
    int r = (int)((1.0f + sqrtf(1.0f + 8.0f * (float)k)) * 0.5f);  // estimate, corrected below
    while (r > 1 && r * (r - 1) / 2 > k) r--;
    while ((r + 1) * r / 2 <= k) r++;
    b = r;
    a = k - r * (r - 1) / 2;
}

__global__ void __launch_bounds__(PCHB_THREADS) k_pchb_build(const DevInst *__restrict__ Ip, double ppair,
                                                             double2 *__restrict__ meta,
                                                             ulonglong2 *__restrict__ ent, u64 ss_base)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ u64 red[2 * (PCHB_THREADS / 32)];
    __shared__ double Ssh;
    const DevInst &I = *Ip;
    const int N = I.norb, t = blockIdx.x, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const bool ss = t >= N * N;
    int i, j, K;
    u64 off;
    if (!ss) {
        i = t / N; j = t % N; K = N * N; off = (u64)t * (u64)K;
    } else {
        const int p = t - N * N;
        ss_pair(p, i, j);
        K = N * (N - 1) / 2;
        off = ss_base + (u64)p * (u64)K;
    }
    double *q = (double *)smem;
    unsigned short *stk = (unsigned short *)(q + K);
    unsigned short *al = stk + K;

    // 1. |H| of every entry and the exact sum
    i128 acc = 0;
    for (int k = tid; k < K; k += PCHB_THREADS) {
        int a, b;
        double v;
        if (!ss) {
            a = k / N; b = k % N;
            v = (a == i || b == j) ? 0.0 : eri4(I, a, i, b, j);
        } else {
            ss_pair(k, a, b);
            v = (a == i || a == j || b == i || b == j) ? 0.0 : eri4(I, a, i, b, j) - eri4(I, a, j, b, i);
        }
        const double av = bitsd(dbits(v) & ~SIGN64);
        q[k] = av;
        al[k] = (unsigned short)k;
        acc += to_fixed(av, I.F);
    }
    for (int m = 16; m >= 1; m >>= 1) acc += shfl_xor_i128(acc, m);
    if (lane == 0) { red[2 * wid] = (u64)acc; red[2 * wid + 1] = (u64)((u128)acc >> 64); }
    __syncthreads();
    if (tid == 0) {
        i128 s = 0;
        for (int w = 0; w < PCHB_THREADS / 32; w++) s += (i128)(((u128)red[2 * w + 1] << 64) | (u128)red[2 * w]);
        const double S = fixed_to_double(s, I.F);
        Ssh = S;
        meta[t] = make_double2((I.tau * S) / ppair, S);
    }
    __syncthreads();
    const double S = Ssh;

    if (S > 0.0) {
        // 2. scaled weights, then the alias construction (one thread, fixed order)
        const double Kd = (double)K;
        for (int k = tid; k < K; k += PCHB_THREADS) q[k] = (q[k] / S) * Kd;
        __syncthreads();
        if (tid == 0) {
            int ns = 0, nl = 0;  // small grows from stk[0], large from stk[K-1] downwards
            for (int k = 0; k < K; k++) {
                if (q[k] < 1.0) stk[ns++] = (unsigned short)k;
                else stk[K - 1 - nl++] = (unsigned short)k;
            }
            while (ns > 0 && nl > 0) {
                const int s = stk[--ns];
                const int l = stk[K - nl];
                nl--;
                al[s] = (unsigned short)l;  // prob_s = q_s stays in q[s]
                q[l] = (q[l] + q[s]) - 1.0;
                if (q[l] < 1.0) stk[ns++] = (unsigned short)l;
                else stk[K - 1 - nl++] = (unsigned short)l;
            }
            for (int x = 0; x < ns; x++) q[stk[x]] = 1.0;
            for (int x = 0; x < nl; x++) q[stk[K - 1 - x]] = 1.0;
        }
        __syncthreads();
    }

    // 3. thresholds and hole pairs
    for (int k = tid; k < K; k += PCHB_THREADS) {
        u64 thr = 0;
        unsigned own, alt;
        int a, b;
        if (S > 0.0) {
            const double pk = q[k];
            thr = !(pk > 0.0) ? 0ULL : (pk >= 1.0 ? (1ULL << 53) : (u64)ceil(pk * 0x1p53));
        }
        if (!ss) { a = k / N; b = k % N; } else ss_pair(k, a, b);
        own = (unsigned)a | ((unsigned)b << 8);
        const int kk = al[k];
        if (!ss) { a = kk / N; b = kk % N; } else ss_pair(kk, a, b);
        alt = (unsigned)a | ((unsigned)b << 8);
        ent[off + k] = make_ulonglong2(thr, (u64)(own | (alt << 16)));
    }
}

cudaError_t launch_pchb_build(const DevInst *dinst, int norb, double ppair, double2 *meta, ulonglong2 *ent,
                              u64 ss_base, cudaStream_t s)
{
    const int N = norb;
    const int nt = N * N + N * (N - 1) / 2;
    const size_t smem = (size_t)N * N * (sizeof(double) + 2 * sizeof(unsigned short));
    cudaError_t e = cudaFuncSetAttribute(k_pchb_build, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_pchb_build<<<nt, PCHB_THREADS, smem, s>>>(dinst, ppair, meta, ent, ss_base);
    return cudaGetLastError();
}

}  // namespace fq
