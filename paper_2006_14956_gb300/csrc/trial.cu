// trial.cu -- set-up of the trial-wave-function energy estimator (Sec. IV):
//   E_Trial = <Psi^T|H|Psi> / <Psi^T|Psi>,
// Psi^T the lowest eigenvector of H projected into the trial space T.
//   k_trial_dense  H^T (CSR from the semi-stochastic builder) as a dense
//                  matrix, padded to an even order;
//   k_jacobi       its lowest eigenpair by Jacobi rotations in the parallel
//                  round-robin order (Brent and Luk 1985): n/2 disjoint
//                  planes rotated at once, each plane's angle from
//                  theta = (A_qq - A_pp) / (2 A_pq),
//                  t = sign(theta) / (|theta| + sqrt(theta^2 + 1)), sweeps
//                  until the off-diagonal part is below 1e-15 of the norm;
//   k_trial_w      W_j = <D_j|H - E_ref|Psi^T> for every determinant in T and
//                  connected to it, accumulated in an open-addressing table
//                  that the annihilation kernel probes every iteration.
#include <cuda_runtime.h>

#include "fq_device.cuh"

namespace fq {

constexpr int JAC_THREADS = 1024;
constexpr int JAC_MAX = 1024;  // largest trial space

__global__ void k_trial_dense(const long long *__restrict__ rowptr, const int *__restrict__ col,
                              const double *__restrict__ val, int nt, int n2, double *A, double *hdiag)
{
    for (int r = blockIdx.x; r < nt; r += gridDim.x)
        for (long long q = rowptr[r] + threadIdx.x; q < rowptr[r + 1]; q += blockDim.x) {
            const int c = col[q];
            A[(size_t)r * n2 + c] = val[q];
            if (c == r) hdiag[r] = val[q];
        }
}

// one block; A (n2 x n2, row-major, symmetric, destroyed) and V in global memory
__global__ void __launch_bounds__(JAC_THREADS) k_jacobi(double *A, double *V, int n, int n2, double *E, double *v,
                                                        int *sweeps)
{
    __shared__ double cs[JAC_MAX / 2], sn[JAC_MAX / 2];
    __shared__ int P[JAC_MAX / 2], Q[JAC_MAX / 2];
    __shared__ double red[JAC_THREADS / 32];
    __shared__ int s_done;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5, h = n2 / 2;
    for (size_t x = t; x < (size_t)n2 * n2; x += JAC_THREADS) V[x] = (x / n2 == x % n2) ? 1.0 : 0.0;
    // Frobenius norm
    double acc = 0.0;
    for (size_t x = t; x < (size_t)n2 * n2; x += JAC_THREADS) acc = acc + A[x] * A[x];
    for (int m = 16; m >= 1; m >>= 1) acc = acc + __shfl_xor_sync(0xffffffffu, acc, m);
    if (lane == 0) red[warp] = acc;
    __syncthreads();
    double norm = 0.0;
    for (int k = 0; k < JAC_THREADS / 32; k++) norm = norm + red[k];
    __syncthreads();
    int sweep = 0;
    for (; sweep < 60; sweep++) {
        // off-diagonal part
        double off = 0.0;
        for (size_t x = t; x < (size_t)n2 * n2; x += JAC_THREADS)
            if (x / n2 < x % n2) off = off + A[x] * A[x];
        for (int m = 16; m >= 1; m >>= 1) off = off + __shfl_xor_sync(0xffffffffu, off, m);
        if (lane == 0) red[warp] = off;
        __syncthreads();
        if (t == 0) {
            double o = 0.0;
            for (int k = 0; k < JAC_THREADS / 32; k++) o = o + red[k];
            s_done = !(o > 1e-30 * norm);
        }
        __syncthreads();
        if (s_done) break;
        for (int r = 0; r < n2 - 1; r++) {
            // round r of the round-robin: slot 0 fixed, slots 1..n2-1 rotated by r
            for (int k = t; k < h; k += JAC_THREADS) {
                const int j1 = k, j2 = n2 - 1 - k;
                const int p0 = j1 == 0 ? 0 : ((j1 - 1 + r) % (n2 - 1)) + 1;
                const int q0 = ((j2 - 1 + r) % (n2 - 1)) + 1;
                const int p = min(p0, q0), q = max(p0, q0);
                const double apq = A[(size_t)p * n2 + q];
                double c = 1.0, s = 0.0;
                if (apq != 0.0) {
                    const double theta = (A[(size_t)q * n2 + q] - A[(size_t)p * n2 + p]) / (2.0 * apq);
                    const double tt = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                    c = 1.0 / sqrt(tt * tt + 1.0);
                    s = tt * c;
                }
                P[k] = p; Q[k] = q; cs[k] = c; sn[k] = s;
            }
            __syncthreads();
            // columns of A and V, then rows of A (A <- J^T A J)
            for (size_t x = t; x < (size_t)h * n2; x += JAC_THREADS) {
                const int k = (int)(x / n2), i = (int)(x % n2);
                const int p = P[k], q = Q[k];
                const double c = cs[k], s = sn[k];
                if (s == 0.0) continue;
                const double aip = A[(size_t)i * n2 + p], aiq = A[(size_t)i * n2 + q];
                A[(size_t)i * n2 + p] = c * aip - s * aiq;
                A[(size_t)i * n2 + q] = s * aip + c * aiq;
                const double vip = V[(size_t)i * n2 + p], viq = V[(size_t)i * n2 + q];
                V[(size_t)i * n2 + p] = c * vip - s * viq;
                V[(size_t)i * n2 + q] = s * vip + c * viq;
            }
            __syncthreads();
            for (size_t x = t; x < (size_t)h * n2; x += JAC_THREADS) {
                const int k = (int)(x / n2), j = (int)(x % n2);
                const int p = P[k], q = Q[k];
                const double c = cs[k], s = sn[k];
                if (s == 0.0) continue;
                const double apj = A[(size_t)p * n2 + j], aqj = A[(size_t)q * n2 + j];
                A[(size_t)p * n2 + j] = c * apj - s * aqj;
                A[(size_t)q * n2 + j] = s * apj + c * aqj;
            }
            __syncthreads();
        }
    }
    if (t == 0) {
        int lo = 0;
        for (int i = 1; i < n; i++)
            if (A[(size_t)i * n2 + i] < A[(size_t)lo * n2 + lo]) lo = i;
        *E = A[(size_t)lo * n2 + lo];
        P[0] = lo;
        *sweeps = sweep;
    }
    __syncthreads();
    const int lo = P[0];
    for (int i = t; i < n; i += JAC_THREADS) v[i] = V[(size_t)i * n2 + lo];
}

// determinants connected to one determinant by one application of H, in the
// order of the reference coupling sum: alpha singles, beta singles,
// opposite-spin doubles, alpha-alpha doubles, beta-beta doubles (the
// same-spin index grids include every ordered pair; only i < j, a < b count)
long long connections_per_det(int na, int nb, int ma, int mb)
{
    const long long s1 = (long long)na * ma, s2 = (long long)nb * mb, s3 = (long long)na * nb * ma * mb;
    const long long s4 = (long long)na * na * ma * ma, s5 = (long long)nb * nb * mb * mb;
    return s1 + s2 + s3 + s4 + s5;
}

// item q of determinant (ra, rb): target (ta, tb), or false if the item is
// not a distinct excitation
__device__ __forceinline__ bool connection(const DevInst &I, u64 ra, u64 rb, long long q, u64 &ta, u64 &tb)
{
    const u64 va = ~ra & I.normask, vb = ~rb & I.normask;
    const long long na = I.na, nb = I.nb, ma = I.ma, mb = I.mb;
    const long long s1 = na * ma, s2 = nb * mb, s3 = na * nb * ma * mb, s4 = na * na * ma * ma;
    ta = ra; tb = rb;
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
        if (!(i < j && a < b)) return false;
        ta ^= (1ULL << nth_set(ra, i)) | (1ULL << nth_set(ra, j)) | (1ULL << nth_set(va, a)) | (1ULL << nth_set(va, b));
    } else {
        q -= s4;
        const int b = (int)(q % mb); q /= mb;
        const int a = (int)(q % mb); q /= mb;
        const int j = (int)(q % nb), i = (int)(q / nb);
        if (!(i < j && a < b)) return false;
        tb ^= (1ULL << nth_set(rb, i)) | (1ULL << nth_set(rb, j)) | (1ULL << nth_set(vb, a)) | (1ULL << nth_set(vb, b));
    }
    return true;
}

// find-or-insert key (a, b); the claimer writes the key, then publishes the
// slot.  A reader that meets a slot being written waits a bounded time.
__device__ int trial_slot(unsigned *state, TrialEnt *tab, int bits, u64 a, u64 b, unsigned long long *count, int *err)
{
    const u64 mask = (1ULL << bits) - 1;
    u64 s = det_hash(a, b) & mask;
    for (u64 probe = 0; probe <= mask; probe++) {
        unsigned st = *(volatile unsigned *)(state + s);
        if (st == 0) {
            if (atomicCAS(state + s, 0u, 1u) == 0u) {
                tab[s].a = a;
                tab[s].b = b;
                __threadfence();
                atomicExch(state + s, 2u);
                atomicAdd(count, 1ULL);
                return (int)s;
            }
            st = *(volatile unsigned *)(state + s);
        }
        for (int spin = 0; st == 1u; spin++) {
            if (spin > (1 << 22)) { atomicOr(err, 1); return -1; }
            st = *(volatile unsigned *)(state + s);
        }
        __threadfence();
        const u64 ka = *(volatile u64 *)&tab[s].a, kb = *(volatile u64 *)&tab[s].b;
        if (ka == a && kb == b) return (int)s;
        s = (s + 1) & mask;
    }
    atomicOr(err, 2);
    return -1;
}

// item x = i (per_det + 1) + q: q < per_det the q-th connection of T_i, q =
// per_det the diagonal term of T_i (and its component of Psi^T)
__global__ void k_trial_w(const DevInst *__restrict__ Ip, const ulonglong2 *__restrict__ tkey,
                          const double *__restrict__ cT, const double *__restrict__ hdiag, int nt, long long per_det,
                          unsigned *state, TrialEnt *tab, int bits, unsigned long long *count, int *err)
{
    const DevInst &I = *Ip;
    const long long total = (long long)nt * (per_det + 1);
    for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < total;
         x += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(x / (per_det + 1));
        const long long q = x % (per_det + 1);
        const ulonglong2 k = tkey[i];
        const double c = cT[i];
        if (q == per_det) {
            const int s = trial_slot(state, tab, bits, k.x, k.y, count, err);
            if (s < 0) return;
            atomicAdd(&tab[s].w, hdiag[i] * c);
            tab[s].cT = c;
            continue;
        }
        u64 ta, tb;
        if (!connection(I, k.x, k.y, q, ta, tb)) continue;
        const double hv = hoff_generic(I, k.x, k.y, ta, tb);
        if (is_zero(hv)) continue;
        const int s = trial_slot(state, tab, bits, ta, tb, count, err);
        if (s < 0) return;
        atomicAdd(&tab[s].w, hv * c);
    }
}

cudaError_t launch_trial_dense(const long long *rowptr, const int *col, const double *val, int nt, int n2, double *A,
                               double *hdiag, cudaStream_t s)
{
    k_trial_dense<<<nt > 0 ? nt : 1, 128, 0, s>>>(rowptr, col, val, nt, n2, A, hdiag);
    return cudaGetLastError();
}

cudaError_t launch_jacobi_lowest(double *A, double *V, int n, int n2, double *E, double *v, int *sweeps,
                                 cudaStream_t s)
{
    if (n2 > JAC_MAX || (n2 & 1)) return cudaErrorInvalidValue;
    k_jacobi<<<1, JAC_THREADS, 0, s>>>(A, V, n, n2, E, v, sweeps);
    return cudaGetLastError();
}

cudaError_t launch_trial_w(const DevInst *dinst, const ulonglong2 *tkey, const double *cT, const double *hdiag, int nt,
                           long long per_det, unsigned *state, TrialEnt *tab, int bits, unsigned long long *count,
                           int *err, cudaStream_t s)
{
    int dev = 0, sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sm, cudaDevAttrMultiProcessorCount, dev);
    const long long total = (long long)nt * (per_det + 1);
    long long blocks = (total + 255) / 256;
    if (blocks > (long long)sm * 16) blocks = (long long)sm * 16;
    if (blocks < 1) blocks = 1;
    k_trial_w<<<(unsigned)blocks, 256, 0, s>>>(dinst, tkey, cT, hdiag, nt, per_det, state, tab, bits, count, err);
    return cudaGetLastError();
}

}  // namespace fq
