// noalloc.cu -- an entry point that allocates no device memory.
//
// fciqmc_ref_offdiag_sum_noalloc computes the same quantity as the handle
// path (fciqmc_create's sum_j |<D_j|H|D_ref>|, returned by
// fciqmc_ref_offdiag_sum) from integrals the caller already holds in device
// memory.  Its scratch -- the per-block partial sums and the exponent range of
// the integrals -- lives in a file-scope device array instead of memory from
// cudaMalloc, so it can serve callers that must not allocate: frameworks that
// own every byte of device memory through their own pool, jobs held to a
// fixed device-memory budget, or loops that must not enter the CUDA driver's
// allocator (cudaMalloc can synchronise the whole device).
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "fq_device.cuh"

namespace fq {

// Scratch layout (bytes): [0, 512) 64 block partial sums; [512, 528) the
// smallest significand-lsb exponent, the largest exponent and an error flag
// of the integral scan.  Every GPU that loads the library keeps this array
// until the process exits.
constexpr int NOALLOC_BLOCKS = 64;
constexpr size_t NOALLOC_SCRATCH_BYTES = 1024;
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

// exponent range of the non-zero integrals: lsb exponent of each value's
// significand (after removing trailing zeros) and its binary exponent
__global__ void k_noalloc_scan(const double *__restrict__ h1, long long nh, const double *__restrict__ eri,
                               long long ne, int *ints)
{
    int lmin = 1 << 20, mmax = -(1 << 20), bad = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nh + ne;
         i += (long long)gridDim.x * blockDim.x) {
        const double x = i < nh ? h1[i] : eri[i - nh];
        const u64 b = dbits(x);
        const int ex = (int)((b >> 52) & 0x7ff);
        u64 m = b & 0xFFFFFFFFFFFFFULL;
        if (ex == 0x7ff) { bad = 1; continue; }
        if (ex == 0 && m == 0) continue;
        int e = ex ? ex - 1075 : -1074;
        if (ex) m |= 1ULL << 52;
        lmin = min(lmin, e + __ffsll((long long)m) - 1);
        mmax = max(mmax, (ex ? ex - 1023 : (e + 63 - __clzll((long long)m))));
    }
    atomicMin(ints + 0, lmin);
    atomicMax(ints + 1, mmax);
    if (bad) atomicOr(ints + 2, 1);
}

// the enumeration of k_ref_abs_sum, with the scale F taken from the scan
__global__ void __launch_bounds__(256) k_noalloc_ref_sum(DevInst Ia, const int *ints, double *partial)
{
    __shared__ DevInst Is;
    __shared__ double sm[8];
    if (threadIdx.x == 0) {
        Is = Ia;
        Is.F = max(0, -ints[0]);
    }
    __syncthreads();
    const DevInst &I = Is;
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
    for (int m = 16; m >= 1; m >>= 1) acc = acc + __shfl_xor_sync(0xffffffffu, acc, m);
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int k = 0; k < 8; k++) s = s + sm[k];
        partial[blockIdx.x] = s;
    }
}

// the partial sums added in block order, as the handle path does on the host
__global__ void k_noalloc_total(const double *partial, double *out)
{
    double acc = 0.0;
    for (int k = 0; k < NOALLOC_BLOCKS; k++) acc = acc + partial[k];
    *out = acc;
}

// the array's device address per device, looked up by the first call on that
// device and kept for the process (stale after the device's primary context
// is destroyed, e.g. by cudaDeviceReset)
static std::mutex g_noalloc_mu;
static unsigned char *g_noalloc_ptr[256];

}  // namespace fq

using namespace fq;

extern "C" int fciqmc_ref_offdiag_sum_noalloc(int32_t norb, int32_t n_alpha, int32_t n_beta, const double *d_h1,
                                              const double *d_eri, uint64_t ref_alpha, uint64_t ref_beta,
                                              double *d_out, void *stream)
{
    if (norb < 1 || norb > 64 || n_alpha < 0 || n_beta < 0 || n_alpha > norb || n_beta > norb || !d_h1 || !d_eri ||
        !d_out)
        return FCIQMC_ERR_INVALID_ARG;
    const u64 normask = norb >= 64 ? ~0ULL : ((1ULL << norb) - 1);
    if (__builtin_popcountll(ref_alpha) != n_alpha || __builtin_popcountll(ref_beta) != n_beta ||
        ((ref_alpha | ref_beta) & ~normask))
        return FCIQMC_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    // set-up, once per device, with that device current: the host-side name of
    // the array is not a device address, so the kernels get this pointer
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return FCIQMC_ERR_CUDA;
    unsigned char *base;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        if (!g_noalloc_ptr[dev]) {
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return FCIQMC_ERR_CUDA;
            g_noalloc_ptr[dev] = (unsigned char *)p;
        }
        base = g_noalloc_ptr[dev];
    }
    double *partial = (double *)base;
    int *ints = (int *)(base + 512);
    const int init[4] = {1 << 20, -(1 << 20), 0, 0};
    // the array keeps the previous call's contents: reset the scan results
    if (cudaMemcpyAsync(ints, init, sizeof(init), cudaMemcpyHostToDevice, s) != cudaSuccess) return FCIQMC_ERR_CUDA;
    const long long N = norb, np = N * (N + 1) / 2, ne = np * (np + 1) / 2;
    k_noalloc_scan<<<NOALLOC_BLOCKS, 256, 0, s>>>(d_h1, N * N, d_eri, ne, ints);
    int hi[4];
    if (cudaMemcpyAsync(hi, ints, sizeof(hi), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return FCIQMC_ERR_CUDA;
    if (hi[2]) return FCIQMC_ERR_INVALID_ARG;  // a non-finite integral
    const int n = n_alpha + n_beta;
    int terms_bits = 0;
    while ((1LL << terms_bits) < (long long)n * n + 2 * n + 4) terms_bits++;
    const int F = hi[0] > (1 << 19) ? 0 : (hi[0] < 0 ? -hi[0] : 0);
    if (hi[1] > -(1 << 19) && hi[1] + F + terms_bits + 2 > 125) return FCIQMC_ERR_UNSUPPORTED;
    DevInst I;
    memset(&I, 0, sizeof(I));
    I.kind = FCIQMC_ABINITIO;
    I.norb = norb; I.na = n_alpha; I.nb = n_beta; I.n = n; I.ma = norb - n_alpha; I.mb = norb - n_beta;
    I.h = d_h1; I.eri = d_eri;
    I.ref_a = ref_alpha; I.ref_b = ref_beta; I.normask = normask;
    k_noalloc_ref_sum<<<NOALLOC_BLOCKS, 256, 0, s>>>(I, ints, partial);
    k_noalloc_total<<<1, 1, 0, s>>>(partial, d_out);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) return FCIQMC_ERR_CUDA;
    return FCIQMC_OK;
}
