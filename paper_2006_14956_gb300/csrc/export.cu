// export.cu -- moving the walker list between the host and the bucket layout.
// Import: the compact input is checked, counted per bucket (to choose the
// bucket count) and placed on the device, each determinant into the next free
// slot of its bucket (order inside a bucket affects no result: every draw is
// keyed and every sum exact), and its slot listed for the H_ii kernel.
// Export, in (alpha, beta) order: the occupied slots of every bucket are compacted,
// sorted by a least-significant-digit radix sort over the orbital bits in use
// (8-bit digits, beta word first, each pass stable), and C, H_ii - E_ref and
// the flags are gathered in that order.  Only the n live entries then cross
// to the host.
#include <cuda_runtime.h>

#include "fq_device.cuh"

namespace fq {

constexpr int XS_THREADS = 256;  // one thread per digit value in the scatter
constexpr int XS_ROUNDS = 8;
constexpr int XS_TILE = XS_THREADS * XS_ROUNDS;

// occupied slots of bucket b go to [off[b], off[b] + cnt[b])
__global__ void k_export_compact(const ulonglong2 *__restrict__ key, const int *__restrict__ cnt,
                                 const long long *__restrict__ off, int nbk, u64 *ka, u64 *kb, u64 *idx)
{
    for (int b = blockIdx.x; b < nbk; b += gridDim.x) {
        const int m = cnt[b];
        const long long o = off[b];
        for (int e = threadIdx.x; e < m; e += blockDim.x) {
            const size_t s = (size_t)b * CAP_M + e;
            const ulonglong2 k = key[s];
            ka[o + e] = k.x;
            kb[o + e] = k.y;
            idx[o + e] = s;
        }
    }
}

__device__ __forceinline__ int digit_of(const u64 *ka, const u64 *kb, long long i, int word, int shift)
{
    return (int)(((word ? ka[i] : kb[i]) >> shift) & 255u);
}

// digit counts of every tile, stored digit-major: hist[d * ntiles + tile]
__global__ void __launch_bounds__(XS_THREADS) k_export_hist(const u64 *__restrict__ ka, const u64 *__restrict__ kb,
                                                            long long n, int word, int shift, int *hist, int ntiles)
{
    __shared__ int s_h[256];
    const int t = threadIdx.x;
    s_h[t] = 0;
    __syncthreads();
    const long long i0 = (long long)blockIdx.x * XS_TILE;
    for (int r = 0; r < XS_ROUNDS; r++) {
        const long long i = i0 + (long long)r * XS_THREADS + t;
        if (i < n) atomicAdd(&s_h[digit_of(ka, kb, i, word, shift)], 1);
    }
    __syncthreads();
    hist[(size_t)t * ntiles + blockIdx.x] = s_h[t];
}

// exclusive scan of each digit's row of tile counts, hist[d * ntiles ..
// (d + 1) * ntiles), in place (block d), and the row total in dtot[d]
__global__ void __launch_bounds__(XS_THREADS) k_export_scan(int *hist, int ntiles, int *dtot)
{
    __shared__ int s_w[XS_THREADS / 32];
    __shared__ int s_carry;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    int *row = hist + (size_t)blockIdx.x * ntiles;
    if (t == 0) s_carry = 0;
    __syncthreads();
    for (int q0 = 0; q0 < ntiles; q0 += XS_THREADS) {
        const int q = q0 + t;
        const int v = q < ntiles ? row[q] : 0;
        int incl = v;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) s_w[warp] = incl;
        __syncthreads();
        int before = s_carry;
        for (int w = 0; w < warp; w++) before += s_w[w];
        if (q < ntiles) row[q] = before + incl - v;
        __syncthreads();
        if (t == XS_THREADS - 1) s_carry = before + incl;
        __syncthreads();
    }
    if (t == 0) dtot[blockIdx.x] = s_carry;
}

// stable scatter of one tile: rounds of XS_THREADS keys in index order; the
// rank of a key among the equal digits before it is its tile's offset for
// the digit, plus the counts of the earlier warps of the round, plus its
// rank among the lanes of its warp that share the digit
__global__ void __launch_bounds__(XS_THREADS) k_export_scatter(const u64 *__restrict__ ka, const u64 *__restrict__ kb,
                                                               const u64 *__restrict__ idx, long long n, int word,
                                                               int shift, const int *__restrict__ hist, int ntiles,
                                                               const int *__restrict__ dtot, u64 *ka2, u64 *kb2,
                                                               u64 *idx2)
{
    constexpr int NW = XS_THREADS / 32;
    __shared__ int s_base[256];
    __shared__ int s_w[NW][256];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    {  // keys with a smaller digit (exclusive scan of the digit totals), then this tile's row prefix
        const int v = dtot[t];
        int incl = v;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) s_w[0][warp] = incl;
        __syncthreads();
        int before = 0;
        for (int w = 0; w < warp; w++) before += s_w[0][w];
        s_base[t] = before + incl - v + hist[(size_t)t * ntiles + blockIdx.x];
        __syncthreads();
    }
    const long long i0 = (long long)blockIdx.x * XS_TILE;
    const unsigned below = (1u << lane) - 1u;
    for (int r = 0; r < XS_ROUNDS; r++) {
        const long long i = i0 + (long long)r * XS_THREADS + t;
        const bool valid = i < n;
        u64 a = 0, b = 0, x = 0;
        int d = 256;  // invalid lanes share a value no key has
        if (valid) {
            a = ka[i];
            b = kb[i];
            x = idx[i];
            d = (int)(((word ? a : b) >> shift) & 255u);
        }
        for (int q = t; q < NW * 256; q += XS_THREADS) (&s_w[0][0])[q] = 0;
        __syncthreads();
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        if (valid && lane == __ffs(peers) - 1) s_w[warp][d] = __popc(peers);
        __syncthreads();
        {  // thread t: digit t, prefix over the warps for this batch of keys
            int s = s_base[t];
            for (int w = 0; w < NW; w++) {
                const int c = s_w[w][t];
                s_w[w][t] = s;
                s += c;
            }
            s_base[t] = s;
        }
        __syncthreads();
        if (valid) {
            const int o = s_w[warp][d] + __popc(peers & below);
            ka2[o] = a;
            kb2[o] = b;
            idx2[o] = x;
        }
        __syncthreads();
    }
}

__global__ void k_export_gather(const u64 *__restrict__ idx, long long n, const double *__restrict__ c,
                                const double *__restrict__ hd, const uint8_t *__restrict__ fl, double *oc, double *ohd,
                                int32_t *ofl)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const u64 s = idx[i];
        oc[i] = c[s];
        ohd[i] = hd[s];
        ofl[i] = fl[s];
    }
}

// import, step 1: flags bit 0 = an entry with a wrong electron count, an
// orbital beyond norb or a non-finite amplitude; bit 1 = the reference present
__global__ void k_import_check(const u64 *__restrict__ a, const u64 *__restrict__ b, const double *__restrict__ c,
                               long long n, int na, int nb, u64 normask, u64 ra, u64 rb, int *flags)
{
    int f = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const u64 x = a[i], y = b[i];
        const bool finite = (dbits(c[i]) & 0x7ff0000000000000ULL) != 0x7ff0000000000000ULL;
        if (__popcll(x) != na || __popcll(y) != nb || ((x | y) & ~normask) || !finite) f |= 1;
        if (x == ra && y == rb) f |= 2;
    }
    f = __reduce_or_sync(0xffffffffu, f);
    if ((threadIdx.x & 31) == 0 && f) atomicOr(flags, f);
}

// import, step 2: bucket counts at 2^bb buckets; *over = 1 once a bucket
// holds more than half its capacity
__global__ void k_import_count(const u64 *__restrict__ a, const u64 *__restrict__ b, long long n, int bb, int *cnt,
                               int *over)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int o = atomicAdd(&cnt[bucket_of(det_hash(a[i], b[i]), bb)], 1);
        if (o == CAP_M / 2) atomicOr(over, 1);
    }
}

// import, step 3: each determinant into the next free slot of its bucket
// (fill = the zeroed counts of the list), flags (the reference's), and its
// slot into list[i]
__global__ void k_import_place(const u64 *__restrict__ a, const u64 *__restrict__ b, const double *__restrict__ c,
                               long long n, int bb, u64 ra, u64 rb, int *fill, ulonglong2 *key, double *oc,
                               uint8_t *ofl, unsigned *list)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const u64 x = a[i], y = b[i];
        const int bk = bucket_of(det_hash(x, y), bb);
        const size_t s = (size_t)bk * CAP_M + (size_t)atomicAdd(&fill[bk], 1);
        key[s] = make_ulonglong2(x, y);
        oc[s] = c[i];
        ofl[s] = (uint8_t)((x == ra && y == rb) ? DFLAG_REF : 0);
        list[i] = (unsigned)s;
    }
}

static unsigned grid_for(long long n)
{
    const long long g = (n + 255) / 256;
    return (unsigned)(g < 1 ? 1 : (g < 4096 ? g : 4096));
}

cudaError_t launch_import_check(const u64 *a, const u64 *b, const double *c, long long n, int na, int nb, u64 normask,
                                u64 ra, u64 rb, int *flags, cudaStream_t s)
{
    if (n > 0) k_import_check<<<grid_for(n), 256, 0, s>>>(a, b, c, n, na, nb, normask, ra, rb, flags);
    return cudaGetLastError();
}

cudaError_t launch_import_count(const u64 *a, const u64 *b, long long n, int bb, int *cnt, int *over, cudaStream_t s)
{
    k_import_count<<<grid_for(n), 256, 0, s>>>(a, b, n, bb, cnt, over);
    return cudaGetLastError();
}

cudaError_t launch_import_place(const u64 *a, const u64 *b, const double *c, long long n, int bb, u64 ra, u64 rb,
                                int *fill, ulonglong2 *key, double *oc, uint8_t *ofl, unsigned *list, cudaStream_t s)
{
    k_import_place<<<grid_for(n), 256, 0, s>>>(a, b, c, n, bb, ra, rb, fill, key, oc, ofl, list);
    return cudaGetLastError();
}

size_t export_scratch_bytes(long long n)
{
    const long long ntiles = (n + XS_TILE - 1) / XS_TILE;
    return (size_t)n * (6 * sizeof(u64) + 2 * sizeof(double) + sizeof(int32_t)) + (size_t)ntiles * 256 * sizeof(int) +
           256 * sizeof(int) + 8 * 256;
}

// the n occupied determinants of list `par` sorted by (alpha, beta) into
// device arrays carved from `scratch` (export_scratch_bytes(n) bytes); the
// sorted keys end in *oa / *ob, the gathered values in *oc, *ohd, *ofl
cudaError_t export_sorted(const ulonglong2 *key, const double *c, const double *hd, const uint8_t *fl, const int *cnt,
                          const long long *off, int nbk, long long n, int norb, void *scratch, const u64 **oa,
                          const u64 **ob, const double **oc, const double **ohd, const int32_t **ofl, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    if (n > 0x7fffffffLL) return cudaErrorInvalidValue;  // 32-bit positions in the scatter
    const long long ntiles = (n + XS_TILE - 1) / XS_TILE;
    unsigned char *p = (unsigned char *)scratch;
    u64 *ka[2], *kb[2], *ix[2];
    for (int k = 0; k < 2; k++) {
        ka[k] = (u64 *)p; p += (size_t)n * sizeof(u64);
        kb[k] = (u64 *)p; p += (size_t)n * sizeof(u64);
        ix[k] = (u64 *)p; p += (size_t)n * sizeof(u64);
    }
    double *dc = (double *)p; p += (size_t)n * sizeof(double);
    double *dh = (double *)p; p += (size_t)n * sizeof(double);
    int32_t *df = (int32_t *)p; p += (size_t)n * sizeof(int32_t);
    p = (unsigned char *)(((uintptr_t)p + 255) & ~(uintptr_t)255);
    int *dtot = (int *)p;
    p += 256 * sizeof(int);
    int *hist = (int *)p;

    k_export_compact<<<nbk < 4096 ? nbk : 4096, 256, 0, s>>>(key, cnt, off, nbk, ka[0], kb[0], ix[0]);
    int cur = 0;
    for (int word = 0; word < 2; word++)  // beta first: the less significant word
        for (int shift = 0; shift < norb; shift += 8) {
            k_export_hist<<<(unsigned)ntiles, XS_THREADS, 0, s>>>(ka[cur], kb[cur], n, word, shift, hist, (int)ntiles);
            k_export_scan<<<256, XS_THREADS, 0, s>>>(hist, (int)ntiles, dtot);
            k_export_scatter<<<(unsigned)ntiles, XS_THREADS, 0, s>>>(ka[cur], kb[cur], ix[cur], n, word, shift, hist,
                                                                      (int)ntiles, dtot, ka[cur ^ 1], kb[cur ^ 1],
                                                                      ix[cur ^ 1]);
            cur ^= 1;
        }
    const int gb = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
    k_export_gather<<<gb, 256, 0, s>>>(ix[cur], n, c, hd, fl, dc, dh, df);
    *oa = ka[cur];
    *ob = kb[cur];
    *oc = dc;
    *ohd = dh;
    *ofl = df;
    return cudaGetLastError();
}

}  // namespace fq
