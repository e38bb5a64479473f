// capi.cu -- host side of the C ABI in include/fciqmc.h.
//
// Owns the device memory of each run, prepares the integrals (including the
// fixed-point tables used for exact diagonal sums), sizes the bucketed
// buffers, captures one projector iteration as a CUDA graph, replays it, and
// grows the buffers when a capacity flag comes back.  Statistics (blocking
// analysis of the projected energy) are computed here on the host.
#include <cuda_runtime.h>

#include <algorithm>
#include <new>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "fq_internal.h"

using namespace fq;

namespace {

thread_local std::string g_create_error;

struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
};

}  // namespace

struct fciqmc_handle {
    // system (host copies)
    int kind = 0, norb = 0, na = 0, nb = 0;
    double ecore = 0.0;
    std::vector<double> h, eri;
    std::vector<int> nbr;
    int z = 0;
    double t = 0.0, U = 0.0;
    u64 ref_a = 0, ref_b = 0;
    double eref = 0.0;
    fciqmc_params p{};
    // device
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::vector<DevBuf> bufs;
    size_t bytes = 0;
    DevInst hi{};                 // host image of the device descriptor
    DevInst *dinst = nullptr;     // device copy
    int *dunit = nullptr;         // unit_start {0, nb}
    IterState *dstate = nullptr;
    cudaGraphExec_t graph = nullptr;
    int graph_kernels = 0;  // kernel nodes of the captured iteration
    int graph_gen = -1;     // launch-configuration generation the graph was captured with
    bool profiling = false;
    double ktime[6] = {0, 0, 0, 0, 0, 0};  // spawn, heavy, annihilate, finalize, semistoch, new-determinant H_jj
    // layout
    int bb = 0;
    int heavy_cap = 0;
    int ring_cap = 4096;  // a power of two (the finalize kernel masks the iteration)
    // host-side history
    std::vector<fciqmc_iter_stats> hist;
    IterState hst{};
    std::string err;
    // semi-stochastic space
    int nd = 0;
    long long nnz = 0;
    double ref_sum = 0.0;
    // trial-wave-function estimator
    long long trial_nt = 0, trial_nw = 0;
    double trial_ET = 0.0;
    const ulonglong2 *trial_key = nullptr;
    const double *trial_cT = nullptr;
    // adaptive shift: list index and weight sums to rebuild at the next upload
    bool kidx_dirty = false;
    int step_rc = 0;  // error of the last step that failed on this run (cleared by the next good step)
    // replica pair: the other replica (owned by the first), replica index
    fciqmc_handle *partner = nullptr;
    bool secondary = false;
    bool paired = false;
    int side_nbk = 0;
    // asynchronous stepping
    bool pending = false;
    long long async_base = 0, async_target = 0;
};

// ------------------------------------------------------------------ helpers
static int fail(fciqmc_handle *h, int code, const std::string &msg)
{
    if (h) h->err = msg; else g_create_error = msg;
    return code;
}

#define CUDA_TRY(h, call)                                                                         \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess) return fail(h, e_ == cudaErrorMemoryAllocation ? FCIQMC_ERR_OUT_OF_MEMORY \
                                              : FCIQMC_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

static void *dev_alloc(fciqmc_handle *h, size_t bytes)
{
    if (bytes == 0) bytes = 16;
    bytes = (bytes + 255) & ~(size_t)255;
    if (h->p.max_device_bytes > 0 && h->bytes + bytes > (size_t)h->p.max_device_bytes) return nullptr;
    void *ptr = nullptr;
    if (h->p.alloc) ptr = h->p.alloc(bytes, h->p.alloc_ctx);
    else if (cudaMalloc(&ptr, bytes) != cudaSuccess) ptr = nullptr;
    if (ptr) {
        h->bufs.push_back({ptr, bytes});
        h->bytes += bytes;
    }
    return ptr;
}

static void dev_free(fciqmc_handle *h, void *ptr)
{
    if (!ptr) return;
    for (size_t i = 0; i < h->bufs.size(); i++)
        if (h->bufs[i].p == ptr) {
            h->bytes -= h->bufs[i].bytes;
            h->bufs.erase(h->bufs.begin() + i);
            break;
        }
    if (h->p.free) h->p.free(ptr, h->p.alloc_ctx);
    else cudaFree(ptr);
}

static int64_t pair_index(int64_t i, int64_t j) { return i >= j ? i * (i + 1) / 2 + j : j * (j + 1) / 2 + i; }

// binary64 -> (mantissa, exponent) with x = m 2^e, m odd (or 0)
static void decompose(double x, u64 *m, int *e)
{
    u64 bits;
    memcpy(&bits, &x, 8);
    int ex = (int)((bits >> 52) & 0x7ff);
    u64 mm = bits & 0xFFFFFFFFFFFFFULL;
    int ee;
    if (ex == 0) ee = -1074; else { mm |= 1ULL << 52; ee = ex - 1075; }
    if (mm == 0) { *m = 0; *e = 0; return; }
    while (!(mm & 1ULL)) { mm >>= 1; ee++; }
    *m = mm;
    *e = ee;
}

// exact placement of x on the grid 2^-F (caller guarantees it fits)
static i128 host_fixed(double x, int F)
{
    u64 m;
    int e;
    decompose(x, &m, &e);
    if (m == 0) return 0;
    int sh = e + F;
    u128 v = sh >= 0 ? ((u128)m << sh) : (u128)(m >> (-sh));
    return std::signbit(x) ? -(i128)v : (i128)v;
}

// nearest binary64 to v 2^-F, ties to even
static double host_fixed_to_double(i128 v, int F)
{
    if (v == 0) return 0.0;
    bool neg = v < 0;
    u128 u = neg ? (u128)(-v) : (u128)v;
    int msb = 127;
    while (!((u >> msb) & 1)) msb--;
    u64 mant;
    int e2;
    if (msb <= 52) { mant = (u64)u; e2 = 0; }
    else {
        int sh = msb - 52;
        u128 q = u >> sh;
        mant = (u64)q;
        u128 rem = u - (q << sh), half = (u128)1 << (sh - 1);
        if (rem > half || (rem == half && (mant & 1))) mant++;
        e2 = sh;
    }
    double r = std::ldexp((double)mant, e2 - F);
    return neg ? -r : r;
}

static int exponent_of(double x)
{
    int e;
    std::frexp(x, &e);
    return e - 1;  // x in [2^e, 2^(e+1))
}

// generation probability of class c (App. A uniform generator, spin-conditioned)
static double pgen_class(const fciqmc_handle *h, int c)
{
    int n = h->na + h->nb, N = h->norb;
    int64_t ma = N - h->na, mb = N - h->nb, nn = (int64_t)n * (n - 1);
    double ps = h->p.p_single;
    switch (c) {
    case CLS_SINGLE_A: return ps / ((double)n * (double)ma);
    case CLS_SINGLE_B: return ps / ((double)n * (double)mb);
    case CLS_DOUBLE_AB: return ((1.0 - ps) * 2.0) / ((double)nn * (double)(ma * mb));
    case CLS_DOUBLE_AA: return ((1.0 - ps) * 4.0) / ((double)nn * (double)(ma * (ma - 1)));
    case CLS_DOUBLE_BB: return ((1.0 - ps) * 4.0) / ((double)nn * (double)(mb * (mb - 1)));
    case CLS_HOP: return 1.0 / ((double)n * (double)h->z);
    }
    return 0.0;
}

// ------------------------------------------------------------------ layout
static int alloc_layout(fciqmc_handle *h, DevInst &I, int bb)
{
    const size_t nbk = (size_t)1 << bb;
    const size_t nm = nbk * CAP_M, ns = nbk * (size_t)I.cap_s;
    for (int k = 0; k < 2; k++) {
        I.key[k] = (ulonglong2 *)dev_alloc(h, nm * sizeof(ulonglong2));
        I.c[k] = (double *)dev_alloc(h, nm * sizeof(double));
        I.hd[k] = (double *)dev_alloc(h, nm * sizeof(double));
        I.fl[k] = (uint8_t *)dev_alloc(h, nm);
        I.cnt[k] = (int *)dev_alloc(h, nbk * sizeof(int));
        if (!I.key[k] || !I.c[k] || !I.hd[k] || !I.fl[k] || !I.cnt[k]) return FCIQMC_ERR_OUT_OF_MEMORY;
        if (cudaMemsetAsync(I.cnt[k], 0, nbk * sizeof(int), h->stream) != cudaSuccess) return FCIQMC_ERR_CUDA;
    }
    I.skey = (ulonglong2 *)dev_alloc(h, ns * sizeof(ulonglong2));
    I.sw = (double *)dev_alloc(h, ns * sizeof(double));
    I.scnt_i = (int *)dev_alloc(h, nbk * sizeof(int));
    I.scnt_n = (int *)dev_alloc(h, nbk * sizeof(int));
    I.part = (Partial *)dev_alloc(h, nbk * sizeof(Partial));
    I.big_list = (int *)dev_alloc(h, nbk * sizeof(int));
    I.newdet = (unsigned *)dev_alloc(h, nm * sizeof(unsigned));
    if (!I.skey || !I.sw || !I.scnt_i || !I.scnt_n || !I.part || !I.big_list || !I.newdet) return FCIQMC_ERR_OUT_OF_MEMORY;
    if (h->p.adaptive_shift)
        for (int k = 0; k < 2; k++) {
            I.facc[k] = (u64 *)dev_alloc(h, nm * 4 * sizeof(u64));
            I.kidx[k] = (unsigned short *)dev_alloc(h, nbk * KIDX * sizeof(unsigned short));
            if (!I.facc[k] || !I.kidx[k]) return FCIQMC_ERR_OUT_OF_MEMORY;
            if (cudaMemsetAsync(I.kidx[k], 0, nbk * KIDX * sizeof(unsigned short), h->stream) != cudaSuccess ||
                cudaMemsetAsync(I.facc[k], 0, nm * 4 * sizeof(u64), h->stream) != cudaSuccess)
                return FCIQMC_ERR_CUDA;
        }
    cudaMemsetAsync(I.scnt_i, 0, nbk * sizeof(int), h->stream);
    cudaMemsetAsync(I.scnt_n, 0, nbk * sizeof(int), h->stream);
    cudaMemsetAsync(I.part, 0, nbk * sizeof(Partial), h->stream);
    I.bb = bb;
    I.unit0 = 0;
    return FCIQMC_OK;
}

static void free_layout(fciqmc_handle *h, DevInst &I)
{
    for (int k = 0; k < 2; k++) {
        dev_free(h, I.key[k]); dev_free(h, I.c[k]); dev_free(h, I.hd[k]); dev_free(h, I.fl[k]); dev_free(h, I.cnt[k]);
        I.key[k] = nullptr; I.c[k] = nullptr; I.hd[k] = nullptr; I.fl[k] = nullptr; I.cnt[k] = nullptr;
    }
    dev_free(h, I.skey); dev_free(h, I.sw); dev_free(h, I.scnt_i); dev_free(h, I.scnt_n); dev_free(h, I.part);
    dev_free(h, I.big_list); dev_free(h, I.newdet);
    for (int k = 0; k < 2; k++) {
        dev_free(h, I.facc[k]); dev_free(h, I.kidx[k]);
        I.facc[k] = nullptr; I.kidx[k] = nullptr;
    }
    I.skey = nullptr; I.sw = nullptr; I.scnt_i = nullptr; I.scnt_n = nullptr; I.part = nullptr; I.big_list = nullptr;
    I.newdet = nullptr;
}

static int upload_inst(fciqmc_handle *h)
{
    CUDA_TRY(h, cudaMemcpyAsync(h->dinst, &h->hi, sizeof(DevInst), cudaMemcpyHostToDevice, h->stream));
    int us[2] = {0, 1 << h->bb};
    CUDA_TRY(h, cudaMemcpyAsync(h->dunit, us, sizeof(us), cudaMemcpyHostToDevice, h->stream));
    if (h->p.adaptive_shift && h->kidx_dirty) {  // index of the current list, zeroed weight sums
        launch_build_kidx(h->dinst, h->hst.parity, 1 << h->bb, h->stream);
        CUDA_TRY(h, cudaGetLastError());
        h->kidx_dirty = false;
    }
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    return FCIQMC_OK;
}

static int enqueue_iteration(fciqmc_handle *h, cudaEvent_t *ev)
{
    const int units = 1 << h->bb;
    if (ev) cudaEventRecord(ev[0], h->stream);
    const bool st = staged_spawn_fits(h->hi), split = st && h->hi.qcnt != nullptr && spawn_split_selected();
    launch_spawn(h->dinst, h->dunit, 1, units, st, split, h->stream);
    if (split) launch_spawn_eval(h->dinst, 1, h->stream);
    if (ev) cudaEventRecord(ev[1], h->stream);
    launch_spawn_heavy(h->dinst, 1, h->stream);
    if (ev) cudaEventRecord(ev[2], h->stream);
    if (h->nd > 0) launch_semistoch(h->dinst, 1, h->nd, h->stream);
    if (ev) cudaEventRecord(ev[3], h->stream);
    cudaError_t e = launch_annihilate(h->dinst, h->dunit, 1, units, h->hi.side || h->hi.adaptive,
                                      staged_annihilation_fits(h->hi), h->stream);
    if (e != cudaSuccess) return fail(h, FCIQMC_ERR_CUDA, std::string("annihilation launch: ") + cudaGetErrorString(e));
    launch_annihilate_big(h->dinst, 1, h->stream);
    if (ev) cudaEventRecord(ev[4], h->stream);
    launch_new_diag(h->dinst, 1, h->stream);
    if (ev) cudaEventRecord(ev[5], h->stream);
    launch_finalize(h->dinst, 1, h->stream);
    if (ev) cudaEventRecord(ev[6], h->stream);
    return FCIQMC_OK;
}

// kernel launches recorded in a captured graph
static int count_kernel_nodes(cudaGraph_t g)
{
    size_t n = 0;
    if (cudaGraphGetNodes(g, nullptr, &n) != cudaSuccess || n == 0) return 0;
    std::vector<cudaGraphNode_t> nodes(n);
    if (cudaGraphGetNodes(g, nodes.data(), &n) != cudaSuccess) return 0;
    int k = 0;
    for (size_t i = 0; i < n; i++) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(nodes[i], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) k++;
    }
    return k;
}

// the attempt queues of split spawning, allocated when that mode is selected
// (and the run's arrays suit the staged kernels): min(draw grid, buckets)
// segments per class, each sized from the requested count (need, per class),
// at least 4096 entries (two determinants' worth of light attempts)
static int ensure_queues(fciqmc_handle *h, long long need0 = 0, long long need1 = 0)
{
    DevInst &I = h->hi;
    if (!spawn_split_selected() || !staged_spawn_fits(I)) return FCIQMC_OK;
    bool changed = false;
    const int nseg = std::min(draw_segments(), 1 << h->bb);
    if (I.qcnt && I.qnseg != nseg) {  // more buckets or another grid: new queues
        dev_free(h, I.qcnt);
        dev_free(h, I.qrec[0]);
        dev_free(h, I.qrec[1]);
        I.qcnt = nullptr;
        I.qrec[0] = I.qrec[1] = nullptr;
        I.qcap[0] = I.qcap[1] = 0;
    }
    if (!I.qcnt) {
        I.qcnt = (int *)dev_alloc(h, 2 * (size_t)nseg * sizeof(int));
        if (!I.qcnt) return fail(h, FCIQMC_ERR_OUT_OF_MEMORY, "out of device memory (attempt queues)");
        CUDA_TRY(h, cudaMemsetAsync(I.qcnt, 0, 2 * (size_t)nseg * sizeof(int), h->stream));
        I.qnseg = nseg;
        changed = true;
    }
    const long long want[2] = {std::max<long long>(4096, need0), std::max<long long>(4096, need1)};
    for (int c = 0; c < 2; c++) {
        if (I.qrec[c] && I.qcap[c] >= want[c]) continue;
        long long cap = I.qcap[c] > 0 ? I.qcap[c] : 4096;
        while (cap < want[c]) cap = cap + cap / 2;
        if (cap > (1LL << 30)) return fail(h, FCIQMC_ERR_CAPACITY, "attempt queue limit reached");
        dev_free(h, I.qrec[c]);
        I.qrec[c] = (QRec *)dev_alloc(h, (size_t)nseg * (size_t)cap * sizeof(QRec));
        if (!I.qrec[c]) {
            I.qcap[c] = 0;
            return fail(h, FCIQMC_ERR_OUT_OF_MEMORY, "out of device memory (attempt queues)");
        }
        I.qcap[c] = cap;
        changed = true;
    }
    return changed ? upload_inst(h) : FCIQMC_OK;  // the device copy of the descriptor follows
}

static int capture_graph(fciqmc_handle *h)
{
    if (h->graph) { cudaGraphExecDestroy(h->graph); h->graph = nullptr; }
    cudaGraph_t g;
    {
        const int rq = ensure_queues(h);
        if (rq) return rq;
    }
    CUDA_TRY(h, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
    int rc = enqueue_iteration(h, nullptr);
    cudaError_t e = cudaStreamEndCapture(h->stream, &g);
    if (rc) return rc;
    if (e != cudaSuccess) return fail(h, FCIQMC_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    h->graph_kernels = count_kernel_nodes(g);
    h->graph_gen = launch_geometry_generation();
    e = cudaGraphInstantiate(&h->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(h, FCIQMC_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    return FCIQMC_OK;
}

static int read_state(fciqmc_handle *h)
{
    CUDA_TRY(h, cudaMemcpyAsync(&h->hst, h->dstate, sizeof(IterState), cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    return FCIQMC_OK;
}

static int write_state(fciqmc_handle *h)
{
    CUDA_TRY(h, cudaMemcpyAsync(h->dstate, &h->hst, sizeof(IterState), cudaMemcpyHostToDevice, h->stream));
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    return FCIQMC_OK;
}

// split every bucket in two (one more hash bit)
static int grow_buckets(fciqmc_handle *h)
{
    if (h->bb >= MAX_BB) return fail(h, FCIQMC_ERR_CAPACITY, "walker list exceeds 2^22 buckets");
    DevInst nI = h->hi;
    if (nI.cap_s > CAP_S0) nI.cap_s /= 2;  // each new bucket receives about half the spawns
    int rc = alloc_layout(h, nI, h->bb + 1);
    if (rc) return fail(h, rc, "out of device memory while growing the walker buffers");
    DevInst *tmp = (DevInst *)dev_alloc(h, 2 * sizeof(DevInst));
    if (!tmp) return fail(h, FCIQMC_ERR_OUT_OF_MEMORY, "out of device memory");
    CUDA_TRY(h, cudaMemcpyAsync(tmp, &h->hi, sizeof(DevInst), cudaMemcpyHostToDevice, h->stream));
    CUDA_TRY(h, cudaMemcpyAsync(tmp + 1, &nI, sizeof(DevInst), cudaMemcpyHostToDevice, h->stream));
    const int par = h->hst.parity;
    launch_rebucket(tmp, tmp + 1, 1 << h->bb, par, h->stream);
    if (h->p.adaptive_shift) launch_build_kidx(tmp + 1, par, 1 << nI.bb, h->stream);
    CUDA_TRY(h, cudaGetLastError());
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    int rc2 = read_state(h);
    if (rc2) return rc2;
    dev_free(h, tmp);
    free_layout(h, h->hi);
    h->hi = nI;
    h->bb = nI.bb;
    if (h->hst.err & ERRB_MAIN_CAP) return fail(h, FCIQMC_ERR_CAPACITY, "bucket overflow while splitting");
    return FCIQMC_OK;
}

// larger spawn regions per bucket; buckets that no longer fit in shared
// memory are annihilated from a global scratch slice per block
static int grow_spawn_capacity(fciqmc_handle *h, long long need)
{
    DevInst &I = h->hi;
    const size_t nbk = (size_t)1 << h->bb;
    long long want = std::max<long long>(2LL * I.cap_s, need + need / 4);
    int ncap = I.cap_s;
    while (ncap < want && ncap < (1 << 30)) ncap *= 2;
    if ((size_t)ncap * nbk > ((size_t)1 << 33)) return fail(h, FCIQMC_ERR_CAPACITY, "spawn buffer limit reached");
    ulonglong2 *nk = (ulonglong2 *)dev_alloc(h, nbk * (size_t)ncap * sizeof(ulonglong2));
    double *nw = (double *)dev_alloc(h, nbk * (size_t)ncap * sizeof(double));
    const int Ecap = CAP_M + ncap;
    int tabbits = TABBITS;
    while ((1 << tabbits) < 2 * Ecap) tabbits++;
    size_t stride = (size_t)Ecap * (sizeof(ulonglong2) + sizeof(double) + 8 + 8 + 4 + 4 + 4) + ((size_t)4 << tabbits);
    stride = (stride + 255) & ~(size_t)255;
    unsigned char *scr = (unsigned char *)dev_alloc(h, stride * BIG_BLOCKS);
    if (!nk || !nw || !scr) return fail(h, FCIQMC_ERR_OUT_OF_MEMORY, "out of device memory (spawn buffers)");
    dev_free(h, I.skey); dev_free(h, I.sw); dev_free(h, I.big_scratch);
    I.skey = nk; I.sw = nw; I.cap_s = ncap;
    I.big_scratch = scr; I.big_stride = stride; I.big_tabbits = tabbits;
    return FCIQMC_OK;
}

// per-bucket determinant lists of a replica pair, sized for the current layout
static int ensure_side(fciqmc_handle *h)
{
    if (!h->paired) return FCIQMC_OK;
    DevInst &I = h->hi;
    const int nbk = 1 << h->bb, cap = CAP_M + I.cap_s;
    if (I.side && I.side_cap == cap && h->side_nbk == nbk) return FCIQMC_OK;
    dev_free(h, I.side);
    dev_free(h, I.side_cnt);
    I.side = (SideEnt *)dev_alloc(h, (size_t)nbk * cap * sizeof(SideEnt));
    I.side_cnt = (int *)dev_alloc(h, (size_t)nbk * sizeof(int));
    if (!I.side || !I.side_cnt) return fail(h, FCIQMC_ERR_OUT_OF_MEMORY, "out of device memory (replica lists)");
    CUDA_TRY(h, cudaMemsetAsync(I.side_cnt, 0, (size_t)nbk * sizeof(int), h->stream));
    I.side_cap = cap;
    h->side_nbk = nbk;
    return FCIQMC_OK;
}

static int grow_heavy(fciqmc_handle *h)
{
    int ncap = h->heavy_cap * 4;
    HeavyChunk *nh = (HeavyChunk *)dev_alloc(h, (size_t)ncap * sizeof(HeavyChunk));
    if (!nh) return fail(h, FCIQMC_ERR_OUT_OF_MEMORY, "out of device memory (heavy queue)");
    dev_free(h, h->hi.heavy);
    h->hi.heavy = nh;
    h->hi.heavy_cap = ncap;
    h->heavy_cap = ncap;
    return FCIQMC_OK;
}

static int reset_after_error(fciqmc_handle *h)
{
    const size_t nbk = (size_t)1 << h->bb;
    CUDA_TRY(h, cudaMemsetAsync(h->hi.scnt_i, 0, nbk * sizeof(int), h->stream));
    CUDA_TRY(h, cudaMemsetAsync(h->hi.scnt_n, 0, nbk * sizeof(int), h->stream));
    h->hst.err = 0;
    h->hst.heavy_n = 0;
    h->hst.big_n = 0;
    h->hst.need_spawn = 0;
    h->hst.need_main = 0;
    h->hst.n_spawn_over = 0;
    h->hst.new_n = 0;
    h->hst.need_queue[0] = 0;
    h->hst.need_queue[1] = 0;
    if (h->hi.qcnt) CUDA_TRY(h, cudaMemsetAsync(h->hi.qcnt, 0, 2 * (size_t)h->hi.qnseg * sizeof(int), h->stream));
    CUDA_TRY(h, cudaMemsetAsync(h->hi.acc, 0, NSHARD * ACC_STRIDE * sizeof(u64), h->stream));  // partial totals
    // the failed iteration's adaptive-shift weight sums are discarded when the
    // descriptor is next uploaded (the device copy may still describe an old
    // layout here)
    h->kidx_dirty = true;
    return write_state(h);
}

static int pull_history(fciqmc_handle *h, long long from, long long to)
{
    if (to <= from) return FCIQMC_OK;
    std::vector<fciqmc_iter_stats> rows((size_t)(to - from));
    for (long long it = from; it < to;) {
        long long slot = it % h->ring_cap;
        long long n = std::min<long long>(to - it, h->ring_cap - slot);
        CUDA_TRY(h, cudaMemcpyAsync(rows.data() + (it - from), h->hi.ring + slot, n * sizeof(fciqmc_iter_stats),
                                    cudaMemcpyDeviceToHost, h->stream));
        it += n;
    }
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    // the history is indexed by iteration; a retried iteration overwrites,
    // and rows that fell out of the ring are kept as placeholders
    if ((long long)h->hist.size() > from) h->hist.resize((size_t)from);
    while ((long long)h->hist.size() < from) {
        fciqmc_iter_stats z;
        memset(&z, 0, sizeof z);
        z.iteration = -1;
        h->hist.push_back(z);
    }
    h->hist.insert(h->hist.end(), rows.begin(), rows.end());
    return FCIQMC_OK;
}

// ------------------------------------------------------------------ semi-stochastic set-up (Sec. III)
// D = the N_D determinants of largest |C| (ties: ascending key), found by a
// 16-bit-digit radix selection over the bit patterns of |C| on the device;
// H^D in CSR built on the device; the main list flags D and pins it.
// the `count` determinants of largest |C| (ties: ascending key), returned
// in ascending key order: a radix selection on the bit patterns of |C|
// (16-bit digit histograms on the device), then the ties at the threshold
static int select_top(fciqmc_handle *h, long long count, std::vector<ulonglong2> &sel, long long *nsel)
{
    const int par = h->hst.parity, nbk = 1 << h->bb;
    std::vector<int> cnt(nbk);
    CUDA_TRY(h, cudaMemcpy(cnt.data(), h->hi.cnt[par], nbk * sizeof(int), cudaMemcpyDeviceToHost));
    long long ndet = 0;
    for (int c : cnt) ndet += c;
    const long long nd = std::min<long long>(count, ndet);
    *nsel = nd;
    sel.clear();
    if (nd <= 0) return FCIQMC_OK;
    unsigned *dhist = (unsigned *)dev_alloc(h, 65536 * sizeof(unsigned));
    if (!dhist) return fail(h, FCIQMC_ERR_OUT_OF_MEMORY, "out of device memory (selection)");
    std::vector<unsigned> hist(65536);
    u64 prefix = 0;
    long long need = nd, ties = 0;
    for (int shift = 0; shift < 64; shift += 16) {
        CUDA_TRY(h, cudaMemsetAsync(dhist, 0, 65536 * sizeof(unsigned), h->stream));
        launch_abs_hist(h->dinst, par, nbk, shift, prefix, dhist, h->stream);
        CUDA_TRY(h, cudaMemcpyAsync(hist.data(), dhist, 65536 * sizeof(unsigned), cudaMemcpyDeviceToHost, h->stream));
        CUDA_TRY(h, cudaStreamSynchronize(h->stream));
        long long acc = 0;
        int d = 65535;
        for (; d > 0; d--) {
            if (acc + hist[d] >= need) break;
            acc += hist[d];
        }
        need -= acc;
        ties = hist[d];
        prefix = (prefix << 16) | (u64)d;
    }
    const u64 thr = prefix;  // bit pattern of the count-th largest |C|
    const int cap = (int)(nd - need + ties);
    ulonglong2 *ckeys = (ulonglong2 *)dev_alloc(h, (size_t)cap * sizeof(ulonglong2));
    u64 *cmags = (u64 *)dev_alloc(h, (size_t)cap * sizeof(u64));
    int *dn = (int *)dev_alloc(h, sizeof(int));
    if (!ckeys || !cmags || !dn) return fail(h, FCIQMC_ERR_OUT_OF_MEMORY, "out of device memory (selection)");
    CUDA_TRY(h, cudaMemsetAsync(dn, 0, sizeof(int), h->stream));
    launch_abs_collect(h->dinst, par, nbk, thr, ckeys, cmags, dn, cap, h->stream);
    std::vector<ulonglong2> keys(cap);
    std::vector<u64> mags(cap);
    int ncol = 0;
    CUDA_TRY(h, cudaMemcpyAsync(&ncol, dn, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(h, cudaMemcpyAsync(keys.data(), ckeys, (size_t)cap * sizeof(ulonglong2), cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(h, cudaMemcpyAsync(mags.data(), cmags, (size_t)cap * sizeof(u64), cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    if (ncol != cap) return fail(h, FCIQMC_ERR_CUDA, "selection count mismatch");
    std::vector<ulonglong2> tie;
    for (int i = 0; i < cap; i++) (mags[i] > thr ? sel : tie).push_back(keys[i]);
    auto kless = [](const ulonglong2 &x, const ulonglong2 &y) { return x.x < y.x || (x.x == y.x && x.y < y.y); };
    std::sort(tie.begin(), tie.end(), kless);
    for (long long i = 0; i < need; i++) sel.push_back(tie[(size_t)i]);
    std::sort(sel.begin(), sel.end(), kless);
    dev_free(h, dhist); dev_free(h, ckeys); dev_free(h, cmags); dev_free(h, dn);
    return FCIQMC_OK;
}

// H^S (diagonal relative to E_ref) of the sorted keys dkey in CSR on the device
static int build_hsub(fciqmc_handle *h, const ulonglong2 *dkey, long long nd, long long **rowptr, int **dcol,
                      double **dval, long long *nnz_out)
{
    long long *rowcnt = (long long *)dev_alloc(h, (size_t)nd * sizeof(long long));
    *rowptr = (long long *)dev_alloc(h, (size_t)(nd + 1) * sizeof(long long));
    if (!rowcnt || !*rowptr) return fail(h, FCIQMC_ERR_OUT_OF_MEMORY, "out of device memory (sparse H)");
    launch_build_hd(h->dinst, (int)nd, dkey, rowcnt, nullptr, nullptr, nullptr, 0, h->stream);
    std::vector<long long> rc((size_t)nd), rp((size_t)nd + 1, 0);
    CUDA_TRY(h, cudaMemcpyAsync(rc.data(), rowcnt, (size_t)nd * sizeof(long long), cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    for (long long r = 0; r < nd; r++) rp[r + 1] = rp[r] + rc[r];
    const long long nnz = rp[nd];
    *dcol = (int *)dev_alloc(h, (size_t)std::max(1LL, nnz) * sizeof(int));
    *dval = (double *)dev_alloc(h, (size_t)std::max(1LL, nnz) * sizeof(double));
    if (!*dcol || !*dval) return fail(h, FCIQMC_ERR_OUT_OF_MEMORY, "out of device memory (sparse H)");
    CUDA_TRY(h, cudaMemcpy(*rowptr, rp.data(), (size_t)(nd + 1) * sizeof(long long), cudaMemcpyHostToDevice));
    launch_build_hd(h->dinst, (int)nd, dkey, rowcnt, *rowptr, *dcol, *dval, 1, h->stream);
    CUDA_TRY(h, cudaGetLastError());
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    dev_free(h, rowcnt);
    *nnz_out = nnz;
    return FCIQMC_OK;
}

static int build_semistochastic(fciqmc_handle *h)
{
    DevInst &I = h->hi;
    const int par = h->hst.parity, nbk = 1 << h->bb;
    h->hst.semi_built = 1;
    std::vector<ulonglong2> sel;
    long long nd = 0;
    int rcs = select_top(h, h->p.semistoch_size, sel, &nd);
    if (rcs) return rcs;
    if (nd <= 0) return FCIQMC_OK;
    // open-addressing set of D keys
    int hb = 1;
    while ((1LL << hb) < 2 * nd) hb++;
    std::vector<u64> tabk((size_t)2 << hb, 0ULL);
    std::vector<int> tabi((size_t)1 << hb, -1);  // position of the key in D (ascending key order)
    for (size_t q = 0; q < sel.size(); q++) {
        const auto &k = sel[q];
        u64 sl = det_hash_host(k.x, k.y) & (((u64)1 << hb) - 1);
        while (tabk[2 * sl] || tabk[2 * sl + 1]) sl = (sl + 1) & (((u64)1 << hb) - 1);
        tabk[2 * sl] = k.x;
        tabk[2 * sl + 1] = k.y;
        tabi[sl] = (int)q;
    }
    ulonglong2 *dkey = (ulonglong2 *)dev_alloc(h, (size_t)nd * sizeof(ulonglong2));
    u64 *dtab = (u64 *)dev_alloc(h, tabk.size() * sizeof(u64));
    int *dtabi = (int *)dev_alloc(h, tabi.size() * sizeof(int));
    double *dcn = (double *)dev_alloc(h, (size_t)nd * sizeof(double));
    double *dcc = (double *)dev_alloc(h, (size_t)nd * sizeof(double));
    double *dcc2 = (double *)dev_alloc(h, (size_t)nd * sizeof(double));
    if (!dkey || !dtab || !dtabi || !dcn || !dcc || !dcc2)
        return fail(h, FCIQMC_ERR_OUT_OF_MEMORY, "out of device memory (D)");
    CUDA_TRY(h, cudaMemcpy(dkey, sel.data(), (size_t)nd * sizeof(ulonglong2), cudaMemcpyHostToDevice));
    CUDA_TRY(h, cudaMemcpy(dtab, tabk.data(), tabk.size() * sizeof(u64), cudaMemcpyHostToDevice));
    CUDA_TRY(h, cudaMemcpy(dtabi, tabi.data(), tabi.size() * sizeof(int), cudaMemcpyHostToDevice));
    long long *rowptr = nullptr, nnz = 0;
    int *dcol = nullptr;
    double *dval = nullptr;
    rcs = build_hsub(h, dkey, nd, &rowptr, &dcol, &dval, &nnz);
    if (rcs) return rcs;
    I.nd = (int)nd; I.dkey = dkey; I.drow = rowptr; I.dcol = dcol; I.dval = dval; I.dc_new = dcn;
    I.dc_buf[0] = dcc; I.dc_buf[1] = dcc2;
    I.dhash_keys = dtab; I.dhash_idx = dtabi; I.dhash_bits = hb;
    int rc2 = upload_inst(h);
    if (rc2) return rc2;
    launch_mark_d(h->dinst, par, nbk, h->stream);
    CUDA_TRY(h, cudaGetLastError());
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    h->nd = (int)nd;
    h->nnz = nnz;
    return capture_graph(h);
}

// trial-wave-function estimator (Sec. IV): T, H^T, its lowest eigenvector,
// and the table of W_j over T and the space connected to it
static int build_trial(fciqmc_handle *h)
{
    DevInst &I = h->hi;
    h->hst.trial_built = 1;
    std::vector<ulonglong2> sel;
    long long nt = 0;
    int rc = select_top(h, h->p.trial_size, sel, &nt);
    if (rc) return rc;
    if (nt <= 0) return FCIQMC_OK;
    ulonglong2 *tkey = (ulonglong2 *)dev_alloc(h, (size_t)nt * sizeof(ulonglong2));
    double *cT = (double *)dev_alloc(h, (size_t)nt * sizeof(double));
    double *hdiag = (double *)dev_alloc(h, (size_t)nt * sizeof(double));
    double *dE = (double *)dev_alloc(h, sizeof(double));
    int *dsw = (int *)dev_alloc(h, 2 * sizeof(int));
    if (!tkey || !cT || !hdiag || !dE || !dsw) return fail(h, FCIQMC_ERR_OUT_OF_MEMORY, "out of device memory (trial space)");
    CUDA_TRY(h, cudaMemcpy(tkey, sel.data(), (size_t)nt * sizeof(ulonglong2), cudaMemcpyHostToDevice));
    long long *rowptr = nullptr, nnz = 0;
    int *col = nullptr;
    double *val = nullptr;
    rc = build_hsub(h, tkey, nt, &rowptr, &col, &val, &nnz);
    if (rc) return rc;
    // dense H^T (order padded to even), lowest eigenpair
    const int n2 = (int)(nt + (nt & 1));
    double *A = (double *)dev_alloc(h, (size_t)n2 * n2 * sizeof(double));
    double *V = (double *)dev_alloc(h, (size_t)n2 * n2 * sizeof(double));
    if (!A || !V) return fail(h, FCIQMC_ERR_OUT_OF_MEMORY, "out of device memory (trial eigenproblem)");
    CUDA_TRY(h, cudaMemsetAsync(A, 0, (size_t)n2 * n2 * sizeof(double), h->stream));
    CUDA_TRY(h, launch_trial_dense(rowptr, col, val, (int)nt, n2, A, hdiag, h->stream));
    CUDA_TRY(h, launch_jacobi_lowest(A, V, (int)nt, n2, dE, cT, dsw, h->stream));
    int sweeps = 0;
    CUDA_TRY(h, cudaMemcpyAsync(&h->trial_ET, dE, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(h, cudaMemcpyAsync(&sweeps, dsw, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    if (sweeps >= 60) return fail(h, FCIQMC_ERR_NUMERIC, "trial eigenproblem did not converge");
    dev_free(h, A); dev_free(h, V); dev_free(h, rowptr); dev_free(h, col); dev_free(h, val);
    // W table: at most nt (connections + 1) determinants, at most half full
    const long long per = connections_per_det(h->na, h->nb, h->norb - h->na, h->norb - h->nb);
    int bits = 4;
    while ((1LL << bits) < 2 * nt * (per + 1) && bits < 40) bits++;
    const size_t slots = (size_t)1 << bits;
    unsigned *state = (unsigned *)dev_alloc(h, slots * sizeof(unsigned));
    TrialEnt *tab = (TrialEnt *)dev_alloc(h, slots * sizeof(TrialEnt));
    unsigned long long *dcount = (unsigned long long *)dev_alloc(h, sizeof(unsigned long long));
    int *derr = (int *)dev_alloc(h, sizeof(int));
    if (!state || !tab || !dcount || !derr) return fail(h, FCIQMC_ERR_OUT_OF_MEMORY, "out of device memory (trial table)");
    CUDA_TRY(h, cudaMemsetAsync(state, 0, slots * sizeof(unsigned), h->stream));
    CUDA_TRY(h, cudaMemsetAsync(tab, 0, slots * sizeof(TrialEnt), h->stream));
    CUDA_TRY(h, cudaMemsetAsync(dcount, 0, sizeof(unsigned long long), h->stream));
    CUDA_TRY(h, cudaMemsetAsync(derr, 0, sizeof(int), h->stream));
    CUDA_TRY(h, launch_trial_w(h->dinst, tkey, cT, hdiag, (int)nt, per, state, tab, bits, dcount, derr, h->stream));
    unsigned long long cnt = 0;
    int terr = 0;
    CUDA_TRY(h, cudaMemcpyAsync(&cnt, dcount, sizeof(cnt), cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(h, cudaMemcpyAsync(&terr, derr, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    if (terr) return fail(h, FCIQMC_ERR_TIMEOUT, "trial table construction failed (wait limit or table full)");
    h->trial_nt = nt;
    h->trial_nw = (long long)cnt;
    h->trial_key = tkey;
    h->trial_cT = cT;
    I.trial_bits = bits;
    I.trial_state = state;
    I.trial_tab = tab;
    int rc2 = upload_inst(h);
    if (rc2) return rc2;
    return capture_graph(h);
}

// ------------------------------------------------------------------ C ABI
extern "C" {

const char *fciqmc_last_error(const fciqmc_handle *h) { return h ? h->err.c_str() : g_create_error.c_str(); }

static void destroy_run(fciqmc_handle *h)
{
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    if (h->graph) cudaGraphExecDestroy(h->graph);
    while (!h->bufs.empty()) dev_free(h, h->bufs.back().p);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    delete h;
}

// the second replica of a pair belongs to the first and is released with it
void fciqmc_destroy(fciqmc_handle *h)
{
    if (!h || h->secondary) return;
    if (h->partner) destroy_run(h->partner);
    destroy_run(h);
}

fciqmc_handle *fciqmc_replica(fciqmc_handle *h, int32_t r)
{
    if (!h || h->secondary) return nullptr;
    if (r == 0) return h;
    if (r == 1) return h->partner;
    return nullptr;
}

static int create_run(const fciqmc_system *sys, const fciqmc_params *prm, u64 replica, fciqmc_handle **out)
{
    if (!out) return fail(nullptr, FCIQMC_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!sys || !prm) return fail(nullptr, FCIQMC_ERR_INVALID_ARG, "system or params is NULL");
    fciqmc_handle *h = new fciqmc_handle();
    h->p = *prm;
    auto bail = [&](int rc, const std::string &msg) {
        g_create_error = msg;
        fciqmc_destroy(h);
        return rc;
    };
    const fciqmc_params &P = h->p;
    if (!(P.tau == P.tau) || !(P.c_min > 0.0) || !(P.initial_walkers > 0.0) || P.shift_interval < 1 ||
        !(P.p_single >= 0.0 && P.p_single <= 1.0) || !(P.initiator_threshold >= 0.0) || !(P.shift_damping >= 0.0) ||
        !(P.target_walkers > 0.0) || !std::isfinite(P.initial_shift))
        return bail(FCIQMC_ERR_INVALID_ARG, "invalid parameters (tau, c_min, initial_walkers, shift_interval, p_single, "
                                            "initiator_threshold, shift_damping, target_walkers must be positive/finite)");
    if (P.trial_size < 0 || P.trial_size > 1024 || (P.trial_size > 0 && P.trial_start < 1))
        return bail(FCIQMC_ERR_INVALID_ARG, "trial_size must be in [0, 1024] and trial_start >= 1");
    h->kind = sys->kind;
    h->na = sys->n_alpha;
    h->nb = sys->n_beta;
    h->ecore = sys->ecore;
    int N;
    if (sys->kind == FCIQMC_ABINITIO) {
        N = sys->norb;
        if (N < 1 || N > 64 || !sys->h1 || !sys->eri) return bail(FCIQMC_ERR_INVALID_ARG, "ab initio system needs 1 <= norb <= 64, h1 and eri");
        int64_t np = (int64_t)N * (N + 1) / 2, ne = np * (np + 1) / 2;
        h->h.assign(sys->h1, sys->h1 + (size_t)N * N);
        h->eri.assign(sys->eri, sys->eri + ne);
    } else if (sys->kind == FCIQMC_HUBBARD) {
        int lx = sys->lx, ly = sys->ly;
        N = lx * ly;
        if (lx < 1 || ly < 1 || N > 64 || (sys->periodic_x && lx == 2) || (sys->periodic_y && ly == 2))
            return bail(FCIQMC_ERR_INVALID_ARG, "Hubbard lattice needs lx*ly <= 64 and periodic lengths of 1 or >= 3");
        h->z = ly > 1 ? 4 : 2;
        h->t = sys->t;
        h->U = sys->U;
        h->nbr.assign((size_t)4 * N, -1);
        for (int y = 0; y < ly; y++)
            for (int x = 0; x < lx; x++) {
                int p = x + lx * y;
                int *q = &h->nbr[4 * p];
                q[0] = x > 0 ? p - 1 : (sys->periodic_x && lx > 1 ? p + lx - 1 : -1);
                q[1] = x < lx - 1 ? p + 1 : (sys->periodic_x && lx > 1 ? p - (lx - 1) : -1);
                q[2] = y > 0 ? p - lx : (sys->periodic_y && ly > 1 ? p + lx * (ly - 1) : -1);
                q[3] = y < ly - 1 ? p + lx : (sys->periodic_y && ly > 1 ? p - lx * (ly - 1) : -1);
            }
        int64_t np = (int64_t)N * (N + 1) / 2, ne = np * (np + 1) / 2;
        h->h.assign((size_t)N * N, 0.0);
        h->eri.assign((size_t)ne, 0.0);
        for (int p = 0; p < N; p++)
            for (int k = 0; k < h->z; k++)
                if (h->nbr[4 * p + k] >= 0) h->h[(size_t)p * N + h->nbr[4 * p + k]] = -sys->t;
        for (int p = 0; p < N; p++) h->eri[pair_index(pair_index(p, p), pair_index(p, p))] = sys->U;
    } else {
        return bail(FCIQMC_ERR_INVALID_ARG, "unknown system kind");
    }
    h->norb = N;
    if (h->na < 0 || h->nb < 0 || h->na > N || h->nb > N || h->na + h->nb < 1)
        return bail(FCIQMC_ERR_INVALID_ARG, "electron counts out of range");
    const u64 normask = N >= 64 ? ~0ULL : ((1ULL << N) - 1);
    if (sys->has_ref) {
        h->ref_a = sys->ref_alpha;
        h->ref_b = sys->ref_beta;
    } else if (sys->kind == FCIQMC_ABINITIO) {
        h->ref_a = h->na >= 64 ? ~0ULL : ((1ULL << h->na) - 1);
        h->ref_b = h->nb >= 64 ? ~0ULL : ((1ULL << h->nb) - 1);
    } else {
        for (int y = 0; y < sys->ly; y++)
            for (int x = 0; x < sys->lx; x++) {
                if (((x + y) & 1) == 0) h->ref_a |= 1ULL << (x + sys->lx * y);
                else h->ref_b |= 1ULL << (x + sys->lx * y);
            }
    }
    if (__builtin_popcountll(h->ref_a) != h->na || __builtin_popcountll(h->ref_b) != h->nb ||
        ((h->ref_a | h->ref_b) & ~normask))
        return bail(FCIQMC_ERR_INVALID_ARG, "reference determinant does not match the electron counts");

    // exact-sum scale F: every integral (and E_core) must lie on the grid 2^-F
    int lsb_min = 0, msb_max = -1100;
    bool any = false;
    auto scan = [&](double x) {
        if (x == 0.0) return true;
        if (!std::isfinite(x)) return false;
        u64 m;
        int e;
        decompose(x, &m, &e);
        lsb_min = any ? std::min(lsb_min, e) : e;
        msb_max = any ? std::max(msb_max, exponent_of(std::fabs(x))) : exponent_of(std::fabs(x));
        any = true;
        return true;
    };
    for (double x : h->h) if (!scan(x)) return bail(FCIQMC_ERR_INVALID_ARG, "non-finite one-electron integral");
    for (double x : h->eri) if (!scan(x)) return bail(FCIQMC_ERR_INVALID_ARG, "non-finite two-electron integral");
    if (!scan(h->ecore)) return bail(FCIQMC_ERR_INVALID_ARG, "non-finite core energy");
    const int n = h->na + h->nb;
    int F = any ? std::max(0, -lsb_min) : 0;
    int terms_bits = 0;
    while ((1LL << terms_bits) < (long long)n * n + 2 * n + 4) terms_bits++;
    // Integral grid: the exact sums (H_ii, single excitations, heat-bath table
    // sums of up to N^2 terms) must fit 125 bits.  Where the integrals' own
    // finest bit lies below what that allows (FCIDUMP files print values of
    // 1e-17 .. 1e-20 next to O(10) Eh), every integral and E_core is rounded
    // to the nearest multiple of 2^-G (ties to even), G = 125 - msb - 2 -
    // max(terms, table bits), before any use; otherwise nothing changes.
    int table_bits = 0;
    while ((1LL << table_bits) < (long long)N * N) table_bits++;
    const int G = 125 - msb_max - 2 - std::max(terms_bits, table_bits + 2);
    if (any && F > G) {
        if (G < 0) return bail(FCIQMC_ERR_UNSUPPORTED, "integrals too large for the 128-bit exact accumulator");
        auto to_grid = [G](double x) { return std::ldexp(std::nearbyint(std::ldexp(x, G)), -G); };
        for (double &x : h->h) x = to_grid(x);
        for (double &x : h->eri) x = to_grid(x);
        h->ecore = to_grid(h->ecore);
        msb_max = -1100;
        any = false;
        lsb_min = 0;
        for (double x : h->h) scan(x);
        for (double x : h->eri) scan(x);
        scan(h->ecore);
        F = any ? std::max(0, -lsb_min) : 0;
    }
    if (any && msb_max + F + terms_bits + 2 > 125)
        return bail(FCIQMC_ERR_UNSUPPORTED, "integral dynamic range too wide for the 128-bit exact accumulator");
    const int ecm = exponent_of(P.c_min);
    const int Fw = 52 - ecm;
    if (Fw + 31 + 14 > 125 || Fw + 31 < 0)
        return bail(FCIQMC_ERR_UNSUPPORTED, "c_min outside the supported range (about 1e-9 .. 1e9)");

    // device, stream
    if (init_kernels() != cudaSuccess) {
        cudaGetLastError();
        return bail(FCIQMC_ERR_CUDA, "no usable CUDA device (kernel attribute setup failed)");
    }
    if (P.stream) h->stream = (cudaStream_t)P.stream;
    else {
        if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess)
            return bail(FCIQMC_ERR_CUDA, "cannot create a CUDA stream (no usable GPU?)");
        h->own_stream = true;
    }

    // fixed-point tables for the exact diagonal sums
    std::vector<ulonglong2> hfx(N), Jfx((size_t)N * N), JKfx((size_t)N * N);
    auto put = [](ulonglong2 &d, i128 v) { d.x = (u64)(u128)v; d.y = (u64)((u128)v >> 64); };
    for (int p = 0; p < N; p++) {
        put(hfx[p], host_fixed(h->h[(size_t)p * N + p], F));
        for (int q = 0; q < N; q++) {
            put(Jfx[(size_t)p * N + q], host_fixed(h->eri[pair_index(pair_index(p, p), pair_index(q, q))], F));
            put(JKfx[(size_t)p * N + q], host_fixed(h->eri[pair_index(pair_index(p, p), pair_index(q, q))], F) -
                                             host_fixed(h->eri[pair_index(pair_index(p, q), pair_index(q, p))], F));
        }
    }
    // single-excitation terms: (ai|kk) and (ai|kk) - (ak|ki) per (a, i, k)
    std::vector<ulonglong2> Sfx((size_t)N * N * N * 2);
    for (int a = 0; a < N; a++)
        for (int i = 0; i < N; i++)
            for (int k = 0; k < N; k++) {
                const i128 c = host_fixed(h->eri[pair_index(pair_index(a, i), pair_index(k, k))], F);
                const i128 x = host_fixed(h->eri[pair_index(pair_index(a, k), pair_index(k, i))], F);
                const size_t o = (((size_t)a * N + i) * N + k) * 2;
                put(Sfx[o], c);
                put(Sfx[o + 1], c - x);
            }
    // X(ref): sum over occupied orbitals and occupied pairs
    std::vector<std::pair<int, int>> occ;
    for (int p = 0; p < N; p++) if ((h->ref_a >> p) & 1) occ.push_back({p, 0});
    for (int p = 0; p < N; p++) if ((h->ref_b >> p) & 1) occ.push_back({p, 1});
    i128 xref = 0;
    for (size_t i = 0; i < occ.size(); i++) {
        xref += host_fixed(h->h[(size_t)occ[i].first * N + occ[i].first], F);
        for (size_t j = i + 1; j < occ.size(); j++) {
            int p = occ[i].first, q = occ[j].first;
            xref += host_fixed(h->eri[pair_index(pair_index(p, p), pair_index(q, q))], F);
            if (occ[i].second == occ[j].second) xref -= host_fixed(h->eri[pair_index(pair_index(p, q), pair_index(q, p))], F);
        }
    }
    h->eref = host_fixed_to_double(xref + host_fixed(h->ecore, F), F);

    DevInst &I = h->hi;
    I.replica = replica;
    I.partner = -1;
    I.kind = h->kind; I.norb = N; I.na = h->na; I.nb = h->nb; I.n = n; I.ma = N - h->na; I.mb = N - h->nb; I.z = h->z;
    I.F = F; I.Fw = Fw;
    {
        // E_num total on the grid 2^-Fe: |H_ref,j| < (2n + 1) 2^(msb_max + 1), |C_j| < 2^31 and at most
        // 2^34 determinants, so |E_num| 2^Fe stays below 2^126 with Fe = 60 - msb_max - ceil(log2(2n + 1))
        int L = 0;
        while ((1LL << L) < 2LL * n + 1) L++;
        const int fe = any ? 60 - msb_max - L : 64;
        I.Fe = fe > 64 ? 64 : fe;
    }
    I.ref_a = h->ref_a; I.ref_b = h->ref_b; I.normask = normask;
    I.xref_lo = (u64)(u128)xref; I.xref_hi = (u64)((u128)xref >> 64);
    const bool auto_tau = !(P.tau > 0.0);
    I.tmt = -h->t;
    {
        double q = P.p_single * 0x1p53;  // exact
        I.tsingle = (u64)std::ceil(q);
    }
    {
        // ceil(2^64 / d) of the generators' fixed divisors (0 for d <= 1)
        auto magic = [](long long d) -> u64 { return d > 1 ? (u64)(~0ULL / (u64)d) + 1ULL : 0ULL; };
        I.mg_n1 = magic(n - 1);
        I.mg_mb = magic(I.mb);
        I.mg_ma1 = magic(I.ma - 1);
        I.mg_mb1 = magic(I.mb - 1);
    }
    I.seed = P.seed; I.cmin = P.c_min; I.n_a = P.initiator_threshold;
    {
        int e2;
        double fr = std::frexp(P.c_min, &e2);
        I.cmin_pow2 = fr == 0.5;  // c_min = 2^(e2-1)
        I.cmin_log2 = e2 - 1;
    }

    I.target = P.target_walkers; I.A = P.shift_interval;
    I.semi_start = P.semistoch_start; I.semi_size = P.semistoch_size;
    I.trial_size = P.trial_size; I.trial_start = P.trial_start;
    I.adaptive = P.adaptive_shift ? 1 : 0;
    I.ring_cap = h->ring_cap;

    // integrals and tables on the device
    double *dh = (double *)dev_alloc(h, h->h.size() * sizeof(double));
    double *deri = (double *)dev_alloc(h, h->eri.size() * sizeof(double));
    ulonglong2 *dhfx = (ulonglong2 *)dev_alloc(h, hfx.size() * sizeof(ulonglong2));
    ulonglong2 *dJ = (ulonglong2 *)dev_alloc(h, Jfx.size() * sizeof(ulonglong2));
    ulonglong2 *dK = (ulonglong2 *)dev_alloc(h, JKfx.size() * sizeof(ulonglong2));
    ulonglong2 *dS = (ulonglong2 *)dev_alloc(h, Sfx.size() * sizeof(ulonglong2));
    int *dnbr = (int *)dev_alloc(h, std::max<size_t>(1, h->nbr.size()) * sizeof(int));
    h->dinst = (DevInst *)dev_alloc(h, sizeof(DevInst));
    h->dunit = (int *)dev_alloc(h, 2 * sizeof(int));
    h->dstate = (IterState *)dev_alloc(h, sizeof(IterState));
    I.ring = (fciqmc_iter_stats *)dev_alloc(h, (size_t)h->ring_cap * sizeof(fciqmc_iter_stats));
    I.acc = (u64 *)dev_alloc(h, NSHARD * ACC_STRIDE * sizeof(u64));
    if (!dh || !deri || !dhfx || !dJ || !dK || !dS || !dnbr || !h->dinst || !h->dunit || !h->dstate || !I.ring || !I.acc)
        return bail(FCIQMC_ERR_OUT_OF_MEMORY, "out of device memory (integrals)");
    cudaMemsetAsync(I.acc, 0, NSHARD * ACC_STRIDE * sizeof(u64), h->stream);
    cudaMemcpyAsync(dh, h->h.data(), h->h.size() * sizeof(double), cudaMemcpyHostToDevice, h->stream);
    cudaMemcpyAsync(deri, h->eri.data(), h->eri.size() * sizeof(double), cudaMemcpyHostToDevice, h->stream);
    cudaMemcpyAsync(dhfx, hfx.data(), hfx.size() * sizeof(ulonglong2), cudaMemcpyHostToDevice, h->stream);
    cudaMemcpyAsync(dJ, Jfx.data(), Jfx.size() * sizeof(ulonglong2), cudaMemcpyHostToDevice, h->stream);
    cudaMemcpyAsync(dK, JKfx.data(), JKfx.size() * sizeof(ulonglong2), cudaMemcpyHostToDevice, h->stream);
    cudaMemcpyAsync(dS, Sfx.data(), Sfx.size() * sizeof(ulonglong2), cudaMemcpyHostToDevice, h->stream);
    if (!h->nbr.empty()) cudaMemcpyAsync(dnbr, h->nbr.data(), h->nbr.size() * sizeof(int), cudaMemcpyHostToDevice, h->stream);
    I.h = dh; I.eri = deri; I.hfx = dhfx; I.Jfx = dJ; I.JKfx = dK; I.Sfx = dS; I.nbr = dnbr;
    I.st = h->dstate;
    // time step: given, or 0.5 / sum_j |H_ref,j| (computed on the device)
    {
        double *dpart = (double *)dev_alloc(h, 64 * sizeof(double));
        if (!dpart) return bail(FCIQMC_ERR_OUT_OF_MEMORY, "out of device memory");
        if (cudaMemcpyAsync(h->dinst, &I, sizeof(DevInst), cudaMemcpyHostToDevice, h->stream) != cudaSuccess ||
            ref_abs_sum(h->dinst, dpart, &h->ref_sum, h->stream) != cudaSuccess)
            return bail(FCIQMC_ERR_CUDA, "reference coupling sum failed");
        dev_free(h, dpart);
        if (auto_tau) {
            if (!(h->ref_sum > 0.0)) return bail(FCIQMC_ERR_INVALID_ARG, "tau <= 0 needs a reference with couplings");
            h->p.tau = 0.5 / h->ref_sum;
        }
        I.tau = h->p.tau;
        for (int c = 0; c < NCLS; c++) I.lam[c] = h->p.tau / pgen_class(h, c);
        I.cz = P.shift_damping / ((double)P.shift_interval * h->p.tau);
    }

    // pre-computed heat-bath tables (generator 1, ab initio systems with a double)
    if (P.generator == 1 && h->kind == FCIQMC_ABINITIO && n >= 2) {
        // the exact table sums add up to N^2 terms of |(ai|bj) - (aj|bi)| < 2^(msb_max + 2)
        int kb = 0;
        while ((1LL << kb) < (long long)N * N) kb++;
        if (any && msb_max + 2 + F + kb + 2 > 125)
            return bail(FCIQMC_ERR_UNSUPPORTED, "integral dynamic range too wide for the exact heat-bath table sums");
        const u64 nab = (u64)N * N, kss = (u64)N * (N - 1) / 2;
        const u64 ss_base = nab * nab;
        const u64 nent = ss_base + kss * kss;
        double2 *meta = (double2 *)dev_alloc(h, (size_t)(nab + kss) * sizeof(double2));
        ulonglong2 *ent = (ulonglong2 *)dev_alloc(h, (size_t)nent * sizeof(ulonglong2));
        if (!meta || !ent) return bail(FCIQMC_ERR_OUT_OF_MEMORY, "out of device memory (heat-bath tables)");
        // probability of one unordered electron pair: (1 - p_single) 2 / (n (n - 1))
        const double ppair = ((1.0 - P.p_single) * 2.0) / ((double)n * (double)(n - 1));
        if (cudaMemcpyAsync(h->dinst, &I, sizeof(DevInst), cudaMemcpyHostToDevice, h->stream) != cudaSuccess ||
            launch_pchb_build(h->dinst, N, ppair, meta, ent, ss_base, h->stream) != cudaSuccess ||
            cudaStreamSynchronize(h->stream) != cudaSuccess)
            return bail(FCIQMC_ERR_CUDA, "heat-bath table construction failed");
        I.pchb = 1;
        I.pchb_meta = meta;
        I.pchb_ent = ent;
        I.pchb_ss_base = ss_base;
    } else if (P.generator != 0 && P.generator != 1) {
        return bail(FCIQMC_ERR_INVALID_ARG, "generator must be 0 (uniform) or 1 (pre-computed heat-bath)");
    }

    // bucket layout: average occupancy well below the per-bucket capacity
    // start at the expected size (capped: buffers grow on demand)
    double dets_hint = P.max_dets > 0 ? (double)P.max_dets : std::min(std::max(4096.0, P.target_walkers), 8388608.0);
    {
        double fci = 1.0;  // C(N, n_alpha) C(N, n_beta)
        for (int k = 0; k < h->na; k++) fci *= (double)(N - k) / (double)(k + 1);
        for (int k = 0; k < h->nb; k++) fci *= (double)(N - k) / (double)(k + 1);
        if (P.max_dets <= 0) dets_hint = std::min(dets_hint, std::max(1.0, fci));
    }
    int bb = 0;
    while (((double)(1LL << bb)) * 640.0 < dets_hint && bb < MAX_BB) bb++;
    I.cap_s = CAP_S0;
    int rc = alloc_layout(h, I, bb);
    if (rc) return bail(rc, "out of device memory (walker buffers)");
    h->bb = bb;
    h->heavy_cap = std::max(4096, (int)std::min(1e6, 4.0 * P.target_walkers / HEAVY_ATT));
    I.heavy = (HeavyChunk *)dev_alloc(h, (size_t)h->heavy_cap * sizeof(HeavyChunk));
    I.heavy_cap = h->heavy_cap;
    if (!I.heavy) return bail(FCIQMC_ERR_OUT_OF_MEMORY, "out of device memory (heavy queue)");

    // initial state: initial_walkers on the reference determinant
    {
        const int b0 = bb ? (int)(det_hash_host(h->ref_a, h->ref_b) >> (64 - bb)) : 0;
        ulonglong2 k;
        k.x = h->ref_a; k.y = h->ref_b;
        double c = P.initial_walkers, hd0 = 0.0;
        uint8_t f = DFLAG_REF;
        int one = 1;
        size_t o = (size_t)b0 * CAP_M;
        cudaMemcpyAsync(I.key[0] + o, &k, sizeof(k), cudaMemcpyHostToDevice, h->stream);
        cudaMemcpyAsync(I.c[0] + o, &c, sizeof(c), cudaMemcpyHostToDevice, h->stream);
        cudaMemcpyAsync(I.hd[0] + o, &hd0, sizeof(hd0), cudaMemcpyHostToDevice, h->stream);
        cudaMemcpyAsync(I.fl[0] + o, &f, 1, cudaMemcpyHostToDevice, h->stream);
        cudaMemcpyAsync(I.cnt[0] + b0, &one, sizeof(int), cudaMemcpyHostToDevice, h->stream);
        if (cudaStreamSynchronize(h->stream) != cudaSuccess) return bail(FCIQMC_ERR_CUDA, "initial upload failed");
    }
    memset(&h->hst, 0, sizeof(IterState));
    h->hst.S = P.initial_shift;
    h->hst.stop_iter = LLONG_MAX;
    if (write_state(h)) return bail(FCIQMC_ERR_CUDA, h->err);
    if (upload_inst(h)) return bail(FCIQMC_ERR_CUDA, h->err);
    if (P.adaptive_shift) {
        launch_build_kidx(h->dinst, 0, 1 << bb, h->stream);
        if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(h->stream) != cudaSuccess)
            return bail(FCIQMC_ERR_CUDA, "adaptive-shift index set-up failed");
    }
    if (capture_graph(h)) return bail(FCIQMC_ERR_CUDA, h->err);
    *out = h;
    return FCIQMC_OK;
}

static int create_impl(const fciqmc_system *sys, const fciqmc_params *prm, fciqmc_handle **out)
{
    if (prm && (prm->replicas < 0 || prm->replicas > 2)) {
        if (out) *out = nullptr;
        return fail(nullptr, FCIQMC_ERR_INVALID_ARG, "replicas must be 1 or 2");
    }
    int rc = create_run(sys, prm, 0, out);
    if (rc || prm->replicas != 2) return rc;
    // the second replica: same system and parameters, Philox key word 1 = 1,
    // on the first replica's stream
    fciqmc_handle *h = *out, *h2 = nullptr;
    fciqmc_params p2 = *prm;
    p2.stream = h->stream;
    rc = create_run(sys, &p2, 1, &h2);
    if (rc) {
        fciqmc_destroy(h);
        *out = nullptr;
        return rc;
    }
    h->partner = h2; h2->partner = h; h2->secondary = true;
    h->paired = h2->paired = true;
    rc = replica_kernel_init() == cudaSuccess ? FCIQMC_OK : fail(h, FCIQMC_ERR_CUDA, "replica kernel set-up failed");
    if (!rc) rc = ensure_side(h);
    if (!rc) rc = ensure_side(h2);
    if (!rc) rc = upload_inst(h);
    if (!rc) rc = upload_inst(h2);
    if (!rc) rc = capture_graph(h);
    if (!rc) rc = capture_graph(h2);
    if (rc) {
        g_create_error = h->err;
        fciqmc_destroy(h);
        *out = nullptr;
    }
    return rc;
}

int fciqmc_create(const fciqmc_system *sys, const fciqmc_params *prm, fciqmc_handle **out)
{
    try {
        return create_impl(sys, prm, out);
    } catch (const std::bad_alloc &) {
        return fail(nullptr, FCIQMC_ERR_OUT_OF_MEMORY, "host allocation failed");
    } catch (...) {
        return fail(nullptr, FCIQMC_ERR_OUT_OF_MEMORY, "host exception");
    }
}

int fciqmc_set_profiling(fciqmc_handle *h, int32_t on)
{
    if (!h) return FCIQMC_ERR_INVALID_ARG;
    h->profiling = on != 0;
    return FCIQMC_OK;
}

int fciqmc_kernel_times(fciqmc_handle *h, double out[6])
{
    if (!h || !out) return FCIQMC_ERR_INVALID_ARG;
    for (int k = 0; k < 6; k++) out[k] = h->ktime[k];
    return FCIQMC_OK;
}

int fciqmc_layout(fciqmc_handle *h, int64_t out[4])
{
    if (!h || !out) return FCIQMC_ERR_INVALID_ARG;
    out[0] = 1LL << h->bb; out[1] = CAP_M; out[2] = h->hi.cap_s; out[3] = (int64_t)h->bytes;
    return FCIQMC_OK;
}

int32_t fciqmc_graph_kernels(fciqmc_handle *h) { return h ? h->graph_kernels : -1; }

int fciqmc_device_memory(int32_t device, int64_t out[2])
{
    if (!out) return FCIQMC_ERR_INVALID_ARG;
    int clk = 0, bus = 0;
    if (cudaDeviceGetAttribute(&clk, cudaDevAttrMemoryClockRate, device) != cudaSuccess ||
        cudaDeviceGetAttribute(&bus, cudaDevAttrGlobalMemoryBusWidth, device) != cudaSuccess) {
        cudaGetLastError();
        return FCIQMC_ERR_CUDA;
    }
    out[0] = clk;
    out[1] = bus;
    return FCIQMC_OK;
}

int fciqmc_set_launch_config(int32_t spawn, int32_t heavy, int32_t annihilate)
{
    const bool sp_ok = spawn == 0 || spawn == 1 || spawn == 2 || spawn == 4 || spawn == 8 || spawn == 16;
    const bool hv_ok = heavy >= 1 && heavy <= 16;
    const bool an_ok = annihilate == 0 || annihilate == 3 || annihilate == 9 || annihilate == 24;
    if (!sp_ok || !hv_ok || !an_ok) return FCIQMC_ERR_INVALID_ARG;
    set_launch_geometry(spawn, heavy, annihilate);
    return FCIQMC_OK;
}

int fciqmc_get_launch_config(int32_t out[3])
{
    if (!out) return FCIQMC_ERR_INVALID_ARG;
    int a, b, c;
    get_launch_geometry(&a, &b, &c);
    out[0] = a; out[1] = b; out[2] = c;
    return FCIQMC_OK;
}

int64_t fciqmc_semistoch_info(fciqmc_handle *h, int64_t *nnz)
{
    if (!h) return FCIQMC_ERR_INVALID_ARG;
    if (nnz) *nnz = h->nd > 0 ? (int64_t)h->nnz : 0;
    return h->nd;
}

static int step_to(fciqmc_handle *h, long long target_iter);

static int step_impl(fciqmc_handle *h, int64_t n_iter)
{
    if (!h || n_iter < 0) return FCIQMC_ERR_INVALID_ARG;
    if (h->secondary) return fail(h, FCIQMC_ERR_INVALID_ARG, "step a replica pair through its first replica");
    if (h->partner) {  // both replicas in one launch per kernel, in lockstep
        fciqmc_handle *pair[2] = {h, h->partner};
        return fciqmc_step_batch(pair, 2, n_iter);
    }
    if (h->pending) {
        int rc = fciqmc_sync(h);
        if (rc) return rc;
    }
    int rc = read_state(h);
    if (rc) return rc;
    if (h->graph && h->graph_gen != launch_geometry_generation()) {  // the launch configuration changed
        rc = capture_graph(h);
        if (rc) return rc;
    }
    return step_to(h, h->hst.iter + n_iter);
}

int fciqmc_step(fciqmc_handle *h, int64_t n_iter)
{
    try {
        return step_impl(h, n_iter);
    } catch (const std::bad_alloc &) {
        return fail(h, FCIQMC_ERR_OUT_OF_MEMORY, "host allocation failed");
    } catch (...) {
        return fail(h, FCIQMC_ERR_OUT_OF_MEMORY, "host exception");
    }
}

static int step_async_impl(fciqmc_handle *h, int64_t n_iter)
{
    if (!h || n_iter < 0) return FCIQMC_ERR_INVALID_ARG;
    if (h->partner) return fail(h, FCIQMC_ERR_UNSUPPORTED, "replica pairs are stepped with fciqmc_step");
    if (!h->pending) {
        int rc = read_state(h);
        if (rc) return rc;
        h->async_base = h->hst.iter;
        h->async_target = h->hst.iter;
        if (h->graph && h->graph_gen != launch_geometry_generation()) {  // the launch configuration changed
            rc = capture_graph(h);
            if (rc) return rc;
        }
    }
    for (int64_t k = 0; k < n_iter; k++) CUDA_TRY(h, cudaGraphLaunch(h->graph, h->stream));
    h->async_target += n_iter;
    h->pending = true;
    return FCIQMC_OK;
}

int fciqmc_step_async(fciqmc_handle *h, int64_t n_iter)
{
    try {
        return step_async_impl(h, n_iter);
    } catch (const std::bad_alloc &) {
        return fail(h, FCIQMC_ERR_OUT_OF_MEMORY, "host allocation failed");
    } catch (...) {
        return fail(h, FCIQMC_ERR_OUT_OF_MEMORY, "host exception");
    }
}

static int sync_impl(fciqmc_handle *h)
{
    if (!h) return FCIQMC_ERR_INVALID_ARG;
    if (!h->pending) return FCIQMC_OK;
    h->pending = false;
    int rc = read_state(h);
    if (rc) return rc;
    // rows of the iterations that completed; beyond the ring only the last ring_cap are kept
    long long from = std::max<long long>(h->async_base, h->hst.iter - h->ring_cap);
    rc = pull_history(h, from, h->hst.iter);
    if (rc) return rc;
    if (!h->hst.err) return FCIQMC_OK;
    return step_to(h, h->async_target);
}

int fciqmc_sync(fciqmc_handle *h)
{
    try {
        return sync_impl(h);
    } catch (const std::bad_alloc &) {
        return fail(h, FCIQMC_ERR_OUT_OF_MEMORY, "host allocation failed");
    } catch (...) {
        return fail(h, FCIQMC_ERR_OUT_OF_MEMORY, "host exception");
    }
}

void *fciqmc_stream(fciqmc_handle *h) { return h ? (void *)h->stream : nullptr; }

// Runs iterations until target_iter, in chunks of graph replays; after each
// chunk reads the device state and reacts to its flags (capacity growth with
// a bit-identical repeat, semi-stochastic set-up, or a fatal error).
static int handle_flags(fciqmc_handle *h, int *retries);

static int step_to(fciqmc_handle *h, long long target_iter)
{
    int rc;
    int retries = 0;
    std::vector<cudaEvent_t> evs;
    double kt[6] = {0, 0, 0, 0, 0, 0};
    static const int slot_of[6] = {0, 1, 4, 2, 5, 3};  // event interval -> ktime slot
    long long kn = 0;
    long long chunk_max = 16;  // grows after clean chunks; an error costs at most one chunk of no-op replays
    for (;;) {
        if (h->hst.err) {
            chunk_max = 16;
            rc = handle_flags(h, &retries);
            if (rc) return rc;
            continue;
        }
        if (h->hst.iter >= target_iter) break;
        const long long start = h->hst.iter;
        const long long chunk = std::min<long long>(std::min<long long>(target_iter - start, h->ring_cap), chunk_max);
        chunk_max = std::min<long long>(chunk_max * 2, h->ring_cap);
        if (h->profiling) {
            evs.resize((size_t)chunk * 7);
            for (auto &e : evs) cudaEventCreate(&e);
            for (long long k = 0; k < chunk; k++) {
                rc = enqueue_iteration(h, evs.data() + 7 * k);
                if (rc) return rc;
            }
        } else {
            for (long long k = 0; k < chunk; k++) CUDA_TRY(h, cudaGraphLaunch(h->graph, h->stream));
        }
        rc = read_state(h);
        if (rc) return rc;
        if (h->profiling) {
            const long long done = h->hst.iter - start;
            for (long long k = 0; k < done; k++)
                for (int j = 0; j < 6; j++) {
                    float ms = 0.f;
                    cudaEventElapsedTime(&ms, evs[7 * k + j], evs[7 * k + j + 1]);
                    kt[slot_of[j]] += ms;
                }
            kn += done;
            for (auto &e : evs) cudaEventDestroy(e);
            evs.clear();
        }
        rc = pull_history(h, start, h->hst.iter);
        if (rc) return rc;
        if (!h->hst.err && !h->hist.empty() && h->hist.back().ndet > (1LL << h->bb) * (long long)(CAP_M / 2) &&
            h->bb < MAX_BB) {
            // keep head-room in the main buckets: split once the average
            // occupancy passes half the capacity
            rc = grow_buckets(h);
            if (rc) return rc;
            rc = reset_after_error(h);
            if (rc) return rc;
            rc = upload_inst(h);
            if (rc) return rc;
            rc = capture_graph(h);
            if (rc) return rc;
        }
    }
    if (h->profiling && kn > 0)
        for (int j = 0; j < 6; j++) h->ktime[j] = kt[j] / (double)kn;
    return FCIQMC_OK;
}

static int handle_flags(fciqmc_handle *h, int *retries)
{
    int rc;
    if (h->hst.err & ERRB_STOP) {  // left by a batch: clear and continue
        h->hst.err &= ~ERRB_STOP;
        h->hst.stop_iter = LLONG_MAX;
        rc = write_state(h);
        if (rc) return rc;
        if (!h->hst.err) return FCIQMC_OK;
    }
    const int err = h->hst.err;
    if (err & ERRB_NUMERIC)
        return fail(h, FCIQMC_ERR_NUMERIC, "numeric error (NaN/Inf or |C| >= 2^31) at iteration " + std::to_string(h->hst.iter));
    if (err & ERRB_TIMEOUT) return fail(h, FCIQMC_ERR_TIMEOUT, "device wait timed out");
    if (err && !(err & ~(ERRB_PAUSE_SEMI | ERRB_PAUSE_TRIAL))) {
        if (err & ERRB_PAUSE_SEMI) {
            rc = build_semistochastic(h);
            if (rc) return rc;
        }
        if (err & ERRB_PAUSE_TRIAL) {
            rc = build_trial(h);
            if (rc) return rc;
        }
        h->hst.err = 0;
        return write_state(h);
    }
    if (err == ERRB_PARTNER) {  // the other replica failed: repeat the iteration as it was
        rc = reset_after_error(h);
        if (rc) return rc;
        return upload_inst(h);
    }
    if (++*retries > 64) return fail(h, FCIQMC_ERR_CAPACITY, "capacity growth did not converge");
    const long long need = h->hst.need_spawn;
    const int n_over = h->hst.n_spawn_over;
    const long long needq0 = h->hst.need_queue[0], needq1 = h->hst.need_queue[1];
    rc = reset_after_error(h);
    if (rc) return rc;
    if (err & (ERRB_SPAWN_CAP | ERRB_MAIN_CAP)) {
        // a new list too large for its bucket, or spawns spread evenly over
        // crowded buckets: split buckets.  Spawns concentrated on a few
        // determinants: enlarge the spawn regions to what was needed.
        const long long nbk = 1LL << h->bb;
        const bool even = (long long)n_over * 16 > nbk;  // many buckets overflowed: the load is spread
        if ((err & ERRB_MAIN_CAP) || ((err & ERRB_SPAWN_CAP) && even)) rc = grow_buckets(h);
        else rc = grow_spawn_capacity(h, need);
        if (rc) return rc;
        rc = reset_after_error(h);
        if (rc) return rc;
    }
    if (err & ERRB_HEAVY_CAP) {
        rc = grow_heavy(h);
        if (rc) return rc;
    }
    if (err & ERRB_QUEUE_CAP) {  // a segment of the attempt queues was too short: a quarter above the need
        rc = ensure_queues(h, needq0 + needq0 / 4, needq1 + needq1 / 4);
        if (rc) return rc;
    }
    rc = ensure_side(h);
    if (rc) return rc;
    // a replica pair keeps one bucket layout: the other replica follows a split
    fciqmc_handle *pt = h->partner;
    if (pt && pt->bb < h->bb) {
        // its pending iteration (not committed: the replicas move in lockstep)
        // is repeated after the split; its own flags come back if still due
        rc = read_state(pt);
        if (rc) return rc;
        const int keep = pt->hst.err & (ERRB_STOP | ERRB_PAUSE_SEMI | ERRB_PAUSE_TRIAL);
        rc = reset_after_error(pt);
        if (rc) return rc;
        if (keep) {
            pt->hst.err = keep;
            rc = write_state(pt);
            if (rc) return rc;
        }
        while (pt->bb < h->bb) {
            rc = grow_buckets(pt);
            if (rc) return rc;
        }
        rc = ensure_side(pt);
        if (rc) return rc;
        rc = upload_inst(pt);
        if (rc) return rc;
        rc = capture_graph(pt);
        if (rc) return rc;
    }
    rc = upload_inst(h);
    if (rc) return rc;
    return capture_graph(h);
}

int64_t fciqmc_num_dets(fciqmc_handle *h)
{
    if (!h) return -1;
    int nbk = 1 << h->bb;
    std::vector<int> cnt(nbk);
    if (read_state(h)) return -1;
    if (cudaMemcpy(cnt.data(), h->hi.cnt[h->hst.parity], nbk * sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return -1;
    int64_t s = 0;
    for (int c : cnt) s += c;
    return s;
}

static int export_state_impl(fciqmc_handle *h, int64_t cap, uint64_t *alpha, uint64_t *beta, double *c, double *hdiag,
                        int32_t *flags, int64_t *n_out)
{
    if (!h || !n_out) return FCIQMC_ERR_INVALID_ARG;
    int rc = read_state(h);
    if (rc) return rc;
    const int par = h->hst.parity;
    const size_t nbk = (size_t)1 << h->bb, nm = nbk * CAP_M;
    std::vector<int> cnt(nbk);
    CUDA_TRY(h, cudaMemcpy(cnt.data(), h->hi.cnt[par], nbk * sizeof(int), cudaMemcpyDeviceToHost));
    int64_t n = 0;
    for (int x : cnt) n += x;
    *n_out = n;
    if (n > cap) return fail(h, FCIQMC_ERR_CAPACITY, "export buffer too small");
    if (n > 0 && (!alpha || !beta || !c)) return FCIQMC_ERR_INVALID_ARG;
    if (n == 0) return FCIQMC_OK;
    // on the device: compaction, radix sort by (alpha, beta), gather; only the
    // n live entries are copied out.  Transient scratch from the run's
    // allocator; where it cannot be had, the same order is produced on the host.
    {
        std::vector<long long> off(nbk + 1, 0);
        for (size_t b = 0; b < nbk; b++) off[b + 1] = off[b] + cnt[b];
        const size_t off_bytes = ((nbk + 1) * sizeof(long long) + 255) & ~(size_t)255;
        unsigned char *scr = (unsigned char *)dev_alloc(h, off_bytes + export_scratch_bytes(n));
        if (scr) {
            const u64 *oa, *ob;
            const double *oc, *ohd;
            const int32_t *ofl;
            cudaError_t e = cudaMemcpyAsync(scr, off.data(), (nbk + 1) * sizeof(long long), cudaMemcpyHostToDevice,
                                            h->stream);
            if (e == cudaSuccess)
                e = export_sorted(h->hi.key[par], h->hi.c[par], h->hi.hd[par], h->hi.fl[par], h->hi.cnt[par],
                                  (const long long *)scr, (int)nbk, n, h->norb, scr + off_bytes, &oa, &ob, &oc, &ohd,
                                  &ofl, h->stream);
            if (e == cudaSuccess) e = cudaMemcpyAsync(alpha, oa, n * sizeof(u64), cudaMemcpyDeviceToHost, h->stream);
            if (e == cudaSuccess) e = cudaMemcpyAsync(beta, ob, n * sizeof(u64), cudaMemcpyDeviceToHost, h->stream);
            if (e == cudaSuccess) e = cudaMemcpyAsync(c, oc, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
            if (e == cudaSuccess && hdiag)
                e = cudaMemcpyAsync(hdiag, ohd, n * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
            if (e == cudaSuccess && flags)
                e = cudaMemcpyAsync(flags, ofl, n * sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
            dev_free(h, scr);
            if (e != cudaSuccess) return fail(h, FCIQMC_ERR_CUDA, std::string("export: ") + cudaGetErrorString(e));
            return FCIQMC_OK;
        }
    }
    std::vector<ulonglong2> k(nm);
    std::vector<double> cc(nm), hh(nm);
    std::vector<uint8_t> ff(nm);
    CUDA_TRY(h, cudaMemcpy(k.data(), h->hi.key[par], nm * sizeof(ulonglong2), cudaMemcpyDeviceToHost));
    CUDA_TRY(h, cudaMemcpy(cc.data(), h->hi.c[par], nm * sizeof(double), cudaMemcpyDeviceToHost));
    CUDA_TRY(h, cudaMemcpy(hh.data(), h->hi.hd[par], nm * sizeof(double), cudaMemcpyDeviceToHost));
    CUDA_TRY(h, cudaMemcpy(ff.data(), h->hi.fl[par], nm, cudaMemcpyDeviceToHost));
    std::vector<size_t> idx;
    idx.reserve((size_t)n);
    for (size_t b = 0; b < nbk; b++)
        for (int e = 0; e < cnt[b]; e++) idx.push_back(b * CAP_M + e);
    std::sort(idx.begin(), idx.end(), [&](size_t x, size_t y) {
        return k[x].x < k[y].x || (k[x].x == k[y].x && k[x].y < k[y].y);
    });
    for (size_t i = 0; i < idx.size(); i++) {
        alpha[i] = k[idx[i]].x;
        beta[i] = k[idx[i]].y;
        c[i] = cc[idx[i]];
        if (hdiag) hdiag[i] = hh[idx[i]];
        if (flags) flags[i] = ff[idx[i]];
    }
    return FCIQMC_OK;
}

int fciqmc_export_state(fciqmc_handle *h, int64_t cap, uint64_t *alpha, uint64_t *beta, double *c, double *hdiag,
                        int32_t *flags, int64_t *n_out)
{
    try {
        return export_state_impl(h, cap, alpha, beta, c, hdiag, flags, n_out);
    } catch (const std::bad_alloc &) {
        return fail(h, FCIQMC_ERR_OUT_OF_MEMORY, "host allocation failed");
    } catch (...) {
        return fail(h, FCIQMC_ERR_OUT_OF_MEMORY, "host exception");
    }
}

int fciqmc_export_shift(fciqmc_handle *h, int64_t *iteration, double *S, int32_t *vary, int64_t *shift_start,
                        int64_t *cnt, uint64_t *nw_last_hi, uint64_t *nw_last_lo)
{
    if (!h) return FCIQMC_ERR_INVALID_ARG;
    int rc = read_state(h);
    if (rc) return rc;
    if (iteration) *iteration = h->hst.iter;
    if (S) *S = h->hst.S;
    if (vary) *vary = h->hst.vary;
    if (shift_start) *shift_start = h->hst.shift_start;
    if (cnt) *cnt = h->hst.cnt;
    if (nw_last_hi) *nw_last_hi = h->hst.nwl_hi;
    if (nw_last_lo) *nw_last_lo = h->hst.nwl_lo;
    return FCIQMC_OK;
}

// import on the device: the compact input in `scr` ((n + 1) keys, amplitudes
// and four flag words), checked, counted per bucket to choose the bucket
// count, and placed; the slots are listed in newdet for the H_ii kernel
static int import_device(fciqmc_handle *h, int64_t n, const uint64_t *alpha, const uint64_t *beta, const double *c,
                         u64 normask, unsigned char *scr, int64_t *nt_out)
{
    cudaStream_t s = h->stream;
    u64 *da = (u64 *)scr, *db = da + (n + 1);
    double *dc = (double *)(db + (n + 1));
    int *dflag = (int *)(dc + (n + 1));
    CUDA_TRY(h, cudaMemsetAsync(dflag, 0, 4 * sizeof(int), s));
    if (n > 0) {
        CUDA_TRY(h, cudaMemcpyAsync(da, alpha, (size_t)n * sizeof(u64), cudaMemcpyHostToDevice, s));
        CUDA_TRY(h, cudaMemcpyAsync(db, beta, (size_t)n * sizeof(u64), cudaMemcpyHostToDevice, s));
        CUDA_TRY(h, cudaMemcpyAsync(dc, c, (size_t)n * sizeof(double), cudaMemcpyHostToDevice, s));
    }
    CUDA_TRY(h, launch_import_check(da, db, dc, n, h->na, h->nb, normask, h->ref_a, h->ref_b, dflag, s));
    int flags = 0;
    CUDA_TRY(h, cudaMemcpyAsync(&flags, dflag, sizeof(int), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(h, cudaStreamSynchronize(s));
    if (flags & 1) return fail(h, FCIQMC_ERR_INVALID_ARG, "imported determinant with wrong electron count or bad amplitude");
    int64_t nt = n;
    const u64 ra = h->ref_a, rb = h->ref_b;
    const double zero = 0.0;
    if (!(flags & 2)) {  // the reference, when absent, is appended as entry n with C = 0
        CUDA_TRY(h, cudaMemcpyAsync(da + n, &ra, sizeof(u64), cudaMemcpyHostToDevice, s));
        CUDA_TRY(h, cudaMemcpyAsync(db + n, &rb, sizeof(u64), cudaMemcpyHostToDevice, s));
        CUDA_TRY(h, cudaMemcpyAsync(dc + n, &zero, sizeof(double), cudaMemcpyHostToDevice, s));
        nt = n + 1;
    }
    int rc = read_state(h);  // also completes the copies above
    if (rc) return rc;
    // the fewest buckets (at least the current number) that hold every
    // bucket's determinants within half the main capacity; one allocation
    int bb = h->bb;
    for (;; bb++) {
        int *cntb = (int *)dev_alloc(h, ((size_t)1 << bb) * sizeof(int));
        if (!cntb) return fail(h, FCIQMC_ERR_OUT_OF_MEMORY, "out of device memory (import counts)");
        int over = 0;
        cudaError_t e = cudaMemsetAsync(cntb, 0, ((size_t)1 << bb) * sizeof(int), s);
        if (e == cudaSuccess) e = cudaMemsetAsync(dflag + 1, 0, sizeof(int), s);
        if (e == cudaSuccess) e = launch_import_count(da, db, nt, bb, cntb, dflag + 1, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&over, dflag + 1, sizeof(int), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        dev_free(h, cntb);
        if (e != cudaSuccess) return fail(h, FCIQMC_ERR_CUDA, std::string("import: ") + cudaGetErrorString(e));
        if (!over) break;
        if (bb >= MAX_BB)  // distinct keys crowd one bucket at the largest bucket count only if duplicated
            return fail(h, FCIQMC_ERR_INVALID_ARG, "imported keys crowd one bucket (duplicate determinants?)");
    }
    if (bb != h->bb) {
        DevInst nI = h->hi;
        rc = alloc_layout(h, nI, bb);
        if (rc) return fail(h, rc, "out of device memory");
        free_layout(h, h->hi);
        h->hi = nI;
        h->bb = nI.bb;
    }
    const int par = 0;
    CUDA_TRY(h, cudaMemsetAsync(h->hi.cnt[par], 0, ((size_t)1 << h->bb) * sizeof(int), s));
    CUDA_TRY(h, launch_import_place(da, db, dc, nt, h->bb, ra, rb, h->hi.cnt[par], h->hi.key[par], h->hi.c[par],
                                    h->hi.fl[par], h->hi.newdet, s));
    CUDA_TRY(h, cudaStreamSynchronize(s));
    *nt_out = nt;
    return FCIQMC_OK;
}

// import on the host (when no device scratch can be had): the same checks and
// bucket count, the padded layout built here and copied
static int import_host(fciqmc_handle *h, int64_t n, const uint64_t *alpha, const uint64_t *beta, const double *c,
                       u64 normask)
{
    std::vector<u64> hash((size_t)n + 1);
    bool has_ref = false;
    for (int64_t i = 0; i < n; i++) {
        const u64 a = alpha[i], b = beta[i];
        if (__builtin_popcountll(a) != h->na || __builtin_popcountll(b) != h->nb || ((a | b) & ~normask) ||
            !std::isfinite(c[i]))
            return fail(h, FCIQMC_ERR_INVALID_ARG, "imported determinant with wrong electron count or bad amplitude");
        has_ref |= a == h->ref_a && b == h->ref_b;
        hash[i] = det_hash_host(a, b);
    }
    const int64_t nt = n + (has_ref ? 0 : 1);  // the reference, when absent, as entry n with C = 0
    if (!has_ref) hash[n] = det_hash_host(h->ref_a, h->ref_b);
    auto key_a = [&](int64_t i) { return i < n ? (u64)alpha[i] : h->ref_a; };
    auto key_b = [&](int64_t i) { return i < n ? (u64)beta[i] : h->ref_b; };
    int rc = read_state(h);
    if (rc) return rc;
    int bb = h->bb;
    for (;; bb++) {
        std::vector<int> cnt_b((size_t)1 << bb, 0);
        bool over = false;
        for (int64_t i = 0; i < nt && !over; i++)
            if (++cnt_b[bb ? (size_t)(hash[i] >> (64 - bb)) : 0] > CAP_M / 2) over = true;
        if (!over) break;
        if (bb >= MAX_BB)
            return fail(h, FCIQMC_ERR_INVALID_ARG, "imported keys crowd one bucket (duplicate determinants?)");
    }
    if (bb != h->bb) {
        DevInst nI = h->hi;
        rc = alloc_layout(h, nI, bb);
        if (rc) return fail(h, rc, "out of device memory");
        free_layout(h, h->hi);
        h->hi = nI;
        h->bb = nI.bb;
    }
    const size_t nbk = (size_t)1 << h->bb, nm = nbk * CAP_M;
    std::vector<int> cnt_b(nbk, 0);
    std::vector<ulonglong2> k(nm);
    std::vector<double> cc(nm, 0.0);
    std::vector<uint8_t> ff(nm, 0);
    for (int64_t i = 0; i < nt; i++) {
        const size_t b = h->bb ? (size_t)(hash[i] >> (64 - h->bb)) : 0;
        const size_t o = b * CAP_M + (size_t)cnt_b[b]++;
        k[o].x = key_a(i);
        k[o].y = key_b(i);
        cc[o] = i < n ? c[i] : 0.0;
    }
    const int par = 0;
    CUDA_TRY(h, cudaMemcpy(h->hi.key[par], k.data(), nm * sizeof(ulonglong2), cudaMemcpyHostToDevice));
    CUDA_TRY(h, cudaMemcpy(h->hi.c[par], cc.data(), nm * sizeof(double), cudaMemcpyHostToDevice));
    CUDA_TRY(h, cudaMemcpy(h->hi.fl[par], ff.data(), nm, cudaMemcpyHostToDevice));
    CUDA_TRY(h, cudaMemcpy(h->hi.cnt[par], cnt_b.data(), nbk * sizeof(int), cudaMemcpyHostToDevice));
    return FCIQMC_OK;
}

static int import_state_impl(fciqmc_handle *h, int64_t n, const uint64_t *alpha, const uint64_t *beta, const double *c,
                        int64_t iteration, double S, int32_t vary, int64_t shift_start, int64_t cnt, uint64_t nw_last_hi,
                        uint64_t nw_last_lo)
{
    if (!h || n < 0 || (n > 0 && (!alpha || !beta || !c)) || iteration < 0) return FCIQMC_ERR_INVALID_ARG;
    const u64 normask = h->norb >= 64 ? ~0ULL : ((1ULL << h->norb) - 1);
    const int par = 0;
    // on the device (transient scratch from the run's allocator); where that
    // scratch cannot be had, on the host
    int64_t nt = 0;
    unsigned char *scr = (unsigned char *)dev_alloc(h, ((size_t)n + 1) * 24 + 4 * sizeof(int));
    const bool listed = scr != nullptr;  // H_ii from the list of placed slots
    int rc = listed ? import_device(h, n, alpha, beta, c, normask, scr, &nt) : import_host(h, n, alpha, beta, c, normask);
    if (scr) dev_free(h, scr);
    if (rc) return rc;
    const size_t nbk = (size_t)1 << h->bb;
    CUDA_TRY(h, cudaMemset(h->hi.scnt_i, 0, nbk * sizeof(int)));
    CUDA_TRY(h, cudaMemset(h->hi.scnt_n, 0, nbk * sizeof(int)));
    rc = ensure_side(h);
    if (rc) return rc;
    rc = upload_inst(h);
    if (rc) return rc;
    if (listed) launch_diag_list(h->dinst, par, h->hi.newdet, (int)nt, h->stream);
    else launch_diag(h->dinst, par, (int)nbk, h->stream);
    if (h->p.adaptive_shift) launch_build_kidx(h->dinst, par, (int)nbk, h->stream);
    CUDA_TRY(h, cudaGetLastError());
    memset(&h->hst, 0, sizeof(IterState));
    CUDA_TRY(h, cudaMemsetAsync(h->hi.acc, 0, NSHARD * ACC_STRIDE * sizeof(u64), h->stream));
    h->hst.stop_iter = LLONG_MAX;
    h->hst.iter = iteration; h->hst.parity = par; h->hst.S = S; h->hst.vary = vary;
    h->hst.shift_start = shift_start; h->hst.cnt = cnt; h->hst.nwl_hi = nw_last_hi; h->hst.nwl_lo = nw_last_lo;
    h->hst.semi_built = h->hi.nd > 0;
    h->hst.trial_built = h->trial_nt > 0;
    rc = write_state(h);
    if (rc) return rc;
    // a space due at the imported iteration is built now (the kernels raise
    // its pause at the end of the iteration before)
    if (vary && h->p.semistoch_size > 0 && !h->hst.semi_built && iteration == shift_start + h->p.semistoch_start) {
        rc = build_semistochastic(h);
        if (rc) return rc;
    }
    if (vary && h->p.trial_size > 0 && !h->hst.trial_built && iteration == shift_start + h->p.trial_start) {
        rc = build_trial(h);
        if (rc) return rc;
    }
    rc = write_state(h);
    if (rc) return rc;
    h->hist.clear();
    h->hist.resize((size_t)iteration);
    for (int64_t i = 0; i < iteration; i++) { memset(&h->hist[i], 0, sizeof(fciqmc_iter_stats)); h->hist[i].iteration = -1; }
    return capture_graph(h);
}

int fciqmc_import_state(fciqmc_handle *h, int64_t n, const uint64_t *alpha, const uint64_t *beta, const double *c,
                        int64_t iteration, double S, int32_t vary, int64_t shift_start, int64_t cnt, uint64_t nw_last_hi,
                        uint64_t nw_last_lo)
{
    try {
        return import_state_impl(h, n, alpha, beta, c, iteration, S, vary, shift_start, cnt, nw_last_hi, nw_last_lo);
    } catch (const std::bad_alloc &) {
        return fail(h, FCIQMC_ERR_OUT_OF_MEMORY, "host allocation failed");
    } catch (...) {
        return fail(h, FCIQMC_ERR_OUT_OF_MEMORY, "host exception");
    }
}

int64_t fciqmc_iter_stats_count(fciqmc_handle *h) { return h ? (int64_t)h->hist.size() : -1; }

// Many runs per launch: one descriptor table covering the buckets of all
// runs, one captured iteration graph; each run stops at its own target via
// the stop iteration, and capacity flags are handled run by run.
static int step_batch_impl(fciqmc_handle **hs, int32_t k, int64_t n_iter)
{
    if (!hs || k < 1 || n_iter < 0) return FCIQMC_ERR_INVALID_ARG;
    for (int i = 0; i < k; i++) {
        if (!hs[i]) return FCIQMC_ERR_INVALID_ARG;
        for (int j = 0; j < i; j++)
            if (hs[j] == hs[i]) return fail(hs[0], FCIQMC_ERR_INVALID_ARG, "a handle appears twice in the batch");
    }
    std::vector<int> pidx(k, -1);  // position of each run's replica partner in the batch
    bool any_pair = false;
    for (int i = 0; i < k; i++) {
        if (!hs[i]->partner) continue;
        for (int j = 0; j < k; j++)
            if (hs[j] == hs[i]->partner) pidx[i] = j;
        if (pidx[i] < 0) return fail(hs[0], FCIQMC_ERR_INVALID_ARG, "a replica is stepped without its partner");
        any_pair = true;
    }
    fciqmc_handle *h0 = hs[0];
    std::vector<long long> target(k);
    for (int i = 0; i < k; i++) {
        fciqmc_handle *h = hs[i];
        int rc = h->pending ? fciqmc_sync(h) : FCIQMC_OK;
        if (rc) return rc;
        rc = read_state(h);
        if (rc) return rc;
        if (h->hst.err) {  // leftover flags (e.g. a pending semi-stochastic set-up)
            int retries = 0;
            rc = handle_flags(h, &retries);
            if (rc) return rc;
        }
        CUDA_TRY(h, cudaStreamSynchronize(h->stream));
        target[i] = h->hst.iter + n_iter;
    }
    DevInst *dinst = (DevInst *)dev_alloc(h0, (size_t)k * sizeof(DevInst));
    int *dunit = (int *)dev_alloc(h0, (size_t)(k + 1) * sizeof(int));
    if (!dinst || !dunit) return fail(h0, FCIQMC_ERR_OUT_OF_MEMORY, "out of device memory (batch table)");
    cudaGraphExec_t gexec = nullptr;
    int units = 0, max_nd = 0;
    auto cleanup = [&]() {
        if (gexec) cudaGraphExecDestroy(gexec);
        gexec = nullptr;
    };
    auto rebuild = [&]() -> int {
        std::vector<DevInst> tab(k);
        std::vector<int> us(k + 1);
        units = 0;
        max_nd = 0;
        int max_bk = 1;
        for (int i = 0; i < k; i++) {
            int rq = ensure_queues(hs[i]);
            if (rq) return rq;
            tab[i] = hs[i]->hi;
            tab[i].partner = pidx[i];
            max_bk = std::max(max_bk, 1 << hs[i]->bb);
            tab[i].unit0 = units;
            us[i] = units;
            units += 1 << hs[i]->bb;
            max_nd = std::max(max_nd, hs[i]->nd);
        }
        us[k] = units;
        CUDA_TRY(h0, cudaMemcpy(dinst, tab.data(), (size_t)k * sizeof(DevInst), cudaMemcpyHostToDevice));
        CUDA_TRY(h0, cudaMemcpy(dunit, us.data(), (size_t)(k + 1) * sizeof(int), cudaMemcpyHostToDevice));
        cleanup();
        cudaGraph_t g;
        CUDA_TRY(h0, cudaStreamBeginCapture(h0->stream, cudaStreamCaptureModeThreadLocal));
        bool sp_staged = true, split = spawn_split_selected();
        for (int i = 0; i < k; i++) {
            sp_staged = sp_staged && staged_spawn_fits(tab[i]);
            split = split && tab[i].qcnt != nullptr;
        }
        launch_spawn(dinst, dunit, k, units, sp_staged, split, h0->stream);
        if (split && sp_staged) launch_spawn_eval(dinst, k, h0->stream);
        launch_spawn_heavy(dinst, k, h0->stream);
        if (max_nd > 0) launch_semistoch(dinst, k, max_nd, h0->stream);
        bool general = false, staged = true;
        for (int i = 0; i < k; i++) {
            general = general || tab[i].side || tab[i].adaptive;
            staged = staged && staged_annihilation_fits(tab[i]);
        }
        cudaError_t le = launch_annihilate(dinst, dunit, k, units, general, staged, h0->stream);
        launch_annihilate_big(dinst, k, h0->stream);
        launch_new_diag(dinst, k, h0->stream);
        cudaError_t xe = any_pair ? launch_replica_cross(dinst, k, max_bk, h0->stream) : cudaSuccess;
        launch_finalize(dinst, k, h0->stream);
        cudaError_t e = cudaStreamEndCapture(h0->stream, &g);
        if (le != cudaSuccess || xe != cudaSuccess || e != cudaSuccess)
            return fail(h0, FCIQMC_ERR_CUDA, "batch graph capture failed");
        e = cudaGraphInstantiate(&gexec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return fail(h0, FCIQMC_ERR_CUDA, "batch graph instantiate failed");
        return FCIQMC_OK;
    };
    int rc = FCIQMC_OK;
    for (int i = 0; i < k && !rc; i++) {
        hs[i]->hst.stop_iter = target[i];
        if (hs[i]->hst.iter >= target[i]) hs[i]->hst.err |= ERRB_STOP;
        rc = write_state(hs[i]);
    }
    if (!rc) rc = rebuild();
    long long chunk_max = 16;
    std::vector<int> retries(k, 0);
    while (!rc) {
        long long remaining = 0;
        for (int i = 0; i < k; i++) remaining = std::max(remaining, target[i] - hs[i]->hst.iter);
        if (remaining <= 0) break;
        const long long chunk = std::min<long long>(std::min<long long>(remaining, chunk_max), h0->ring_cap);
        chunk_max = std::min<long long>(chunk_max * 2, h0->ring_cap);
        std::vector<long long> start(k);
        for (int i = 0; i < k; i++) start[i] = hs[i]->hst.iter;
        for (long long c = 0; c < chunk && !rc; c++)
            if (cudaGraphLaunch(gexec, h0->stream) != cudaSuccess) rc = fail(h0, FCIQMC_ERR_CUDA, "batch graph launch failed");
        if (rc) break;
        if (cudaStreamSynchronize(h0->stream) != cudaSuccess) { rc = fail(h0, FCIQMC_ERR_CUDA, "batch synchronisation failed"); break; }
        bool changed = false;
        for (int i = 0; i < k && !rc; i++) {
            fciqmc_handle *h = hs[i];
            rc = read_state(h);
            if (rc) break;
            rc = pull_history(h, start[i], h->hst.iter);
            if (rc) break;
            const int err = h->hst.err & ~ERRB_STOP;
            if (err) {
                chunk_max = 16;
                const int bb0 = h->bb, nd0 = h->nd, cap0 = h->hi.cap_s, hc0 = h->heavy_cap;
                h->hst.err = err;  // keep the stop flag off while handling
                rc = handle_flags(h, &retries[i]);
                if (rc) { h->step_rc = rc; break; }
                if (h->bb != bb0 || h->nd != nd0 || h->hi.cap_s != cap0 || h->heavy_cap != hc0) changed = true;
                h->hst.stop_iter = target[i];
                if (h->hst.iter >= target[i]) h->hst.err |= ERRB_STOP;
                rc = write_state(h);
                changed = true;
            } else if (!(h->hst.err & ERRB_STOP) && h->hst.iter >= target[i]) {
                h->hst.err |= ERRB_STOP;
                rc = write_state(h);
            }
        }
        if (!rc && changed) rc = rebuild();
    }
    // restore the single-run state: no stop flag, own graph
    for (int i = 0; i < k; i++) {
        fciqmc_handle *h = hs[i];
        if (read_state(h)) continue;
        h->hst.err &= ~ERRB_STOP;
        h->hst.stop_iter = LLONG_MAX;
        write_state(h);
        capture_graph(h);
    }
    cleanup();
    dev_free(h0, dinst);
    dev_free(h0, dunit);
    if (!rc)
        for (int i = 0; i < k; i++) hs[i]->step_rc = 0;
    return rc;
}

int fciqmc_step_batch(fciqmc_handle **hs, int32_t k, int64_t n_iter)
{
    try {
        return step_batch_impl(hs, k, n_iter);
    } catch (const std::bad_alloc &) {
        return fail((hs ? hs[0] : nullptr), FCIQMC_ERR_OUT_OF_MEMORY, "host allocation failed");
    } catch (...) {
        return fail((hs ? hs[0] : nullptr), FCIQMC_ERR_OUT_OF_MEMORY, "host exception");
    }
}

int fciqmc_iter_stats_get(fciqmc_handle *h, int64_t first, int64_t count, fciqmc_iter_stats *out)
{
    if (!h || !out || first < 0 || count < 0 || first + count > (int64_t)h->hist.size()) return FCIQMC_ERR_INVALID_ARG;
    memcpy(out, h->hist.data() + first, (size_t)count * sizeof(fciqmc_iter_stats));
    return FCIQMC_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ statistics
// Error analysis of the estimators (the paper gives none): Flyvbjerg-Petersen
// blocking (J. Chem. Phys. 91, 461 (1989)) -- level k+1 holds the means of
// neighbouring pairs of level k, an odd last element dropped, down to two
// elements; the standard error of level k is sqrt(var_pop / (n_k - 1)) -- with
// the block length chosen by the rule of Lee et al. (Phys. Rev. E 83, 066706
// (2011)): the smallest level k with (2^k)^3 > 2 n_0 (SE_k / SE_0)^4 (the last
// level if none qualifies; level 0 for a constant series).
static std::vector<std::vector<double>> blocking_levels(const std::vector<double> &x)
{
    std::vector<std::vector<double>> lev;
    std::vector<double> y = x;
    while (y.size() >= 2) {
        std::vector<double> z(y.size() / 2);
        for (size_t i = 0; i < z.size(); i++) z[i] = 0.5 * (y[2 * i] + y[2 * i + 1]);
        lev.push_back(std::move(y));
        y = std::move(z);
    }
    return lev;
}

static double mean_of(const std::vector<double> &y)
{
    double m = 0.0;
    for (double v : y) m += v;
    return m / (double)y.size();
}

// (co)variance of the means of two equally long levels, their elements taken as independent
static double level_cov(const std::vector<double> &y, const std::vector<double> &z)
{
    const double my = mean_of(y), mz = mean_of(z);
    double c = 0.0;
    for (size_t i = 0; i < y.size(); i++) c += (y[i] - my) * (z[i] - mz);
    return c / (double)y.size() / (double)(y.size() - 1);
}

static int optimal_level(const std::vector<std::vector<double>> &lev)
{
    if (lev.empty()) return -1;
    const double n0 = (double)lev[0].size(), se0 = std::sqrt(level_cov(lev[0], lev[0]));
    if (se0 == 0.0) return 0;
    for (size_t k = 0; k < lev.size(); k++) {
        const double q = std::sqrt(level_cov(lev[k], lev[k])) / se0;
        const double b = std::ldexp(1.0, (int)k);
        if (b * b * b > 2.0 * n0 * (q * q) * (q * q)) return (int)k;
    }
    return (int)lev.size() - 1;
}

static double blocking_sigma(const std::vector<double> &x)
{
    const auto lev = blocking_levels(x);
    if (lev.empty()) return NAN;
    const int k = optimal_level(lev);
    return std::sqrt(level_cov(lev[k], lev[k]));
}

// ratio of the means of num and den; delta-method error
// (s_n^2 - 2 r c + r^2 s_d^2) / mean(den)^2 with the variances and the
// covariance of the two means at one level, the larger of the two optimal levels
static void ratio_blocking(const std::vector<double> &num, const std::vector<double> &den, double *ratio, double *sigma)
{
    const double mn = mean_of(num), md = mean_of(den), r = mn / md;
    *ratio = r;
    const auto ln = blocking_levels(num), ld = blocking_levels(den);
    if (ln.empty()) { *sigma = NAN; return; }
    const int k = std::max(optimal_level(ln), optimal_level(ld));
    const double vn = level_cov(ln[k], ln[k]), vd = level_cov(ld[k], ld[k]), c = level_cov(ln[k], ld[k]);
    *sigma = std::sqrt(std::max(vn - 2.0 * r * c + r * r * vd, 0.0)) / std::fabs(md);
}

static int energy_impl(fciqmc_handle *h, fciqmc_stats *out)
{
    if (!h || !out) return FCIQMC_ERR_INVALID_ARG;
    memset(out, 0, sizeof(*out));
    int rc = read_state(h);
    if (rc) return rc;
    out->iteration = h->hst.iter;
    out->eref = h->eref;
    out->shift = h->eref + h->hst.S;
    out->vary = h->hst.vary;
    out->equil_start = h->hst.vary ? h->hst.shift_start + 500 : -1;
    out->e_proj_mean = NAN;
    out->e_proj_sigma = NAN;
    out->shift_mean = NAN;
    out->shift_sigma = NAN;
    for (const auto &r : h->hist) {
        if (r.iteration < 0) continue;
        out->attempts_total += r.attempts;
        out->spawns_total += r.spawns;
        out->rejected_total += r.rejected;
        out->annihilated_total += r.annihilated;
    }
    if (!h->hist.empty()) {
        const auto &r = h->hist.back();
        out->nw = r.nw;
        out->ndet = r.ndet;
        out->e_proj_inst = r.e_den != 0.0 ? h->eref + r.e_num / r.e_den : NAN;
    }
    if (out->equil_start >= 0) {
        std::vector<double> num, den, sh;
        for (const auto &r : h->hist)
            if (r.iteration >= out->equil_start) { num.push_back(r.e_num); den.push_back(r.e_den); sh.push_back(r.shift); }
        out->n_samples = (int64_t)num.size();
        if (num.size() >= 8) {
            double ms = 0, r, sg;
            for (size_t i = 0; i < sh.size(); i++) ms += sh[i];
            ms /= sh.size();
            ratio_blocking(num, den, &r, &sg);
            out->e_proj_mean = h->eref + r;
            out->e_proj_sigma = sg;
            out->shift_mean = h->eref + ms;
            out->shift_sigma = blocking_sigma(sh);
        }
    }
    // replica pair (first replica): variational energy and PT2 correction
    out->e_var_mean = NAN;
    out->e_var_sigma = NAN;
    out->pt2_mean = NAN;
    out->pt2_sigma = NAN;
    if (h->partner && !h->secondary && out->equil_start >= 0 && h->partner->hst.vary) {
        const long long t0 = std::max<long long>(out->equil_start, h->partner->hst.shift_start + 500);
        std::vector<double> ov, vn, pt;
        for (const auto &r : h->hist)
            if (r.iteration >= t0 && r.x_overlap != 0.0) {
                ov.push_back(r.x_overlap);
                vn.push_back(r.x_var_num);
                pt.push_back(r.x_pt2);
            }
        out->pair_samples = (int64_t)ov.size();
        if (ov.size() >= 8) {
            double r, sg;
            ratio_blocking(vn, ov, &r, &sg);
            out->e_var_mean = h->eref + r;
            out->e_var_sigma = sg;
            ratio_blocking(pt, ov, &r, &sg);
            out->pt2_mean = r;
            out->pt2_sigma = sg;
        }
    }
    // trial-wave-function estimator (Sec. IV)
    out->e_trial_mean = NAN;
    out->e_trial_sigma = NAN;
    out->e_trial_T = h->trial_nt > 0 ? h->eref + h->trial_ET : NAN;
    if (h->trial_nt > 0 && out->equil_start >= 0) {
        const long long t0 = std::max<long long>(out->equil_start, h->hst.shift_start + h->p.trial_start);
        std::vector<double> num, den;
        for (const auto &r : h->hist)
            if (r.iteration >= t0 && r.trial_den != 0.0) { num.push_back(r.trial_num); den.push_back(r.trial_den); }
        out->trial_samples = (int64_t)num.size();
        if (num.size() >= 8) {
            double r, sg;
            ratio_blocking(num, den, &r, &sg);
            out->e_trial_mean = h->eref + r;
            out->e_trial_sigma = sg;
        }
    }
    return FCIQMC_OK;
}

extern "C" int fciqmc_energy(fciqmc_handle *h, fciqmc_stats *out)
{
    try {
        return energy_impl(h, out);
    } catch (const std::bad_alloc &) {
        return fail(h, FCIQMC_ERR_OUT_OF_MEMORY, "host allocation failed");
    } catch (...) {
        return fail(h, FCIQMC_ERR_OUT_OF_MEMORY, "host exception");
    }
}

extern "C" int64_t fciqmc_trial_info(fciqmc_handle *h, int64_t *n_w, double *ET, uint64_t *t_alpha, uint64_t *t_beta,
                                     double *cT, int64_t cap)
{
    if (!h || cap < 0) return FCIQMC_ERR_INVALID_ARG;
    if (n_w) *n_w = h->trial_nw;
    if (ET) *ET = h->trial_ET;
    const long long m = std::min<long long>(cap, h->trial_nt);
    if (m > 0 && (t_alpha || t_beta)) {
        std::vector<ulonglong2> k((size_t)m);
        if (cudaMemcpy(k.data(), h->trial_key, (size_t)m * sizeof(ulonglong2), cudaMemcpyDeviceToHost) != cudaSuccess)
            return fail(h, FCIQMC_ERR_CUDA, "trial copy failed");
        for (long long i = 0; i < m; i++) {
            if (t_alpha) t_alpha[i] = k[(size_t)i].x;
            if (t_beta) t_beta[i] = k[(size_t)i].y;
        }
    }
    if (m > 0 && cT &&
        cudaMemcpy(cT, h->trial_cT, (size_t)m * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
        return fail(h, FCIQMC_ERR_CUDA, "trial copy failed");
    return h->trial_nt;
}

// ------------------------------------------------------------------ time step
extern "C" int fciqmc_ref_offdiag_sum(fciqmc_handle *h, double *out)
{
    if (!h || !out) return FCIQMC_ERR_INVALID_ARG;
    *out = h->ref_sum;
    return FCIQMC_OK;
}

extern "C" double fciqmc_tau(fciqmc_handle *h) { return h ? h->p.tau : NAN; }

extern "C" int64_t fciqmc_pchb_table(fciqmc_handle *h, int32_t same_spin, int32_t i, int32_t j, double *S, double *lam,
                                     uint64_t *threshold, uint32_t *holes, int64_t cap)
{
    if (!h || !h->hi.pchb) return FCIQMC_ERR_INVALID_ARG;
    const int N = h->norb;
    if (i < 0 || j < 0 || i >= N || j >= N || (same_spin && i >= j) || cap < 0) return FCIQMC_ERR_INVALID_ARG;
    int64_t t, K;
    u64 off;
    if (!same_spin) {
        t = (int64_t)i * N + j;
        K = (int64_t)N * N;
        off = (u64)t * (u64)K;
    } else {
        const int64_t p = (int64_t)j * (j - 1) / 2 + i;
        t = (int64_t)N * N + p;
        K = (int64_t)N * (N - 1) / 2;
        off = h->hi.pchb_ss_base + (u64)p * (u64)K;
    }
    double2 mt;
    if (cudaMemcpy(&mt, h->hi.pchb_meta + t, sizeof(mt), cudaMemcpyDeviceToHost) != cudaSuccess)
        return fail(h, FCIQMC_ERR_CUDA, "heat-bath table copy failed");
    if (lam) *lam = mt.x;
    if (S) *S = mt.y;
    const int64_t m = std::min(K, cap);
    if (m > 0 && (threshold || holes)) {
        std::vector<ulonglong2> e((size_t)m);
        if (cudaMemcpy(e.data(), h->hi.pchb_ent + off, (size_t)m * sizeof(ulonglong2), cudaMemcpyDeviceToHost) !=
            cudaSuccess)
            return fail(h, FCIQMC_ERR_CUDA, "heat-bath table copy failed");
        for (int64_t k = 0; k < m; k++) {
            if (threshold) threshold[k] = e[k].x;
            if (holes) holes[k] = (uint32_t)e[k].y;
        }
    }
    return K;
}

// ------------------------------------------------------------------ serving
#include <chrono>
#include <deque>
#include <map>

namespace {

struct Request {
    int64_t id = 0;
    fciqmc_system sys{};
    std::vector<double> h1, eri;
    fciqmc_params p{};
    double target_sigma = 1e-3;
    int64_t max_iters = 0;
    fciqmc_request_status st{};
    fciqmc_handle *h = nullptr;
    int64_t est_bytes = 0;
};

}  // namespace

struct fciqmc_server {
    int64_t budget = 0;
    int max_active = 0;
    void *stream = nullptr;
    std::chrono::steady_clock::time_point t0;
    int64_t next_id = 1;
    std::deque<int64_t> queue;
    std::vector<int64_t> running;
    std::map<int64_t, Request> req;
    std::string err;
    double now() const { return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count(); }
};

// device memory a request needs when admitted: its initial layout and
// integrals, the attempt queues, and the first growth of the spawn regions (to 4 CAP_S0 slots per
// bucket, old and new buffers held together, with the large-bucket scratch)
static int64_t estimate_bytes(const Request &r)
{
    const int N = r.sys.kind == FCIQMC_HUBBARD ? r.sys.lx * r.sys.ly : r.sys.norb;
    const double np = (double)N * (N + 1) / 2, ne = np * (np + 1) / 2;
    double dets = r.p.max_dets > 0 ? (double)r.p.max_dets : std::min(std::max(4096.0, r.p.target_walkers), 8388608.0);
    int bb = 0;
    while (((double)(1LL << bb)) * (CAP_M / 2.5) < dets && bb < MAX_BB) bb++;
    const double per_bucket = 2.0 * CAP_M * (16 + 8 + 8 + 1) + 5.0 * CAP_S0 * 24.0 + 2 * 8 + sizeof(Partial) + 3 * 4 +
                              4.0 * CAP_M;
    const double ecap = CAP_M + 4.0 * CAP_S0;
    int tb = TABBITS;
    while ((double)(1 << tb) < 2.0 * ecap) tb++;
    const double scratch = (double)BIG_BLOCKS * (ecap * 52.0 + 4.0 * (double)(1 << tb) + 256.0);
    // the attempt queues of split spawning at their first size
    const double queues = 2.0 * (double)std::min(draw_segments(), 1 << bb) * (4096.0 * sizeof(QRec) + 4.0);
    return (int64_t)((double)(1LL << bb) * per_bucket + scratch + queues + 8.0 * (N * N + ne) + 48.0 * N * N +
                     4096.0 * 88 + 1.0e6);
}

extern "C" {

int fciqmc_server_create(int64_t mem_budget_bytes, int32_t max_active, void *stream, fciqmc_server **out)
{
    if (!out || mem_budget_bytes <= 0 || max_active < 1) return FCIQMC_ERR_INVALID_ARG;
    fciqmc_server *s = new fciqmc_server();
    s->budget = mem_budget_bytes;
    s->max_active = max_active;
    s->stream = stream;
    s->t0 = std::chrono::steady_clock::now();
    *out = s;
    return FCIQMC_OK;
}

double fciqmc_server_clock(fciqmc_server *srv) { return srv ? srv->now() : NAN; }

static int server_submit_impl(fciqmc_server *srv, const fciqmc_system *sys, const fciqmc_params *params, double target_sigma,
                              double t_arrival, int64_t max_iters, int64_t *id)
{
    if (!srv || !sys || !params || !id || !(target_sigma > 0.0) || max_iters < 1) return FCIQMC_ERR_INVALID_ARG;
    if (params->replicas > 1) return FCIQMC_ERR_UNSUPPORTED;  // the server batches single runs
    Request r;
    r.id = srv->next_id++;
    r.sys = *sys;
    if (sys->kind == FCIQMC_ABINITIO) {
        if (sys->norb < 1 || sys->norb > 64 || !sys->h1 || !sys->eri) return FCIQMC_ERR_INVALID_ARG;
        const int64_t N = sys->norb, np = N * (N + 1) / 2, ne = np * (np + 1) / 2;
        r.h1.assign(sys->h1, sys->h1 + N * N);
        r.eri.assign(sys->eri, sys->eri + ne);
    }
    r.p = *params;
    r.p.stream = srv->stream;
    r.target_sigma = target_sigma;
    r.max_iters = max_iters;
    r.est_bytes = estimate_bytes(r);
    r.st.state = 0;
    r.st.t_submit = srv->now();
    r.st.t_arrival = (t_arrival >= 0.0) ? t_arrival : r.st.t_submit;  // NaN compares false: now
    r.st.energy = NAN;
    r.st.sigma = NAN;
    *id = r.id;
    const double ta = r.st.t_arrival;
    srv->req[r.id] = std::move(r);
    // queued in order of arrival (ties: order of submission)
    auto pos = srv->queue.end();
    while (pos != srv->queue.begin() && srv->req[*(pos - 1)].st.t_arrival > ta) --pos;
    srv->queue.insert(pos, *id);
    return FCIQMC_OK;
}

int fciqmc_server_submit(fciqmc_server *srv, const fciqmc_system *sys, const fciqmc_params *params, double target_sigma,
                         double t_arrival, int64_t max_iters, int64_t *id)
{
    try {
        return server_submit_impl(srv, sys, params, target_sigma, t_arrival, max_iters, id);
    } catch (const std::bad_alloc &) {
        return fail(nullptr, FCIQMC_ERR_OUT_OF_MEMORY, "host allocation failed");
    } catch (...) {
        return fail(nullptr, FCIQMC_ERR_OUT_OF_MEMORY, "host exception");
    }
}

// the energy a request reports: E_Trial when it has enough samples and the
// smaller error, else E_proj; returns its sample count
static int64_t best_energy(const fciqmc_stats &st, fciqmc_request_status &o)
{
    const bool trial = st.trial_samples >= 200 && std::isfinite(st.e_trial_sigma) &&
                       !(st.e_proj_sigma <= st.e_trial_sigma);
    o.energy = trial ? st.e_trial_mean : st.e_proj_mean;
    o.sigma = trial ? st.e_trial_sigma : st.e_proj_sigma;
    o.estimator = trial ? 1 : 0;
    return trial ? st.trial_samples : st.n_samples;
}

static void retire(fciqmc_server *srv, Request &r, int state)
{
    fciqmc_stats st;
    if (r.h && fciqmc_energy(r.h, &st) == FCIQMC_OK) {
        r.st.iterations = st.iteration;
        best_energy(st, r.st);
        r.st.shift = st.shift;
        r.st.attempts = st.attempts_total;
    }
    if (r.h) {
        r.st.device_bytes = std::max<int64_t>(r.st.device_bytes, (int64_t)r.h->bytes);
        fciqmc_destroy(r.h);
    }
    r.h = nullptr;
    r.st.state = state;
    r.st.t_done = srv->now();
}

static int server_tick_impl(fciqmc_server *srv, int64_t n_iter, int32_t *n_active)
{
    if (!srv || n_iter < 1) return FCIQMC_ERR_INVALID_ARG;
    // 1. admission: first come, first served, by device memory
    int64_t used = 0;
    for (int64_t id : srv->running) used += (int64_t)srv->req[id].h->bytes;
    const double now = srv->now();
    while (!srv->queue.empty() && (int)srv->running.size() < srv->max_active) {
        Request &r = srv->req[srv->queue.front()];
        if (r.st.t_arrival > now) break;  // not arrived yet
        if (!srv->running.empty() && used + r.est_bytes > srv->budget) break;
        srv->queue.pop_front();
        fciqmc_system sys = r.sys;
        if (sys.kind == FCIQMC_ABINITIO) { sys.h1 = r.h1.data(); sys.eri = r.eri.data(); }
        fciqmc_params p = r.p;
        if (p.max_device_bytes <= 0) p.max_device_bytes = std::max<int64_t>(srv->budget - used, r.est_bytes);
        int rc = fciqmc_create(&sys, &p, &r.h);
        r.st.t_start = srv->now();
        if (rc) {
            r.st.state = 4;
            r.st.error = rc;
            r.st.t_done = r.st.t_start;
            continue;
        }
        r.st.state = 1;
        r.st.tau = r.h->p.tau;
        used += (int64_t)r.h->bytes;
        srv->running.push_back(r.id);
    }
    // 2. advance every running request together
    if (!srv->running.empty()) {
        std::vector<fciqmc_handle *> hs;
        for (int64_t id : srv->running) hs.push_back(srv->req[id].h);
        int rc = fciqmc_step_batch(hs.data(), (int32_t)hs.size(), n_iter);
        if (rc) {
            // the failing run(s): a recorded step error, a flag left up, or no
            // readable energy; when none can be told apart every run of the
            // batch is retired, so that a tick never repeats a failing batch
            int n_retired = 0;
            for (int64_t id : srv->running) {
                Request &r = srv->req[id];
                fciqmc_stats st;
                if (r.h->step_rc || fciqmc_energy(r.h, &st) != FCIQMC_OK ||
                    r.h->hst.err & ~(ERRB_STOP | ERRB_PAUSE_SEMI | ERRB_PAUSE_TRIAL)) {
                    r.st.error = r.h->step_rc ? r.h->step_rc : rc;
                    retire(srv, r, 4);
                    n_retired++;
                }
            }
            if (!n_retired)
                for (int64_t id : srv->running) {
                    Request &r = srv->req[id];
                    r.st.error = rc;
                    retire(srv, r, 4);
                }
        }
    }
    // 3. retire converged or exhausted requests
    std::vector<int64_t> still;
    for (int64_t id : srv->running) {
        Request &r = srv->req[id];
        if (!r.h) continue;
        r.st.device_bytes = std::max<int64_t>(r.st.device_bytes, (int64_t)r.h->bytes);
        fciqmc_stats st;
        if (fciqmc_energy(r.h, &st) != FCIQMC_OK) { retire(srv, r, 4); continue; }
        r.st.iterations = st.iteration;
        const int64_t ns = best_energy(st, r.st);
        r.st.attempts = st.attempts_total;
        if (ns >= 200 && r.st.sigma < r.target_sigma) retire(srv, r, 2);
        else if (st.iteration >= r.max_iters) retire(srv, r, 3);
        else still.push_back(id);
    }
    srv->running.swap(still);
    if (n_active) *n_active = (int32_t)(srv->running.size() + srv->queue.size());
    return FCIQMC_OK;
}

int fciqmc_server_tick(fciqmc_server *srv, int64_t n_iter, int32_t *n_active)
{
    try {
        return server_tick_impl(srv, n_iter, n_active);
    } catch (const std::bad_alloc &) {
        return fail(nullptr, FCIQMC_ERR_OUT_OF_MEMORY, "host allocation failed");
    } catch (...) {
        return fail(nullptr, FCIQMC_ERR_OUT_OF_MEMORY, "host exception");
    }
}

int fciqmc_server_poll(fciqmc_server *srv, int64_t id, fciqmc_request_status *out)
{
    if (!srv || !out) return FCIQMC_ERR_INVALID_ARG;
    auto it = srv->req.find(id);
    if (it == srv->req.end()) return FCIQMC_ERR_INVALID_ARG;
    *out = it->second.st;
    return FCIQMC_OK;
}

void fciqmc_server_destroy(fciqmc_server *srv)
{
    if (!srv) return;
    for (auto &kv : srv->req)
        if (kv.second.h) fciqmc_destroy(kv.second.h);
    delete srv;
}

}  // extern "C"

// ------------------------------------------------------------------ FCIDUMP
#include <cctype>
#include <fstream>
#include <sstream>

static bool namelist_int(const std::string &nl, const char *key, long long *v)
{
    std::string up;
    for (char c : nl) up += (char)std::toupper((unsigned char)c);
    std::string k(key);
    size_t pos = 0;
    while ((pos = up.find(k, pos)) != std::string::npos) {
        const bool left_ok = pos == 0 || !std::isalnum((unsigned char)up[pos - 1]);
        size_t q = pos + k.size();
        while (q < up.size() && std::isspace((unsigned char)up[q])) q++;
        if (left_ok && q < up.size() && up[q] == '=') {
            q++;
            while (q < up.size() && std::isspace((unsigned char)up[q])) q++;
            char *end = nullptr;
            const long long x = std::strtoll(up.c_str() + q, &end, 10);
            if (end != up.c_str() + q) { *v = x; return true; }
        }
        pos += k.size();
    }
    return false;
}

static int read_fcidump_impl(const char *path, fciqmc_system *out)
{
    if (!path || !out) return FCIQMC_ERR_INVALID_ARG;
    std::ifstream f(path);
    if (!f) { g_create_error = std::string("cannot open ") + path; return FCIQMC_ERR_INVALID_ARG; }
    std::string line, nl;
    bool done = false;
    while (!done && std::getline(f, line)) {
        nl += line + " ";
        std::string up;
        for (char c : line) up += (char)std::toupper((unsigned char)c);
        if (up.find("&END") != std::string::npos || up.find('/') != std::string::npos) done = true;
    }
    long long norb = 0, nelec = 0, ms2 = 0;
    if (!done || !namelist_int(nl, "NORB", &norb) || !namelist_int(nl, "NELEC", &nelec)) {
        g_create_error = "FCIDUMP namelist without NORB/NELEC";
        return FCIQMC_ERR_INVALID_ARG;
    }
    namelist_int(nl, "MS2", &ms2);
    if (norb < 1 || norb > 64 || nelec < 1 || (nelec + ms2) % 2 || nelec + ms2 < 0 || nelec - ms2 < 0 ||
        (nelec + ms2) / 2 > norb || (nelec - ms2) / 2 > norb) {
        g_create_error = "FCIDUMP sizes outside 1 <= NORB <= 64 or inconsistent NELEC/MS2";
        return FCIQMC_ERR_INVALID_ARG;
    }
    const long long N = norb, np = N * (N + 1) / 2, ne = np * (np + 1) / 2;
    double *h = (double *)std::calloc((size_t)(N * N), sizeof(double));
    double *eri = (double *)std::calloc((size_t)ne, sizeof(double));
    if (!h || !eri) { std::free(h); std::free(eri); return FCIQMC_ERR_OUT_OF_MEMORY; }
    double ecore = 0.0;
    while (std::getline(f, line)) {
        for (char &c : line) if (c == 'D' || c == 'd') c = 'E';  // Fortran exponents
        std::istringstream is(line);
        double v;
        long long i, j, k, l;
        if (!(is >> v >> i >> j >> k >> l)) continue;
        if (i < 0 || j < 0 || k < 0 || l < 0 || i > N || j > N || k > N || l > N) {
            std::free(h); std::free(eri);
            g_create_error = "FCIDUMP index out of range";
            return FCIQMC_ERR_INVALID_ARG;
        }
        if (i == 0 && j == 0 && k == 0 && l == 0) ecore = v;
        else if (k == 0 && l == 0) {
            if (i == 0 || j == 0) continue;  // orbital energies: not part of H
            h[(i - 1) * N + (j - 1)] = v;
            h[(j - 1) * N + (i - 1)] = v;
        } else if (i && j && k && l) {
            eri[pair_index(pair_index(i - 1, j - 1), pair_index(k - 1, l - 1))] = v;
        }
    }
    memset(out, 0, sizeof(*out));
    out->kind = FCIQMC_ABINITIO;
    out->norb = (int32_t)N;
    out->n_alpha = (int32_t)((nelec + ms2) / 2);
    out->n_beta = (int32_t)((nelec - ms2) / 2);
    out->ecore = ecore;
    out->h1 = h;
    out->eri = eri;
    return FCIQMC_OK;
}

extern "C" int fciqmc_read_fcidump(const char *path, fciqmc_system *out)
{
    try {
        return read_fcidump_impl(path, out);
    } catch (const std::bad_alloc &) {
        return fail(nullptr, FCIQMC_ERR_OUT_OF_MEMORY, "host allocation failed");
    } catch (...) {
        return fail(nullptr, FCIQMC_ERR_OUT_OF_MEMORY, "host exception");
    }
}

extern "C" void fciqmc_free_system(fciqmc_system *sys)
{
    if (!sys) return;
    std::free((void *)sys->h1);
    std::free((void *)sys->eri);
    sys->h1 = nullptr;
    sys->eri = nullptr;
}

// ------------------------------------------------------------------ autotuner
static int autotune_impl(fciqmc_handle **hs, int32_t k, int64_t n_iter, int32_t out[3])
{
    if (!hs || k < 1 || n_iter < 1 || !out) return FCIQMC_ERR_INVALID_ARG;
    // annihilation: 0 = the staged kernel (bulk copies one bucket ahead, two
    // blocks per SM), else the plain-load kernel with that many blocks per SM
    const int spawn_c[] = {0, 1, 2, 4, 8, 16}, anni_c[] = {0, 3, 9, 24}, heavy_c[] = {1, 2, 4};
    int best_s = 1, best_h = 2, best_a = 0;
    double best = 1e300;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    auto timed = [&](int sb, int hb, int ab, double *ms) -> int {
        set_launch_geometry(sb, hb, ab);
        for (int i = 0; i < k; i++) {
            int rc = capture_graph(hs[i]);
            if (rc) return rc;
        }
        cudaStream_t st = hs[0]->stream;
        cudaEventRecord(e0, st);
        int rc = fciqmc_step_batch(hs, k, n_iter);
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        float m = 0.f;
        cudaEventElapsedTime(&m, e0, e1);
        *ms = m;
        return rc;
    };
    // one sweep per kernel, the others held at their current best
    for (int sb : spawn_c) {
        double ms;
        int rc = timed(sb, best_h, best_a, &ms);
        if (rc) return rc;
        if (ms < best) { best = ms; best_s = sb; }
    }
    best = 1e300;
    for (int ab : anni_c) {
        double ms;
        int rc = timed(best_s, best_h, ab, &ms);
        if (rc) return rc;
        if (ms < best) { best = ms; best_a = ab; }
    }
    best = 1e300;
    for (int hb : heavy_c) {
        double ms;
        int rc = timed(best_s, hb, best_a, &ms);
        if (rc) return rc;
        if (ms < best) { best = ms; best_h = hb; }
    }
    set_launch_geometry(best_s, best_h, best_a);
    for (int i = 0; i < k; i++) capture_graph(hs[i]);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    out[0] = best_s; out[1] = best_h; out[2] = best_a;
    return FCIQMC_OK;
}

extern "C" int fciqmc_autotune(fciqmc_handle **hs, int32_t k, int64_t n_iter, int32_t out[3])
{
    try {
        return autotune_impl(hs, k, n_iter, out);
    } catch (const std::bad_alloc &) {
        return fail((hs ? hs[0] : nullptr), FCIQMC_ERR_OUT_OF_MEMORY, "host allocation failed");
    } catch (...) {
        return fail((hs ? hs[0] : nullptr), FCIQMC_ERR_OUT_OF_MEMORY, "host exception");
    }
}
