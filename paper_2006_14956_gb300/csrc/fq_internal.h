// fq_internal.h -- layout shared by the host driver (capi.cu) and the kernels
// (kernels.cu) of the GB300 FCIQMC library.  Not part of the public ABI.
#pragma once
#include <stdint.h>
#include <cuda_runtime.h>

#include "../../include/fciqmc.h"

namespace fq {

typedef unsigned long long u64;
typedef __int128 i128;
typedef unsigned __int128 u128;

// excitation classes; lambda_c = tau / p_gen(c)
enum { CLS_SINGLE_A = 0, CLS_SINGLE_B, CLS_DOUBLE_AB, CLS_DOUBLE_AA, CLS_DOUBLE_BB, CLS_HOP, NCLS };
// Philox counter purposes
enum { PURPOSE_SPAWN = 1, PURPOSE_DEATH = 2, PURPOSE_ANNIH = 3 };
// device error bits (IterState::err)
enum {
    ERRB_SPAWN_CAP = 1,   // a bucket received more spawns than it holds
    ERRB_MAIN_CAP = 2,    // a bucket's new list exceeds its capacity
    ERRB_HEAVY_CAP = 4,   // heavy-determinant chunk queue full
    ERRB_NUMERIC = 8,     // NaN/Inf or |C|, |w| beyond 2^31
    ERRB_TIMEOUT = 16,    // bounded wait expired
    ERRB_PAUSE_SEMI = 32, // iteration boundary at which D must be built (not an error)
    ERRB_STOP = 64,       // the run reached its stop iteration inside a batch (not an error)
    ERRB_PAUSE_TRIAL = 128,  // iteration boundary at which the trial space must be built (not an error)
    ERRB_PARTNER = 256,      // the other replica of a pair failed this iteration: repeat it (not an error)
    ERRB_QUEUE_CAP = 512,    // a segment of the attempt queues overflowed (split spawning)
};
// errors raised before the finalize kernel: a replica commits its iteration
// only if neither it nor its partner has one
constexpr int ERRB_STAGE = ERRB_SPAWN_CAP | ERRB_MAIN_CAP | ERRB_HEAVY_CAP | ERRB_NUMERIC | ERRB_TIMEOUT | ERRB_QUEUE_CAP;
enum { DFLAG_REF = 1, DFLAG_D = 2 };

// launch geometry
constexpr int K1_THREADS = 256;
constexpr unsigned HEAVY_ATT = 2048;  // attempts per heavy chunk
constexpr int K3_THREADS = 256;
constexpr int EMAX = 1280;            // main + spawned records staged per bucket in shared memory (3 blocks per SM)
constexpr int CAP_M = 1024;           // main-list capacity per bucket
constexpr int MAX_BB = 22;            // at most 2^22 buckets: slot indices (bucket * CAP_M + position) fit 32 bits
constexpr int CAP_S0 = EMAX - CAP_M;  // initial spawn capacity per bucket (grows at run time)
constexpr int TABBITS = 12;           // shared-memory hash table of the annihilation (2 x EMAX slots)
constexpr int BIG_BLOCKS = 64;        // blocks of the large-bucket annihilation kernel
constexpr int K5_THREADS = 256;
constexpr int KIDX = 2048;            // slots of the per-bucket list index (adaptive shift)
constexpr int STAGED_SCAP = 256;      // spawn records per bucket the staged annihilation holds

struct HeavyChunk {  // a slice of the attempts of one determinant with many walkers
    u64 a, b;
    double cper;
    u64 k0;
    uint32_t count;
    uint32_t flags;  // bit 0: initiator, bit 1: parent in D
    uint32_t slot;   // the determinant's main-list slot (adaptive shift)
    uint32_t pad;
};

// Split spawning: every drawn attempt is queued in global memory by class
// (0: singles and lattice hops, 1: doubles), in the segment of the drawing
// block (bucket b of a run goes to segment b mod the draw kernel's grid), and
// evaluated by a flat kernel with one attempt per thread.
constexpr int NSEG_MAX = 1024;  // segments per class (the draw kernel's grid) at most
struct QRec {  // 48 bytes
    u64 ka, kb;      // parent
    double cper;     // C_i / n_att
    u64 w2, w3;      // hole word, rounding word
    unsigned slot;   // parent's main-list slot (adaptive shift)
    unsigned info;   // electron (single, hop) or pair e1 | e2 << 8 (double) | parent flags << 16
};

struct Partial {  // per-bucket binary64 sums of one iteration (estimators that need them)
    double t_num, t_den;    // trial-wave-function estimator
    double x_ov, x_hd, x_cr, x_pt2;  // replica pair: overlap, diagonal and spawn cross terms, PT2 sum
    double pad[2];
};

// Exact per-iteration totals, accumulated by atomic adds of every bucket's
// share into one of NSHARD 128-byte lines (bucket b uses line b % NSHARD, so
// the adds spread over L2 slices): 128-bit integers as three limbs (bits 0-39
// and 40-79 unsigned, the rest signed), so that no add needs another's result
// and every order gives the same sum; counts as plain 64-bit adds.  k_finalize
// sums the lines and clears them when it commits the iteration; the host
// clears them before a repeated one.
enum {
    ACC_NW = 0,      // N_w * 2^32, three limbs
    ACC_ANN = 3,     // annihilated walkers * 2^32, three limbs
    ACC_ENUM = 6,    // E_num * 2^Fe (every term truncated to the grid), three limbs
    ACC_NDET = 9, ACC_REJ, ACC_SPAWNS, ACC_ATT,
    NACC
};
constexpr int LIMB = 40;
constexpr int NSHARD = 32, ACC_STRIDE = 16;  // lines, words per line (NACC <= ACC_STRIDE)

struct SideEnt {  // one determinant of a bucket in one replica's iteration (pairs only)
    u64 a, b;
    double c0;    // amplitude at the start of the iteration
    double hd;    // H_jj - E_ref if the determinant was in the list, else 0
    double sacc;  // accepted spawns (exact sum, rounded once)
    double srej;  // spawns removed by the initiator rule (exact sum, rounded once)
};

struct IterState {  // device-resident iteration state of one run
    long long iter;
    int parity;
    int vary;
    double S;
    long long shift_start;
    long long cnt;
    u64 nwl_hi, nwl_lo;     // N_w(2^32 units) at the last shift update
    int err;
    int heavy_n;
    double e_den;
    long long semi_built;   // 1 once D exists
    int big_n;              // buckets deferred to the large-bucket kernel
    int need_spawn;         // largest spawn count of an overflowing bucket
    int need_main;          // largest new-list size of an overflowing bucket
    int n_spawn_over;       // buckets whose spawns overflowed
    long long stop_iter;    // K5 raises ERRB_STOP when iter reaches it
    long long trial_built;  // 1 once the trial space exists
    int new_n;              // determinants created in this iteration (their H_jj is computed by k_new_diag)
    int err_at_start;       // err when the iteration's spawning began (nonzero: the iteration was skipped)
    int need_queue[2];      // largest count a queue segment of each class needed (split spawning)
};

struct TrialEnt;

// one run as seen by the kernels
struct DevInst {
    // system
    int kind, norb, na, nb, n, ma, mb, z;
    int F;    // exact-sum scale of the integrals: value = X * 2^-F
    int Fw;   // exact-sum scale of spawned weights
    int Fe;   // fixed-point scale of the E_num total
    const double *h;
    const double *eri;
    const int *nbr;
    const ulonglong2 *hfx;  // h_pp, fixed point (lo, hi)
    const ulonglong2 *Jfx;  // (pp|qq)
    const ulonglong2 *JKfx; // (pp|qq) - (pq|qp)
    const ulonglong2 *Sfx;  // [(a N + i) N + k][2]: (ai|kk), (ai|kk) - (ak|ki); NULL = convert on the fly
    u64 xref_lo, xref_hi;   // exact diagonal sum of the reference
    u64 ref_a, ref_b;
    u64 normask;
    double lam[NCLS];
    double tmt;             // -t (Hubbard hopping matrix element)
    u64 tsingle;            // single excitation iff (w0 >> 11) < tsingle
    // ceil(2^64 / d) for the run's fixed divisors d = n - 1, m_beta,
    // m_alpha - 1, m_beta - 1 (0 for d = 1): x / d = umulhi(x, M) exactly
    // for x < 2^32
    u64 mg_n1, mg_mb, mg_ma1, mg_mb1;
    u64 seed;
    double tau, cmin, n_a;
    int cmin_log2;          // c_min = 2^cmin_log2 when cmin_pow2
    int cmin_pow2;
    double cz;              // shift_damping / (A tau)
    double target;
    long long A;
    long long semi_start;
    long long semi_size;
    // layout
    int bb;                 // buckets = 1 << bb
    int unit0;              // first global unit (bucket) index of this run
    ulonglong2 *key[2];
    double *c[2];
    double *hd[2];
    uint8_t *fl[2];
    int *cnt[2];
    ulonglong2 *skey;
    double *sw;
    int *scnt_i;
    int *scnt_n;
    int cap_s;              // spawn capacity per bucket
    int big_tabbits;        // hash-table bits of the large-bucket path
    int *big_list;          // deferred bucket ids (capacity = buckets)
    unsigned *newdet;       // main-list slots of the determinants created in this iteration
    unsigned char *big_scratch;  // BIG_BLOCKS slices of big_stride bytes
    size_t big_stride;
    HeavyChunk *heavy;
    int heavy_cap;
    QRec *qrec[2];          // attempt queues by class: qnseg segments of qcap[class] entries each
    int *qcnt;              // [2 * qnseg]: entries queued per segment, singles then doubles (cleared by k_finalize)
    int qnseg;              // segments per class
    long long qcap[2];
    Partial *part;
    u64 *acc;  // exact totals of the iteration: NSHARD lines of ACC_STRIDE words (see ACC_*)
    IterState *st;
    fciqmc_iter_stats *ring;
    int ring_cap;
    // semi-stochastic space D (sorted keys, CSR of H^D - E_ref, new amplitudes)
    int nd;
    const ulonglong2 *dkey;
    const long long *drow;
    const int *dcol;
    const double *dval;     // H^D - E_ref on the diagonal
    double *dc_new;         // C_D after the exact projection of this iteration
    double *dc_buf[2];      // C_D after the last completed iteration, by list parity
    const u64 *dhash_keys;  // open-addressing set of D keys (a, b interleaved), size dhash_cap
    const int *dhash_idx;   // per slot of that set: the key's position in dkey
    int dhash_bits;
    // pre-computed heat-bath doubles (generator 1): opposite-spin table of
    // (i alpha, j beta) at meta[i N + j], entries [(i N + j) N^2, +N^2), entry
    // k = a N + b; same-spin table of i < j at meta[N^2 + p], p = j(j-1)/2 + i,
    // entries [ss_base + p K_ss, +K_ss), K_ss = N(N-1)/2, entry k = b(b-1)/2 + a
    // (a < b).  meta = (|H|/p_gen of every entry, sum of |H|); entry =
    // (alias threshold on 53-bit words, own hole pair | alias's hole pair << 16),
    // hole pair = a | b << 8.
    int pchb;
    const double2 *pchb_meta;
    const ulonglong2 *pchb_ent;
    u64 pchb_ss_base;
    // adaptive shift (Sec. V): per main-list slot the exact sums A (accepted)
    // and T (all) of the weights of the iteration's spawns, 4 words (A lo, hi,
    // T lo, hi), by parity; per bucket KIDX slots of list positions + 1 (an
    // open-addressing index of the list on the determinant hash), by parity
    int adaptive;
    u64 *facc[2];
    unsigned short *kidx[2];
    // replica pair: key word 1 of every Philox draw; index of the other
    // replica in the instance table (-1: none); per-bucket lists of the
    // determinants of the iteration (side_cap entries per bucket)
    u64 replica;
    int partner;
    int side_cap;
    SideEnt *side;
    int *side_cnt;
    // trial-wave-function estimator: open-addressing table of W_j and cT_j
    // (slot state 0 empty, 1 being written, 2 ready), 2^trial_bits slots
    long long trial_size, trial_start;
    int trial_bits;
    const unsigned *trial_state;
    const TrialEnt *trial_tab;
};

struct TrialEnt {
    u64 a, b;
    double w;   // <Psi^T|H - E_ref|D_j>
    double cT;  // component of Psi^T (0 outside T)
};

// host-side launchers (kernels.cu)
void launch_spawn(const DevInst *dinst, const int *unit_start, int n_inst, int n_units, bool staged, bool split,
                  cudaStream_t s);
bool spawn_split_selected();
int draw_segments();  // the draw kernel's largest grid: a run needs min(this, buckets) queue segments
void launch_spawn_eval(const DevInst *dinst, int n_inst, cudaStream_t s);
bool staged_spawn_fits(const DevInst &I);
void launch_spawn_heavy(const DevInst *dinst, int n_inst, cudaStream_t s);
void launch_semistoch(const DevInst *dinst, int n_inst, int max_nd, cudaStream_t s);
cudaError_t launch_annihilate(const DevInst *dinst, const int *unit_start, int n_inst, int n_units, bool general,
                              bool staged, cudaStream_t s);
bool staged_annihilation_fits(const DevInst &I);
cudaError_t init_kernels();
size_t annihilate_smem_bytes();
void launch_annihilate_big(const DevInst *dinst, int n_inst, cudaStream_t s);
void launch_finalize(const DevInst *dinst, int n_inst, cudaStream_t s);
void launch_new_diag(const DevInst *dinst, int n_inst, cudaStream_t s);
void launch_build_kidx(const DevInst *dinst, int parity, int nb, cudaStream_t s);
cudaError_t launch_replica_cross(const DevInst *dinst, int n_inst, int max_buckets, cudaStream_t s);
cudaError_t replica_kernel_init();
void launch_rebucket(const DevInst *src, const DevInst *dst, int nb_src, int parity, cudaStream_t s);
void launch_diag(const DevInst *dinst, int parity, int nb, cudaStream_t s);
void launch_diag_list(const DevInst *dinst, int par, const unsigned *list, int nn, cudaStream_t s);
cudaError_t launch_import_check(const u64 *a, const u64 *b, const double *c, long long n, int na, int nb, u64 normask,
                                u64 ra, u64 rb, int *flags, cudaStream_t s);
cudaError_t launch_import_count(const u64 *a, const u64 *b, long long n, int bb, int *cnt, int *over, cudaStream_t s);
cudaError_t launch_import_place(const u64 *a, const u64 *b, const double *c, long long n, int bb, u64 ra, u64 rb,
                                int *fill, ulonglong2 *key, double *oc, uint8_t *ofl, unsigned *list, cudaStream_t s);
void launch_abs_hist(const DevInst *dinst, int par, int nb, int shift, u64 prefix, unsigned *hist, cudaStream_t s);
void launch_abs_collect(const DevInst *dinst, int par, int nb, u64 thr, ulonglong2 *keys, u64 *mags, int *n, int cap,
                        cudaStream_t s);
void launch_build_hd(const DevInst *dinst, int nd, const ulonglong2 *dkey, long long *rowcnt, const long long *rowptr,
                     int *col, double *val, int pass, cudaStream_t s);
void launch_mark_d(const DevInst *dinst, int parity, int nb, cudaStream_t s);

cudaError_t launch_pchb_build(const DevInst *dinst, int norb, double ppair, double2 *meta, ulonglong2 *ent,
                              u64 ss_base, cudaStream_t s);
cudaError_t launch_trial_dense(const long long *rowptr, const int *col, const double *val, int nt, int n2, double *A,
                               double *hdiag, cudaStream_t s);
cudaError_t launch_jacobi_lowest(double *A, double *V, int n, int n2, double *E, double *v, int *sweeps,
                                 cudaStream_t s);
cudaError_t launch_trial_w(const DevInst *dinst, const ulonglong2 *tkey, const double *cT, const double *hdiag, int nt,
                           long long per_det, unsigned *state, TrialEnt *tab, int bits, unsigned long long *count,
                           int *err, cudaStream_t s);
long long connections_per_det(int na, int nb, int ma, int mb);
void set_launch_geometry(int spawn_bps, int heavy_bps, int anni_bps);
int launch_geometry_generation();
void get_launch_geometry(int *spawn_bps, int *heavy_bps, int *anni_bps);
cudaError_t ref_abs_sum(const DevInst *dinst, double *dpartial, double *out, cudaStream_t s);
size_t export_scratch_bytes(long long n);
cudaError_t export_sorted(const ulonglong2 *key, const double *c, const double *hd, const uint8_t *fl, const int *cnt,
                          const long long *off, int nbk, long long n, int norb, void *scratch, const u64 **oa,
                          const u64 **ob, const double **oc, const double **ohd, const int32_t **ofl, cudaStream_t s);

// host helpers shared with capi.cu
u64 det_hash_host(u64 a, u64 b);

}  // namespace fq
