/*
 * fciqmc.h -- C ABI of the GB300 initiator-FCIQMC library.
 *
 * One handle = one FCIQMC run: a sparse walker list of Slater determinants
 * (two uint64 occupation words, alpha and beta) with signed binary64
 * amplitudes, resident in device memory, advanced by the projector
 * psi(t + dt) = (1 - dt (H - S)) psi(t) of Eq. (2) of Guther et al.,
 * J. Chem. Phys. 153, 034107 (2020) (arXiv:2006.14956), in the three steps
 * of its Eq. (4): spawning, death, annihilation, with the initiator rule of
 * Sec. I, stochastic rounding at C_min (Eq. (3)), the shift update and the
 * reference projected energy of Eq. (9).  Deterministic (semi-stochastic)
 * projection inside the space D of Sec. III is optional.
 *
 * Conventions used throughout:
 *  - Determinant: alpha word bit p set <=> spatial orbital p occupied by an
 *    alpha electron; same for beta.  Canonical operator order is alpha_0 ..
 *    alpha_{N-1}, beta_0 .. beta_{N-1}; all fermionic signs follow from it.
 *  - Integrals: chemist notation (pq|rs), 8-fold packed as in FCIDUMP files:
 *    pair(p,q) = max(p,q)(max(p,q)+1)/2 + min(p,q), and
 *    eri[pair(pair(p,q), pair(r,s))] = (pq|rs).
 *  - Random numbers: Philox4x64-10 keyed by (seed, 0) with the counter
 *    (alpha, beta, iteration, (slot << 8) | purpose); every random decision
 *    is a function of the determinant, the iteration and the attempt only,
 *    so results do not depend on list order, batching or launch geometry.
 *  - Buffers passed in are HOST pointers unless stated otherwise; they are
 *    copied, and the caller keeps ownership.  The handle owns all device
 *    memory it allocates.
 *  - No function throws; every error is reported by its return code, with a
 *    message available from fciqmc_last_error().
 *  - Thread safety: a handle may be used by one host thread at a time.
 */
#ifndef FCIQMC_GB300_H
#define FCIQMC_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes (no C++ exception leaves the library: a host allocation that
 * fails inside a call returns FCIQMC_ERR_OUT_OF_MEMORY) */
enum {
    FCIQMC_OK = 0,
    FCIQMC_ERR_INVALID_ARG = 1,   /* bad argument; nothing changed */
    FCIQMC_ERR_OUT_OF_MEMORY = 2, /* device or host allocation failed */
    FCIQMC_ERR_CAPACITY = 3,      /* a fixed-capacity buffer overflowed; the state is unchanged */
    FCIQMC_ERR_NUMERIC = 4,       /* NaN/Inf or a population beyond the representable range */
    FCIQMC_ERR_TIMEOUT = 5,       /* a bounded device-side wait expired */
    FCIQMC_ERR_CUDA = 6,          /* a CUDA runtime call failed */
    FCIQMC_ERR_UNSUPPORTED = 7    /* valid request outside what this build supports */
};

enum { FCIQMC_ABINITIO = 0, FCIQMC_HUBBARD = 1 };

/* The Hamiltonian (Sec. I; Eq. (4)).  For FCIQMC_ABINITIO, h1 and eri are
 * host arrays of binary64 (norb*norb row-major, and the packed 8-fold ERI).
 * For FCIQMC_HUBBARD the library builds h_pq = -t on lattice bonds and
 * (pp|pp) = U itself from lx, ly and the periodic flags; sites are numbered
 * x + lx*y.  A periodic direction must have length 1 or >= 3.
 * ref: the reference determinant of Eq. (9); when has_ref is 0 it is the
 * aufbau determinant (ABINITIO) or the Neel determinant, alpha on sites with
 * even x+y (HUBBARD). */
typedef struct {
    int32_t kind;
    int32_t norb;      /* spatial orbitals (ABINITIO), <= 64 */
    int32_t n_alpha;
    int32_t n_beta;
    double ecore;
    const double *h1;  /* ABINITIO: norb*norb */
    const double *eri; /* ABINITIO: packed (npair*(npair+1)/2), npair = norb(norb+1)/2 */
    int32_t lx, ly;    /* HUBBARD lattice, lx*ly <= 64 */
    int32_t periodic_x, periodic_y;
    double t, U;
    int32_t has_ref;
    int32_t pad0;
    uint64_t ref_alpha, ref_beta;
} fciqmc_system;

/* Run parameters.  tau: time step (Eq. (2)).  Shift (Eq. (2)): S starts at
 * initial_shift and stays there until the walker number N_w first reaches
 * target_walkers; from then on, every shift_interval (A) iterations,
 * S <- S - shift_damping / (A tau) * ln(N_w(t) / N_w(t - A)).
 * initiator_threshold n_a: a determinant is an initiator when |C| > n_a (or
 * it is the reference, or it lies in D); 0 gives plain FCIQMC.  c_min:
 * rounding threshold of Eq. (3); tau <= 0 selects tau = 0.5 / sum_j |H_ref,j|
 * (see fciqmc_ref_offdiag_sum).  p_single: probability of proposing a single
 * excitation (App. A).  semistoch_size: N_D of Sec. III (0 = off), chosen
 * semistoch_start iterations after the shift starts to vary.
 * max_dets / max_spawns: capacity hints (0 = derived from target_walkers);
 * capacities grow automatically when exceeded, up to max_device_bytes.  stream: a cudaStream_t
 * (NULL = the library creates its own).  alloc/free: optional device
 * allocator (for example a framework's caching allocator); NULL = cudaMalloc.
 * trial_size, trial_start: the trial-wave-function energy estimator (Sec. IV):
 * trial_start iterations after the shift starts to vary, T = the trial_size
 * (at most 1024) largest |C| (ties: ascending key), Psi^T = the lowest
 * eigenvector of H projected into T (Jacobi rotations on the device), and
 * every later iteration accumulates <Psi^T|H - E_ref|Psi> and <Psi^T|Psi>.
 * replicas = 2: two independent runs of the same system (the second draws
 * with Philox key word 1 = 1), stepped together in lockstep with one bucket
 * layout; fciqmc_step and fciqmc_energy on the first handle drive and report
 * both (the variational-energy and PT2 estimators of fciqmc_stats), and
 * fciqmc_replica gives the second for read-only queries.
 * adaptive_shift = 1 (Sec. V, adaptive shift): a non-initiator D_i dies with
 * the local shift f_i S instead of S, f_i = A_i / T_i (1 without spawns),
 * where every spawn of D_i in the iteration that survives Eq. (3) adds
 * w = |H_ji| / |H_jj - E_ref - S| (truncated to 2^-64; w >= 2^36 left out)
 * to T_i, and to A_i too if its target is occupied at the start of the
 * iteration (the initiator rule accepts it).
 * generator: how double excitations are proposed (App. A).  0: uniformly
 * (electron pair, then hole pair).  1: pre-computed heat-bath sampling
 * (App. A, p(ab|ij) proportional to |H_ij^ab|): one Walker alias table per
 * pair of occupied spin orbitals over hole pairs of matching spin, built on
 * the device at create time (about 16 (N^4 + (N(N-1)/2)^2) bytes for N
 * spatial orbitals).  Lattice (HUBBARD) systems ignore it: every hop has the
 * same |H|.  Singles stay uniform in both. */
typedef struct {
    double tau;
    double shift_damping;
    double target_walkers;
    double initial_walkers;
    double initial_shift;
    double initiator_threshold;
    double c_min;
    double p_single;
    int64_t shift_interval;
    uint64_t seed;
    int64_t semistoch_size;
    int64_t semistoch_start;
    int64_t max_dets;
    int64_t max_spawns;
    int64_t max_device_bytes; /* growth beyond this fails with FCIQMC_ERR_OUT_OF_MEMORY (0 = no limit) */
    void *stream;
    void *(*alloc)(size_t bytes, void *ctx);
    void (*free)(void *ptr, void *ctx);
    void *alloc_ctx;
    int32_t generator;
    int32_t replicas;    /* 1 (or 0): one run; 2: a replica pair (Sec. V) */
    int64_t trial_size;  /* N_T of the trial-wave-function estimator (0 = off) */
    int64_t trial_start; /* iterations after the shift starts to vary at which T is chosen */
    int32_t adaptive_shift; /* 1: the adaptive shift of Sec. V for non-initiators */
    int32_t pad1;
} fciqmc_params;

/* One row per completed iteration.  nw: walker number N_w = 2^-32 sum
 * floor(|C| 2^32).  shift: S after the iteration (relative to E_ref).
 * e_num = sum_{j != ref} H_ref,j C_j and e_den = C_ref after the iteration
 * (Eq. (9); every term of e_num is the binary64 product truncated toward zero
 * to a multiple of 2^-Fe, Fe = min(64, 60 - floor(log2 max |integral|) -
 * ceil(log2(2n + 1))), and the terms are summed exactly and rounded once, so
 * e_num depends on no order); attempts = sum ceil(|C|); spawns = spawned walkers stored;
 * rejected = spawns removed by the initiator rule; annihilated = walkers
 * removed by summing opposite-sign contributions. */
typedef struct {
    int64_t iteration;
    double nw;
    double shift;
    double e_num;
    double e_den;
    int64_t ndet;
    int64_t attempts;
    int64_t spawns;
    int64_t rejected;
    double annihilated;
    int32_t vary;
    int32_t pad0;
    double trial_num; /* <Psi^T|H - E_ref|Psi> after the iteration (0 before T exists) */
    double trial_den; /* <Psi^T|Psi> */
    /* replica pair (first replica's rows; 0 otherwise), from the amplitudes C^r
     * at the start of the iteration and the spawns S^r of the iteration:
     * x_overlap = sum_j C^1_j C^2_j; x_var_num = sum_j C^1_j (H_jj - E_ref) C^2_j
     * - sum_j (C^1_j S^2_j + C^2_j S^1_j) / (2 tau), an estimate of
     * <Psi^1|H - E_ref|Psi^2>; x_pt2 = sum_j R^1_j R^2_j / (E_0 - H_jj + E_ref) / tau^2
     * over determinants whose spawns R^r were removed by the initiator rule in
     * both replicas (Sec. VI), E_0 the mean of the shifts */
    double x_overlap;
    double x_var_num;
    double x_pt2;
} fciqmc_iter_stats;

/* Summary returned by fciqmc_energy.  Energies are absolute (E_ref added).
 * e_proj_mean / e_proj_sigma: ratio of the means of e_num and e_den over
 * iterations from equil_start on, with a Flyvbjerg-Petersen blocking error;
 * equil_start = the iteration at which the shift started to vary + 500. */
typedef struct {
    int64_t iteration;
    int64_t ndet;
    double nw;
    double eref;
    double shift;
    double e_proj_inst;
    double e_proj_mean;
    double e_proj_sigma;
    double shift_mean;
    double shift_sigma;
    int64_t equil_start;
    int64_t n_samples;
    int64_t attempts_total;
    int64_t spawns_total;
    int64_t rejected_total;
    double annihilated_total;
    int32_t vary;
    int32_t pad0;
    /* trial-wave-function estimator: E_Trial = E_ref + mean(trial_num) /
     * mean(trial_den) over iterations from max(equil_start, T built) on, with
     * its blocking error; e_trial_T = E^T (absolute), the lowest eigenvalue of
     * H^T; trial_samples = 0 when the estimator is off or T is not built yet */
    double e_trial_mean;
    double e_trial_sigma;
    double e_trial_T;
    int64_t trial_samples;
    /* replica pair (first replica only; NaN otherwise): variational energy
     * E_var = E_ref + mean(x_var_num) / mean(x_overlap) and the PT2 correction
     * mean(x_pt2) / mean(x_overlap) (Sec. VI; the replicas are not normalised,
     * so both are divided by <Psi^1|Psi^2>), each with a blocking error, over
     * iterations from 500 after the later of the two shift starts */
    double e_var_mean;
    double e_var_sigma;
    double pt2_mean;
    double pt2_sigma;
    int64_t pair_samples;
} fciqmc_stats;

typedef struct fciqmc_handle fciqmc_handle;

/* Reads an FCIDUMP file (Knowles-Handy format: a namelist with NORB, NELEC,
 * MS2, then lines "value i j k l", 1-based orbitals; i j 0 0 one-electron,
 * 0 0 0 0 core energy) into *out as an FCIQMC_ABINITIO system with
 * n_alpha = (NELEC + MS2) / 2, n_beta = (NELEC - MS2) / 2.  Integrals are
 * chemist (ij|kl); each listed value is placed at all of its 8-fold (or
 * 2-fold for h) symmetric positions.  The arrays are allocated by the library
 * and released by fciqmc_free_system. */
int fciqmc_read_fcidump(const char *path, fciqmc_system *out);
void fciqmc_free_system(fciqmc_system *sys);

/* Creates a run: validates and copies the system, uploads the integrals,
 * places initial_walkers on the reference determinant, sizes the bucketed
 * walker and spawn buffers, and captures one iteration as a CUDA graph.
 * Returns FCIQMC_OK and *out, or an error code (then *out is NULL). */
int fciqmc_create(const fciqmc_system *sys, const fciqmc_params *params, fciqmc_handle **out);

/* Runs n_iter projector iterations on the handle's stream and synchronises
 * once at the end.  On FCIQMC_ERR_CAPACITY the library grows the buffers and
 * repeats the failed iteration, which is bit-identical because every random
 * draw is keyed; other errors stop the run at the last good iteration. */
int fciqmc_step(fciqmc_handle *h, int64_t n_iter);

/* Enqueues n_iter iterations on the handle's stream and returns at once (no
 * host synchronisation, no error check).  The caller must call fciqmc_sync
 * before reading results; fciqmc_sync reports the first error and, after a
 * capacity overflow, grows the buffers and repeats the missing iterations
 * (bit-identical).  Lets a caller overlap host work or bracket single
 * iterations with its own events on fciqmc_stream(h). */
int fciqmc_step_async(fciqmc_handle *h, int64_t n_iter);
int fciqmc_sync(fciqmc_handle *h);

/* The cudaStream_t all work of the handle runs on. */
void *fciqmc_stream(fciqmc_handle *h);

/* Fills *out from the iteration history (host-side statistics). */
int fciqmc_energy(fciqmc_handle *h, fciqmc_stats *out);

/* Frees all resources; NULL is allowed.  The second replica of a pair is
 * released with the first (destroying it directly does nothing). */
void fciqmc_destroy(fciqmc_handle *h);

/* Replica r (0 or 1) of a pair created with replicas = 2 (r = 0 is h itself),
 * for export, statistics and queries; NULL for other r or other handles.
 * The second replica is stepped, and destroyed, through the first. */
fciqmc_handle *fciqmc_replica(fciqmc_handle *h, int32_t r);

/* Message of the last error on this handle (or of the last failed create
 * when h is NULL). */
const char *fciqmc_last_error(const fciqmc_handle *h);

/* Number of occupied determinants after the last completed iteration. */
int64_t fciqmc_num_dets(fciqmc_handle *h);

/* Copies the walker list to host arrays of capacity cap, sorted by (alpha,
 * beta) ascending; hdiag = H_ii - E_ref; flags bit 0 = reference, bit 1 =
 * in D.  *n_out receives the number of determinants (also when it exceeds
 * cap, in which case FCIQMC_ERR_CAPACITY is returned and nothing copied).
 * The list is compacted and radix-sorted on the device in transient scratch
 * (about 68 bytes per determinant, from the run's allocator); when
 * max_device_bytes leaves no room for it the sort runs on the host. */
int fciqmc_export_state(fciqmc_handle *h, int64_t cap, uint64_t *alpha, uint64_t *beta, double *c,
                        double *hdiag, int32_t *flags, int64_t *n_out);

/* Shift state: S, vary flag, iteration at which it started, iterations since
 * the last update, and N_w at the last update as a 128-bit fixed-point
 * integer (N_w * 2^32, high and low words). */
int fciqmc_export_shift(fciqmc_handle *h, int64_t *iteration, double *S, int32_t *vary,
                        int64_t *shift_start, int64_t *cnt, uint64_t *nw_last_hi, uint64_t *nw_last_lo);

/* Replaces the walker list and the shift state (a restart from a checkpoint).
 * Keys must be distinct, with the right electron counts; the reference
 * determinant is kept (added with C = 0 when absent).  The bucket count grows
 * (one allocation) until every bucket holds at most half its capacity.  The
 * entries are checked, counted and placed on the device in transient scratch
 * (about 24 bytes per determinant, from the run's allocator); when
 * max_device_bytes leaves no room for it, on the host.
 * FCIQMC_ERR_INVALID_ARG for a wrong electron count, an orbital beyond norb,
 * a non-finite amplitude, or keys that crowd one bucket even at 2^22 buckets
 * (duplicates); duplicates that do not are not detected. */
int fciqmc_import_state(fciqmc_handle *h, int64_t n, const uint64_t *alpha, const uint64_t *beta,
                        const double *c, int64_t iteration, double S, int32_t vary, int64_t shift_start,
                        int64_t cnt, uint64_t nw_last_hi, uint64_t nw_last_lo);

/* Copies rows first .. first+count-1 of the per-iteration history. */
int fciqmc_iter_stats_get(fciqmc_handle *h, int64_t first, int64_t count, fciqmc_iter_stats *out);
int64_t fciqmc_iter_stats_count(fciqmc_handle *h);

/* Advances k independent handles by n_iter iterations each, sharing every
 * launch: one graph-captured iteration processes the buckets of all k runs.
 * Each run's results are bit-identical to running it alone.  All handles
 * must be distinct; they are synchronised on the first handle's stream. */
int fciqmc_step_batch(fciqmc_handle **hs, int32_t k, int64_t n_iter);

/* sum_j |<D_j|H|D_ref>| over all single and double excitations of the
 * reference, computed on the device in a fixed order (deterministic).  A run
 * created with tau <= 0 uses tau = 0.5 / this sum: a walker spawns
 * tau sum_j |H_ij| walkers per iteration in expectation, and only when that is
 * below 1 can the shift hold the walker number. */
int fciqmc_ref_offdiag_sum(fciqmc_handle *h, double *out);
double fciqmc_tau(fciqmc_handle *h);

/* The trial space of the E_Trial estimator once it is built (trial_size > 0):
 * returns N_T (0 before), *n_w = the number of determinants with a stored
 * W_j = <Psi^T|H - E_ref|D_j> (T and the space connected to it), *ET = E^T -
 * E_ref; the first min(N_T, cap) keys of T in ascending order and their
 * components of Psi^T (unit norm, sign arbitrary) when the arrays are given.
 * Negative status on error. */
int64_t fciqmc_trial_info(fciqmc_handle *h, int64_t *n_w, double *ET, uint64_t *t_alpha, uint64_t *t_beta,
                          double *cT, int64_t cap);

/* Copies one pre-computed heat-bath table (generator 1; App. A) to the host:
 * same_spin = 0: the table of (i alpha, j beta), entry k = a N + b over
 * (a alpha, b beta); same_spin = 1: the table of i < j (either spin), entry
 * k = b (b - 1) / 2 + a over a < b.  *S = sum_k |H_ij^ab| (exact sum rounded
 * once), *lam = tau S / p_pair with p_pair = (1 - p_single) 2 / (n (n - 1)),
 * i.e. |H| / p_gen of every entry.  For each of the first min(K, cap) entries:
 * threshold[k] = ceil(prob_k 2^53), the alias coin keeping entry k when the
 * top 53 bits of the low word of w K are below it; holes[k] = own hole pair
 * | alias's hole pair << 16, a hole pair being a | b << 8.  Returns K (>= 0),
 * or a negative status: FCIQMC_ERR_INVALID_ARG when the run has no tables or
 * (i, j) is out of range, FCIQMC_ERR_CUDA on a copy failure.  Output pointers
 * may be NULL. */
int64_t fciqmc_pchb_table(fciqmc_handle *h, int32_t same_spin, int32_t i, int32_t j, double *S, double *lam,
                          uint64_t *threshold, uint32_t *holes, int64_t cap);

/* The same sum as fciqmc_ref_offdiag_sum, for callers that cannot allocate
 * device memory: frameworks whose memory pool owns every device byte, jobs
 * held to a fixed memory budget, or loops that must not enter the CUDA driver's
 * allocator (cudaMalloc can synchronise the whole device).  No counterpart in
 * the paper: this is an interface
 * convenience of this library.
 *   norb, n_alpha, n_beta: as in fciqmc_system (norb <= 64);
 *   d_h1, d_eri: DEVICE arrays owned by the caller, laid out as h1 / eri of
 *     fciqmc_system (norb*norb, and the packed 8-fold ERI);
 *   ref_alpha, ref_beta: the reference determinant;
 *   d_out: DEVICE pointer to one double, receives the sum;
 *   stream: cudaStream_t (NULL = legacy default stream).
 * Calls no cudaMalloc/cudaFree and no allocating library routine.  Scratch
 * lives in a fixed 1 KB array in the library's device image (64 block
 * partial sums and the integral exponent range); every GPU that loads the
 * library keeps it until the process exits.  The first call on a device looks
 * up that array's device address (cudaGetSymbolAddress) with the device
 * current; make that first call before any stream capture.  The address is
 * kept for the rest of the process: after cudaDeviceReset, or anything else
 * that destroys the device's primary context, it is stale, and the entry
 * point must not be called again on that device.  All calls share
 * the array: calls that overlap on the GPU race and must not be issued
 * concurrently.  Synchronises the stream before returning.  Errors:
 * FCIQMC_ERR_INVALID_ARG for bad sizes/pointers, a reference with the wrong
 * electron counts or a non-finite integral; FCIQMC_ERR_UNSUPPORTED when the
 * integrals' dynamic range exceeds the 128-bit exact accumulator;
 * FCIQMC_ERR_CUDA on a CUDA failure. */
int fciqmc_ref_offdiag_sum_noalloc(int32_t norb, int32_t n_alpha, int32_t n_beta, const double *d_h1,
                                   const double *d_eri, uint64_t ref_alpha, uint64_t ref_beta, double *d_out,
                                   void *stream);

/* ---- serving: runs admitted by device memory and stepped together ----
 * A request is a system + parameters + a target error; the server admits
 * queued requests (first come, first served) while the sum of the device
 * memory of running requests stays within mem_budget_bytes and at most
 * max_active run, advances all running requests together (one batched launch
 * per iteration, fciqmc_step_batch), and retires a request when the blocking
 * error of its energy is below target_sigma with at least 200 samples after
 * equilibration, or after max_iters iterations.  The energy is the projected
 * estimator E_proj, or E_Trial when the request asked for a trial space
 * (trial_size > 0) and it has at least 200 samples with the smaller error.
 * Each result is identical to running the request alone. */
typedef struct fciqmc_server fciqmc_server;
typedef struct {
    int32_t state;        /* 0 queued, 1 running, 2 converged, 3 stopped at max_iters, 4 failed */
    int32_t error;        /* status code of a failed request */
    int64_t iterations;
    double energy;        /* energy mean (absolute): E_proj or E_Trial, see estimator */
    double sigma;         /* its blocking error */
    double shift;
    double t_submit;      /* seconds on the server's clock */
    double t_start;
    double t_done;
    int64_t attempts;
    int64_t device_bytes; /* peak device memory of the run */
    double tau;
    int32_t estimator;    /* 0: E_proj (Eq. (9)), 1: E_Trial (Sec. IV) */
    int32_t pad0;
    double t_arrival;     /* arrival time on the server's clock; latency = t_done - t_arrival */
} fciqmc_request_status;

int fciqmc_server_create(int64_t mem_budget_bytes, int32_t max_active, void *stream, fciqmc_server **out);
/* Copies sys (including the integral arrays) and params; returns the request
 * id.  t_arrival is the request's arrival time in seconds on the server's
 * clock (fciqmc_server_clock); a negative or NaN value means now.  Requests
 * are admitted in order of arrival, never before their arrival time, so a
 * client may hand over a future arrival schedule up front or submit each
 * request when it arrives; its latency counts from t_arrival either way.
 * Errors: FCIQMC_ERR_INVALID_ARG (missing pointers, target_sigma <= 0,
 * max_iters < 1, norb outside 1..64), FCIQMC_ERR_UNSUPPORTED (replicas > 1). */
int fciqmc_server_submit(fciqmc_server *srv, const fciqmc_system *sys, const fciqmc_params *params,
                         double target_sigma, double t_arrival, int64_t max_iters, int64_t *id);
/* one scheduling round: admit, advance every running request by n_iter
 * iterations, retire finished ones; *n_active = running + queued afterwards */
int fciqmc_server_tick(fciqmc_server *srv, int64_t n_iter, int32_t *n_active);
int fciqmc_server_poll(fciqmc_server *srv, int64_t id, fciqmc_request_status *out);
double fciqmc_server_clock(fciqmc_server *srv);
void fciqmc_server_destroy(fciqmc_server *srv);

/* Autotuner of the launch configuration: times n_iter iterations of the
 * batch hs[0..k-1] (advancing it) for each candidate, keeps the fastest for
 * every later launch in the process, and writes it to out[3] (spawn, heavy,
 * annihilation).  Candidates: for the spawning kernel 0 = the staged kernel
 * (256-thread blocks, three per SM, each bucket's keys, amplitudes and flags
 * brought into shared memory by bulk copies one bucket ahead), 1 = split
 * spawning (see fciqmc_set_launch_config) or 2, 4, 8, 16 = the plain-load
 * kernel with that many blocks per SM; the heavy-spawning
 * kernel's grid (1, 2, 4 blocks per SM); for the annihilation 0 = the staged
 * kernel (two 256-thread blocks per SM, bulk copies one bucket ahead) or 3,
 * 9, 24 = the plain-load kernel (three resident per SM) with that grid.
 * Defaults: 1, 2, 0.  Results of the runs do not depend on the
 * configuration. */
int fciqmc_autotune(fciqmc_handle **hs, int32_t k, int64_t n_iter, int32_t out[3]);

/* Sets (or reads) the launch configuration the autotuner chooses from, for
 * every later launch in the process: spawn 0 = the staged kernel, 1 = split
 * spawning (a staged draw kernel queues every attempt in global memory by
 * class, 48 bytes each, in per-run segments owned by its blocks, about 7 GB at
 * 1.2e8 attempts; a flat kernel evaluates them one per thread), 2, 4, 8, 16 =
 * the plain-load kernel with that many blocks per SM;
 * heavy = blocks per SM of the heavy-determinant kernel (1..16); annihilate
 * as for fciqmc_autotune (0, 3, 9, 24).  A handle captures its iteration graph
 * again at its next step.  FCIQMC_ERR_INVALID_ARG for other values.  Results
 * of the runs do not depend on the configuration. */
int fciqmc_set_launch_config(int32_t spawn, int32_t heavy, int32_t annihilate);
int fciqmc_get_launch_config(int32_t out[3]);

/* Device timing of the kernels of the last fciqmc_step call (milliseconds per
 * iteration, averaged), measured with CUDA events on the handle's stream:
 * out[0] spawn, out[1] heavy-determinant spawn, out[2] annihilation,
 * out[3] finalize, out[4] semi-stochastic, out[5] H_jj of the determinants
 * created in the iteration.  Enabled by fciqmc_set_profiling. */
int fciqmc_set_profiling(fciqmc_handle *h, int32_t on);
int fciqmc_kernel_times(fciqmc_handle *h, double out[6]);

/* Internal layout figures used to compute algorithmic bytes and to size
 * buffers: out[0] buckets, out[1] main capacity per bucket, out[2] spawn
 * capacity per bucket, out[3] device bytes allocated. */
int fciqmc_layout(fciqmc_handle *h, int64_t out[4]);

/* Kernel launches in one iteration of the handle's captured CUDA graph (a
 * count of the graph's kernel nodes, taken when the graph was captured;
 * 0 before the first step, -1 for a NULL handle).  One fciqmc_step of n
 * iterations replays the graph n times. */
int32_t fciqmc_graph_kernels(fciqmc_handle *h);

/* The device's memory interface, for the nominal HBM bandwidth
 * 2 x clock x bus width: out[0] the peak memory clock in kHz, out[1] the
 * global-memory bus width in bits, as the CUDA runtime reports them for
 * `device`.  FCIQMC_ERR_INVALID_ARG for a NULL out, FCIQMC_ERR_CUDA when the
 * runtime cannot answer (no such device). */
int fciqmc_device_memory(int32_t device, int64_t out[2]);

/* Size of the semi-stochastic space D (Sec. III) once it has been selected
 * (0 before), and in *nnz (may be NULL) the stored entries of H^D, whose CSR
 * the projection reads every iteration; FCIQMC_ERR_INVALID_ARG for NULL. */
int64_t fciqmc_semistoch_info(fciqmc_handle *h, int64_t *nnz);

#ifdef __cplusplus
}
#endif
#endif
