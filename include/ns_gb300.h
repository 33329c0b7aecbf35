/*
 * ns_gb300.h -- C ABI of the GB300 (sm_103a) batched nested sampler.
 *
 * The library computes the Bayesian evidence
 *     Z = integral_0^1 L(X) dX                       (section 1, eq. 1.1)
 * of a likelihood over a uniform prior box by nested sampling with batched
 * live-point replacement: each iteration removes the m worst live points,
 * draws m replacements by slice sampling in parallel (section 2.2), and
 * repairs the ordering with batch sorting (Algorithm 1) and the history
 * correction (Algorithm 2) of section 3.1.  Clustering of the live points
 * (section 2.1) shapes the slice directions.
 *
 * Conventions shared by every entry point
 *  - Every function returns ns_status (NS_OK = 0, negative on error).  No
 *    entry point aborts, traps or throws.  A device loop that runs out of
 *    its iteration budget reports NS_ERR_BUDGET instead of spinning.
 *  - "host" pointers are read during the call only, unless stated; the
 *    caller keeps ownership.  "device" pointers are CUDA global-memory
 *    pointers on the current device; the caller owns them and they must stay
 *    valid until the work queued on `stream` has finished.
 *  - `stream` is a cudaStream_t passed as void*; NULL means the legacy
 *    default stream.  The step-level calls (ns_philox4x32_10 ... ns_cluster)
 *    are asynchronous on `stream` and allocate nothing.
 *  - Points are stored in unit-cube coordinates x in [0,1]^d; the likelihood
 *    is evaluated at theta = lo + (hi - lo) * x.
 *  - Random numbers: Philox4x32-10 (Salmon et al., SC'11) with key
 *    (seed & 0xffffffff, seed >> 32) and counter (block, purpose, walker, t);
 *    draw n of a stream is word n % 4 of block n / 4.  Purposes: slice step
 *    s (0..0xffff) of walker w at iteration t; NS_PURPOSE_SEED for the
 *    choice of a walker's start point; NS_PURPOSE_KMEANS (walker = tree node)
 *    for the first k-means centre; iteration NS_T_INIT (walker = live slot)
 *    for the initial live points.
 *  - Log-likelihoods are unnormalised (section 3.2).  A NaN likelihood counts
 *    as -infinity (outside every constraint).
 */
#ifndef NS_GB300_H
#define NS_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define NS_MAX_DIM 32          /* largest d a run may have */
#define NS_MAX_MODES 8         /* MIXTURE components */
#define NS_MAX_GMM_MODES 64    /* GMM components */
#define NS_GMM_CAPACITY 512    /* GMM: n_modes x (d rounded up to its register class) */
#define NS_MAX_DEPTH 6         /* cluster tree depth: up to 64 leaves, 127 nodes */
#define NS_MAX_BATCH 256       /* m, walkers per run (one thread, or one warp, each) */
#define NS_MAX_LIVE 65536      /* N_live per run */
#define NS_MAX_HISTORY 64      /* history slots per walker */
#define NS_PURPOSE_SEED 0x10000u
#define NS_PURPOSE_KMEANS 0x20000u
#define NS_T_INIT 0xFFFFFFFFu

typedef enum {
    NS_OK = 0,
    NS_ERR_ARG = -1,      /* an argument is out of range; nothing was queued */
    NS_ERR_CUDA = -2,     /* a CUDA call failed; see ns_last_error */
    NS_ERR_OOM = -3,      /* device allocation failed */
    NS_ERR_BUDGET = -4,   /* a capped loop gave up (step-out, shrink, iterations, dead buffer) */
    NS_ERR_STATE = -5,    /* call out of order (e.g. ns_result before ns_run) */
    NS_ERR_UNSUPPORTED = -6
} ns_status;

typedef enum {
    NS_LIK_GAUSS_ISO = 0,   /* -1/2 sum ((theta-mean)/sigma)^2            (section 3.2) */
    NS_LIK_GAUSS_CORR = 1,  /* -1/2 |L^T (theta-mean)|^2, L L^T = Sigma^-1 */
    NS_LIK_ROSENBROCK = 2,  /* -sum_i (a-theta_i)^2 + b (theta_{i+1}-theta_i^2)^2 (section 4.2) */
    NS_LIK_MIXTURE = 3,     /* log (1/K) sum_k exp(-|theta-c_k|^2 / (2 sigma^2)) (eq. array form) */
    NS_LIK_MLP = 4,         /* -1/2 sum_k ((MLP(theta)_k - data_k)/sigma_k)^2 (section 5 stand-in) */
    NS_LIK_GMM = 5,         /* log sum_k w_k exp(-1/2 sum_i (theta_i-mu_ki)^2 / s_ki^2) (section 2.3, eqs. array, separation) */
    NS_LIK_SHELL = 6        /* -1/2 ((|theta-c| - r0) / w)^2 (section 2.3, eq. shell) */
} ns_lik_kind;

/* Likelihood description; host pointers, copied by ns_create*. */
typedef struct {
    int kind;                  /* ns_lik_kind */
    const double* mean;        /* [d]   GAUSS_ISO, GAUSS_CORR; SHELL: the centre c */
    const double* prec_chol;   /* [d*d] GAUSS_CORR: row-major lower L with L L^T = Sigma^-1 */
    double sigma;              /*       GAUSS_ISO, MIXTURE (> 0); SHELL: the width w (> 0) */
    int n_modes;               /*       MIXTURE 1..NS_MAX_MODES; GMM 1..NS_MAX_GMM_MODES */
    const double* centres;     /* [n_modes*d] MIXTURE, GMM */
    double a, b;               /*       ROSENBROCK; SHELL: a = the radius r0 (>= 0) */
    int n_layers;              /*       MLP: affine layers */
    const int* widths;         /* [n_layers+1], widths[0] = d */
    const float* weights;      /* concatenated [out][in] row-major blocks */
    const float* biases;       /* concatenated [out] blocks */
    const float* data;         /* [widths[n_layers]] */
    const float* sigma_out;    /* [widths[n_layers]] (> 0) */
    const double* mode_var;    /* [n_modes*d] GMM: per-mode diagonal variances (> 0) */
    const double* mode_logw;   /* [n_modes]   GMM: log weights (finite; not normalised) */
} ns_likelihood;

typedef struct {
    int depth;            /* cluster tree depth, 0..NS_MAX_DEPTH (default 0: one cluster) */
    int recluster_every;  /* iterations between re-clusterings; 0 = max(1, 100/m) (section 2.3) */
    int n_min;            /* a child cluster needs more than n_min points; 0 = d + 1 */
    double vol_frac;      /* children must be this much smaller than the parent (0.5) */
    int kmeans_iters;     /* Lloyd iterations per 2-means split (10) */
    int correction;       /* 0 naive, 1 batch sorting, 2 sorting + history (default), 3 best-of-worst */
    int history_iters;    /* K of Algorithm 2 (1) */
    int t_max;            /* history slots per walker, 1..NS_MAX_HISTORY (64) */
    int e_max;            /* step-out expansions per side (64) */
    int s_max;            /* shrink draws per slice step (128) */
    double width;         /* initial bracket width along the direction (1.0) */
    long long max_iter;   /* iterations before NS_ERR_BUDGET (1000000) */
    long long dead_cap;   /* dead-point capacity per run; 0 = 400 * N + 4 * m */
    int chunk_iters;      /* iterations per persistent launch (1000) */
    int precision;        /* MLP only: 0 FP32 on the CUDA cores, 1 BF16 on the tensor cores with FP32
                           * re-evaluation near the threshold, 2 FP32 on the tensor cores (every evaluation with
                           * inputs and activations split exactly into three BF16 parts; networks whose weights
                           * are all BF16 values only, else NS_ERR_ARG) */
    double reeval_margin; /* MLP only: re-evaluate in FP32 when |logL - threshold| <   */
    double reeval_rel;    /*   reeval_margin + reeval_rel |threshold| (2.0 and 4e-3) */
    int reeval_defer;     /* MLP only: rounds a near-threshold candidate may wait so that several are
                           * re-evaluated in one FP32 pass, 0..64 (4; 0 = at once); results do not depend on it */
    int walker_mapping;   /* analytic likelihoods: 0 one walker per thread (default), 1 one walker per warp
                           * (the lanes share the coordinates); ns_autotune picks per run.  The mappings take
                           * the same decisions and draws; only the order of the FP32 sums in log L differs */
    int mlp_batch_cap;    /* MLP precision 1: candidates evaluated per lock-step round, 0..128 (128 = one pass of
                           * the weights per round; walkers beyond it keep their candidate for the next round and go
                           * first there; 0 = every candidate of the round, in equal calls).  Decisions do not
                           * depend on it */
    int mlp_cluster;      /* MLP precision 1 and 2: CTAs (SMs) per run that share its tensor-core evaluations,
                           * each streaming and multiplying a disjoint quarter or half of every layer's weight
                           * tiles: 1, 2 or 4 (every layer's 128-row tile count must be a multiple of it, else
                           * NS_ERR_ARG), or 0 = automatic (4, then 2, while that many CTAs per MLP run fit on the
                           * device's SMs; else 1).  The chi^2 partials of the CTAs are added in rank order, so
                           * results differ from one CTA's in the last bits of log L */
    int two_plane;        /* MLP precision 1, BF16-valued weights: a candidate inside the BF16 margin is first
                           * re-evaluated with 16-bit activations (two BF16 planes, 64 per tensor-core pass) and
                           * goes on to FP32 only if that value lies within reeval2_margin + reeval2_rel
                           * |threshold| of its threshold (1, default), or goes to FP32 at once (0) */
    double reeval2_margin; /* (0.05) */
    double reeval2_rel;    /* (1e-4) */
    int bracket;          /* the unit of the initial slice bracket (section 2.2 gives none): 0 (default) the
                           * walker's cluster Cholesky factor, so the bracket spans `width` standard deviations of
                           * the cluster; 1 that factor times the cluster's bounding radius (the largest
                           * Mahalanobis distance of a member from its centre), so it spans `width` radii.  With
                           * 1 the FP32 factors written to the cluster tables (chol) are the scaled ones; chol64
                           * stays the unscaled factor */
} ns_options;

/* One run of a batch. */
typedef struct {
    const ns_likelihood* lik;
    const double* lo;     /* [d] prior box, lo < hi */
    const double* hi;     /* [d] */
    int d;                /* 1..NS_MAX_DIM */
    int n_live;           /* N, 2..NS_MAX_LIVE */
    int m;                /* batch size, 1 <= m <= N/2, m <= NS_MAX_BATCH */
    int n_slice_steps;    /* slice steps per replacement (5 d in the paper, section 4) */
    double stop_frac;     /* stop when L_max X_k < stop_frac Z, 0 < stop_frac < 1 */
    uint64_t seed;        /* Philox key */
} ns_problem;

typedef struct ns_handle ns_handle;

typedef struct {
    double log_z;         /* log evidence (dead points + final live tail) */
    double log_z_err;     /* sqrt(H / N) (Skilling 2006) */
    double info_h;        /* information H in nats */
    long long n_dead;     /* samples returned: dead points then the final live points */
    long long n_evals;    /* likelihood evaluations, initial draws included */
    long long n_iter;     /* iterations of the batched loop */
    long long n_relaxed;  /* points replaced by Algorithm 2 */
    long long n_reeval;   /* FP32 re-evaluations (MLP precision 1) */
    long long n_capped;   /* walker steps that hit the step-out or shrink cap */
    int status;           /* ns_status of this run */
    int d;
    /* samples: the dead points in death order (ascending logL), then the
     * final live points in slot order */
    const float* dead_x;     /* [n_dead*d] host, owned by the handle */
    const float* dead_logl;  /* [n_dead]   host, owned by the handle */
    const double* dead_logw; /* [n_dead]   host, owned by the handle: log weight (prior mass times L) */
    /* MLP runs: lock-step walker rounds, and the evaluator passes and the
     * candidates they carried, BF16 passes, FP32 ones (tensor-core
     * three-plane or CUDA-core) and 16-bit ones (two planes) apart; 0 for
     * other runs */
    long long n_rounds, n_pass_bf16, n_cand_bf16, n_pass_fp32, n_cand_fp32, n_pass_x2, n_cand_x2;
} ns_result_t;

/* ---- whole runs ------------------------------------------------------- */

/* Batching: each run's execution configuration, picked by measurement --
 * an analytic run's walker-to-lane mapping (one walker per thread, the
 * default, or one per warp), a BF16 MLP run's candidates per weight pass (the
 * N of the tensor-core passes: at most 128 per lock-step round, the default;
 * at most 64; or every candidate of the round in equal calls); FP32 MLP runs
 * keep theirs.  First warm_iters (>= 0) iterations of every unfinished run
 * with its current configuration (ordinary iterations of the run: they are
 * kept), so that the probe sees a live set inside the run rather than the
 * prior; then a device snapshot of every run's state (live set, cluster
 * tables, counters) and, for each configuration, probe_iters (1..1000)
 * iterations followed by the snapshot's restore.  A run leaves its default
 * only for a configuration with at least 5 % fewer SM cycles per iteration
 * in the slice phase (a4-a7).  On return every run is in its state after the
 * warm-up, bit for bit.  The mappings take the same decisions with FP32 sums
 * in another order; the MLP configurations give identical runs.
 * A probe is never allowed to dominate the job it tunes: after the warm-up
 * the iterations left are estimated from each run's stopping rule (with its
 * current lmax and log Z, (N/m)(lmax - k/N - log Z - log stop_frac), at
 * most max_iter minus the iterations done); if the probe's iterations
 * (configurations x probe_iters) exceed a quarter of the longest run's
 * estimate, nothing is probed and every run keeps its configuration
 * (out_ratio NaN).
 * out_choice [n_runs] (host, may be NULL): analytic runs 1 = per warp, 0 =
 * per thread; MLP runs the candidate cap (128, 64, or 0 = equal calls).
 * out_ratio [n_runs] (host, may be NULL): the second configuration's cycles
 * per iteration over the default's (warp over thread; 64 over 128), NaN
 * where not measured (runs that had stopped, FP32 MLP runs).  The choices
 * are not part of a checkpoint.  Allocates the snapshot with cudaMalloc for
 * the duration of the call (NS_ERR_OOM if it cannot). */
ns_status ns_autotune(ns_handle* h, int warm_iters, int probe_iters, int* out_choice, double* out_ratio,
                      void* stream);

/* Set run `run`'s walker mapping (0 one walker per thread, 1 one walker per
 * warp; analytic runs only) for the iterations that follow. */
ns_status ns_set_walker_mapping(ns_handle* h, int run, int warp);

/* Fill `opt` with the defaults listed above. */
ns_status ns_default_options(ns_options* opt);

/* One run.  Validates every argument (NS_ERR_ARG, nothing allocated, on the
 * first bad one), copies the likelihood to the device, allocates the run's
 * device state (live set, dead buffer, history, cluster table) with
 * cudaMalloc on the current device, and returns a handle.  `opt` NULL means
 * defaults. */
ns_status ns_create(const ns_likelihood* lik, const double* lo, const double* hi, int d,
                    int n_live, int m, int n_slice_steps, double stop_frac, uint64_t seed,
                    const ns_options* opt, ns_handle** out);

/* Several independent runs (any mix of d, N, m and likelihood) sampled
 * together: one persistent thread block per run. */
ns_status ns_create_batch(int n_runs, const ns_problem* runs, const ns_options* opt,
                          ns_handle** out);

/* Runs every run of the handle to its stopping rule (or budget), queued on
 * `stream`, and waits for it.  Per-chunk host/device traffic is one status
 * word per run. */
ns_status ns_run(ns_handle* h, void* stream);

/* Advances every unfinished run of the handle by at most n_iters iterations
 * (one persistent launch per register class), queued on `stream`, and waits
 * for it; ns_run or further ns_step calls continue from there.  The result
 * of a run does not depend on how its iterations were split into calls.
 * NS_ERR_ARG for n_iters < 1. */
ns_status ns_step(ns_handle* h, int n_iters, void* stream);

/* Checkpoint / resume.  Every random number of a run is a Philox draw keyed
 * by (seed, iteration, walker, step), so a run's whole state is its device
 * memory: ns_checkpoint copies it (with a fingerprint of the batch's shapes
 * and options) into the caller's host buffer of ns_checkpoint_bytes(h)
 * bytes; ns_restore loads such a checkpoint into a handle created by
 * ns_create_batch with the same runs and options (in this or another
 * process), after which ns_run finishes every run exactly as the
 * checkpointed handle would have.  NS_ERR_ARG if the buffer is too small or
 * the checkpoint comes from a batch of another shape.  Both wait for
 * `stream`. */
size_t ns_checkpoint_bytes(const ns_handle* h);
ns_status ns_checkpoint(ns_handle* h, void* host_buf, size_t bytes, void* stream);
ns_status ns_restore(ns_handle* h, const void* host_buf, size_t bytes, void* stream);

/* Returns every run of the handle to its initial state (same seeds) so that
 * ns_run can be repeated on the allocated memory; asynchronous on `stream`. */
ns_status ns_reset(ns_handle* h, void* stream);

/* Result of run `run` (0-based).  Copies that run's samples to host memory
 * owned by the handle on first call; pointers stay valid until ns_destroy. */
ns_status ns_result(ns_handle* h, int run, ns_result_t* out);

/* The scalars of ns_result (log Z, error, H, counts, status) without
 * copying any sample to the host; the three sample pointers are NULL. */
ns_status ns_summary(const ns_handle* h, int run, ns_result_t* out);

/* Tracing: SM cycles spent by run `run` in each step of its iterations,
 * accumulated over all its iterations since creation or ns_reset, as seen
 * by thread 0 of its block between barriers.  out[0..5] = clustering,
 * selection, slice walkers, Algorithms 1-2, live/dead update, evidence and
 * stop test; out[6..7] = within the slice phase: MLP runs, the batch
 * evaluations (BF16 or FP32 path) and the FP32 re-evaluations; other runs,
 * the first warp's direction draws and its walk.
 * Valid after ns_run. */
ns_status ns_phase_cycles(const ns_handle* h, int run, long long* out);

/* Tracing: a copy of one of run `run`'s device buffers, as the last
 * iteration left it (call between ns_step / ns_run calls; asynchronous on
 * `stream`, which this call synchronises).  `which` names the buffer; its
 * size in bytes is ns_run_buffer_bytes(h, run, which) and `bytes` must equal
 * it (NS_ERR_ARG otherwise):
 *   NS_BUF_LIVE_X       float [d][n_pad]      live points, unit cube, n_pad = N rounded up to 32
 *   NS_BUF_LIVE_L       float [N]             their log L
 *   NS_BUF_LIVE_CID     int   [N]             their cluster-tree leaf
 *   NS_BUF_NEW_X        float [m][d]          the last iteration's walker outputs (a4-a6): new points
 *   NS_BUF_NEW_L        float [m]             their log L
 *   NS_BUF_HIST_L       float [m][t_max]      shrink history of each walker's last slice step
 *   NS_BUF_HIST_X       float [m][t_max][d]   its points
 *   NS_BUF_HIST_LEN     int   [m]             entries used
 *   NS_BUF_WALKER_EVALS int   [m]             likelihood evaluations of each walker (in-box candidates)
 *   NS_BUF_WALKER_FLAGS int   [m]             bit 0: a step-out cap was hit, bit 1: a shrink cap
 *   NS_BUF_CHOL         float [n_nodes][d][d] the cluster tree's Cholesky factors (row-major, lower)
 *   NS_BUF_CENTRES      float [n_nodes][d]    its centres
 *   NS_BUF_MASK         int   [n_nodes]       its accepted leaves
 * The walker buffers are the step level's (ns_slice_replace) for the
 * iteration's selection; together with the live set read before that
 * iteration they let a caller replay each walker on the CPU. */
typedef enum {
    NS_BUF_LIVE_X = 0, NS_BUF_LIVE_L, NS_BUF_LIVE_CID, NS_BUF_NEW_X, NS_BUF_NEW_L, NS_BUF_HIST_L,
    NS_BUF_HIST_X, NS_BUF_HIST_LEN, NS_BUF_WALKER_EVALS, NS_BUF_WALKER_FLAGS, NS_BUF_CHOL,
    NS_BUF_CENTRES, NS_BUF_MASK, NS_BUF_COUNT_
} ns_buffer;
size_t ns_run_buffer_bytes(const ns_handle* h, int run, int which);
ns_status ns_copy_run_buffer(ns_handle* h, int run, int which, void* host, size_t bytes, void* stream);

/* How many runs of dimension d, batch m and tree depth one SM of the
 * current device holds at once (one thread block each); -1 on error.
 * ns_create_batch with (this) x (SM count) runs of that shape fills the
 * GPU in a single wave. */
int ns_resident_runs_per_sm(int d, int m, int depth);

/* Number of runs in the handle, or -1 for NULL. */
int ns_n_runs(const ns_handle* h);

/* Device time of the last ns_run in milliseconds (CUDA events). */
ns_status ns_last_run_ms(const ns_handle* h, double* ms);

/* Counters of the last ns_run (and of ns_create / ns_result for the byte
 * counts): run_ms = device time of the whole call; kernel_ms = summed
 * device time of the run-kernel launches (CUDA events around each launch
 * group, on the run's stream); launches = run-kernel launches; h2d_bytes =
 * bytes copied host->device by ns_create; d2h_bytes = bytes copied
 * device->host by the last ns_run plus every ns_result since. */
typedef struct {
    double run_ms;
    double kernel_ms;
    long long launches;
    long long h2d_bytes;
    long long d2h_bytes;
} ns_stats;
ns_status ns_get_stats(const ns_handle* h, ns_stats* out);

/* Last error message of the handle (or of the library if h is NULL). */
const char* ns_last_error(const ns_handle* h);

/* Frees every device and host resource of the handle.  NULL is ignored. */
void ns_destroy(ns_handle* h);

/* ---- a whole run without any device allocation -------------------------
 * The paper has no counterpart to this call; it exists for callers that
 * cannot use cudaMalloc: a library loaded into a host program whose device
 * memory is already reserved by another allocator (so a fresh cudaMalloc
 * fails or fragments that pool), or code on a latency-critical path where
 * cudaMalloc's implicit device-wide synchronisation would stall other work.
 *
 * ns_run_noalloc does what ns_create + ns_run + ns_summary do for one run,
 * but all of its working memory (live set, walker staging, history, cluster
 * tables, run state) lives in one file-scope device array of
 * NS_NOALLOC_SCRATCH_BYTES that every GPU loading the library holds until
 * the process exits.  It calls no cudaMalloc, cudaFree or other allocating
 * routine.  The caller provides the outputs: dead_x [dead_cap*d],
 * dead_logl [dead_cap] and dead_logw [dead_cap] in device memory, filled as
 * in ns_result (dead points in death order, then the final live points), and
 * `out` on the host, whose three sample pointers are set to NULL (the
 * samples are in the caller's device arrays).  `problem` and `opt` are host
 * structs as for ns_create_batch (opt NULL = defaults; opt->dead_cap is
 * ignored, dead_cap sizes the caller's arrays).
 *
 * Limits and errors: the run's working set is, to within a few KB of
 * descriptors and 256-byte rounding,
 *   4 m (n_slice_steps r + t_max (d + 1) + 2 d + 2)        walkers
 *   + 4 n_pad (d + 2) [+ 4 n_pad (d + 1) if depth > 0]      live set
 *   + 12 n_nodes d^2 (+ the tree scratch of a spilled run)  cluster tables
 * bytes, with r = c + 4 rounded up to a multiple of 4 (the per-step
 * direction row; c = d rounded up to its register class 2,4,6,8,10,12,16,
 * 20,24,28,32), n_pad = N rounded up to 32, n_nodes = 2^(depth+1) - 1.  The slice steps usually dominate: d = 32,
 * N = 4096, m = 128, 160 slice steps, depth 0 needs about 4.6 MB and fits;
 * the same run with m = 256 needs about 8.7 MB and does not.  A run that
 * does not fit is rejected with NS_ERR_ARG and a message giving the bytes
 * it needs; so is dead_cap < N + m.  Every call shares the one array: it is
 * re-initialised at the start of each call, and calls whose GPU work
 * overlaps (two host threads, or two streams) race on it and give wrong
 * results -- serialise them.  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress) with that device current
 * and keeps it for the life of the process; make that first call before
 * any stream capture begins.  The kept address belongs to the device's
 * primary context: after cudaDeviceReset it is stale, so a program that
 * resets a device must not call ns_run_noalloc on it again.  The call waits
 * for the run to finish on `stream`. */
#define NS_NOALLOC_SCRATCH_BYTES (8u << 20)
ns_status ns_run_noalloc(const ns_problem* problem, const ns_options* opt, float* dead_x, float* dead_logl,
                         double* dead_logw, long long dead_cap, ns_result_t* out, void* stream);

/* ---- step-level calls (device buffers, asynchronous, no allocation) ----
 * These run the same device code as ns_run, one step at a time, on caller
 * buffers.  Layouts: live_x is structure-of-arrays [d][n_pad] (n_pad >= N);
 * everything else is dense row-major as written. */

/* Raw generator: out[4i..4i+3] = Philox4x32-10(ctr[4i..4i+3], key). */
ns_status ns_philox4x32_10(const uint32_t* ctr, uint32_t key0, uint32_t key1, int n,
                           uint32_t* out, void* stream);

/* FP32 log-likelihood of n points x [n][d] (device) -> logl [n] (device). */
ns_status ns_loglike(const ns_likelihood* lik, const double* lo, const double* hi, int d,
                     int n, const float* x, float* logl, void* stream);

/* a1-a2 (Algorithm 1 "sorted", S_W, "RNG.choose"): for each of n_runs runs
 * with N live log-likelihoods logl [n_runs][N] (device), the m lowest by
 * (logL, slot) in ascending order -> worst [n_runs][m] (device), their
 * values -> W [n_runs][m], and each walker's start slot, drawn uniformly from
 * the N - m survivors in ascending slot order with stream
 * (t, walker, NS_PURPOSE_SEED) -> seed_slot [n_runs][m].  seeds [n_runs]
 * (host) are the runs' Philox seeds. */
ns_status ns_select_worst(int n_runs, int N, int m, const float* logl, const uint64_t* seeds,
                          uint32_t t, int* worst, float* W, int* seed_slot, void* stream);

/* a4-a7 (section 2.2 and 3.1): one run's m walkers, each n_steps slice
 * steps from live point seed_slot[i] with direction chol[cid[seed]] z/|z|
 * (chol: [n_nodes][d][d] row-major lower, device FP32), expansion against
 * W[0] and shrinkage against W[i] (W[m-1] for both under correction 3).
 * Outputs (device): new_x [m][d], new_l [m], the last step's shrink history
 * hist_l [m][t_max], hist_x [m][t_max][d], hist_len [m], evals [m] and
 * flags [m] (bit0 step-out cap, bit1 shrink cap).  dir_scratch: device
 * working memory of ns_slice_scratch_bytes(d, m, n_steps) bytes, 16-byte
 * aligned, owned by the caller (it receives the drawn directions). */
ns_status ns_slice_replace(const ns_likelihood* lik, const double* lo, const double* hi, int d,
                           int N, int n_pad, int m, int n_steps, const ns_options* opt,
                           uint64_t seed, uint32_t t, const float* live_x, const float* live_l,
                           const int* seed_slot, const float* W, const float* chol, const int* cid,
                           float* new_x, float* new_l, float* hist_l, float* hist_x, int* hist_len,
                           long long* evals, int* flags, float* dir_scratch, void* stream);

/* Bytes of dir_scratch that ns_slice_replace needs (0 for bad sizes). */
size_t ns_slice_scratch_bytes(int d, int m, int n_steps);

/* a8-a9 (Algorithms 1 and 2): 2m candidates -- the removed points W [m]
 * (candidates 0..m-1) and the new points new_l [m] of walkers 0..m-1
 * (candidates m..2m-1, parent threshold W[i]) -- sorted by (logL,
 * candidate); the m lowest die, the m highest live; then up to K history
 * iterations.  Outputs (device, ascending): acc_* [m] and rej_* [m] with the
 * candidate index (src), history slot used (hpos, -1 none), logL and parent
 * threshold (P, -1 for removed points); n_relaxed [1]. */
ns_status ns_batch_correct(int m, int K, int correction, const float* W, const float* new_l,
                           const float* hist_l, const int* hist_len, int t_max,
                           int* acc_src, int* acc_hpos, float* acc_l, float* acc_P,
                           int* rej_src, int* rej_hpos, float* rej_l, float* rej_P,
                           int* n_relaxed, void* stream);

/* a11 (eq. 1.1 as a sum): FP64 evidence update with n dead points of
 * ascending logL dead_l [n] (device) for N live points.  state [3] (device,
 * FP64) holds (log Z, H, k) and is updated in place; logw [n] (device)
 * receives each point's log weight.  live = 1 treats the points as the final
 * live tail (each gets X_k / N) instead of dead points. */
ns_status ns_evidence_update(int N, int n, const float* dead_l, double* state, double* logw,
                             int live, void* stream);

/* a3 (section 2.1): cluster tree of one live set live_x [d][n_pad] (device)
 * at iteration t: the root is the whole set; for depth >= 1 every node is
 * split by 2-means (points whitened by the root's Cholesky factor; first
 * centre the Philox-chosen member of stream (t, node, NS_PURPOSE_KMEANS),
 * second the member farthest from it; Lloyd iterations to a fixed point or
 * kmeans_iters), then the tree is pruned bottom-up (children replace their
 * parent only if both hold more than n_min points and their bounding-
 * ellipsoid volumes add up to less than (1 - vol_frac) of the parent's).
 * Outputs (device): node centres [n_nodes][d], Cholesky factors chol
 * [n_nodes][d][d] (FP32) and chol64 (FP64), log volumes [n_nodes] (unit-ball
 * constant dropped), counts [n_nodes], split flags [n_nodes], accepted-leaf
 * mask [n_nodes] and each point's leaf cid [N].  n_nodes = 2^(depth+1) - 1.
 * scratch: ns_cluster_scratch_bytes(N, n_pad, d) bytes of device memory
 * (unused, may be NULL, at depth 0): the whitened points and child bits,
 * then room for the tree's FP64 node statistics when a deep tree of large
 * d does not fit in shared memory. */
ns_status ns_cluster(int N, int n_pad, int d, const float* live_x, const ns_options* opt,
                     uint64_t seed, uint32_t t, float* centres, float* chol, double* chol64,
                     float* logvol, int* count, int* split, int* mask, int* cid, void* scratch,
                     void* stream);

/* Bytes of scratch that ns_cluster needs at any depth up to NS_MAX_DEPTH
 * (0 for bad sizes). */
size_t ns_cluster_scratch_bytes(int N, int n_pad, int d);

/* a7, MLP likelihood (the emulator of section 5, replaced by a SiLU MLP and
 * a chi^2 against a data vector).  The weights live on the device as one
 * packed image: BF16 copies in the tensor cores' 128-byte-swizzled tile
 * layout (128 output features x 64 inputs per 16 KB tile), then FP32 biases,
 * data, 1/sigma and the FP32 weights.  Hidden layers up to 512 wide; the
 * output layer any width.
 * ns_mlp_image_bytes: size of that image for `lik` (0 if it does not fit).
 * ns_mlp_pack: builds the image on the host and copies it to `image`
 *   (device, 1024-byte aligned, caller-owned); synchronous on `stream`. */
size_t ns_mlp_image_bytes(const ns_likelihood* lik, int d);
ns_status ns_mlp_pack(const ns_likelihood* lik, int d, void* image, void* stream);

/* log L of n points x [n][d] (device, unit cube) -> logl [n] (device):
 * precision 1 = BF16 inputs, weights and activations on the tensor cores
 * (tcgen05, FP32 accumulation in tensor memory), up to 128 points per call;
 * precision 0 = FP32 on the CUDA cores;
 * precision 2 = FP32 accuracy on the tensor cores, for networks whose
 * weights are all BF16 values (NS_ERR_ARG otherwise): inputs and
 * activations split exactly into three BF16 parts whose products with the
 * weights are exact in FP32, FP32 accumulation and FP32 epilogues (the MLP
 * runs re-evaluate near-threshold points this way when the weights allow);
 * precision 3 = 16-bit accuracy on the tensor cores (two BF16 planes per
 * input and activation, relative rounding 2^-17; BF16-valued weights only),
 * the intermediate stage of the MLP runs' re-evaluation.
 * A block whose tensor-core pipeline stalls past its wait budget writes NaN
 * for its points. */
ns_status ns_mlp_loglike(const ns_likelihood* lik, const double* lo, const double* hi, int d,
                         const void* image, int n, const float* x, float* logl, int precision,
                         void* stream);

/* The tensor-core evaluators of ns_mlp_loglike (precision 1: BF16;
 * precision 2: FP32 accuracy, BF16-valued weights only) split over a
 * thread-block cluster of `cluster` (2 or 4) CTAs on as many SMs: each CTA
 * streams and multiplies the weight tiles of a disjoint share of every
 * layer's 128-row output tiles (tile t goes to CTA t % cluster), passes its
 * slice of each hidden layer's activations to the other CTAs through
 * distributed shared memory, and CTA 0 adds the CTAs' partial chi^2 in rank
 * order.  This is how one MLP run's batches are evaluated when its
 * ns_options.mlp_cluster is above 1 (section 5: one emulator inference on
 * several SMs).  Same arguments, layouts and results as ns_mlp_loglike up to
 * the order of that last sum; NS_ERR_ARG if a layer's tile count is not a
 * multiple of `cluster`. */
ns_status ns_mlp_loglike_cluster(const ns_likelihood* lik, const double* lo, const double* hi, int d,
                                 const void* image, int n, const float* x, float* logl, int precision, int cluster,
                                 void* stream);

#ifdef __cplusplus
}
#endif
#endif /* NS_GB300_H */
