/*
 * ns_oracle.h -- plain FP64 CPU reference of the batched nested sampler
 * ("Fast and efficient nested sampling with BEST", arXiv 2608.28514).
 *
 * TEST INFRASTRUCTURE ONLY.  This oracle exists so that the CUDA path can be
 * checked against something slow and obviously correct.  Only the test suite,
 * the smoke check and the CPU-baseline leg of the benchmark may load it; the
 * product path never does.  It shares no code with the CUDA sources.
 *
 * Conventions (same as the library's public header, restated here on purpose):
 *  - points live in unit-cube coordinates x in [0,1]^d; the likelihood sees
 *    theta = lo + (hi - lo) * x;
 *  - every random number comes from Philox4x32-10 (Salmon et al., SC'11)
 *    with key = (seed low word, seed high word) and counter
 *    (block, purpose, walker, iteration); draw n of a stream is word n%4 of
 *    block n/4;
 *  - log-likelihoods are unnormalised (section 3.2, eq. for the Gaussian).
 */
#ifndef NS_ORACLE_H
#define NS_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- random numbers ---------------------------------------------------- */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
/* n draws of stream (t, walker, purpose) starting at draw `first`. */
void orc_stream_draws(const uint32_t key[2], uint32_t t, uint32_t walker, uint32_t purpose,
                      uint32_t first, int n, uint32_t* out);

/* ---- likelihoods ------------------------------------------------------- */
enum { ORC_LIK_GAUSS_ISO = 0, ORC_LIK_GAUSS_CORR = 1, ORC_LIK_ROSENBROCK = 2,
       ORC_LIK_MIXTURE = 3, ORC_LIK_MLP = 4, ORC_LIK_GMM = 5, ORC_LIK_SHELL = 6 };

typedef struct {
    int kind;
    int d;
    const double* lo;          /* [d] prior box */
    const double* hi;          /* [d] */
    const double* mean;        /* [d] GAUSS_ISO, GAUSS_CORR */
    const double* prec_chol;   /* [d*d] row-major lower L, inverse covariance = L L^T */
    double sigma;              /* GAUSS_ISO, MIXTURE */
    int n_modes;               /* MIXTURE */
    const double* centres;     /* [n_modes*d] */
    double a, b;               /* ROSENBROCK */
    int n_layers;              /* MLP: number of affine layers */
    const int* widths;         /* [n_layers+1] */
    const double* weights;     /* concatenated [out][in] row-major blocks */
    const double* biases;      /* concatenated [out] blocks */
    const double* data;        /* [widths[n_layers]] */
    const double* sigma_out;   /* [widths[n_layers]] */
    const double* mode_var;    /* [n_modes*d] GMM: per-mode diagonal variances */
    const double* mode_logw;   /* [n_modes]   GMM: log weights (not normalised) */
} orc_lik;

double orc_loglike(const orc_lik* L, const double* x_unit);
/* out[j] = orc_loglike(L, x + j d), j < n */
void orc_loglike_batch(const orc_lik* L, int n, const double* x_unit, double* out);

/* ---- sampler options ---------------------------------------------------- */
typedef struct {
    int depth;           /* cluster tree depth (0 = one cluster) */
    int recluster_every; /* iterations between re-clusterings */
    int n_min;           /* a child needs more than n_min points (<=0: d+1) */
    double vol_frac;     /* children must be this fraction smaller than parent */
    int kmeans_iters;    /* Lloyd iterations per 2-means split */
    int history_iters;   /* K of Algorithm 2 (0 = sorting only) */
    int t_max;           /* history slots per walker */
    int e_max;           /* step-out expansions per side */
    int s_max;           /* shrink draws per slice step */
    double width;        /* initial bracket width along the direction */
    long long max_iter;  /* safety cap on iterations */
    long long dead_cap;  /* capacity of the caller's dead arrays */
    int correction;      /* 0 naive, 1 sorting (Alg. 1), 2 sorting + history (Alg. 2) */
    int bracket;         /* initial slice bracket: 0 = width in units of the cluster's
                            Cholesky factor (reading c3); 1 = width in units of the
                            cluster's bounding radius, the factor scaled by the largest
                            Mahalanobis distance of a member from the centre (reading c18) */
} orc_opts;

void orc_default_opts(orc_opts* o, int d, int m);

/* ---- a2: selection of the m worst and of the slice seeds --------------- */
void orc_select(int N, int m, const double* logl, const uint32_t key[2], uint32_t t,
                int* worst, int* seed_slot);

/* ---- a4-a7: one walker's slice-sampling replacement --------------------- */
typedef struct {
    double min_l_margin;   /* smallest |logL - threshold| met in a comparison */
    double min_box_margin; /* smallest distance of a candidate coordinate to 0 or 1 */
    long long n_evals;
    int flags;             /* bit0: step-out cap hit, bit1: shrink cap hit */
} orc_walker_info;

void orc_slice_walker(const orc_lik* L, const orc_opts* o, int n_steps,
                      const uint32_t key[2], uint32_t t, int walker,
                      const double* x_seed, double l_seed, const double* chol,
                      double thr_out, double thr_in,
                      double* x_out, double* l_out,
                      double* hist_l, double* hist_x, int* hist_len,
                      orc_walker_info* info);

/* ---- a8-a9: Algorithm 1 (batch sorting) and Algorithm 2 (history) ------- */
/* Candidate c in 0..2m-1: c < m is the old point W[c]; c >= m is walker c-m.
 * hpos = -1 means "the point as produced", else the history slot used. */
void orc_batch_correct(int m, int K, int correction, const double* W, const double* newl,
                       const double* hist_l, const int* hist_len, int t_max,
                       int* acc_src, int* acc_hpos, double* acc_l, double* acc_P,
                       int* rej_src, int* rej_hpos, double* rej_l, double* rej_P,
                       int* n_relaxed);

/* ---- a11: evidence bookkeeping ------------------------------------------ */
typedef struct { double logz; double info; long long k; int n_live; } orc_evid;
void orc_evid_init(orc_evid* e, int n_live);
double orc_evid_add_dead(orc_evid* e, double l);                 /* returns log w */
double orc_evid_add_live(orc_evid* e, double l);                 /* final live tail */
int orc_evid_should_stop(const orc_evid* e, double lmax, double stop_frac);

/* ---- a3: clustering ----------------------------------------------------- */
/* Nodes in heap order (root 0, children 2n+1, 2n+2); 2^(depth+1)-1 nodes.
 * x is [N][d] row-major.  radius (may be NULL): per node the largest
 * Mahalanobis distance of a member from the node's centre, in the node's
 * own Cholesky units (0 for an empty node). */
int orc_cluster(int N, int d, const double* x, const orc_opts* o,
                const uint32_t key[2], uint32_t t,
                double* centres, double* chol, double* logvol, int* count,
                int* split, int* mask, int* assign, double* radius);
int orc_nearest_leaf(int d, int n_nodes, const double* centres, const int* mask,
                     const double* x);
/* Regularised Cholesky of a covariance (section 2.1): returns 1 if the
 * eigenvalue-clipping branch was taken. */
int orc_reg_cholesky(int d, const double* cov, double* chol);

/* ---- whole runs --------------------------------------------------------- */
typedef struct {
    double logz, logz_err, info;
    long long n_dead;      /* dead points written (live tail included) */
    long long n_evals, n_iter, n_relaxed;
    int status;            /* 0 ok, 1 max_iter reached, 2 dead_cap reached, 3 walker cap hit */
} orc_result;

/* Batched sampler of Algorithms 1-2.  dead_* are caller arrays of dead_cap. */
void orc_run(const orc_lik* L, int N, int m, int n_steps, double stop_frac, uint64_t seed,
             const orc_opts* o, double* dead_x, double* dead_l, double* dead_logw,
             orc_result* res);
/* Plain sequential nested sampling (one death per iteration, no batch logic). */
void orc_run_sequential(const orc_lik* L, int N, int n_steps, double stop_frac, uint64_t seed,
                        const orc_opts* o, double* dead_x, double* dead_l, double* dead_logw,
                        orc_result* res);

#ifdef __cplusplus
}
#endif
#endif
