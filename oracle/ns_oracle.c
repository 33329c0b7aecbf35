/*
 * ns_oracle.c -- plain, slow, FP64 CPU reference of the batched nested
 * sampler of arXiv 2608.28514 ("Fast and efficient nested sampling with
 * BEST").
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark, never by the product path.  It shares no
 * code, header, table or helper with the CUDA sources.
 *
 * Every function cites the passage of the paper it follows.  Where the paper
 * is silent the reading taken is stated at the function.  Library primitives
 * used as single steps: qsort (sorting), libm (exp, log, sqrt, erf, cos, sin).
 */
#include "ns_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORC_PURPOSE_SEED 0x10000u
#define ORC_PURPOSE_KMEANS 0x20000u
#define ORC_T_INIT 0xFFFFFFFFu
#define ORC_MAX_DEPTH 6
#define ORC_MAX_NODES ((1 << (ORC_MAX_DEPTH + 1)) - 1)

/* ======================================================================= */
/* Philox4x32-10 counter-based generator, as published by Salmon, Moraes,   */
/* Dror and Shaw, "Parallel random numbers: as easy as 1, 2, 3" (SC'11).    */
/* Ten rounds of two 32x32->64 multiplications; the key is bumped by the    */
/* Weyl constants between rounds.                                           */
/* ======================================================================= */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Draw n of stream (t, walker, purpose) is word n%4 of the block with
 * counter (n/4, purpose, walker, t). */
static uint32_t orc_draw_at(const uint32_t key[2], uint32_t t, uint32_t walker,
                            uint32_t purpose, uint32_t n)
{
    uint32_t ctr[4] = {n / 4u, purpose, walker, t};
    uint32_t out[4];
    orc_philox4x32_10(ctr, key, out);
    return out[n % 4u];
}

void orc_stream_draws(const uint32_t key[2], uint32_t t, uint32_t walker, uint32_t purpose,
                      uint32_t first, int n, uint32_t* out)
{
    for (int i = 0; i < n; ++i) out[i] = orc_draw_at(key, t, walker, purpose, first + (uint32_t)i);
}

/* 24-bit uniforms: exactly representable in FP32 and FP64. */
static double u24(uint32_t w) { return (double)(w >> 8) * (1.0 / 16777216.0); }          /* [0,1) */
static double u24_open0(uint32_t w) { return ((double)(w >> 8) + 1.0) * (1.0 / 16777216.0); } /* (0,1] */
/* Uniform integer in [0, n) by the high word of w*n. */
static int u_index(uint32_t w, int n) { return (int)(((uint64_t)w * (uint64_t)n) >> 32); }

/* ======================================================================= */
/* Likelihoods (unnormalised, reading c1).                                   */
/*  - Gaussian: section 3.2, eq. (gaussian), generalised to a mean, width   */
/*    and full covariance (the correlated workload).                        */
/*  - Rosenbrock: section 4.2; for d > 2 the chained sum over neighbours.   */
/*  - Mixture: equal-weight isotropic Gaussians, in the form of eq. (array).*/
/*  - MLP: section 5's emulator replaced by a SiLU MLP and a chi^2.         */
/* ======================================================================= */
static double silu(double z) { return z / (1.0 + exp(-z)); }

double orc_loglike(const orc_lik* L, const double* x)
{
    const int d = L->d;
    double th[64];
    if (d > 64) return -INFINITY;
    for (int i = 0; i < d; ++i) th[i] = L->lo[i] + (L->hi[i] - L->lo[i]) * x[i];

    double ll = -INFINITY;
    switch (L->kind) {
    case ORC_LIK_GAUSS_ISO: {
        double s = 0.0;
        for (int i = 0; i < d; ++i) {
            double u = (th[i] - L->mean[i]) / L->sigma;
            s += u * u;
        }
        ll = -0.5 * s;
        break;
    }
    case ORC_LIK_GAUSS_CORR: {
        /* (theta-mu)^T Sigma^{-1} (theta-mu) = |L^T (theta-mu)|^2 */
        double y[64];
        for (int i = 0; i < d; ++i) y[i] = th[i] - L->mean[i];
        double s = 0.0;
        for (int j = 0; j < d; ++j) {
            double z = 0.0;
            for (int i = j; i < d; ++i) z += L->prec_chol[i * d + j] * y[i];
            s += z * z;
        }
        ll = -0.5 * s;
        break;
    }
    case ORC_LIK_ROSENBROCK: {
        double s = 0.0;
        for (int i = 0; i + 1 < d; ++i) {
            double p = L->a - th[i];
            double q = th[i + 1] - th[i] * th[i];
            s += p * p + L->b * q * q;
        }
        ll = -s;
        break;
    }
    case ORC_LIK_MIXTURE: {
        double e[64];
        int K = L->n_modes;
        double emax = -INFINITY;
        for (int k = 0; k < K && k < 64; ++k) {
            double s = 0.0;
            for (int i = 0; i < d; ++i) {
                double u = th[i] - L->centres[k * d + i];
                s += u * u;
            }
            e[k] = -s / (2.0 * L->sigma * L->sigma);
            if (e[k] > emax) emax = e[k];
        }
        double acc = 0.0;
        for (int k = 0; k < K && k < 64; ++k) acc += exp(e[k] - emax);
        ll = emax + log(acc / (double)K);
        break;
    }
    case ORC_LIK_GMM: {
        /* Test 1 / Test 2 of section 2.3: log sum_k w_k exp(-1/2 sum_i
         * (theta_i - mu_ki)^2 / s_ki^2), weights as given (eqs. array and
         * separation) */
        int K = L->n_modes;
        double e[256];
        double emax = -INFINITY;
        for (int k = 0; k < K && k < 256; ++k) {
            double s = 0.0;
            for (int i = 0; i < d; ++i) {
                double u = th[i] - L->centres[k * d + i];
                s += u * u / L->mode_var[k * d + i];
            }
            e[k] = L->mode_logw[k] - 0.5 * s;
            if (e[k] > emax) emax = e[k];
        }
        double acc = 0.0;
        for (int k = 0; k < K && k < 256; ++k) acc += exp(e[k] - emax);
        ll = emax + log(acc);
        break;
    }
    case ORC_LIK_SHELL: {
        /* Test 3 of section 2.3: -1/2 ((|theta - c| - r0) / w)^2 */
        double r2 = 0.0;
        for (int i = 0; i < d; ++i) {
            double u = th[i] - L->mean[i];
            r2 += u * u;
        }
        double z = (sqrt(r2) - L->a) / L->sigma;
        ll = -0.5 * z * z;
        break;
    }
    case ORC_LIK_MLP: {
        int maxw = 0;
        for (int l = 0; l <= L->n_layers; ++l)
            if (L->widths[l] > maxw) maxw = L->widths[l];
        double* h = (double*)malloc(sizeof(double) * (size_t)maxw);
        double* g = (double*)malloc(sizeof(double) * (size_t)maxw);
        for (int i = 0; i < d; ++i) h[i] = th[i];
        const double* W = L->weights;
        const double* B = L->biases;
        for (int l = 0; l < L->n_layers; ++l) {
            int nin = L->widths[l], nout = L->widths[l + 1];
            for (int o = 0; o < nout; ++o) {
                double s = B[o];
                for (int i = 0; i < nin; ++i) s += W[(size_t)o * nin + i] * h[i];
                g[o] = (l + 1 < L->n_layers) ? silu(s) : s;
            }
            W += (size_t)nin * nout;
            B += nout;
            double* tmp = h; h = g; g = tmp;
        }
        int nout = L->widths[L->n_layers];
        double chi2 = 0.0;
        for (int o = 0; o < nout; ++o) {
            double r = (h[o] - L->data[o]) / L->sigma_out[o];
            chi2 += r * r;
        }
        free(h);
        free(g);
        ll = -0.5 * chi2;
        break;
    }
    default:
        ll = -INFINITY;
    }
    if (ll != ll) ll = -INFINITY; /* NaN counts as outside the constraint */
    return ll;
}

void orc_loglike_batch(const orc_lik* L, int n, const double* x_unit, double* out)
{
    for (int j = 0; j < n; ++j) out[j] = orc_loglike(L, x_unit + (size_t)j * L->d);
}

/* ======================================================================= */
/* Options                                                                   */
/* ======================================================================= */
void orc_default_opts(orc_opts* o, int d, int m)
{
    o->depth = 0;
    /* Section 2.3 re-clusters every 100 iterations of one death each; the
     * same number of deaths between re-clusterings at batch size m. */
    o->recluster_every = m >= 100 ? 1 : 100 / (m > 0 ? m : 1);
    o->n_min = d + 1;
    o->vol_frac = 0.5;
    o->kmeans_iters = 10;
    o->history_iters = 1;
    o->t_max = 64;
    o->e_max = 64;
    o->s_max = 128;
    o->width = 1.0;
    o->max_iter = 1000000;
    o->dead_cap = 0;
    o->correction = 2;
    o->bracket = 0;
}

/* ======================================================================= */
/* a2: the m worst live points and the slice seeds (Algorithm 1:            */
/* "sorted", S_W = first m, "RNG.choose").                                  */
/* Reading c2: seeds are drawn, with replacement, from the N-m survivors,   */
/* taken in ascending slot order.                                           */
/* ======================================================================= */
typedef struct { double l; int slot; } orc_ls;

static int cmp_ls(const void* pa, const void* pb)
{
    const orc_ls* a = (const orc_ls*)pa;
    const orc_ls* b = (const orc_ls*)pb;
    if (a->l < b->l) return -1;
    if (a->l > b->l) return 1;
    return (a->slot > b->slot) - (a->slot < b->slot);
}

void orc_select(int N, int m, const double* logl, const uint32_t key[2], uint32_t t,
                int* worst, int* seed_slot)
{
    orc_ls* s = (orc_ls*)malloc(sizeof(orc_ls) * (size_t)N);
    for (int j = 0; j < N; ++j) { s[j].l = logl[j]; s[j].slot = j; }
    qsort(s, (size_t)N, sizeof(orc_ls), cmp_ls);
    char* dead = (char*)calloc((size_t)N, 1);
    for (int i = 0; i < m; ++i) { worst[i] = s[i].slot; dead[s[i].slot] = 1; }
    int* surv = (int*)malloc(sizeof(int) * (size_t)N);
    int ns = 0;
    for (int j = 0; j < N; ++j)
        if (!dead[j]) surv[ns++] = j;
    for (int i = 0; i < m; ++i) {
        uint32_t w = orc_draw_at(key, t, (uint32_t)i, ORC_PURPOSE_SEED, 0);
        seed_slot[i] = surv[u_index(w, ns)];
    }
    free(surv);
    free(dead);
    free(s);
}

/* ======================================================================= */
/* a4-a7: slice sampling of one walker (section 2.2, after Neal 2000), with */
/* the two thresholds of section 3.1: the expansion phase uses the batch's  */
/* worst value (thr_out = W[0]), the shrink phase the walker's own          */
/* (thr_in = W[i]); the shrink samples of the last step are kept as the     */
/* history of Algorithm 2.                                                  */
/* Readings (c3, c4): direction = chol * z/|z| with z standard normal (Box- */
/* Muller on 24-bit uniforms); bracket [-r w, (1-r) w]; a candidate outside */
/* the unit cube is never evaluated and fails; history keeps the first      */
/* t_max-1 samples of the last step plus always the accepted one.           */
/* ======================================================================= */
static int inside_unit(int d, const double* x)
{
    for (int i = 0; i < d; ++i)
        if (!(x[i] >= 0.0 && x[i] <= 1.0)) return 0;
    return 1;
}

static double box_margin(int d, const double* x)
{
    double mg = INFINITY;
    for (int i = 0; i < d; ++i) {
        double a = fabs(x[i]), b = fabs(1.0 - x[i]);
        if (a < mg) mg = a;
        if (b < mg) mg = b;
    }
    return mg;
}

static void note_margin(orc_walker_info* info, double l, double thr)
{
    if (!isfinite(l) || !isfinite(thr)) return;
    double scale = fabs(thr) > fabs(l) ? fabs(thr) : fabs(l);
    if (scale < 1.0) scale = 1.0;
    double mg = fabs(l - thr) / scale;
    if (mg < info->min_l_margin) info->min_l_margin = mg;
}

void orc_slice_walker(const orc_lik* L, const orc_opts* o, int n_steps,
                      const uint32_t key[2], uint32_t t, int walker,
                      const double* x_seed, double l_seed, const double* chol,
                      double thr_out, double thr_in,
                      double* x_out, double* l_out,
                      double* hist_l, double* hist_x, int* hist_len,
                      orc_walker_info* info)
{
    const int d = L->d;
    double x[64], z[64], v[64], xp[64];
    double l = l_seed;
    memcpy(x, x_seed, sizeof(double) * (size_t)d);
    info->min_l_margin = INFINITY;
    info->min_box_margin = INFINITY;
    info->n_evals = 0;
    info->flags = 0;
    if (hist_len) *hist_len = 0;

    for (int s = 0; s < n_steps; ++s) {
        const int last = (s == n_steps - 1);
        uint32_t n = 0; /* draw counter of stream (t, walker, s) */
        /* random isotropic direction */
        for (int p = 0; 2 * p < d; ++p) {
            double u1 = u24_open0(orc_draw_at(key, t, (uint32_t)walker, (uint32_t)s, n++));
            double u2 = u24(orc_draw_at(key, t, (uint32_t)walker, (uint32_t)s, n++));
            double rho = sqrt(-2.0 * log(u1));
            z[2 * p] = rho * cos(2.0 * M_PI * u2);
            if (2 * p + 1 < d) z[2 * p + 1] = rho * sin(2.0 * M_PI * u2);
        }
        double nz = 0.0;
        for (int i = 0; i < d; ++i) nz += z[i] * z[i];
        nz = sqrt(nz);
        if (!(nz > 0.0)) {
            for (int i = 0; i < d; ++i) z[i] = 0.0;
            z[0] = 1.0;
            nz = 1.0;
        }
        /* transformed by the cluster's Cholesky factor (section 2.2) */
        for (int i = 0; i < d; ++i) {
            double acc = 0.0;
            for (int k = 0; k <= i; ++k) acc += chol[i * d + k] * (z[k] / nz);
            v[i] = acc;
        }
        /* initial bracket */
        double r = u24(orc_draw_at(key, t, (uint32_t)walker, (uint32_t)s, n++));
        double a = -r * o->width;
        double b = (1.0 - r) * o->width;
        /* stepping out, always against the batch's worst value */
        for (int side = 0; side < 2; ++side) {
            double* end = side == 0 ? &a : &b;
            for (int e = 0;; ++e) {
                for (int i = 0; i < d; ++i) xp[i] = x[i] + (*end) * v[i];
                double bm = box_margin(d, xp);
                if (bm < info->min_box_margin) info->min_box_margin = bm;
                if (!inside_unit(d, xp)) break;
                double le = orc_loglike(L, xp);
                info->n_evals++;
                note_margin(info, le, thr_out);
                if (!(le > thr_out)) break;
                if (e == o->e_max) { info->flags |= 1; break; }
                *end += side == 0 ? -o->width : o->width;
            }
        }
        /* shrinkage against the walker's own threshold */
        int accepted = 0;
        for (int j = 0; j < o->s_max; ++j) {
            double u = u24(orc_draw_at(key, t, (uint32_t)walker, (uint32_t)s, n++));
            double tp = a + u * (b - a);
            for (int i = 0; i < d; ++i) xp[i] = x[i] + tp * v[i];
            double bm = box_margin(d, xp);
            if (bm < info->min_box_margin) info->min_box_margin = bm;
            int in = inside_unit(d, xp);
            double lp = -INFINITY;
            if (in) {
                lp = orc_loglike(L, xp);
                info->n_evals++;
                note_margin(info, lp, thr_in);
            }
            if (last && hist_l && j < o->t_max - 1) {
                hist_l[j] = lp;
                memcpy(hist_x + (size_t)j * d, xp, sizeof(double) * (size_t)d);
                *hist_len = j + 1;
            }
            if (in && lp > thr_in) {
                memcpy(x, xp, sizeof(double) * (size_t)d);
                l = lp;
                accepted = 1;
                if (last && hist_l && j >= o->t_max - 1) {
                    hist_l[o->t_max - 1] = lp;
                    memcpy(hist_x + (size_t)(o->t_max - 1) * d, xp, sizeof(double) * (size_t)d);
                    *hist_len = o->t_max;
                }
                break;
            }
            if (tp < 0.0) a = tp; else b = tp;
        }
        if (!accepted) info->flags |= 2;
    }
    memcpy(x_out, x, sizeof(double) * (size_t)d);
    *l_out = l;
}

/* ======================================================================= */
/* a8-a9: Algorithm 1 (batch sorting) and Algorithm 2 (history correction).  */
/* Readings: ties in the sort are broken by candidate index (old points,   */
/* in W order, before new points, in walker order) (c5); the i-th faulty    */
/* point is paired with the i-th instant death, up to the smaller count     */
/* (c6).  correction: 0 naive, 1 sorting only, 2 sorting + K history        */
/* iterations, 3 best-of-worst (section 3.1: common threshold, no sort).    */
/* ======================================================================= */
typedef struct { double l, P; int H, src, hpos; } orc_cand;

static int cmp_cand(const void* pa, const void* pb)
{
    const orc_cand* a = (const orc_cand*)pa;
    const orc_cand* b = (const orc_cand*)pb;
    if (a->l < b->l) return -1;
    if (a->l > b->l) return 1;
    return (a->src > b->src) - (a->src < b->src);
}

void orc_batch_correct(int m, int K, int correction, const double* W, const double* newl,
                       const double* hist_l, const int* hist_len, int t_max,
                       int* acc_src, int* acc_hpos, double* acc_l, double* acc_P,
                       int* rej_src, int* rej_hpos, double* rej_l, double* rej_P,
                       int* n_relaxed)
{
    orc_cand* C = (orc_cand*)malloc(sizeof(orc_cand) * (size_t)(2 * m));
    orc_cand* r = C;     /* C[0:m]  */
    orc_cand* a = C + m; /* C[m:2m] */
    int relaxed = 0;
    for (int i = 0; i < m; ++i) {
        C[i].l = W[i]; C[i].P = -1.0; C[i].H = -1; C[i].src = i; C[i].hpos = -1;
        C[m + i].l = newl[i]; C[m + i].P = W[i]; C[m + i].H = i; C[m + i].src = m + i; C[m + i].hpos = -1;
    }
    if (correction == 0 || correction == 3) {
        /* the m removed points die, the m new points go live */
        qsort(a, (size_t)m, sizeof(orc_cand), cmp_cand);
    } else {
        qsort(C, (size_t)(2 * m), sizeof(orc_cand), cmp_cand); /* Alg1.sort */
        if (correction == 2) {
            int* JF = (int*)malloc(sizeof(int) * (size_t)m);
            double* I = (double*)malloc(sizeof(double) * (size_t)m);
            for (int k = 1; k <= K; ++k) {
                int nF = 0, nI = 0;
                for (int j = 0; j < m; ++j)
                    if (a[j].H >= 0 && a[j].P >= a[0].l) JF[nF++] = j;
                if (nF == 0) break;
                for (int j = 0; j < m; ++j)
                    if (r[j].H >= 0) I[nI++] = r[j].l; /* r is sorted: I ascending */
                int np = nF < nI ? nF : nI;
                for (int i = 0; i < np; ++i) {
                    orc_cand* c = &a[JF[i]];
                    int w = c->H;
                    for (int h = 0; h < hist_len[w]; ++h) {
                        double hl = hist_l[(size_t)w * t_max + h];
                        if (hl > I[i]) {
                            c->l = hl;
                            c->hpos = h;
                            c->P = I[i];
                            relaxed++;
                            break;
                        }
                    }
                }
                qsort(C, (size_t)(2 * m), sizeof(orc_cand), cmp_cand);
            }
            free(I);
            free(JF);
        }
    }
    for (int j = 0; j < m; ++j) {
        acc_src[j] = a[j].src; acc_hpos[j] = a[j].hpos; acc_l[j] = a[j].l; acc_P[j] = a[j].P;
        rej_src[j] = r[j].src; rej_hpos[j] = r[j].hpos; rej_l[j] = r[j].l; rej_P[j] = r[j].P;
    }
    if (n_relaxed) *n_relaxed = relaxed;
    free(C);
}

/* ======================================================================= */
/* a11: evidence (eq. 1.1 as a sum over the dead points).  Reading c10:      */
/* X_k = exp(-k/N); rectangle weights X_{k-1} - X_k; the final live points  */
/* share X_K equally; information H after Skilling (2006); error sqrt(H/N). */
/* ======================================================================= */
void orc_evid_init(orc_evid* e, int n_live)
{
    e->logz = -INFINITY;
    e->info = 0.0;
    e->k = 0;
    e->n_live = n_live;
}

static double logaddexp(double a, double b)
{
    if (a == -INFINITY) return b;
    if (b == -INFINITY) return a;
    double mx = a > b ? a : b;
    return mx + log1p(exp(-fabs(a - b)));
}

static void evid_accumulate(orc_evid* e, double l, double logw)
{
    double logz_new = logaddexp(e->logz, logw);
    double info = 0.0;
    if (logz_new > -INFINITY) {
        double wl = exp(logw - logz_new);
        info = (isfinite(l) ? wl * l : 0.0) - logz_new;
        if (e->logz > -INFINITY) info += exp(e->logz - logz_new) * (e->info + e->logz);
    }
    e->logz = logz_new;
    e->info = info;
}

double orc_evid_add_dead(orc_evid* e, double l)
{
    const double N = (double)e->n_live;
    e->k += 1;
    /* log(X_{k-1} - X_k) = -(k-1)/N + log(1 - exp(-1/N)) */
    double logdx = -(double)(e->k - 1) / N + log(-expm1(-1.0 / N));
    double logw = l + logdx;
    evid_accumulate(e, l, logw);
    return logw;
}

double orc_evid_add_live(orc_evid* e, double l)
{
    const double N = (double)e->n_live;
    double logw = l - (double)e->k / N - log(N);
    evid_accumulate(e, l, logw);
    return logw;
}

/* Reading c11: stop when L_max X_k < stop_frac * Z. */
int orc_evid_should_stop(const orc_evid* e, double lmax, double stop_frac)
{
    if (e->logz == -INFINITY) return 0;
    return lmax - (double)e->k / (double)e->n_live - e->logz < log(stop_frac);
}

/* ======================================================================= */
/* a3: clustering (section 2.1).                                            */
/* ======================================================================= */
static int cholesky_plain(int d, const double* A, double* Lo)
{
    memset(Lo, 0, sizeof(double) * (size_t)d * d);
    for (int j = 0; j < d; ++j) {
        double s = A[j * d + j];
        for (int k = 0; k < j; ++k) s -= Lo[j * d + k] * Lo[j * d + k];
        if (!(s > 0.0) || !isfinite(s)) return 0;
        double ljj = sqrt(s);
        Lo[j * d + j] = ljj;
        for (int i = j + 1; i < d; ++i) {
            double u = A[i * d + j];
            for (int k = 0; k < j; ++k) u -= Lo[i * d + k] * Lo[j * d + k];
            Lo[i * d + j] = u / ljj;
        }
    }
    return 1;
}

/* Cyclic Jacobi eigendecomposition of a symmetric d x d matrix:
 * A = Q diag(lam) Q^T (Q's columns are eigenvectors). */
static void jacobi_eigen(int d, const double* A0, double* lam, double* Q)
{
    double* A = (double*)malloc(sizeof(double) * (size_t)d * d);
    memcpy(A, A0, sizeof(double) * (size_t)d * d);
    for (int i = 0; i < d * d; ++i) Q[i] = 0.0;
    for (int i = 0; i < d; ++i) Q[i * d + i] = 1.0;
    for (int sweep = 0; sweep < 100; ++sweep) {
        /* converged once the off-diagonal mass is at FP64 rounding level
         * relative to the diagonal */
        double off = 0.0, dia = 0.0;
        for (int p = 0; p < d; ++p) {
            dia += A[p * d + p] * A[p * d + p];
            for (int q = p + 1; q < d; ++q) off += A[p * d + q] * A[p * d + q];
        }
        if (!(off > 1e-30 * dia)) break;
        for (int p = 0; p < d; ++p) {
            for (int q = p + 1; q < d; ++q) {
                double apq = A[p * d + q];
                if (apq == 0.0) continue;
                double theta = (A[q * d + q] - A[p * d + p]) / (2.0 * apq);
                double tt = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                double c = 1.0 / sqrt(tt * tt + 1.0), s = tt * c;
                for (int k = 0; k < d; ++k) { /* A <- A J */
                    double akp = A[k * d + p], akq = A[k * d + q];
                    A[k * d + p] = c * akp - s * akq;
                    A[k * d + q] = s * akp + c * akq;
                }
                for (int k = 0; k < d; ++k) { /* A <- J^T A */
                    double apk = A[p * d + k], aqk = A[q * d + k];
                    A[p * d + k] = c * apk - s * aqk;
                    A[q * d + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < d; ++k) { /* Q <- Q J */
                    double qkp = Q[k * d + p], qkq = Q[k * d + q];
                    Q[k * d + p] = c * qkp - s * qkq;
                    Q[k * d + q] = s * qkp + c * qkq;
                }
            }
        }
    }
    for (int i = 0; i < d; ++i) lam[i] = A[i * d + i];
    free(A);
}

/* Section 2.1: a covariance that is not numerically positive definite is
 * moved to the nearest PSD matrix by clipping its eigenvalues and then
 * regularised to PD.  Reading c7: the plain Cholesky of C + delta I with
 * delta = 1e-10 tr(C)/d is tried first; only if it fails are eigenvalues
 * clipped at 1e-10 lambda_max. */
int orc_reg_cholesky(int d, const double* cov, double* chol)
{
    double tr = 0.0;
    for (int i = 0; i < d; ++i) tr += cov[i * d + i];
    if (!(tr > 0.0) || !isfinite(tr)) {
        memset(chol, 0, sizeof(double) * (size_t)d * d);
        for (int i = 0; i < d; ++i) chol[i * d + i] = 1e-6;
        return 2;
    }
    double delta = 1e-10 * tr / d;
    double* A = (double*)malloc(sizeof(double) * (size_t)d * d);
    memcpy(A, cov, sizeof(double) * (size_t)d * d);
    for (int i = 0; i < d; ++i) A[i * d + i] += delta;
    int ok = cholesky_plain(d, A, chol);
    int clipped = 0;
    if (!ok) {
        double* lam = (double*)malloc(sizeof(double) * (size_t)d);
        double* Q = (double*)malloc(sizeof(double) * (size_t)d * d);
        jacobi_eigen(d, cov, lam, Q);
        double lmax = 0.0;
        for (int i = 0; i < d; ++i)
            if (lam[i] > lmax) lmax = lam[i];
        for (int i = 0; i < d; ++i)
            if (lam[i] < 1e-10 * lmax) lam[i] = 1e-10 * lmax;
        for (int i = 0; i < d; ++i)
            for (int j = 0; j < d; ++j) {
                double s = 0.0;
                for (int k = 0; k < d; ++k) s += Q[i * d + k] * lam[k] * Q[j * d + k];
                A[i * d + j] = s + (i == j ? delta : 0.0);
            }
        if (!cholesky_plain(d, A, chol)) {
            memset(chol, 0, sizeof(double) * (size_t)d * d);
            for (int i = 0; i < d; ++i) chol[i * d + i] = sqrt(A[i * d + i] > 0 ? A[i * d + i] : 1e-12);
        }
        clipped = 1;
        free(Q);
        free(lam);
    }
    free(A);
    return clipped;
}

/* forward substitution: y = L^{-1} r */
static void lower_solve(int d, const double* Lo, const double* r, double* y)
{
    for (int i = 0; i < d; ++i) {
        double s = r[i];
        for (int k = 0; k < i; ++k) s -= Lo[i * d + k] * y[k];
        y[i] = s / Lo[i * d + i];
    }
}

/* Per-node statistics: mean, covariance (1/n normalisation), regularised
 * Cholesky and the log volume of the ellipsoid of that shape scaled to
 * enclose every member (the unit-ball constant is dropped; it cancels in
 * the pruning comparison). */
static void node_stats(int d, const double* x, const int* members, int n,
                       double* centre, double* chol, double* logvol, double* m2_out)
{
    double* cov = (double*)calloc((size_t)d * d, sizeof(double));
    for (int i = 0; i < d; ++i) centre[i] = 0.0;
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < d; ++i) centre[i] += x[(size_t)members[j] * d + i];
    for (int i = 0; i < d; ++i) centre[i] /= (n > 0 ? n : 1);
    for (int j = 0; j < n; ++j) {
        const double* p = x + (size_t)members[j] * d;
        for (int a = 0; a < d; ++a)
            for (int b = 0; b < d; ++b) cov[a * d + b] += (p[a] - centre[a]) * (p[b] - centre[b]);
    }
    for (int i = 0; i < d * d; ++i) cov[i] /= (n > 0 ? n : 1);
    orc_reg_cholesky(d, cov, chol);
    double r[64], y[64];
    double m2 = 0.0;
    for (int j = 0; j < n; ++j) {
        for (int i = 0; i < d; ++i) r[i] = x[(size_t)members[j] * d + i] - centre[i];
        lower_solve(d, chol, r, y);
        double s = 0.0;
        for (int i = 0; i < d; ++i) s += y[i] * y[i];
        if (s > m2) m2 = s;
    }
    double lv = 0.0;
    for (int i = 0; i < d; ++i) lv += log(chol[i * d + i]);
    *logvol = n > 0 ? lv + 0.5 * d * log(m2) : -INFINITY;
    *m2_out = m2;
    free(cov);
}

/* 2-means split of one node's members.  Reading c7: points are whitened by
 * the Cholesky factor of the whole live set (the root node), so that every
 * split of the tree works in one scale-free space; the first centre is a
 * Philox-chosen member, the second the member farthest from it; a fixed
 * number of Lloyd iterations (assign, then move the centres). */
static void kmeans_split(int d, const double* x, const int* members, int n,
                         const double* centre, const double* chol, int iters,
                         const uint32_t key[2], uint32_t t, int node, int* side)
{
    double* y = (double*)malloc(sizeof(double) * (size_t)n * d);
    double r[64];
    for (int j = 0; j < n; ++j) {
        for (int i = 0; i < d; ++i) r[i] = x[(size_t)members[j] * d + i] - centre[i];
        lower_solve(d, chol, r, y + (size_t)j * d);
    }
    double c[2][64];
    int p = u_index(orc_draw_at(key, t, (uint32_t)node, ORC_PURPOSE_KMEANS, 0), n);
    for (int i = 0; i < d; ++i) c[0][i] = y[(size_t)p * d + i];
    int q = 0;
    double best = -1.0;
    for (int j = 0; j < n; ++j) {
        double s = 0.0;
        for (int i = 0; i < d; ++i) {
            double u = y[(size_t)j * d + i] - c[0][i];
            s += u * u;
        }
        if (s > best) { best = s; q = j; }
    }
    for (int i = 0; i < d; ++i) c[1][i] = y[(size_t)q * d + i];
    for (int it = 0; it < iters; ++it) {
        for (int j = 0; j < n; ++j) {
            double s0 = 0.0, s1 = 0.0;
            for (int i = 0; i < d; ++i) {
                double u0 = y[(size_t)j * d + i] - c[0][i];
                double u1 = y[(size_t)j * d + i] - c[1][i];
                s0 += u0 * u0;
                s1 += u1 * u1;
            }
            side[j] = s1 < s0 ? 1 : 0;
        }
        for (int k = 0; k < 2; ++k) {
            double acc[64] = {0};
            int cnt = 0;
            for (int j = 0; j < n; ++j)
                if (side[j] == k) {
                    for (int i = 0; i < d; ++i) acc[i] += y[(size_t)j * d + i];
                    cnt++;
                }
            if (cnt > 0)
                for (int i = 0; i < d; ++i) c[k][i] = acc[i] / cnt;
        }
    }
    free(y);
}

/* Binary tree of 2-means splits to the full depth, then bottom-up pruning:
 * two children replace their parent only if both hold more than n_min
 * points and their (effective) volumes add up to less than (1 - vol_frac)
 * times the parent's volume.  Returns the number of accepted leaves. */
int orc_cluster(int N, int d, const double* x, const orc_opts* o,
                const uint32_t key[2], uint32_t t,
                double* centres, double* chol, double* logvol, int* count,
                int* split, int* mask, int* assign, double* radius)
{
    const int D = o->depth;
    const int n_nodes = (1 << (D + 1)) - 1;
    const int n_min = o->n_min > 0 ? o->n_min : d + 1;
    /* path[j][k]: the node at depth k that point j belongs to on the full tree */
    int* path = (int*)malloc(sizeof(int) * (size_t)N * (D + 1));
    int* members = (int*)malloc(sizeof(int) * (size_t)N);
    int* side = (int*)malloc(sizeof(int) * (size_t)N);
    for (int j = 0; j < N; ++j) {
        for (int k = 0; k <= D; ++k) path[(size_t)j * (D + 1) + k] = -1;
        path[(size_t)j * (D + 1)] = 0;
    }
    double veff[ORC_MAX_NODES];

    for (int nd = 0; nd < n_nodes; ++nd) {
        int depth_nd = 0;
        for (int k = nd; k > 0; k = (k - 1) / 2) depth_nd++;
        int n = 0;
        for (int j = 0; j < N; ++j)
            if (path[(size_t)j * (D + 1) + depth_nd] == nd) members[n++] = j;
        count[nd] = n;
        double m2 = 0.0;
        node_stats(d, x, members, n, centres + (size_t)nd * d, chol + (size_t)nd * d * d, &logvol[nd], &m2);
        if (radius) radius[nd] = n > 0 ? sqrt(m2) : 0.0;
        if (depth_nd < D) {
            if (n >= 2) {
                kmeans_split(d, x, members, n, centres, chol, o->kmeans_iters, key, t, nd, side);
            } else {
                for (int j = 0; j < n; ++j) side[j] = 0;
            }
            for (int j = 0; j < n; ++j) {
                int child = 2 * nd + 1 + side[j];
                path[(size_t)members[j] * (D + 1) + depth_nd + 1] = child;
            }
        }
    }
    /* bottom-up pruning */
    for (int nd = n_nodes - 1; nd >= 0; --nd) {
        int c1 = 2 * nd + 1, c2 = 2 * nd + 2;
        if (c1 >= n_nodes) {
            split[nd] = 0;
            veff[nd] = logvol[nd];
            continue;
        }
        double vc = logaddexp(veff[c1], veff[c2]);
        int ok = count[c1] > n_min && count[c2] > n_min && vc < log(1.0 - o->vol_frac) + logvol[nd];
        split[nd] = ok;
        veff[nd] = ok ? vc : logvol[nd];
    }
    /* accepted leaves: active nodes that are not split */
    int active[ORC_MAX_NODES];
    int n_leaves = 0;
    for (int nd = 0; nd < n_nodes; ++nd) {
        active[nd] = nd == 0 ? 1 : (active[(nd - 1) / 2] && split[(nd - 1) / 2]);
        mask[nd] = active[nd] && !split[nd];
        n_leaves += mask[nd];
    }
    for (int j = 0; j < N; ++j) {
        int nd = 0, dep = 0;
        while (split[nd]) {
            dep++;
            nd = path[(size_t)j * (D + 1) + dep];
        }
        assign[j] = nd;
    }
    free(side);
    free(members);
    free(path);
    return n_leaves;
}

/* Section 2.1: a new point joins the accepted cluster with the closest
 * centre (reading c8: Euclidean, unit-cube coordinates; ties to the lower
 * node index). */
int orc_nearest_leaf(int d, int n_nodes, const double* centres, const int* mask, const double* x)
{
    int best = -1;
    double bd = INFINITY;
    for (int nd = 0; nd < n_nodes; ++nd) {
        if (!mask[nd]) continue;
        double s = 0.0;
        for (int i = 0; i < d; ++i) {
            double u = x[i] - centres[(size_t)nd * d + i];
            s += u * u;
        }
        if (s < bd) { bd = s; best = nd; }
    }
    return best < 0 ? 0 : best;
}

/* ======================================================================= */
/* Whole runs                                                               */
/* ======================================================================= */
typedef struct {
    int d, N, n_nodes;
    double *x, *l;  /* live set [N][d], [N] */
    int* cid;
    double *centres, *chol, *logvol, *radius;
    int *count, *split, *mask, *assign;
} orc_live;

static void live_alloc(orc_live* s, int N, int d, int depth)
{
    s->d = d;
    s->N = N;
    s->n_nodes = (1 << (depth + 1)) - 1;
    s->x = (double*)malloc(sizeof(double) * (size_t)N * d);
    s->l = (double*)malloc(sizeof(double) * (size_t)N);
    s->cid = (int*)calloc((size_t)N, sizeof(int));
    s->centres = (double*)calloc((size_t)s->n_nodes * d, sizeof(double));
    s->chol = (double*)calloc((size_t)s->n_nodes * d * d, sizeof(double));
    s->logvol = (double*)calloc((size_t)s->n_nodes, sizeof(double));
    s->radius = (double*)calloc((size_t)s->n_nodes, sizeof(double));
    s->count = (int*)calloc((size_t)s->n_nodes, sizeof(int));
    s->split = (int*)calloc((size_t)s->n_nodes, sizeof(int));
    s->mask = (int*)calloc((size_t)s->n_nodes, sizeof(int));
    s->assign = (int*)calloc((size_t)N, sizeof(int));
}

static void live_free(orc_live* s)
{
    free(s->x); free(s->l); free(s->cid); free(s->centres); free(s->chol); free(s->logvol); free(s->radius);
    free(s->count); free(s->split); free(s->mask); free(s->assign);
}

/* Initial live set: N uniform draws in the prior box (unit cube), each
 * coordinate a 24-bit uniform on [0, 1). */
static void live_init(orc_live* s, const orc_lik* L, const uint32_t key[2], long long* n_evals)
{
    const int d = s->d;
    for (int j = 0; j < s->N; ++j) {
        for (int i = 0; i < d; ++i)
            s->x[(size_t)j * d + i] = u24(orc_draw_at(key, ORC_T_INIT, (uint32_t)j, 0, (uint32_t)i));
        s->l[j] = orc_loglike(L, s->x + (size_t)j * d);
    }
    *n_evals += s->N;
}

/* Reading c18 (bracket = 1): the slice bracket's width is counted in units
 * of the walker's cluster's bounding radius, i.e. the direction factor is the
 * cluster's Cholesky factor times its radius (a node with no positive finite
 * radius keeps its factor).  The unscaled factors stay in the tree itself. */
static void live_recluster(orc_live* s, const orc_opts* o, const uint32_t key[2], uint32_t t)
{
    orc_cluster(s->N, s->d, s->x, o, key, t, s->centres, s->chol, s->logvol, s->count,
                s->split, s->mask, s->assign, s->radius);
    memcpy(s->cid, s->assign, sizeof(int) * (size_t)s->N);
    if (o->bracket == 1) {
        const int dd = s->d * s->d;
        for (int nd = 0; nd < s->n_nodes; ++nd) {
            const double r = s->radius[nd];
            if (!(r > 0.0) || !isfinite(r)) continue;
            for (int q = 0; q < dd; ++q) s->chol[(size_t)nd * dd + q] *= r;
        }
    }
}

static double live_max(const orc_live* s)
{
    double mx = -INFINITY;
    for (int j = 0; j < s->N; ++j)
        if (s->l[j] > mx) mx = s->l[j];
    return mx;
}

/* Final live tail in ascending (logL, slot) order. */
static void live_finalise(orc_live* s, orc_evid* ev, double* dead_x, double* dead_l,
                          double* dead_logw, orc_result* res)
{
    const int d = s->d;
    orc_ls* o = (orc_ls*)malloc(sizeof(orc_ls) * (size_t)s->N);
    for (int j = 0; j < s->N; ++j) { o[j].l = s->l[j]; o[j].slot = j; }
    qsort(o, (size_t)s->N, sizeof(orc_ls), cmp_ls);
    for (int j = 0; j < s->N; ++j) {
        long long q = res->n_dead++;
        memcpy(dead_x + (size_t)q * d, s->x + (size_t)o[j].slot * d, sizeof(double) * (size_t)d);
        dead_l[q] = o[j].l;
        dead_logw[q] = orc_evid_add_live(ev, o[j].l);
    }
    free(o);
}

void orc_run(const orc_lik* L, int N, int m, int n_steps, double stop_frac, uint64_t seed,
             const orc_opts* o, double* dead_x, double* dead_l, double* dead_logw,
             orc_result* res)
{
    const int d = L->d;
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    orc_live s;
    live_alloc(&s, N, d, o->depth);
    memset(res, 0, sizeof(*res));
    orc_evid ev;
    orc_evid_init(&ev, N);
    live_init(&s, L, key, &res->n_evals);

    int* worst = (int*)malloc(sizeof(int) * (size_t)m);
    int* seeds = (int*)malloc(sizeof(int) * (size_t)m);
    double* W = (double*)malloc(sizeof(double) * (size_t)m);
    double* nx = (double*)malloc(sizeof(double) * (size_t)m * d);
    double* nl = (double*)malloc(sizeof(double) * (size_t)m);
    double* hl = (double*)malloc(sizeof(double) * (size_t)m * o->t_max);
    double* hx = (double*)malloc(sizeof(double) * (size_t)m * o->t_max * d);
    int* hn = (int*)malloc(sizeof(int) * (size_t)m);
    int *as = (int*)malloc(sizeof(int) * (size_t)m), *ah = (int*)malloc(sizeof(int) * (size_t)m);
    int *rs = (int*)malloc(sizeof(int) * (size_t)m), *rh = (int*)malloc(sizeof(int) * (size_t)m);
    double *al = (double*)malloc(sizeof(double) * (size_t)m), *aP = (double*)malloc(sizeof(double) * (size_t)m);
    double *rl = (double*)malloc(sizeof(double) * (size_t)m), *rP = (double*)malloc(sizeof(double) * (size_t)m);
    double* ax = (double*)malloc(sizeof(double) * (size_t)m * d);
    int* acid = (int*)malloc(sizeof(int) * (size_t)m);

    for (uint32_t t = 0;; ++t) {
        if ((long long)t >= o->max_iter) { res->status = 1; break; }
        if (res->n_dead + m + N > o->dead_cap) { res->status = 2; break; }
        if (o->recluster_every > 0 && t % (uint32_t)o->recluster_every == 0) live_recluster(&s, o, key, t);
        orc_select(N, m, s.l, key, t, worst, seeds);
        for (int i = 0; i < m; ++i) W[i] = s.l[worst[i]];
        const double thr_out = o->correction == 3 ? W[m - 1] : W[0];
        for (int i = 0; i < m; ++i) {
            const double thr_in = o->correction == 3 ? W[m - 1] : W[i];
            const int sd = seeds[i];
            orc_walker_info info;
            orc_slice_walker(L, o, n_steps, key, t, i, s.x + (size_t)sd * d, s.l[sd],
                             s.chol + (size_t)s.cid[sd] * d * d, thr_out, thr_in,
                             nx + (size_t)i * d, &nl[i], hl + (size_t)i * o->t_max,
                             hx + (size_t)i * o->t_max * d, &hn[i], &info);
            res->n_evals += info.n_evals;
            if (info.flags) res->status = 3;
        }
        int nrel = 0;
        orc_batch_correct(m, o->history_iters, o->correction, W, nl, hl, hn, o->t_max,
                          as, ah, al, aP, rs, rh, rl, rP, &nrel);
        res->n_relaxed += nrel;
        /* rejected points die, in ascending order */
        for (int j = 0; j < m; ++j) {
            const double* px;
            if (rs[j] < m) px = s.x + (size_t)worst[rs[j]] * d;
            else if (rh[j] < 0) px = nx + (size_t)(rs[j] - m) * d;
            else px = hx + ((size_t)(rs[j] - m) * o->t_max + rh[j]) * d;
            long long q = res->n_dead++;
            memcpy(dead_x + (size_t)q * d, px, sizeof(double) * (size_t)d);
            dead_l[q] = rl[j];
            dead_logw[q] = orc_evid_add_dead(&ev, rl[j]);
        }
        /* accepted points take the slots of S_W, in ascending order */
        for (int j = 0; j < m; ++j) {
            const double* px;
            if (as[j] < m) {
                px = s.x + (size_t)worst[as[j]] * d;
                acid[j] = s.cid[worst[as[j]]];
            } else {
                if (ah[j] < 0) px = nx + (size_t)(as[j] - m) * d;
                else px = hx + ((size_t)(as[j] - m) * o->t_max + ah[j]) * d;
                acid[j] = orc_nearest_leaf(d, s.n_nodes, s.centres, s.mask, px);
            }
            memcpy(ax + (size_t)j * d, px, sizeof(double) * (size_t)d);
        }
        for (int j = 0; j < m; ++j) {
            memcpy(s.x + (size_t)worst[j] * d, ax + (size_t)j * d, sizeof(double) * (size_t)d);
            s.l[worst[j]] = al[j];
            s.cid[worst[j]] = acid[j];
        }
        res->n_iter = (long long)t + 1;
        if (orc_evid_should_stop(&ev, live_max(&s), stop_frac)) break;
    }
    if (res->status != 2) live_finalise(&s, &ev, dead_x, dead_l, dead_logw, res);
    res->logz = ev.logz;
    res->info = ev.info;
    res->logz_err = sqrt(ev.info > 0 ? ev.info / N : 0.0);

    free(acid); free(ax); free(rP); free(rl); free(aP); free(al); free(rh); free(rs);
    free(ah); free(as); free(hn); free(hx); free(hl); free(nl); free(nx); free(W);
    free(seeds); free(worst);
    live_free(&s);
}

/* Textbook sequential nested sampling (section 1): one worst point dies,
 * one replacement is drawn above it.  Written without the batch machinery
 * so that the batched sampler at m = 1 can be checked against it. */
void orc_run_sequential(const orc_lik* L, int N, int n_steps, double stop_frac, uint64_t seed,
                        const orc_opts* o, double* dead_x, double* dead_l, double* dead_logw,
                        orc_result* res)
{
    const int d = L->d;
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    orc_live s;
    live_alloc(&s, N, d, o->depth);
    memset(res, 0, sizeof(*res));
    orc_evid ev;
    orc_evid_init(&ev, N);
    live_init(&s, L, key, &res->n_evals);
    double* xn = (double*)malloc(sizeof(double) * (size_t)d);
    for (uint32_t t = 0;; ++t) {
        if ((long long)t >= o->max_iter) { res->status = 1; break; }
        if (res->n_dead + 1 + N > o->dead_cap) { res->status = 2; break; }
        if (o->recluster_every > 0 && t % (uint32_t)o->recluster_every == 0) live_recluster(&s, o, key, t);
        int w = 0;
        for (int j = 1; j < N; ++j)
            if (s.l[j] < s.l[w]) w = j; /* first minimum: lowest slot among ties */
        const double thr = s.l[w];
        int pick = u_index(orc_draw_at(key, t, 0, ORC_PURPOSE_SEED, 0), N - 1);
        int sd = pick < w ? pick : pick + 1; /* pick-th slot other than w */
        double ln;
        orc_walker_info info;
        orc_slice_walker(L, o, n_steps, key, t, 0, s.x + (size_t)sd * d, s.l[sd],
                         s.chol + (size_t)s.cid[sd] * d * d, thr, thr, xn, &ln, NULL, NULL, NULL, &info);
        res->n_evals += info.n_evals;
        if (info.flags) res->status = 3;
        long long q = res->n_dead++;
        memcpy(dead_x + (size_t)q * d, s.x + (size_t)w * d, sizeof(double) * (size_t)d);
        dead_l[q] = thr;
        dead_logw[q] = orc_evid_add_dead(&ev, thr);
        memcpy(s.x + (size_t)w * d, xn, sizeof(double) * (size_t)d);
        s.l[w] = ln;
        s.cid[w] = orc_nearest_leaf(d, s.n_nodes, s.centres, s.mask, xn);
        res->n_iter = (long long)t + 1;
        if (orc_evid_should_stop(&ev, live_max(&s), stop_frac)) break;
    }
    if (res->status != 2) live_finalise(&s, &ev, dead_x, dead_l, dead_logw, res);
    res->logz = ev.logz;
    res->info = ev.info;
    res->logz_err = sqrt(ev.info > 0 ? ev.info / N : 0.0);
    free(xn);
    live_free(&s);
}
