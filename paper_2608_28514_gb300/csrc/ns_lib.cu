// ns_lib.cu -- kernels and C ABI of the GB300 batched nested sampler
// (arXiv 2608.28514: slice-sampling replacement, section 2.2; batch sorting
// and history correction, Algorithms 1-2 of section 3.1; clustering, section
// 2.1; evidence, eq. 1.1).
//
// Execution model: one persistent thread block per run.  A launch advances
// each of its runs by up to `chunk_iters` iterations (select -> slice
// walkers -> Algorithms 1/2 -> live/dead update -> FP64 evidence -> stop
// test) with no host involvement; the host reads one status word per run
// between launches.  Walkers are threads of the run's block.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "../../include/ns_gb300.h"
#include "ns_run.cuh"

using namespace nsd;

// From ns_mlp.cu.
bool ns_mlp_make_desc(const ns_likelihood& L, const double* lo, const double* hi, int d, MlpDesc* M,
                      std::string* msg);
void ns_mlp_pack_host(const ns_likelihood& L, const MlpDesc& M, std::vector<uint8_t>& img);

namespace {

// ---------------------------------------------------------------------------
// Step-level kernels (same device code, caller buffers)
// ---------------------------------------------------------------------------
__global__ void k_philox(const uint32_t* __restrict__ ctr, uint32_t k0, uint32_t k1, int n,
                         uint32_t* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const U4 r = philox(ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3], k0, k1);
  out[4 * i] = r.x;
  out[4 * i + 1] = r.y;
  out[4 * i + 2] = r.z;
  out[4 * i + 3] = r.w;
}

struct SelectArgs {
  uint32_t keys[2 * 128];
};

__global__ void k_select(int N, int m, const float* __restrict__ logl, const SelectArgs K, uint32_t t,
                         int* worst, float* W, int* seed_slot) {
  extern __shared__ __align__(16) char sm[];
  __shared__ BlockScratch S;
  __shared__ SelectScratch X;
  int* sel_slot = reinterpret_cast<int*>(sm);
  uint32_t* sel_key = reinterpret_cast<uint32_t*>(sm + al16(sizeof(int) * m));
  const int r = blockIdx.x;
  select_worst(logl + (size_t)r * N, N, m, K.keys[2 * r], K.keys[2 * r + 1], t, sel_slot, sel_key,
               worst + (size_t)r * m, W + (size_t)r * m, seed_slot + (size_t)r * m, X, S);
}

__global__ void k_correct(int m, int K, int correction, const float* __restrict__ W,
                          const float* __restrict__ new_l, const float* __restrict__ hist_l,
                          const int* __restrict__ hist_len, int t_max, int* acc_src, int* acc_hpos,
                          float* acc_l, float* acc_P, int* rej_src, int* rej_hpos, float* rej_l,
                          float* rej_P, int* n_relaxed) {
  extern __shared__ __align__(16) char sm[];
  __shared__ BlockScratch S;
  __shared__ int ctr;
  const size_t cb = al16((sizeof(float) * 2 + sizeof(int) * 3) * 2 * m + 64);
  const Cand A = cand_at(sm, m);
  const Cand Bf = cand_at(sm + cb, m);
  const Cand Tm = cand_at(sm + 2 * cb, m);
  int* list = reinterpret_cast<int*>(sm + 3 * cb);
  float* vals = reinterpret_cast<float*>(sm + 3 * cb + al16(sizeof(int) * 2 * m));
  const int rel = batch_correct(m, K, correction, W, new_l, hist_l, hist_len, t_max, A, Bf, Tm, list, vals, &ctr, S);
  for (int j = threadIdx.x; j < m; j += blockDim.x) {
    rej_src[j] = A.src[j];
    rej_hpos[j] = A.hp[j];
    rej_l[j] = A.l[j];
    rej_P[j] = A.P[j];
    acc_src[j] = A.src[m + j];
    acc_hpos[j] = A.hp[m + j];
    acc_l[j] = A.l[m + j];
    acc_P[j] = A.P[m + j];
  }
  if (threadIdx.x == 0) *n_relaxed = rel;
}

__global__ void k_evidence(int N, int n, const float* __restrict__ l, double* state, double* logw, int live) {
  __shared__ BlockScratch S;
  __shared__ EvidState E;
  if (threadIdx.x == 0) {
    E.logz = state[0];
    E.info = state[1];
    E.k = (long long)state[2];
  }
  __syncthreads();
  evidence_add(E, N, n, l, logw, live != 0, S);
  if (threadIdx.x == 0) {
    state[0] = E.logz;
    state[1] = E.info;
    state[2] = (double)E.k;
  }
}

__global__ void k_cluster(RunDesc R, uint32_t t) {
  extern __shared__ __align__(16) char sm[];
  __shared__ BlockScratch S;
  const Carve cv = make_carve(R.d, 1, R.n_nodes, kMaxDim, false, R.spill != 0);
  cluster_phase(R, t, sm, cv, S);
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
std::mutex g_err_mu;
std::string g_err;

void set_err(std::string* dst, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  std::lock_guard<std::mutex> lk(g_err_mu);
  g_err = buf;
  if (dst) *dst = buf;
}

#define NS_CUDA(call, errdst)                                                                  \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess) {                                                                   \
      set_err(errdst, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
      return e_ == cudaErrorMemoryAllocation ? NS_ERR_OOM : NS_ERR_CUDA;                       \
    }                                                                                          \
  } while (0)

struct ClassFns {
  int dmax;
  cudaError_t (*run)(const RunDesc*, const int*, int, int, size_t, int, cudaStream_t);
  cudaError_t (*ll)(const LikParams&, int, const float*, float*, cudaStream_t);
  cudaError_t (*sl)(const LikParams&, const SliceCfg&, int, int, int, const float*, const float*, const int*,
                    const float*, const float*, const int*, float*, float*, float*, float*, int*, long long*, int*,
                    float*, int, cudaStream_t);
  cudaError_t (*occ)(int, size_t, int*);
};
#define NS_CLASS_ENTRY(D) {D, launch_run_##D, launch_loglike_##D, launch_slice_##D, occupancy_run_##D},
const ClassFns kClasses[] = {NS_FOR_EACH_CLASS(NS_CLASS_ENTRY)};
constexpr int kNumClasses = sizeof(kClasses) / sizeof(kClasses[0]);

int class_index(int d) {
  for (int c = 0; c < kNumClasses; ++c)
    if (d <= kClasses[c].dmax) return c;
  return kNumClasses - 1;
}
int dmax_class(int d) { return kClasses[class_index(d)].dmax; }

// True when two MLP likelihoods describe the same network and data (equal
// widths, weights, biases, data and sigma_out; pointer-equal arrays are
// taken as equal without a comparison).
bool same_network(const ns_likelihood& a, const ns_likelihood& b) {
  if (a.n_layers != b.n_layers) return false;
  for (int l = 0; l <= a.n_layers; ++l)
    if (a.widths[l] != b.widths[l]) return false;
  size_t nw = 0, nb = 0;
  for (int l = 0; l < a.n_layers; ++l) {
    nw += (size_t)a.widths[l] * a.widths[l + 1];
    nb += (size_t)a.widths[l + 1];
  }
  const size_t no = (size_t)a.widths[a.n_layers];
  auto eq = [](const float* x, const float* y, size_t n) {
    return x == y || std::memcmp(x, y, sizeof(float) * n) == 0;
  };
  return eq(a.weights, b.weights, nw) && eq(a.biases, b.biases, nb) && eq(a.data, b.data, no) &&
         eq(a.sigma_out, b.sigma_out, no);
}

// Dynamic shared memory a run kernel may take (the static part stays below 3 KB).
constexpr size_t kRunSmemBudget = 227 * 1024 - 3072;

// A run whose cluster tables do not fit in shared memory keeps them in
// global memory (make_carve's spill).
bool run_spills(const ns_problem& p, int n_nodes) {
  const bool mlp = p.lik->kind == NS_LIK_MLP;
  return make_carve(p.d, p.m, n_nodes, dmax_class(p.d), mlp, false).total > kRunSmemBudget;
}

// Global tree scratch of a spilled run, sized for the widest block (the MLP
// run kernel's warps).
size_t tree_ws_bytes(int d, int n_nodes) { return tree_bytes(d, n_nodes, kMlpThreads / 32, tree_chol_warps(d, 8)); }

// FNV-1a over the shape of a batch (what fixes the arena layout): a
// checkpoint restores only into a handle of the same shape.
uint64_t batch_fingerprint(int n_runs, const ns_problem* runs, const ns_options& o, size_t total) {
  uint64_t h = 1469598103934665603ull;
  auto mix = [&](const void* p, size_t n) {
    const unsigned char* b = static_cast<const unsigned char*>(p);
    for (size_t i = 0; i < n; ++i) h = (h ^ b[i]) * 1099511628211ull;
  };
  mix(&n_runs, sizeof(n_runs));
  mix(&total, sizeof(total));
  for (int r = 0; r < n_runs; ++r) {
    const ns_problem& p = runs[r];
    const int v[6] = {p.d, p.n_live, p.m, p.n_slice_steps, p.lik->kind,
                      p.lik->kind == NS_LIK_MLP ? p.lik->n_layers : p.lik->n_modes};
    mix(v, sizeof(v));
    mix(&p.seed, sizeof(p.seed));
    mix(&p.stop_frac, sizeof(p.stop_frac));
  }
  const long long w[12] = {o.depth, o.recluster_every, o.n_min, o.kmeans_iters, o.correction, o.history_iters,
                           o.t_max, o.e_max, o.s_max, o.max_iter, o.dead_cap, o.precision};
  mix(w, sizeof(w));
  return h;
}

// Header of a checkpoint (ns_checkpoint).
struct CheckpointHeader {
  char magic[8];
  uint64_t fingerprint, total, off_desc, desc_bytes, off_state;
  int n_runs, pad;
};
constexpr char kCkptMagic[8] = {'N', 'S', 'C', 'K', 'P', 'T', '0', '1'};

int block_for_m(int m) {
  int b = ((m + 31) / 32) * 32;
  if (b < 128) b = 128;
  if (b > 256) b = 256;
  return b;
}

bool finite_pos(double v) { return std::isfinite(v) && v > 0; }

ns_status check_lik(const ns_likelihood* L, int d, std::string* err) {
  if (!L) {
    set_err(err, "likelihood is NULL");
    return NS_ERR_ARG;
  }
  switch (L->kind) {
    case NS_LIK_GAUSS_ISO:
      if (!L->mean || !finite_pos(L->sigma)) {
        set_err(err, "GAUSS_ISO needs mean and sigma > 0");
        return NS_ERR_ARG;
      }
      for (int i = 0; i < d; ++i)
        if (!std::isfinite(L->mean[i])) {
          set_err(err, "mean[%d] is not finite", i);
          return NS_ERR_ARG;
        }
      return NS_OK;
    case NS_LIK_GAUSS_CORR:
      if (!L->mean || !L->prec_chol) {
        set_err(err, "GAUSS_CORR needs mean and prec_chol");
        return NS_ERR_ARG;
      }
      for (int i = 0; i < d; ++i) {
        if (!std::isfinite(L->mean[i]) || !finite_pos(L->prec_chol[i * d + i])) {
          set_err(err, "GAUSS_CORR: mean[%d] not finite or prec_chol diagonal not positive", i);
          return NS_ERR_ARG;
        }
        for (int j = 0; j <= i; ++j)
          if (!std::isfinite(L->prec_chol[i * d + j])) {
            set_err(err, "prec_chol[%d][%d] is not finite", i, j);
            return NS_ERR_ARG;
          }
      }
      return NS_OK;
    case NS_LIK_ROSENBROCK:
      if (!std::isfinite(L->a) || !std::isfinite(L->b) || L->b < 0 || d < 2) {
        set_err(err, "ROSENBROCK needs finite a, b >= 0 and d >= 2");
        return NS_ERR_ARG;
      }
      return NS_OK;
    case NS_LIK_MIXTURE:
      if (!L->centres || L->n_modes < 1 || L->n_modes > NS_MAX_MODES || !finite_pos(L->sigma)) {
        set_err(err, "MIXTURE needs 1..%d centres and sigma > 0", NS_MAX_MODES);
        return NS_ERR_ARG;
      }
      for (int k = 0; k < L->n_modes * d; ++k)
        if (!std::isfinite(L->centres[k])) {
          set_err(err, "centres[%d] is not finite", k);
          return NS_ERR_ARG;
        }
      return NS_OK;
    case NS_LIK_GMM:
      if (!L->centres || !L->mode_var || !L->mode_logw || L->n_modes < 1 || L->n_modes > NS_MAX_GMM_MODES ||
          L->n_modes * dmax_class(d) > NS_GMM_CAPACITY) {
        set_err(err, "GMM needs centres, mode_var, mode_logw and 1..%d modes with n_modes x %d <= %d",
                NS_MAX_GMM_MODES, dmax_class(d), NS_GMM_CAPACITY);
        return NS_ERR_ARG;
      }
      for (int k = 0; k < L->n_modes; ++k) {
        if (!std::isfinite(L->mode_logw[k])) {
          set_err(err, "mode_logw[%d] is not finite", k);
          return NS_ERR_ARG;
        }
        for (int i = 0; i < d; ++i)
          if (!std::isfinite(L->centres[k * d + i]) || !finite_pos(L->mode_var[k * d + i])) {
            set_err(err, "GMM mode %d: centre not finite or variance not positive", k);
            return NS_ERR_ARG;
          }
      }
      return NS_OK;
    case NS_LIK_SHELL:
      if (!L->mean || !finite_pos(L->sigma) || !std::isfinite(L->a) || L->a < 0) {
        set_err(err, "SHELL needs the centre (mean), a radius a >= 0 and a width sigma > 0");
        return NS_ERR_ARG;
      }
      for (int i = 0; i < d; ++i)
        if (!std::isfinite(L->mean[i])) {
          set_err(err, "mean[%d] is not finite", i);
          return NS_ERR_ARG;
        }
      return NS_OK;
    case NS_LIK_MLP: {
      MlpDesc M;
      std::string msg;
      std::vector<double> lo(d, 0.0), hi(d, 1.0);
      if (!ns_mlp_make_desc(*L, lo.data(), hi.data(), d, &M, &msg)) {
        set_err(err, "%s", msg.c_str());
        return NS_ERR_ARG;
      }
      return NS_OK;
    }
    default:
      set_err(err, "unknown likelihood kind %d", L->kind);
      return NS_ERR_ARG;
  }
}

ns_status check_opts(const ns_options& o, std::string* err) {
  if (o.depth < 0 || o.depth > NS_MAX_DEPTH) {
    set_err(err, "depth must be in 0..%d", NS_MAX_DEPTH);
    return NS_ERR_ARG;
  }
  if (o.recluster_every < 0 || o.kmeans_iters < 0 || o.history_iters < 0 || o.e_max < 0 || o.s_max < 1 ||
      o.t_max < 1 || o.t_max > NS_MAX_HISTORY || !(o.width > 0) || !std::isfinite(o.width) ||
      o.correction < 0 || o.correction > 3 || o.max_iter < 1 || o.dead_cap < 0 || o.chunk_iters < 0 ||
      !(o.vol_frac >= 0 && o.vol_frac < 1) || o.precision < 0 || o.precision > 2 || !(o.reeval_margin >= 0) ||
      !std::isfinite(o.reeval_margin) || !(o.reeval_rel >= 0) || !std::isfinite(o.reeval_rel) ||
      o.reeval_defer < 0 || o.reeval_defer > 64 || o.walker_mapping < 0 || o.walker_mapping > 1 ||
      o.mlp_batch_cap < 0 || o.mlp_batch_cap > kMlpNbMax ||
      !(o.mlp_cluster == 0 || o.mlp_cluster == 1 || o.mlp_cluster == 2 || o.mlp_cluster == 4) ||
      o.two_plane < 0 || o.two_plane > 1 || !(o.reeval2_margin >= 0) || !std::isfinite(o.reeval2_margin) ||
      !(o.reeval2_rel >= 0) || !std::isfinite(o.reeval2_rel) || o.bracket < 0 || o.bracket > 1) {
    set_err(err, "an option is out of range");
    return NS_ERR_ARG;
  }
  return NS_OK;
}

ns_status check_problem(const ns_problem& p, std::string* err) {
  if (p.d < 1 || p.d > NS_MAX_DIM) {
    set_err(err, "d = %d outside 1..%d", p.d, NS_MAX_DIM);
    return NS_ERR_ARG;
  }
  if (p.n_live < 2 || p.n_live > NS_MAX_LIVE) {
    set_err(err, "n_live = %d outside 2..%d", p.n_live, NS_MAX_LIVE);
    return NS_ERR_ARG;
  }
  if (p.m < 1 || 2 * p.m > p.n_live || p.m > NS_MAX_BATCH) {
    set_err(err, "m = %d must satisfy 1 <= m <= n_live/2 and m <= %d", p.m, NS_MAX_BATCH);
    return NS_ERR_ARG;
  }
  if (p.n_slice_steps < 1 || p.n_slice_steps > 0xFFFF) {
    set_err(err, "n_slice_steps = %d outside 1..65535", p.n_slice_steps);
    return NS_ERR_ARG;
  }
  if (!(p.stop_frac > 0 && p.stop_frac < 1)) {
    set_err(err, "stop_frac must be in (0, 1)");
    return NS_ERR_ARG;
  }
  if (!p.lo || !p.hi) {
    set_err(err, "prior box is NULL");
    return NS_ERR_ARG;
  }
  for (int i = 0; i < p.d; ++i)
    if (!std::isfinite(p.lo[i]) || !std::isfinite(p.hi[i]) || !(p.lo[i] < p.hi[i])) {
      set_err(err, "prior box dimension %d needs finite lo < hi", i);
      return NS_ERR_ARG;
    }
  return check_lik(p.lik, p.d, err);
}

LikParams make_lik(const ns_likelihood& L, const double* lo, const double* hi, int d) {
  LikParams P;
  std::memset(&P, 0, sizeof(P));
  P.kind = L.kind;
  P.d = d;
  for (int i = 0; i < d; ++i) {
    P.lo[i] = (float)lo[i];
    P.span[i] = (float)(hi[i] - lo[i]);
  }
  switch (L.kind) {
    case NS_LIK_GAUSS_ISO:
      P.inv2s2 = (float)(1.0 / (2.0 * L.sigma * L.sigma));
      for (int i = 0; i < d; ++i) P.c[i] = (float)(lo[i] - L.mean[i]);
      break;
    case NS_LIK_GAUSS_CORR:
      for (int i = 0; i < d; ++i) {
        P.c[i] = (float)(lo[i] - L.mean[i]);
        for (int j = 0; j <= i; ++j) {
          float2& cell = P.LpP[(j / 2) * kMaxDim + i];
          if (j % 2 == 0) cell.x = (float)L.prec_chol[i * d + j];
          else cell.y = (float)L.prec_chol[i * d + j];
        }
      }
      break;
    case NS_LIK_ROSENBROCK:
      P.a = (float)L.a;
      P.b = (float)L.b;
      for (int i = 0; i + 1 < d; ++i) P.rw[i] = 1.f;
      break;
    case NS_LIK_MIXTURE:
      P.n_modes = L.n_modes;
      P.inv2s2 = (float)(1.0 / (2.0 * L.sigma * L.sigma));
      P.log_k = (float)std::log((double)L.n_modes);
      for (int k = 0; k < L.n_modes; ++k)
        for (int i = 0; i < d; ++i) P.cm[k * kMaxDim + i] = (float)(lo[i] - L.centres[k * d + i]);
      break;
    case NS_LIK_GMM: {
      const int row = dmax_class(d);
      P.n_modes = L.n_modes;
      for (int k = 0; k < L.n_modes; ++k) {
        P.glw[k] = (float)L.mode_logw[k];
        for (int i = 0; i < d; ++i) {
          P.gm[k * row + i] = (float)(lo[i] - L.centres[k * d + i]);
          P.giv[k * row + i] = (float)(0.5 / L.mode_var[k * d + i]);
        }
      }
      break;
    }
    case NS_LIK_SHELL:
      P.a = (float)L.a;
      P.inv2s2 = (float)(1.0 / (2.0 * L.sigma * L.sigma));
      for (int i = 0; i < d; ++i) P.c[i] = (float)(lo[i] - L.mean[i]);
      break;
    default:
      break;
  }
  return P;
}

struct HostRun {
  int d, N, m;
  long long dead_cap;
  bool fetched = false;
  std::vector<float> dead_x, dead_l;
  std::vector<double> dead_logw;
};

struct ClassGroup {
  int dmax = 0, block = 0, n = 0;
  int cluster = 1;  // MLP group: CTAs per run
  bool mlp = false;
  size_t smem = 0;
  int* d_ids = nullptr;
};

cudaError_t launch_class(const ClassGroup& g, const RunDesc* d_runs, int chunk, cudaStream_t s) {
  if (g.mlp) return launch_run_mlp(d_runs, g.d_ids, g.n, g.block, g.smem, chunk, g.cluster, s);
  return kClasses[class_index(g.dmax)].run(d_runs, g.d_ids, g.n, g.block, g.smem, chunk, s);
}

}  // namespace

struct ns_handle {
  int n_runs = 0;
  ns_options opt;
  void* arena = nullptr;
  size_t arena_bytes = 0;
  RunDesc* d_runs = nullptr;
  RunState* d_states = nullptr;
  RunState* h_states = nullptr;  // pinned
  std::vector<RunDesc> runs;
  std::vector<HostRun> host;
  std::vector<ClassGroup> groups;
  // several groups (register classes, MLP) run concurrently: each on its own
  // stream, forked from and joined back into the caller's stream
  std::vector<cudaStream_t> gstreams;
  std::vector<cudaEvent_t> gjoin;
  cudaEvent_t gfork = nullptr;
  // the arena's meaningful bytes: everything but the run descriptors (device
  // pointers into this arena) is position independent and forms a checkpoint
  char* base = nullptr;
  size_t total = 0, off_desc = 0, desc_bytes = 0, off_state = 0;
  uint64_t fingerprint = 0;
  bool ran = false;
  double last_ms = 0;
  double kernel_ms = 0;
  long long launches = 0;
  long long h2d_bytes = 0;
  long long d2h_bytes = 0;
  std::string err;
};

extern "C" {

ns_status ns_default_options(ns_options* o) {
  if (!o) return NS_ERR_ARG;
  std::memset(o, 0, sizeof(*o));
  o->depth = 0;
  o->recluster_every = 0;
  o->n_min = 0;
  o->vol_frac = 0.5;
  o->kmeans_iters = 10;
  o->correction = 2;
  o->history_iters = 1;
  o->t_max = 64;
  o->e_max = 64;
  o->s_max = 128;
  o->width = 1.0;
  o->max_iter = 1000000;
  o->dead_cap = 0;
  o->chunk_iters = 1000;
  o->precision = 0;
  // the BF16 emulator path's log L error is relative in nature (about 0.1 %
  // at the 99th percentile, 0.35 % at most, on the 27-D emulator network)
  o->reeval_margin = 2.0;
  o->reeval_rel = 4e-3;
  o->reeval_defer = 4;
  o->mlp_batch_cap = kMlpNbMax;
  o->mlp_cluster = 0;
  o->two_plane = 1;
  o->reeval2_margin = 0.05;
  o->reeval2_rel = 1e-4;
  return NS_OK;
}

ns_status ns_create_batch(int n_runs, const ns_problem* runs, const ns_options* opt_in, ns_handle** out) {
  if (!out) {
    set_err(nullptr, "out is NULL");
    return NS_ERR_ARG;
  }
  *out = nullptr;
  if (n_runs < 1 || !runs) {
    set_err(nullptr, "n_runs must be >= 1 and runs non-NULL");
    return NS_ERR_ARG;
  }
  ns_options opt;
  if (opt_in) opt = *opt_in;
  else ns_default_options(&opt);
  ns_status st = check_opts(opt, nullptr);
  if (st != NS_OK) return st;
  for (int r = 0; r < n_runs; ++r) {
    st = check_problem(runs[r], nullptr);
    if (st != NS_OK) {
      std::string m;
      {
        std::lock_guard<std::mutex> lk(g_err_mu);
        m = g_err;
      }
      set_err(nullptr, "run %d: %s", r, m.c_str());
      return st;
    }
  }
  ns_handle* h = new ns_handle();
  h->n_runs = n_runs;
  h->opt = opt;
  const int n_nodes = (1 << (opt.depth + 1)) - 1;
  // arena layout
  std::vector<size_t> offs;
  size_t total = 0;
  auto take = [&](size_t bytes) {
    size_t o = total;
    total += (bytes + 255) & ~(size_t)255;
    return o;
  };
  struct Off {
    int mlp_owner;  // the run whose MLP image this run reads (itself if it owns one)
    int spill;      // cluster tables in global memory
    size_t tree_ws;
    size_t lik, mlp_img, mlp_desc, live_x, live_l, live_cid, new_x, new_l, hist_l, hist_x, hist_len, wk_evals,
        wk_flags, stage_x, dirs, wsp, side, dead_x, dead_l, dead_logw, centres, chol, chol64, logvol, count, split,
        mask;
  };
  std::vector<Off> off(n_runs);
  h->host.resize(n_runs);
  h->runs.resize(n_runs);
  for (int r = 0; r < n_runs; ++r) {
    const ns_problem& p = runs[r];
    const int d = p.d, N = p.n_live, m = p.m, n_pad = ((N + 31) / 32) * 32;
    const long long cap = opt.dead_cap > 0 ? opt.dead_cap : 400LL * N + 4LL * m;
    Off& o = off[r];
    o.lik = take(sizeof(LikParams));
    o.mlp_img = 0;
    o.mlp_desc = 0;
    o.mlp_owner = -1;
    if (p.lik->kind == NS_LIK_MLP) {
      // runs of the same network share one image (one L2-resident copy)
      for (int q = 0; q < r && o.mlp_owner < 0; ++q)
        if (runs[q].lik->kind == NS_LIK_MLP && off[q].mlp_owner == q && same_network(*runs[q].lik, *p.lik))
          o.mlp_owner = q;
      if (o.mlp_owner >= 0) {
        o.mlp_img = off[o.mlp_owner].mlp_img;
      } else {
        o.mlp_owner = r;
        total = (total + 1023) & ~(size_t)1023;
        o.mlp_img = take(ns_mlp_image_bytes(p.lik, d));
      }
      o.mlp_desc = take(sizeof(MlpDesc));
    }
    o.live_x = take(sizeof(float) * (size_t)d * n_pad);
    o.live_l = take(sizeof(float) * N);
    o.live_cid = take(sizeof(int) * N);
    o.new_x = take(sizeof(float) * (size_t)m * d);
    o.new_l = take(sizeof(float) * m);
    o.hist_l = take(sizeof(float) * (size_t)m * opt.t_max);
    o.hist_x = take(sizeof(float) * (size_t)m * opt.t_max * d);
    o.hist_len = take(sizeof(int) * m);
    o.wk_evals = take(sizeof(int) * m);
    o.wk_flags = take(sizeof(int) * m);
    o.stage_x = take(sizeof(float) * (size_t)m * d);
    o.dirs = take(sizeof(float) * (size_t)m * p.n_slice_steps *
                  dir_row(p.lik->kind == NS_LIK_MLP ? kMaxDim : dmax_class(d)));
    o.wsp = take(opt.depth > 0 ? sizeof(float) * (size_t)d * n_pad : 16);
    o.side = take(opt.depth > 0 ? sizeof(int) * (size_t)N : 16);
    o.dead_x = take(sizeof(float) * (size_t)cap * d);
    o.dead_l = take(sizeof(float) * (size_t)cap);
    o.dead_logw = take(sizeof(double) * (size_t)cap);
    o.centres = take(sizeof(float) * n_nodes * d);
    o.chol = take(sizeof(float) * n_nodes * d * d);
    o.chol64 = take(sizeof(double) * n_nodes * d * d);
    o.logvol = take(sizeof(float) * n_nodes);
    o.count = take(sizeof(int) * n_nodes);
    o.split = take(sizeof(int) * n_nodes);
    o.mask = take(sizeof(int) * n_nodes);
    o.spill = run_spills(p, n_nodes) ? 1 : 0;
    o.tree_ws = o.spill ? take(tree_ws_bytes(d, n_nodes)) : 0;
    HostRun& hr = h->host[r];
    hr.d = d;
    hr.N = N;
    hr.m = m;
    hr.dead_cap = cap;
  }
  const size_t off_desc = take(sizeof(RunDesc) * n_runs);
  const size_t off_state = take(sizeof(RunState) * n_runs);
  // class groups
  // one launch group per register class, plus one for MLP runs (index kNumClasses)
  std::vector<int> counts(kNumClasses + 1, 0);
  std::vector<std::vector<int>> members(kNumClasses + 1);
  for (int r = 0; r < n_runs; ++r) {
    const int ci = runs[r].lik->kind == NS_LIK_MLP ? kNumClasses : class_index(runs[r].d);
    members[ci].push_back(r);
    counts[ci]++;
  }
  std::vector<size_t> off_ids(kNumClasses + 1);
  for (int ci = 0; ci <= kNumClasses; ++ci) off_ids[ci] = take(sizeof(int) * std::max(1, counts[ci]));
  h->arena_bytes = total + 1024;
  cudaError_t e = cudaMalloc(&h->arena, total + 1024);
  if (e != cudaSuccess) {
    set_err(&h->err, "cudaMalloc of %zu bytes failed: %s", total, cudaGetErrorString(e));
    delete h;
    return e == cudaErrorMemoryAllocation ? NS_ERR_OOM : NS_ERR_CUDA;
  }
  char* base = reinterpret_cast<char*>((reinterpret_cast<uintptr_t>(h->arena) + 1023) & ~(uintptr_t)1023);
  h->base = base;
  h->total = total;
  h->off_desc = off_desc;
  h->desc_bytes = sizeof(RunDesc) * n_runs;
  h->off_state = off_state;
  h->fingerprint = batch_fingerprint(n_runs, runs, opt, total);
  e = cudaMallocHost(&h->h_states, sizeof(RunState) * n_runs);
  if (e != cudaSuccess) {
    set_err(&h->err, "cudaMallocHost failed: %s", cudaGetErrorString(e));
    cudaFree(h->arena);
    delete h;
    return NS_ERR_CUDA;
  }
  std::vector<LikParams> liks(n_runs);
  for (int r = 0; r < n_runs; ++r) {
    const ns_problem& p = runs[r];
    const Off& o = off[r];
    RunDesc& R = h->runs[r];
    std::memset(&R, 0, sizeof(R));
    R.d = p.d;
    R.N = p.n_live;
    R.m = p.m;
    R.n_pad = ((p.n_live + 31) / 32) * 32;
    R.n_steps = p.n_slice_steps;
    R.depth = opt.depth;
    R.n_nodes = n_nodes;
    R.recluster_every = opt.recluster_every > 0 ? opt.recluster_every : std::max(1, 100 / p.m);
    R.n_min = opt.n_min > 0 ? opt.n_min : p.d + 1;
    R.kmeans_iters = opt.kmeans_iters;
    R.correction = opt.correction;
    R.K = opt.history_iters;
    R.t_max = opt.t_max;
    R.e_max = opt.e_max;
    R.s_max = opt.s_max;
    R.k0 = (uint32_t)(p.seed & 0xFFFFFFFFull);
    R.k1 = (uint32_t)(p.seed >> 32);
    R.width = (float)opt.width;
    R.vol_frac = (float)opt.vol_frac;
    R.log_stop = std::log(p.stop_frac);
    R.max_iter = opt.max_iter;
    R.dead_cap = h->host[r].dead_cap;
    R.lik = reinterpret_cast<const LikParams*>(base + o.lik);
    R.live_x = reinterpret_cast<float*>(base + o.live_x);
    R.live_l = reinterpret_cast<float*>(base + o.live_l);
    R.live_cid = reinterpret_cast<int*>(base + o.live_cid);
    R.new_x = reinterpret_cast<float*>(base + o.new_x);
    R.new_l = reinterpret_cast<float*>(base + o.new_l);
    R.hist_l = reinterpret_cast<float*>(base + o.hist_l);
    R.hist_x = reinterpret_cast<float*>(base + o.hist_x);
    R.hist_len = reinterpret_cast<int*>(base + o.hist_len);
    R.wk_evals = reinterpret_cast<int*>(base + o.wk_evals);
    R.wk_flags = reinterpret_cast<int*>(base + o.wk_flags);
    R.stage_x = reinterpret_cast<float*>(base + o.stage_x);
    R.dirs = reinterpret_cast<float*>(base + o.dirs);
    R.wsp = reinterpret_cast<float*>(base + o.wsp);
    R.side = reinterpret_cast<int*>(base + o.side);
    R.dead_x = reinterpret_cast<float*>(base + o.dead_x);
    R.dead_l = reinterpret_cast<float*>(base + o.dead_l);
    R.dead_logw = reinterpret_cast<double*>(base + o.dead_logw);
    R.centres = reinterpret_cast<float*>(base + o.centres);
    R.chol = reinterpret_cast<float*>(base + o.chol);
    R.chol64 = reinterpret_cast<double*>(base + o.chol64);
    R.logvol = reinterpret_cast<float*>(base + o.logvol);
    R.count = reinterpret_cast<int*>(base + o.count);
    R.split = reinterpret_cast<int*>(base + o.split);
    R.mask = reinterpret_cast<int*>(base + o.mask);
    R.st = reinterpret_cast<RunState*>(base + off_state) + r;
    R.precision = opt.precision;
    R.spill = o.spill;
    R.tree_ws = o.spill ? reinterpret_cast<char*>(base + o.tree_ws) : nullptr;
    R.reeval_margin = (float)opt.reeval_margin;
    R.reeval_rel = (float)opt.reeval_rel;
    R.reeval_defer = opt.reeval_defer;
    R.two_plane = opt.two_plane;
    R.reeval2_margin = (float)opt.reeval2_margin;
    R.reeval2_rel = (float)opt.reeval2_rel;
    R.walker_warp = (p.lik->kind == NS_LIK_MLP) ? 0 : opt.walker_mapping;
    R.mlp_round_cap = opt.mlp_batch_cap;
    R.bracket = opt.bracket;
    if (p.lik->kind == NS_LIK_MLP) {
      R.mlp_tiles = reinterpret_cast<const uint8_t*>(base + o.mlp_img);
      R.mlp_desc = reinterpret_cast<const MlpDesc*>(base + o.mlp_desc);
      MlpDesc M;
      std::string msg;
      ns_mlp_make_desc(*p.lik, p.lo, p.hi, p.d, &M, &msg);
      R.mlp_f32 = reinterpret_cast<const float*>(base + o.mlp_img + M.tile_bytes);
    }
    liks[r] = make_lik(*p.lik, p.lo, p.hi, p.d);
  }
  h->d_runs = reinterpret_cast<RunDesc*>(base + off_desc);
  h->d_states = reinterpret_cast<RunState*>(base + off_state);
  auto fail = [&](ns_status s) {
    cudaFreeHost(h->h_states);
    cudaFree(h->arena);
    delete h;
    return s;
  };
  h->h2d_bytes = (long long)(sizeof(LikParams) + sizeof(RunDesc)) * n_runs;
  for (int r = 0; r < n_runs; ++r) {
    if (runs[r].lik->kind == NS_LIK_MLP) {
      MlpDesc M;
      std::string msg;
      ns_mlp_make_desc(*runs[r].lik, runs[r].lo, runs[r].hi, runs[r].d, &M, &msg);
      e = cudaSuccess;
      if (off[r].mlp_owner == r) {
        std::vector<uint8_t> img;
        ns_mlp_pack_host(*runs[r].lik, M, img);
        e = cudaMemcpy(base + off[r].mlp_img, img.data(), img.size(), cudaMemcpyHostToDevice);
        h->h2d_bytes += (long long)img.size();
      }
      if (e == cudaSuccess) e = cudaMemcpy(base + off[r].mlp_desc, &M, sizeof(M), cudaMemcpyHostToDevice);
      if (e != cudaSuccess) {
        set_err(nullptr, "cudaMemcpy failed: %s", cudaGetErrorString(e));
        return fail(NS_ERR_CUDA);
      }
      h->h2d_bytes += (long long)sizeof(M);
    }
    e = cudaMemcpy(base + off[r].lik, &liks[r], sizeof(LikParams), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      set_err(nullptr, "cudaMemcpy failed: %s", cudaGetErrorString(e));
      return fail(NS_ERR_CUDA);
    }
  }
  e = cudaMemcpy(h->d_runs, h->runs.data(), sizeof(RunDesc) * n_runs, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(h->d_states, 0, sizeof(RunState) * n_runs);
  if (e != cudaSuccess) {
    set_err(nullptr, "device setup failed: %s", cudaGetErrorString(e));
    return fail(NS_ERR_CUDA);
  }
  for (int ci = 0; ci <= kNumClasses; ++ci) {
    if (counts[ci] == 0) continue;
    ClassGroup g;
    g.mlp = (ci == kNumClasses);
    g.dmax = g.mlp ? kMaxDim : kClasses[ci].dmax;
    g.n = counts[ci];
    g.d_ids = reinterpret_cast<int*>(base + off_ids[ci]);
    int maxm = 1;
    size_t smem = 0;
    for (int r : members[ci]) {
      maxm = std::max(maxm, runs[r].m);
      smem = std::max(smem, make_carve(runs[r].d, runs[r].m, n_nodes, g.dmax, g.mlp, off[r].spill != 0).total);
    }
    g.block = block_for_m(maxm);
    if (g.mlp) {
      g.block = std::max(g.block, kMlpThreads);  // the BF16 evaluator's warp roles
      // FP32 on the tensor cores needs BF16-valued weights; CTAs per run
      // (the tile rows of every layer split evenly among them)
      bool fits2 = opt.precision != 0, fits4 = opt.precision != 0;
      for (int r : members[ci]) {
        MlpDesc M;
        std::string msg;
        ns_mlp_make_desc(*runs[r].lik, runs[r].lo, runs[r].hi, runs[r].d, &M, &msg);
        if (opt.precision == 2 && !M.w_bf16) {
          set_err(nullptr, "run %d: precision 2 (FP32 on the tensor cores) needs MLP weights that are BF16 values", r);
          return fail(NS_ERR_ARG);
        }
        fits2 = fits2 && mlp_cluster_fits(M, 2);
        fits4 = fits4 && mlp_cluster_fits(M, 4);
      }
      int dev = 0, n_sm = 1;
      if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) !=
                                                   cudaSuccess)
        n_sm = 1;
      if (opt.mlp_cluster == 0) {
        g.cluster = (fits4 && 4 * g.n <= n_sm) ? 4 : ((fits2 && 2 * g.n <= n_sm) ? 2 : 1);
      } else {
        g.cluster = opt.mlp_cluster;
        if ((g.cluster == 2 && !fits2) || (g.cluster == 4 && !fits4)) {
          set_err(nullptr, "mlp_cluster = %d: every layer's 128-row tile count must be a multiple of it, on the "
                  "tensor-core paths (precision 1 or 2)", g.cluster);
          return fail(NS_ERR_ARG);
        }
      }
    }
    g.smem = smem;
    if (smem > kRunSmemBudget) {
      set_err(nullptr, "runs of dimension class %d need %zu bytes of shared memory (limit 227 KB): "
              "lower the tree depth or m", g.dmax, smem);
      return fail(NS_ERR_ARG);
    }
    e = cudaMemcpy(g.d_ids, members[ci].data(), sizeof(int) * g.n, cudaMemcpyHostToDevice);
    h->h2d_bytes += (long long)sizeof(int) * g.n;
    if (e != cudaSuccess) {
      set_err(nullptr, "cudaMemcpy failed: %s", cudaGetErrorString(e));
      return fail(NS_ERR_CUDA);
    }
    h->groups.push_back(g);
  }
  if (h->groups.size() > 1) {
    e = cudaEventCreateWithFlags(&h->gfork, cudaEventDisableTiming);
    for (size_t gi = 0; gi < h->groups.size() && e == cudaSuccess; ++gi) {
      cudaStream_t gs = nullptr;
      cudaEvent_t ge = nullptr;
      e = cudaStreamCreateWithFlags(&gs, cudaStreamNonBlocking);
      if (e == cudaSuccess) h->gstreams.push_back(gs);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ge, cudaEventDisableTiming);
      if (e == cudaSuccess) h->gjoin.push_back(ge);
    }
    if (e != cudaSuccess) {
      set_err(nullptr, "stream setup failed: %s", cudaGetErrorString(e));
      for (cudaStream_t gs : h->gstreams) cudaStreamDestroy(gs);
      for (cudaEvent_t ge : h->gjoin) cudaEventDestroy(ge);
      if (h->gfork) cudaEventDestroy(h->gfork);
      return fail(NS_ERR_CUDA);
    }
  }
  *out = h;
  return NS_OK;
}

ns_status ns_create(const ns_likelihood* lik, const double* lo, const double* hi, int d, int n_live, int m,
                    int n_slice_steps, double stop_frac, uint64_t seed, const ns_options* opt, ns_handle** out) {
  ns_problem p;
  p.lik = lik;
  p.lo = lo;
  p.hi = hi;
  p.d = d;
  p.n_live = n_live;
  p.m = m;
  p.n_slice_steps = n_slice_steps;
  p.stop_frac = stop_frac;
  p.seed = seed;
  return ns_create_batch(1, &p, opt, out);
}

int ns_n_runs(const ns_handle* h) { return h ? h->n_runs : -1; }

int ns_resident_runs_per_sm(int d, int m, int depth) {
  if (d < 1 || d > NS_MAX_DIM || m < 1 || m > NS_MAX_BATCH || depth < 0 || depth > NS_MAX_DEPTH) return -1;
  const int n_nodes = (1 << (depth + 1)) - 1;
  const int ci = class_index(d);
  int blocks = 0;
  const cudaError_t e =
      kClasses[ci].occ(block_for_m(m), make_carve(d, m, n_nodes, kClasses[ci].dmax).total, &blocks);
  if (e != cudaSuccess) {
    set_err(nullptr, "occupancy query failed: %s", cudaGetErrorString(e));
    return -1;
  }
  return blocks;
}

ns_status ns_reset(ns_handle* h, void* stream) {
  if (!h) return NS_ERR_ARG;
  NS_CUDA(cudaMemsetAsync(h->d_states, 0, sizeof(RunState) * h->n_runs, (cudaStream_t)stream), &h->err);
  for (auto& hr : h->host) {
    hr.fetched = false;
  }
  h->ran = false;
  return NS_OK;
}

namespace {

// Launches every unfinished run for `chunk` iterations per pass; until_done:
// repeat passes until every run has stopped (ns_run), else one pass (ns_step).
ns_status run_impl(ns_handle* h, void* stream_v, int chunk_in, bool until_done) {
  cudaStream_t s = (cudaStream_t)stream_v;
  cudaEvent_t e0, e1, k0, k1;
  NS_CUDA(cudaEventCreate(&e0), &h->err);
  NS_CUDA(cudaEventCreate(&e1), &h->err);
  NS_CUDA(cudaEventCreate(&k0), &h->err);
  NS_CUDA(cudaEventCreate(&k1), &h->err);
  auto cleanup = [&]() {
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaEventDestroy(k0);
    cudaEventDestroy(k1);
  };
  NS_CUDA(cudaEventRecord(e0, s), &h->err);
  const int chunk = chunk_in;
  long long rounds = 0;
  const long long max_rounds = h->opt.max_iter / chunk + 2;
  h->kernel_ms = 0;
  h->launches = 0;
  h->d2h_bytes = 0;
  for (;;) {
    NS_CUDA(cudaEventRecord(k0, s), &h->err);
    const bool fork = h->groups.size() > 1;
    if (fork) NS_CUDA(cudaEventRecord(h->gfork, s), &h->err);
    for (size_t gi = 0; gi < h->groups.size(); ++gi) {
      cudaStream_t gs = fork ? h->gstreams[gi] : s;
      cudaError_t e = fork ? cudaStreamWaitEvent(gs, h->gfork, 0) : cudaSuccess;
      if (e == cudaSuccess) e = launch_class(h->groups[gi], h->d_runs, chunk, gs);
      if (e == cudaSuccess && fork) e = cudaEventRecord(h->gjoin[gi], gs);
      if (e == cudaSuccess && fork) e = cudaStreamWaitEvent(s, h->gjoin[gi], 0);
      if (e != cudaSuccess) {
        set_err(&h->err, "run kernel launch failed: %s", cudaGetErrorString(e));
        cleanup();
        return NS_ERR_CUDA;
      }
      h->launches++;
    }
    NS_CUDA(cudaEventRecord(k1, s), &h->err);
    NS_CUDA(cudaMemcpyAsync(h->h_states, h->d_states, sizeof(RunState) * h->n_runs, cudaMemcpyDeviceToHost, s),
            &h->err);
    NS_CUDA(cudaStreamSynchronize(s), &h->err);
    h->d2h_bytes += (long long)sizeof(RunState) * h->n_runs;
    float kms = 0.f;
    cudaEventElapsedTime(&kms, k0, k1);
    h->kernel_ms += kms;
    ++rounds;
    bool done = true;
    for (int r = 0; r < h->n_runs; ++r)
      if (!h->h_states[r].stopped && h->h_states[r].status == 0) done = false;
    if (done || rounds > max_rounds || !until_done) break;
  }
  NS_CUDA(cudaEventRecord(e1, s), &h->err);
  NS_CUDA(cudaEventSynchronize(e1), &h->err);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  h->last_ms = ms;
  cleanup();
  h->ran = true;
  for (auto& hr : h->host) hr.fetched = false;
  ns_status worst = NS_OK;
  for (int r = 0; r < h->n_runs; ++r)
    if (h->h_states[r].status != 0) worst = (ns_status)h->h_states[r].status;
  if (worst != NS_OK) set_err(&h->err, "a run ended with status %d", (int)worst);
  return worst;
}

}  // namespace

ns_status ns_run(ns_handle* h, void* stream) {
  if (!h) return NS_ERR_ARG;
  return run_impl(h, stream, h->opt.chunk_iters > 0 ? h->opt.chunk_iters : 1000, true);
}

ns_status ns_step(ns_handle* h, int n_iters, void* stream) {
  if (!h || n_iters < 1) return NS_ERR_ARG;
  return run_impl(h, stream, n_iters, false);
}

extern "C++" {
namespace {

// The device buffers of run r that an iteration reads back later: the live
// set, the cluster tables and the state (the dead buffers are appended at
// the state's n_dead, the rest is per-iteration scratch).
template <class F>
void for_each_run_buffer(const ns_handle* h, int r, F&& f) {
  const RunDesc& R = h->runs[r];
  const size_t d = R.d, nn = R.n_nodes;
  f((void*)R.live_x, sizeof(float) * d * R.n_pad);
  f((void*)R.live_l, sizeof(float) * R.N);
  f((void*)R.live_cid, sizeof(int) * R.N);
  f((void*)R.centres, sizeof(float) * nn * d);
  f((void*)R.chol, sizeof(float) * nn * d * d);
  f((void*)R.chol64, sizeof(double) * nn * d * d);
  f((void*)R.logvol, sizeof(float) * nn);
  f((void*)R.count, sizeof(int) * nn);
  f((void*)R.split, sizeof(int) * nn);
  f((void*)R.mask, sizeof(int) * nn);
  f((void*)R.st, sizeof(RunState));
}

}  // namespace
}  // extern "C++"

ns_status ns_set_walker_mapping(ns_handle* h, int run, int warp) {
  if (!h || run < 0 || run >= h->n_runs || warp < 0 || warp > 1) return NS_ERR_ARG;
  if (h->runs[run].mlp_desc != nullptr && warp) {
    set_err(&h->err, "MLP runs keep their lock-step walkers");
    return NS_ERR_ARG;
  }
  h->runs[run].walker_warp = warp;
  NS_CUDA(cudaMemcpy(h->d_runs + run, &h->runs[run], sizeof(RunDesc), cudaMemcpyHostToDevice), &h->err);
  return NS_OK;
}

extern "C++" {
namespace {

// A list of device-to-device copies done by one launch: block b copies
// segment b (sizes are multiples of 4 bytes; 16-byte words where the
// addresses and size allow).
struct CopySeg {
  const char* src;
  char* dst;
  long long bytes;
};
__global__ void k_copy_segments(const CopySeg* __restrict__ seg) {
  const CopySeg S = seg[blockIdx.x];
  const bool v16 = ((reinterpret_cast<uintptr_t>(S.src) | reinterpret_cast<uintptr_t>(S.dst) | (uintptr_t)S.bytes) &
                    15u) == 0;
  if (v16) {
    const int4* a = reinterpret_cast<const int4*>(S.src);
    int4* b = reinterpret_cast<int4*>(S.dst);
    for (long long i = threadIdx.x; i < S.bytes / 16; i += blockDim.x) b[i] = a[i];
  } else {
    const int* a = reinterpret_cast<const int*>(S.src);
    int* b = reinterpret_cast<int*>(S.dst);
    for (long long i = threadIdx.x; i < S.bytes / 4; i += blockDim.x) b[i] = a[i];
  }
}

// ns_autotune's minimum-job guard: the largest share of the remaining job
// (in iterations) a probe may take.
constexpr double kAutotuneMaxProbeFrac = 0.25;

}  // namespace
}  // extern "C++"

ns_status ns_autotune(ns_handle* h, int warm_iters, int probe_iters, int* out_choice, double* out_ratio,
                      void* stream) {
  if (!h || warm_iters < 0 || probe_iters < 1 || probe_iters > 1000) return NS_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const int n = h->n_runs;
  if (warm_iters > 0) {
    const ns_status st = run_impl(h, stream, warm_iters, false);
    if (st != NS_OK) return st;
  }
  // Minimum-job guard: a probe costs modes x probe_iters iterations (the
  // snapshot and its restores are three copy launches); it is skipped, and
  // every run keeps its current configuration, when those iterations exceed
  // a quarter of the job that is left.  The iterations left of run r are
  // estimated from its stopping rule, lmax - k/N - log Z < log(stop_frac):
  // with lmax and log Z frozen at their values now, (N/m) (lmax - k/N -
  // log Z - log stop_frac), at most max_iter - n_iter; the job is its
  // longest run.
  {
    std::vector<RunState> now(n);
    std::vector<std::vector<float>> ll(n);
    NS_CUDA(cudaMemcpyAsync(now.data(), h->d_states, sizeof(RunState) * n, cudaMemcpyDeviceToHost, s), &h->err);
    for (int r = 0; r < n; ++r) {
      ll[r].resize(h->runs[r].N);
      NS_CUDA(cudaMemcpyAsync(ll[r].data(), h->runs[r].live_l, sizeof(float) * h->runs[r].N, cudaMemcpyDeviceToHost,
                              s),
              &h->err);
    }
    NS_CUDA(cudaStreamSynchronize(s), &h->err);
    double left_iters = 0.0;
    int modes_est = 1;
    for (int r = 0; r < n; ++r) {
      const RunState& S = now[r];
      const RunDesc& R = h->runs[r];
      modes_est = std::max(modes_est, R.mlp_desc == nullptr ? 2 : (R.precision == 1 ? 3 : 1));
      if (S.stopped || S.status != 0) continue;
      double left = (double)(R.max_iter - S.n_iter);
      if (S.initialized && std::isfinite(S.logz)) {
        float lmax = -INFINITY;
        for (float v : ll[r]) lmax = std::max(lmax, v);
        const double gap = (double)lmax - (double)S.k / R.N - S.logz - R.log_stop;
        left = std::min(left, std::max(0.0, gap) * (double)R.N / R.m);
      }
      left_iters = std::max(left_iters, left);
    }
    if ((double)modes_est * probe_iters > kAutotuneMaxProbeFrac * left_iters) {
      for (int r = 0; r < n; ++r) {
        if (out_choice)
          out_choice[r] = h->runs[r].mlp_desc == nullptr ? h->runs[r].walker_warp : h->runs[r].mlp_round_cap;
        if (out_ratio) out_ratio[r] = std::nan("");
      }
      return NS_OK;
    }
  }
  // device snapshot of every run's state after the warm-up
  size_t bytes = 0;
  for (int r = 0; r < n; ++r) for_each_run_buffer(h, r, [&](void*, size_t b) { bytes += (b + 255) & ~(size_t)255; });
  char* snap = nullptr;
  size_t n_seg_max = 0;
  for (int r = 0; r < n; ++r) for_each_run_buffer(h, r, [&](void*, size_t) { ++n_seg_max; });
  if (cudaMalloc(&snap, bytes + 2 * sizeof(CopySeg) * n_seg_max) != cudaSuccess) {
    set_err(&h->err, "ns_autotune: cannot allocate %zu bytes for the state snapshot", bytes);
    return NS_ERR_OOM;
  }
  // the snapshot and each restore are one launch of a segment-list copy (a
  // few hundred small buffers per batch of runs: one cudaMemcpyAsync each
  // cost more than the probe itself on short jobs)
  std::vector<CopySeg> seg_save, seg_load;
  {
    size_t o = 0;
    for (int r = 0; r < n; ++r)
      for_each_run_buffer(h, r, [&](void* p, size_t b) {
        seg_save.push_back({static_cast<const char*>(p), snap + o, (long long)b});
        seg_load.push_back({snap + o, static_cast<char*>(p), (long long)b});
        o += (b + 255) & ~(size_t)255;
      });
  }
  const int n_seg = (int)seg_save.size();
  CopySeg* d_seg = reinterpret_cast<CopySeg*>(snap + bytes);
  cudaError_t e0 = cudaMemcpyAsync(d_seg, seg_save.data(), sizeof(CopySeg) * n_seg, cudaMemcpyHostToDevice, s);
  if (e0 == cudaSuccess)
    e0 = cudaMemcpyAsync(d_seg + n_seg, seg_load.data(), sizeof(CopySeg) * n_seg, cudaMemcpyHostToDevice, s);
  auto copy_all = [&](bool save) {
    if (e0 != cudaSuccess) return e0;
    k_copy_segments<<<n_seg, 256, 0, s>>>(d_seg + (save ? 0 : n_seg));
    return cudaGetLastError();
  };
  const std::vector<RunDesc> keep = h->runs;
  // the configurations a run can take, the first being the default: an
  // analytic run's walker mapping (per thread, per warp); a BF16 MLP run's
  // candidates per weight pass (one pass of 128 per round, one of 64, every
  // candidate of the round in equal calls); FP32 MLP runs have one
  auto n_cfg = [&](int r) { return keep[r].mlp_desc == nullptr ? 2 : (keep[r].precision == 1 ? 3 : 1); };
  auto cfg_value = [&](int r, int k) {
    if (keep[r].mlp_desc == nullptr) return k;
    return k == 0 ? kMlpNbMax : (k == 1 ? kMlpNbMax / 2 : 0);
  };
  auto apply = [&](RunDesc& R, int r, int k) {
    if (keep[r].mlp_desc == nullptr) R.walker_warp = cfg_value(r, k);
    else if (keep[r].precision == 1) R.mlp_round_cap = cfg_value(r, k);
  };
  int modes = 1;
  for (int r = 0; r < n; ++r) modes = std::max(modes, n_cfg(r));
  std::vector<RunState> before(n);
  std::vector<std::vector<double>> per_iter(modes, std::vector<double>(n, -1.0));
  ns_status result = NS_OK;
  cudaError_t e = cudaMemcpyAsync(before.data(), h->d_states, sizeof(RunState) * n, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = copy_all(true);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  for (int mode = 0; mode < modes && e == cudaSuccess && result == NS_OK; ++mode) {
    for (int r = 0; r < n; ++r) {
      h->runs[r] = keep[r];
      apply(h->runs[r], r, mode < n_cfg(r) ? mode : 0);
    }
    e = cudaMemcpyAsync(h->d_runs, h->runs.data(), sizeof(RunDesc) * n, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) break;
    result = run_impl(h, stream, probe_iters, false);
    for (int r = 0; r < n; ++r) {
      const RunState& A = before[r];
      const RunState& B = h->h_states[r];
      const long long it = B.n_iter - A.n_iter;
      if (it > 0) per_iter[mode][r] = (double)(B.cycles[kPhSlice] - A.cycles[kPhSlice]) / (double)it;
    }
    if (e == cudaSuccess) e = copy_all(false);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  }
  cudaFree(snap);
  h->runs = keep;
  if (e != cudaSuccess || result != NS_OK) {
    cudaMemcpy(h->d_runs, h->runs.data(), sizeof(RunDesc) * n, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      set_err(&h->err, "ns_autotune: %s", cudaGetErrorString(e));
      return NS_ERR_CUDA;
    }
    return result;
  }
  // a run leaves its default only for a configuration at least 5 % faster
  // in the slice phase
  for (int r = 0; r < n; ++r) {
    int best = 0;
    const double base = per_iter[0][r];
    for (int k = 1; k < n_cfg(r); ++k)
      if (base > 0 && per_iter[k][r] > 0 && per_iter[k][r] < 0.95 * base &&
          (best == 0 || per_iter[k][r] < per_iter[best][r]))
        best = k;
    const bool measured = base > 0 && n_cfg(r) > 1;
    if (measured) apply(h->runs[r], r, best);
    if (out_choice)
      out_choice[r] = keep[r].mlp_desc == nullptr ? h->runs[r].walker_warp : h->runs[r].mlp_round_cap;
    if (out_ratio) out_ratio[r] = measured && per_iter[1][r] > 0 ? per_iter[1][r] / base : std::nan("");
  }
  NS_CUDA(cudaMemcpyAsync(h->d_runs, h->runs.data(), sizeof(RunDesc) * n, cudaMemcpyHostToDevice, s), &h->err);
  NS_CUDA(cudaMemcpyAsync(h->h_states, h->d_states, sizeof(RunState) * n, cudaMemcpyDeviceToHost, s), &h->err);
  NS_CUDA(cudaStreamSynchronize(s), &h->err);
  return NS_OK;
}

size_t ns_checkpoint_bytes(const ns_handle* h) { return h ? sizeof(CheckpointHeader) + h->total : 0; }

ns_status ns_checkpoint(ns_handle* h, void* host_buf, size_t bytes, void* stream) {
  if (!h || !host_buf || bytes < ns_checkpoint_bytes(h)) return NS_ERR_ARG;
  CheckpointHeader hd;
  std::memset(&hd, 0, sizeof(hd));
  std::memcpy(hd.magic, kCkptMagic, 8);
  hd.fingerprint = h->fingerprint;
  hd.total = h->total;
  hd.off_desc = h->off_desc;
  hd.desc_bytes = h->desc_bytes;
  hd.off_state = h->off_state;
  hd.n_runs = h->n_runs;
  std::memcpy(host_buf, &hd, sizeof(hd));
  char* dst = static_cast<char*>(host_buf) + sizeof(hd);
  cudaStream_t s = (cudaStream_t)stream;
  NS_CUDA(cudaMemcpyAsync(dst, h->base, h->total, cudaMemcpyDeviceToHost, s), &h->err);
  NS_CUDA(cudaStreamSynchronize(s), &h->err);
  return NS_OK;
}

ns_status ns_restore(ns_handle* h, const void* host_buf, size_t bytes, void* stream) {
  if (!h || !host_buf || bytes < sizeof(CheckpointHeader)) return NS_ERR_ARG;
  CheckpointHeader hd;
  std::memcpy(&hd, host_buf, sizeof(hd));
  if (std::memcmp(hd.magic, kCkptMagic, 8) != 0 || hd.fingerprint != h->fingerprint || hd.total != h->total ||
      hd.off_desc != h->off_desc || hd.desc_bytes != h->desc_bytes || hd.n_runs != h->n_runs ||
      bytes < sizeof(hd) + hd.total) {
    set_err(&h->err, "ns_restore: the checkpoint was not taken from a batch of this shape");
    return NS_ERR_ARG;
  }
  const char* src = static_cast<const char*>(host_buf) + sizeof(hd);
  cudaStream_t s = (cudaStream_t)stream;
  // everything but the run descriptors, which hold this handle's own pointers
  NS_CUDA(cudaMemcpyAsync(h->base, src, h->off_desc, cudaMemcpyHostToDevice, s), &h->err);
  const size_t tail = h->off_desc + h->desc_bytes;
  NS_CUDA(cudaMemcpyAsync(h->base + tail, src + tail, h->total - tail, cudaMemcpyHostToDevice, s), &h->err);
  NS_CUDA(cudaStreamSynchronize(s), &h->err);
  std::memcpy(h->h_states, src + h->off_state, sizeof(RunState) * h->n_runs);
  for (auto& hr : h->host) hr.fetched = false;
  h->ran = true;
  return NS_OK;
}

ns_status ns_get_stats(const ns_handle* h, ns_stats* out) {
  if (!h || !out) return NS_ERR_ARG;
  out->run_ms = h->last_ms;
  out->kernel_ms = h->kernel_ms;
  out->launches = h->launches;
  out->h2d_bytes = h->h2d_bytes;
  out->d2h_bytes = h->d2h_bytes;
  return NS_OK;
}

ns_status ns_last_run_ms(const ns_handle* h, double* ms) {
  if (!h || !ms) return NS_ERR_ARG;
  if (!h->ran) return NS_ERR_STATE;
  *ms = h->last_ms;
  return NS_OK;
}

ns_status ns_result(ns_handle* h, int run, ns_result_t* out) {
  if (!h || !out || run < 0 || run >= h->n_runs) return NS_ERR_ARG;
  if (!h->ran) {
    set_err(&h->err, "ns_result before ns_run");
    return NS_ERR_STATE;
  }
  const RunState& S = h->h_states[run];
  HostRun& hr = h->host[run];
  const RunDesc& R = h->runs[run];
  if (!hr.fetched) {
    const long long n = S.n_dead;
    hr.dead_x.resize((size_t)std::max(1LL, n) * hr.d);
    hr.dead_l.resize((size_t)std::max(1LL, n));
    hr.dead_logw.resize((size_t)std::max(1LL, n));
    if (n > 0) {
      NS_CUDA(cudaMemcpy(hr.dead_x.data(), R.dead_x, sizeof(float) * (size_t)n * hr.d, cudaMemcpyDeviceToHost),
              &h->err);
      NS_CUDA(cudaMemcpy(hr.dead_l.data(), R.dead_l, sizeof(float) * (size_t)n, cudaMemcpyDeviceToHost), &h->err);
      NS_CUDA(cudaMemcpy(hr.dead_logw.data(), R.dead_logw, sizeof(double) * (size_t)n, cudaMemcpyDeviceToHost),
              &h->err);
      h->d2h_bytes += (long long)n * (long long)(sizeof(float) * hr.d + sizeof(float) + sizeof(double));
    }
    hr.fetched = true;
  }
  out->log_z = S.logz;
  out->log_z_err = std::sqrt(S.info > 0 ? S.info / hr.N : 0.0);
  out->info_h = S.info;
  out->n_dead = S.n_dead;
  out->n_evals = S.n_evals;
  out->n_iter = S.n_iter;
  out->n_relaxed = S.n_relaxed;
  out->n_reeval = S.n_reeval;
  out->n_capped = S.n_capped;
  out->n_rounds = S.mlp_count[0];
  out->n_pass_bf16 = S.mlp_count[1];
  out->n_cand_bf16 = S.mlp_count[2];
  out->n_pass_fp32 = S.mlp_count[3];
  out->n_cand_fp32 = S.mlp_count[4];
  out->n_pass_x2 = S.mlp_count[5];
  out->n_cand_x2 = S.mlp_count[6];
  out->status = S.status;
  out->d = hr.d;
  out->dead_x = hr.dead_x.data();
  out->dead_logl = hr.dead_l.data();
  out->dead_logw = hr.dead_logw.data();
  return NS_OK;
}

ns_status ns_summary(const ns_handle* h, int run, ns_result_t* out) {
  if (!h || !out || run < 0 || run >= h->n_runs) return NS_ERR_ARG;
  if (!h->ran) return NS_ERR_STATE;
  const RunState& S = h->h_states[run];
  const HostRun& hr = h->host[run];
  std::memset(out, 0, sizeof(*out));
  out->log_z = S.logz;
  out->log_z_err = std::sqrt(S.info > 0 ? S.info / hr.N : 0.0);
  out->info_h = S.info;
  out->n_dead = S.n_dead;
  out->n_evals = S.n_evals;
  out->n_iter = S.n_iter;
  out->n_relaxed = S.n_relaxed;
  out->n_reeval = S.n_reeval;
  out->n_capped = S.n_capped;
  out->n_rounds = S.mlp_count[0];
  out->n_pass_bf16 = S.mlp_count[1];
  out->n_cand_bf16 = S.mlp_count[2];
  out->n_pass_fp32 = S.mlp_count[3];
  out->n_cand_fp32 = S.mlp_count[4];
  out->n_pass_x2 = S.mlp_count[5];
  out->n_cand_x2 = S.mlp_count[6];
  out->status = S.status;
  out->d = hr.d;
  return NS_OK;
}

ns_status ns_phase_cycles(const ns_handle* h, int run, long long* out) {
  if (!h || !out || run < 0 || run >= h->n_runs) return NS_ERR_ARG;
  if (!h->ran) return NS_ERR_STATE;
  for (int i = 0; i < 8; ++i) out[i] = h->h_states[run].cycles[i];
  return NS_OK;
}

extern "C++" {
namespace {
// (device address, bytes) of one of run r's buffers (ns_buffer), or {null, 0}.
std::pair<const void*, size_t> run_buffer(const ns_handle* h, int r, int which) {
  const RunDesc& R = h->runs[r];
  const size_t d = R.d, N = R.N, m = R.m, nn = R.n_nodes, T = R.t_max;
  switch (which) {
    case NS_BUF_LIVE_X: return {R.live_x, sizeof(float) * d * R.n_pad};
    case NS_BUF_LIVE_L: return {R.live_l, sizeof(float) * N};
    case NS_BUF_LIVE_CID: return {R.live_cid, sizeof(int) * N};
    case NS_BUF_NEW_X: return {R.new_x, sizeof(float) * m * d};
    case NS_BUF_NEW_L: return {R.new_l, sizeof(float) * m};
    case NS_BUF_HIST_L: return {R.hist_l, sizeof(float) * m * T};
    case NS_BUF_HIST_X: return {R.hist_x, sizeof(float) * m * T * d};
    case NS_BUF_HIST_LEN: return {R.hist_len, sizeof(int) * m};
    case NS_BUF_WALKER_EVALS: return {R.wk_evals, sizeof(int) * m};
    case NS_BUF_WALKER_FLAGS: return {R.wk_flags, sizeof(int) * m};
    case NS_BUF_CHOL: return {R.chol, sizeof(float) * nn * d * d};
    case NS_BUF_CENTRES: return {R.centres, sizeof(float) * nn * d};
    case NS_BUF_MASK: return {R.mask, sizeof(int) * nn};
    default: return {nullptr, 0};
  }
}
}  // namespace
}  // extern "C++"

size_t ns_run_buffer_bytes(const ns_handle* h, int run, int which) {
  if (!h || run < 0 || run >= h->n_runs) return 0;
  return run_buffer(h, run, which).second;
}

ns_status ns_copy_run_buffer(ns_handle* h, int run, int which, void* host, size_t bytes, void* stream) {
  if (!h || !host || run < 0 || run >= h->n_runs) return NS_ERR_ARG;
  const auto b = run_buffer(h, run, which);
  if (!b.first || b.second != bytes) {
    set_err(&h->err, "ns_copy_run_buffer: buffer %d of run %d has %zu bytes, %zu requested", which, run, b.second,
            bytes);
    return NS_ERR_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  NS_CUDA(cudaMemcpyAsync(host, b.first, bytes, cudaMemcpyDeviceToHost, s), &h->err);
  NS_CUDA(cudaStreamSynchronize(s), &h->err);
  h->d2h_bytes += (long long)bytes;
  return NS_OK;
}

const char* ns_last_error(const ns_handle* h) {
  if (h) return h->err.c_str();
  std::lock_guard<std::mutex> lk(g_err_mu);
  static thread_local std::string copy;
  copy = g_err;
  return copy.c_str();
}

void ns_destroy(ns_handle* h) {
  if (!h) return;
  for (cudaStream_t gs : h->gstreams) cudaStreamDestroy(gs);
  for (cudaEvent_t ge : h->gjoin) cudaEventDestroy(ge);
  if (h->gfork) cudaEventDestroy(h->gfork);
  if (h->h_states) cudaFreeHost(h->h_states);
  if (h->arena) cudaFree(h->arena);
  delete h;
}

// ---- a whole run in a static device array (no allocation) -------------------
}  // extern "C"

namespace {

// One fixed array per GPU that loads the library; its host-side name is a
// stand-in, so the device address is looked up once per device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[NS_NOALLOC_SCRATCH_BYTES];
std::mutex g_noalloc_mu;
void* g_noalloc_addr[256] = {};

}  // namespace

extern "C" {

ns_status ns_run_noalloc(const ns_problem* problem, const ns_options* opt_in, float* dead_x, float* dead_logl,
                         double* dead_logw, long long dead_cap, ns_result_t* out, void* stream) {
  if (!problem || !out || !dead_x || !dead_logl || !dead_logw) {
    set_err(nullptr, "ns_run_noalloc: NULL argument");
    return NS_ERR_ARG;
  }
  ns_options opt;
  if (opt_in) opt = *opt_in;
  else ns_default_options(&opt);
  ns_status st = check_opts(opt, nullptr);
  if (st != NS_OK) return st;
  st = check_problem(*problem, nullptr);
  if (st != NS_OK) return st;
  if (problem->lik->kind == NS_LIK_MLP) {
    set_err(nullptr, "ns_run_noalloc: the MLP likelihood needs its weight image; use ns_create");
    return NS_ERR_UNSUPPORTED;
  }
  const ns_problem& p = *problem;
  const int d = p.d, N = p.n_live, m = p.m, n_pad = ((N + 31) / 32) * 32;
  if (dead_cap < (long long)N + m) {
    set_err(nullptr, "ns_run_noalloc: dead_cap = %lld is below N + m = %d", dead_cap, N + m);
    return NS_ERR_ARG;
  }
  const int n_nodes = (1 << (opt.depth + 1)) - 1;
  // layout of the static array for this run
  size_t total = 0;
  auto take = [&](size_t bytes) {
    size_t o = total;
    total += (bytes + 255) & ~(size_t)255;
    return o;
  };
  const size_t o_lik = take(sizeof(LikParams)), o_desc = take(sizeof(RunDesc)), o_state = take(sizeof(RunState)),
               o_ids = take(sizeof(int)), o_live_x = take(sizeof(float) * (size_t)d * n_pad),
               o_live_l = take(sizeof(float) * N), o_live_cid = take(sizeof(int) * N),
               o_new_x = take(sizeof(float) * (size_t)m * d), o_new_l = take(sizeof(float) * m),
               o_hist_l = take(sizeof(float) * (size_t)m * opt.t_max),
               o_hist_x = take(sizeof(float) * (size_t)m * opt.t_max * d), o_hist_len = take(sizeof(int) * m),
               o_stage_x = take(sizeof(float) * (size_t)m * d),
               o_dirs = take(sizeof(float) * (size_t)m * p.n_slice_steps * dir_row(dmax_class(d))),
               o_wsp = take(opt.depth > 0 ? sizeof(float) * (size_t)d * n_pad : 16),
               o_side = take(opt.depth > 0 ? sizeof(int) * (size_t)N : 16),
               o_centres = take(sizeof(float) * n_nodes * d),
               o_chol = take(sizeof(float) * n_nodes * d * d), o_chol64 = take(sizeof(double) * n_nodes * d * d),
               o_logvol = take(sizeof(float) * n_nodes), o_count = take(sizeof(int) * n_nodes),
               o_split = take(sizeof(int) * n_nodes), o_mask = take(sizeof(int) * n_nodes);
  const bool spill = run_spills(p, n_nodes);
  const size_t o_tree = take(spill ? tree_ws_bytes(d, n_nodes) : 16);
  if (total > (size_t)NS_NOALLOC_SCRATCH_BYTES) {
    set_err(nullptr, "ns_run_noalloc: this run needs %zu bytes of working memory; the static array holds %u",
            total, (unsigned)NS_NOALLOC_SCRATCH_BYTES);
    return NS_ERR_ARG;
  }
  int dev = 0;
  NS_CUDA(cudaGetDevice(&dev), nullptr);
  if (dev < 0 || dev >= 256) {
    set_err(nullptr, "ns_run_noalloc: device ordinal %d out of range", dev);
    return NS_ERR_ARG;
  }
  char* base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
      void* ptr = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
      if (e != cudaSuccess || !ptr) {
        set_err(nullptr, "ns_run_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
        return NS_ERR_CUDA;
      }
      g_noalloc_addr[dev] = ptr;
    }
    base = static_cast<char*>(g_noalloc_addr[dev]);
  }
  RunDesc R;
  std::memset(&R, 0, sizeof(R));
  R.d = d;
  R.N = N;
  R.m = m;
  R.n_pad = n_pad;
  R.n_steps = p.n_slice_steps;
  R.depth = opt.depth;
  R.n_nodes = n_nodes;
  R.recluster_every = opt.recluster_every > 0 ? opt.recluster_every : std::max(1, 100 / m);
  R.n_min = opt.n_min > 0 ? opt.n_min : d + 1;
  R.kmeans_iters = opt.kmeans_iters;
  R.correction = opt.correction;
  R.K = opt.history_iters;
  R.t_max = opt.t_max;
  R.e_max = opt.e_max;
  R.s_max = opt.s_max;
  R.k0 = (uint32_t)(p.seed & 0xFFFFFFFFull);
  R.k1 = (uint32_t)(p.seed >> 32);
  R.width = (float)opt.width;
  R.vol_frac = (float)opt.vol_frac;
  R.log_stop = std::log(p.stop_frac);
  R.max_iter = opt.max_iter;
  R.dead_cap = dead_cap;
  R.lik = reinterpret_cast<const LikParams*>(base + o_lik);
  R.live_x = reinterpret_cast<float*>(base + o_live_x);
  R.live_l = reinterpret_cast<float*>(base + o_live_l);
  R.live_cid = reinterpret_cast<int*>(base + o_live_cid);
  R.new_x = reinterpret_cast<float*>(base + o_new_x);
  R.new_l = reinterpret_cast<float*>(base + o_new_l);
  R.hist_l = reinterpret_cast<float*>(base + o_hist_l);
  R.hist_x = reinterpret_cast<float*>(base + o_hist_x);
  R.hist_len = reinterpret_cast<int*>(base + o_hist_len);
  R.stage_x = reinterpret_cast<float*>(base + o_stage_x);
  R.dirs = reinterpret_cast<float*>(base + o_dirs);
  R.wsp = reinterpret_cast<float*>(base + o_wsp);
  R.side = reinterpret_cast<int*>(base + o_side);
  R.dead_x = dead_x;
  R.dead_l = dead_logl;
  R.dead_logw = dead_logw;
  R.centres = reinterpret_cast<float*>(base + o_centres);
  R.chol = reinterpret_cast<float*>(base + o_chol);
  R.chol64 = reinterpret_cast<double*>(base + o_chol64);
  R.logvol = reinterpret_cast<float*>(base + o_logvol);
  R.count = reinterpret_cast<int*>(base + o_count);
  R.split = reinterpret_cast<int*>(base + o_split);
  R.mask = reinterpret_cast<int*>(base + o_mask);
  R.walker_warp = opt.walker_mapping;
  R.bracket = opt.bracket;
  R.spill = spill ? 1 : 0;
  R.tree_ws = spill ? base + o_tree : nullptr;
  R.st = reinterpret_cast<RunState*>(base + o_state);
  const LikParams P = make_lik(*p.lik, p.lo, p.hi, d);
  const int id0 = 0;
  cudaStream_t s = (cudaStream_t)stream;
  // the array keeps the previous call's contents: upload this run's
  // descriptor and start its state from zero
  NS_CUDA(cudaMemcpyAsync(base + o_lik, &P, sizeof(P), cudaMemcpyHostToDevice, s), nullptr);
  NS_CUDA(cudaMemcpyAsync(base + o_desc, &R, sizeof(R), cudaMemcpyHostToDevice, s), nullptr);
  NS_CUDA(cudaMemcpyAsync(base + o_ids, &id0, sizeof(int), cudaMemcpyHostToDevice, s), nullptr);
  NS_CUDA(cudaMemsetAsync(base + o_state, 0, sizeof(RunState), s), nullptr);
  const RunDesc* d_desc = reinterpret_cast<const RunDesc*>(base + o_desc);
  const int* d_ids = reinterpret_cast<const int*>(base + o_ids);
  const int block = block_for_m(m);
  const size_t smem = make_carve(d, m, n_nodes, dmax_class(d), false, spill).total;
  const int chunk = opt.chunk_iters > 0 ? opt.chunk_iters : 1000;
  const long long max_rounds = opt.max_iter / chunk + 2;
  RunState hs;
  std::memset(&hs, 0, sizeof(hs));
  for (long long round = 0;; ++round) {
    const cudaError_t e = kClasses[class_index(d)].run(d_desc, d_ids, 1, block, smem, chunk, s);
    NS_CUDA(e, nullptr);
    NS_CUDA(cudaMemcpyAsync(&hs, base + o_state, sizeof(RunState), cudaMemcpyDeviceToHost, s), nullptr);
    NS_CUDA(cudaStreamSynchronize(s), nullptr);
    if (hs.stopped || hs.status != 0 || round + 1 > max_rounds) break;
  }
  std::memset(out, 0, sizeof(*out));
  out->log_z = hs.logz;
  out->log_z_err = std::sqrt(hs.info > 0 ? hs.info / N : 0.0);
  out->info_h = hs.info;
  out->n_dead = hs.n_dead;
  out->n_evals = hs.n_evals;
  out->n_iter = hs.n_iter;
  out->n_relaxed = hs.n_relaxed;
  out->n_reeval = hs.n_reeval;
  out->n_capped = hs.n_capped;
  out->status = hs.status;
  out->d = d;
  if (hs.status != 0) {
    set_err(nullptr, "ns_run_noalloc: the run ended with status %d", hs.status);
    return (ns_status)hs.status;
  }
  return NS_OK;
}

// ---- step-level entry points ----------------------------------------------
ns_status ns_philox4x32_10(const uint32_t* ctr, uint32_t key0, uint32_t key1, int n, uint32_t* out, void* stream) {
  if (n < 0 || (n > 0 && (!ctr || !out))) {
    set_err(nullptr, "ns_philox4x32_10: bad arguments");
    return NS_ERR_ARG;
  }
  if (n == 0) return NS_OK;
  k_philox<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(ctr, key0, key1, n, out);
  NS_CUDA(cudaGetLastError(), nullptr);
  return NS_OK;
}

ns_status ns_loglike(const ns_likelihood* lik, const double* lo, const double* hi, int d, int n, const float* x,
                     float* logl, void* stream) {
  ns_problem p;
  std::memset(&p, 0, sizeof(p));
  p.lik = lik;
  p.lo = lo;
  p.hi = hi;
  p.d = d;
  p.n_live = 2;
  p.m = 1;
  p.n_slice_steps = 1;
  p.stop_frac = 0.5;
  ns_status st = check_problem(p, nullptr);
  if (st != NS_OK) return st;
  if (lik->kind == NS_LIK_MLP) {
    set_err(nullptr, "ns_loglike: use ns_mlp_loglike for the MLP likelihood");
    return NS_ERR_ARG;
  }
  if (n < 0 || (n > 0 && (!x || !logl))) {
    set_err(nullptr, "ns_loglike: bad arguments");
    return NS_ERR_ARG;
  }
  if (n == 0) return NS_OK;
  const LikParams P = make_lik(*lik, lo, hi, d);
  cudaStream_t s = (cudaStream_t)stream;
  const cudaError_t e = kClasses[class_index(d)].ll(P, n, x, logl, s);
  NS_CUDA(e, nullptr);
  return NS_OK;
}

ns_status ns_select_worst(int n_runs, int N, int m, const float* logl, const uint64_t* seeds, uint32_t t,
                          int* worst, float* W, int* seed_slot, void* stream) {
  if (n_runs < 0 || N < 2 || N > NS_MAX_LIVE || m < 1 || 2 * m > N || m > NS_MAX_BATCH ||
      (n_runs > 0 && (!logl || !seeds || !worst || !W || !seed_slot))) {
    set_err(nullptr, "ns_select_worst: bad arguments (need 1 <= m <= N/2, m <= %d)", NS_MAX_BATCH);
    return NS_ERR_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const size_t smem = al16(sizeof(int) * m) + al16(sizeof(uint32_t) * m);
  for (int r0 = 0; r0 < n_runs; r0 += 128) {
    const int nr = std::min(128, n_runs - r0);
    SelectArgs K;
    for (int r = 0; r < nr; ++r) {
      K.keys[2 * r] = (uint32_t)(seeds[r0 + r] & 0xFFFFFFFFull);
      K.keys[2 * r + 1] = (uint32_t)(seeds[r0 + r] >> 32);
    }
    k_select<<<nr, 256, smem, s>>>(N, m, logl + (size_t)r0 * N, K, t, worst + (size_t)r0 * m, W + (size_t)r0 * m,
                                  seed_slot + (size_t)r0 * m);
    NS_CUDA(cudaGetLastError(), nullptr);
  }
  return NS_OK;
}

ns_status ns_slice_replace(const ns_likelihood* lik, const double* lo, const double* hi, int d, int N, int n_pad,
                           int m, int n_steps, const ns_options* opt_in, uint64_t seed, uint32_t t,
                           const float* live_x, const float* live_l, const int* seed_slot, const float* W,
                           const float* chol, const int* cid, float* new_x, float* new_l, float* hist_l,
                           float* hist_x, int* hist_len, long long* evals, int* flags, float* dir_scratch,
                           void* stream) {
  ns_options opt;
  if (opt_in) opt = *opt_in;
  else ns_default_options(&opt);
  ns_status st = check_opts(opt, nullptr);
  if (st != NS_OK) return st;
  ns_problem p;
  p.lik = lik;
  p.lo = lo;
  p.hi = hi;
  p.d = d;
  p.n_live = N;
  p.m = m;
  p.n_slice_steps = n_steps;
  p.stop_frac = 0.5;
  p.seed = seed;
  st = check_problem(p, nullptr);
  if (st != NS_OK) return st;
  if (lik->kind == NS_LIK_MLP) {
    set_err(nullptr, "ns_slice_replace: the MLP likelihood is sampled by whole runs only");
    return NS_ERR_ARG;
  }
  if (n_pad < N || !live_x || !live_l || !seed_slot || !W || !chol || !cid || !new_x || !new_l || !hist_l ||
      !hist_x || !hist_len || !evals || !flags || !dir_scratch) {
    set_err(nullptr, "ns_slice_replace: NULL buffer or n_pad < N");
    return NS_ERR_ARG;
  }
  const LikParams P = make_lik(*lik, lo, hi, d);
  SliceCfg SC;
  SC.d = d;
  SC.n_steps = n_steps;
  SC.e_max = opt.e_max;
  SC.s_max = opt.s_max;
  SC.t_max = opt.t_max;
  SC.width = (float)opt.width;
  SC.k0 = (uint32_t)(seed & 0xFFFFFFFFull);
  SC.k1 = (uint32_t)(seed >> 32);
  SC.t = t;
  cudaStream_t s = (cudaStream_t)stream;
  const cudaError_t e = kClasses[class_index(d)].sl(P, SC, m, n_pad, opt.correction, live_x, live_l, seed_slot, W,
                                                     chol, cid, new_x, new_l, hist_l, hist_x, hist_len, evals, flags,
                                                     dir_scratch, opt.walker_mapping, s);
  NS_CUDA(e, nullptr);
  return NS_OK;
}

size_t ns_slice_scratch_bytes(int d, int m, int n_steps) {
  if (d < 1 || d > NS_MAX_DIM || m < 1 || n_steps < 1) return 0;
  return sizeof(float) * (size_t)m * n_steps * dir_row(dmax_class(d));
}

ns_status ns_batch_correct(int m, int K, int correction, const float* W, const float* new_l, const float* hist_l,
                           const int* hist_len, int t_max, int* acc_src, int* acc_hpos, float* acc_l, float* acc_P,
                           int* rej_src, int* rej_hpos, float* rej_l, float* rej_P, int* n_relaxed, void* stream) {
  if (m < 1 || m > NS_MAX_BATCH || K < 0 || correction < 0 || correction > 3 || t_max < 1 ||
      t_max > NS_MAX_HISTORY || !W || !new_l || !hist_l || !hist_len || !acc_src || !acc_hpos || !acc_l ||
      !acc_P || !rej_src || !rej_hpos || !rej_l || !rej_P || !n_relaxed) {
    set_err(nullptr, "ns_batch_correct: bad arguments");
    return NS_ERR_ARG;
  }
  const size_t cb = al16((sizeof(float) * 2 + sizeof(int) * 3) * 2 * m + 64);
  const size_t smem = 3 * cb + al16(sizeof(int) * 2 * m) + al16(sizeof(float) * m);
  k_correct<<<1, 256, smem, (cudaStream_t)stream>>>(m, K, correction, W, new_l, hist_l, hist_len, t_max, acc_src,
                                                    acc_hpos, acc_l, acc_P, rej_src, rej_hpos, rej_l, rej_P,
                                                    n_relaxed);
  NS_CUDA(cudaGetLastError(), nullptr);
  return NS_OK;
}

ns_status ns_evidence_update(int N, int n, const float* dead_l, double* state, double* logw, int live,
                             void* stream) {
  if (N < 1 || n < 0 || (n > 0 && (!dead_l || !logw)) || !state) {
    set_err(nullptr, "ns_evidence_update: bad arguments");
    return NS_ERR_ARG;
  }
  if (n == 0) return NS_OK;
  k_evidence<<<1, 256, 0, (cudaStream_t)stream>>>(N, n, dead_l, state, logw, live);
  NS_CUDA(cudaGetLastError(), nullptr);
  return NS_OK;
}

// The whitened points and child bits, then (16-byte aligned) the tree
// scratch of the deepest tree, used when a tree's tables do not fit in
// shared memory.
size_t cluster_points_bytes(int N, int n_pad, int d) {
  return al16(sizeof(float) * (size_t)d * n_pad + sizeof(int) * (size_t)N);
}

size_t ns_cluster_scratch_bytes(int N, int n_pad, int d) {
  if (N < 2 || n_pad < N || d < 1 || d > NS_MAX_DIM) return 0;
  return cluster_points_bytes(N, n_pad, d) + tree_ws_bytes(d, (1 << (NS_MAX_DEPTH + 1)) - 1);
}

ns_status ns_cluster(int N, int n_pad, int d, const float* live_x, const ns_options* opt_in, uint64_t seed,
                     uint32_t t, float* centres, float* chol, double* chol64, float* logvol, int* count, int* split,
                     int* mask, int* cid, void* scratch, void* stream) {
  ns_options opt;
  if (opt_in) opt = *opt_in;
  else ns_default_options(&opt);
  ns_status st = check_opts(opt, nullptr);
  if (st != NS_OK) return st;
  if (N < 2 || n_pad < N || d < 1 || d > NS_MAX_DIM || !live_x || !centres || !chol || !chol64 || !logvol ||
      !count || !split || !mask || !cid || (opt.depth > 0 && !scratch)) {
    set_err(nullptr, "ns_cluster: bad arguments");
    return NS_ERR_ARG;
  }
  RunDesc R;
  std::memset(&R, 0, sizeof(R));
  R.d = d;
  R.N = N;
  R.m = 1;
  R.n_pad = n_pad;
  R.depth = opt.depth;
  R.n_nodes = (1 << (opt.depth + 1)) - 1;
  R.n_min = opt.n_min > 0 ? opt.n_min : d + 1;
  R.kmeans_iters = opt.kmeans_iters;
  R.vol_frac = (float)opt.vol_frac;
  R.bracket = opt.bracket;
  R.k0 = (uint32_t)(seed & 0xFFFFFFFFull);
  R.k1 = (uint32_t)(seed >> 32);
  R.live_x = const_cast<float*>(live_x);
  R.live_cid = cid;
  R.centres = centres;
  R.chol = chol;
  R.chol64 = chol64;
  R.logvol = logvol;
  R.count = count;
  R.split = split;
  R.mask = mask;
  if (opt.depth > 0) {
    R.wsp = static_cast<float*>(scratch);
    R.side = reinterpret_cast<int*>(static_cast<char*>(scratch) + sizeof(float) * (size_t)d * n_pad);
  }
  if (opt.depth > 0 && make_carve(d, 1, R.n_nodes, kMaxDim).total > 227 * 1024) {
    R.spill = 1;
    R.tree_ws = static_cast<char*>(scratch) + cluster_points_bytes(N, n_pad, d);
  }
  const size_t smem = make_carve(d, 1, R.n_nodes, kMaxDim, false, R.spill != 0).total;
  if (smem > 227 * 1024) {
    set_err(nullptr, "ns_cluster: %zu bytes of shared memory needed (limit 227 KB)", smem);
    return NS_ERR_ARG;
  }
  NS_CUDA(cudaFuncSetAttribute(k_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem), nullptr);
  k_cluster<<<1, 256, smem, (cudaStream_t)stream>>>(R, t);
  NS_CUDA(cudaGetLastError(), nullptr);
  return NS_OK;
}

}  // extern "C"
