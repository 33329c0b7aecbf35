// ns_run.cuh -- per-run descriptor, shared-memory layout and the
// persistent run kernel of the batched nested sampler (one thread block per
// run; walkers are the block's threads).  Included by the per-dimension
// instantiation units and by the host library.
#pragma once

#include <cstddef>

#include "../../include/ns_gb300.h"
#include "ns_cluster.cuh"
#include "ns_device.cuh"
#include "ns_mlp.cuh"
#include "ns_mlp_cluster.cuh"

namespace nsd {

// ---------------------------------------------------------------------------
// Per-run device state and descriptor
// ---------------------------------------------------------------------------
// Phases timed by the run kernel (SM cycles, thread 0, between barriers).
enum Phase { kPhCluster = 0, kPhSelect, kPhSlice, kPhCorrect, kPhUpdate, kPhEvidence, kNumPhases };

struct RunState {
  double logz, info;
  long long k, n_dead, n_evals, n_iter, n_relaxed, n_reeval, n_capped;
  long long cycles[8];
  // MLP runs: walker rounds, BF16 passes and their candidates, FP32 passes and
  // theirs, 16-bit (two-plane) passes and theirs
  long long mlp_count[7];
  int t, stopped, status, initialized;
};

struct RunDesc {
  int d, N, m, n_pad, n_steps, depth, n_nodes, recluster_every, n_min, kmeans_iters, correction, K,
      t_max, e_max, s_max;
  uint32_t k0, k1;
  float width, vol_frac;
  double log_stop;
  long long max_iter, dead_cap;
  const LikParams* lik;
  float* live_x;
  float* live_l;
  int* live_cid;
  float* new_x;
  float* new_l;
  float* hist_l;
  float* hist_x;
  int* hist_len;
  int* wk_evals;   // [m] likelihood evaluations of each walker in the last iteration (may be null)
  int* wk_flags;   // [m] its cap flags (bit 0 step-out, bit 1 shrink)
  float* stage_x;
  float* dirs;     // [m][n_steps][dir_row(DMAX of the run's class)] per-step directions and draws
  float* wsp;      // [d][n_pad] whitened live points (cluster tree, depth >= 1)
  int* side;       // [N] child choices of each live point (cluster tree)
  float* dead_x;
  float* dead_l;
  double* dead_logw;
  float* centres;
  float* chol;
  double* chol64;
  float* logvol;
  int* count;
  int* split;
  int* mask;
  RunState* st;
  // MLP likelihood (kind 4): the packed weight image and its description
  const uint8_t* mlp_tiles;
  const float* mlp_f32;
  const MlpDesc* mlp_desc;
  int precision;          // 0 FP32 CUDA cores, 1 BF16 tensor cores + FP32 re-evaluation
  int spill;              // cluster tables in global memory (make_carve)
  char* tree_ws;          // the cluster-tree scratch of a spilled run
  float reeval_margin;    // re-evaluate in FP32 when |logL_bf16 - threshold| <
  float reeval_rel;       //   reeval_margin + reeval_rel |threshold|
  int reeval_defer;       // rounds a near-threshold candidate may wait for a shared FP32 pass
  int two_plane;          // BF16 runs: a 16-bit (two-plane) pass between the BF16 and the FP32 values
  float reeval2_margin;   // FP32 after the 16-bit pass when |logL_16 - threshold| <
  float reeval2_rel;      //   reeval2_margin + reeval2_rel |threshold|
  int walker_warp;        // analytic runs: 1 = one walker per warp, 0 = one walker per thread
  int mlp_round_cap;      // BF16 MLP runs: candidates evaluated per round (0 = all, in equal calls)
  int bracket;            // 1: the direction factors scaled by their cluster's bounding radius
};

// Shared-memory carve of the run kernel, computed identically on host and
// device from the run's sizes.
struct Carve {
  size_t lik, scr, sel, chol, cent, mask, worst, W, seed, sel_slot, sel_key, candA, candB, candT, list, vals, slots,
      ctr, stage_cid, xbuf, lbuf, rlist, tile, acc, c64, l64, work, tree, mlp, total;
  bool chol_global;  // the cluster Cholesky factors live in global memory (MLP runs, spilled runs)
  bool tree_global;  // the cluster-tree scratch lives in global memory (spilled runs)
};

// The BF16 evaluator inside the run kernel: up to 128 candidates per call,
// three weight-tile stages.
constexpr int kRunMlpStages = 3;
using RunMlpSmem = MlpSmem<kMlpNbMax, kRunMlpStages>;

__host__ __device__ inline size_t al16(size_t x) { return (x + 15) & ~(size_t)15; }

// Row stride (floats) of an MLP run's candidate staging buffer.
__host__ __device__ constexpr int mlp_xs(int d) { return (d + 3) & ~3; }

// spill: the run's cluster tables do not fit next to the rest (large d or a
// deep tree); the Cholesky factors and the tree scratch then stay in global
// memory (only the clustering and the direction draws read them).
__host__ __device__ inline Carve make_carve(int d, int m, int n_nodes, int dmax, bool mlp = false,
                                            bool spill = false) {
  Carve c;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    size_t r = o;
    o = al16(o + bytes);
    return r;
  };
  const size_t cand_bytes = (sizeof(float) * 2 + sizeof(int) * 3) * 2 * m + 64;
  c.chol_global = mlp || spill;
  c.tree_global = spill;
  c.lik = take(mlp ? 0 : sizeof(LikParams));
  c.scr = take(sizeof(BlockScratch));
  c.sel = take(sizeof(SelectScratch));
  c.chol = take(c.chol_global ? 0 : sizeof(float) * n_nodes * d * d);
  c.cent = take(sizeof(float) * n_nodes * d);
  c.mask = take(sizeof(int) * n_nodes);
  c.worst = take(sizeof(int) * m);
  c.W = take(sizeof(float) * m);
  c.seed = take(sizeof(int) * m);
  c.sel_slot = take(sizeof(int) * m);
  c.sel_key = take(sizeof(uint32_t) * m);
  c.list = take(sizeof(int) * 2 * m);
  c.vals = take(sizeof(float) * m);
  c.ctr = take(sizeof(int) * 4);
  c.stage_cid = take(sizeof(int) * m);
  // MLP runs: candidate points (two slots per walker, then FP32 staging
  // rows), their log L, the re-evaluation list
  c.xbuf = take(mlp ? sizeof(float) * (size_t)(2 * m + kMlpF32Nb) * mlp_xs(d) : 0);
  c.lbuf = take(mlp ? sizeof(float) * (size_t)(2 * m + kMlpF32Nb) : 0);
  c.rlist = take(mlp ? sizeof(int) * (size_t)(2 * m + kMlpF32Nb) : 0);
  // from here on, scratch of one phase at a time: the clustering, the
  // walker phase (the analytic walkers' row slots; the MLP evaluators) and
  // the batch-correction candidates (Algorithms 1-2 and the update), which
  // never overlap
  const size_t phase0 = o;
  c.tile = take(sizeof(float) * (d * kTileS + d));
  c.acc = take(sizeof(double) * (d + d * d));
  c.c64 = take(sizeof(double) * d * d);
  c.l64 = take(sizeof(double) * d * d);
  c.work = take(sizeof(double) * (3 * d * d + d));
  // per-warp partials for every warp of the block (MLP blocks have kMlpThreads threads, others <= 256)
  c.tree = take(c.tree_global ? 0 : tree_bytes(d, n_nodes, mlp ? kMlpThreads / 32 : 8, tree_chol_warps(d, 8)));
  c.mlp = phase0;
  if (!mlp) {
    const size_t end_cluster = o;
    o = phase0;
    c.slots = take(sizeof(float) * (size_t)dir_row(dmax) * (m + 31) / 32 * 32);
    const size_t end_slots = o;
    o = phase0;
    c.candA = take(cand_bytes);
    c.candB = take(cand_bytes);
    c.candT = take(cand_bytes);
    if (end_cluster > o) o = end_cluster;
    if (end_slots > o) o = end_slots;
  } else {
    c.slots = phase0;
    const size_t end_cluster = o;
    o = phase0;
    c.candA = take(cand_bytes);
    c.candB = take(cand_bytes);
    c.candT = take(cand_bytes);
    const size_t end_cand = o;
    const size_t end_bf16 = phase0 + RunMlpSmem::kBytes + 1024;  // + alignment of the tensor-core region
    const size_t end_f32 = phase0 + mlp_f32_act_bytes(kMlpF32NbWide);
    o = end_cluster;
    if (end_cand > o) o = end_cand;
    if (end_bf16 > o) o = end_bf16;
    if (end_f32 > o) o = end_f32;
  }
  c.total = o;
  return c;
}

__device__ inline Cand cand_at(char* base, int m) {
  Cand c;
  c.l = reinterpret_cast<float*>(base);
  c.P = c.l + 2 * m;
  c.src = reinterpret_cast<int*>(c.P + 2 * m);
  c.H = c.src + 2 * m;
  c.hp = c.H + 2 * m;
  return c;
}

// ---------------------------------------------------------------------------
// Phases of one iteration on one run (whole block)
// ---------------------------------------------------------------------------
template <int DMAX>
inline __device__ void init_live(const RunDesc& R, const LikParams& P) {
  const int d = R.d;
  for (int j = threadIdx.x; j < R.N; j += blockDim.x) {
    float x[DMAX];
#pragma unroll
    for (int i = 0; i < DMAX; ++i) {
      x[i] = (i < d) ? u24(draw_at(R.k0, R.k1, kTInit, (uint32_t)j, 0u, (uint32_t)i)) : 0.f;
      if (i < d) R.live_x[(size_t)i * R.n_pad + j] = x[i];
    }
    R.live_l[j] = loglike_u<DMAX>(P, x);
    R.live_cid[j] = 0;
  }
}

// a3 (section 2.1): the root node is the whole live set (mean, covariance,
// regularised FP64 Cholesky); for depth >= 1 the tree of cluster_tree
// follows.
inline __device__ void cluster_phase(const RunDesc& R, uint32_t t, char* sm, const Carve& cv, BlockScratch& S) {
  const int d = R.d;
  float* tile = reinterpret_cast<float*>(sm + cv.tile);
  double* acc = reinterpret_cast<double*>(sm + cv.acc);
  double* C64 = reinterpret_cast<double*>(sm + cv.c64);
  double* L64 = reinterpret_cast<double*>(sm + cv.l64);
  double* work = reinterpret_cast<double*>(sm + cv.work);
  float* s_chol = cv.chol_global ? R.chol : reinterpret_cast<float*>(sm + cv.chol);
  float* s_cent = reinterpret_cast<float*>(sm + cv.cent);
  int* s_mask = reinterpret_cast<int*>(sm + cv.mask);
  const int n = node_moments(R.live_x, R.n_pad, R.N, d, [](int) { return true; }, tile, acc, S);
  for (int i = threadIdx.x; i < d * d; i += blockDim.x) C64[i] = acc[d + i];
  __syncthreads();
  reg_cholesky(d, C64, L64, work, S);
  for (int i = threadIdx.x; i < d * d; i += blockDim.x) {
    const float f = (float)L64[i];
    s_chol[i] = f;
    R.chol[i] = f;
    R.chol64[i] = L64[i];
  }
  for (int i = threadIdx.x; i < d; i += blockDim.x) {
    s_cent[i] = (float)acc[i];
    R.centres[i] = (float)acc[i];
  }
  if (R.n_nodes == 1 && R.bracket == 1) {
    // the bounding radius of the one cluster: the largest Mahalanobis
    // distance of a live point from the centre, in the root factor's units
    // (the tree computes it for every node); the direction factor is then
    // the Cholesky factor times that radius
    unsigned* m2u = reinterpret_cast<unsigned*>(&S.iw[0]);
    if (threadIdx.x == 0) *m2u = 0u;
    __syncthreads();
    const unsigned mx = max_mahalanobis2(R.live_x, R.n_pad, R.N, d, s_chol, s_cent);
    atomicMax(m2u, mx);
    __syncthreads();
    const float rad = sqrtf(__uint_as_float(*m2u));
    __syncthreads();
    if (rad > 0.f && isfinite(rad))
      for (int i = threadIdx.x; i < d * d; i += blockDim.x) {
        s_chol[i] *= rad;
        R.chol[i] = s_chol[i];
      }
  }
  if (R.n_nodes == 1) {
    if (threadIdx.x == 0) {
      s_mask[0] = 1;
      R.mask[0] = 1;
      R.split[0] = 0;
      R.count[0] = n;
      R.logvol[0] = 0.f;
    }
    for (int j = threadIdx.x; j < R.N; j += blockDim.x) R.live_cid[j] = 0;
    __syncthreads();
    return;
  }
  const int nw = blockDim.x >> 5;
  const int nw_chol = tree_chol_warps(d, 8) < nw ? tree_chol_warps(d, 8) : nw;
  const TreeScratch T = tree_carve(cv.tree_global ? R.tree_ws : sm + cv.tree, d, R.n_nodes, nw, tree_chol_warps(d, 8));
  if (threadIdx.x == 0) T.node_n[0] = n;
  __syncthreads();
  TreeIO io;
  io.x = R.live_x;
  io.y = R.wsp;
  io.side = R.side;
  io.N = R.N;
  io.n_pad = R.n_pad;
  io.d = d;
  io.depth = R.depth;
  io.n_min = R.n_min;
  io.kmeans_iters = R.kmeans_iters;
  io.vol_frac = R.vol_frac;
  io.k0 = R.k0;
  io.k1 = R.k1;
  io.t = t;
  io.centres = R.centres;
  io.chol = R.chol;
  io.chol64 = R.chol64;
  io.logvol = R.logvol;
  io.count = R.count;
  io.split = R.split;
  io.mask = R.mask;
  io.cid = R.live_cid;
  io.s_chol = s_chol;
  io.s_cent = s_cent;
  io.s_mask = s_mask;
  io.bracket = R.bracket;
  cluster_tree(io, T, S, nw_chol);
}

inline __device__ int nearest_leaf(const float* x, int d, int n_nodes, const float* cent, const int* mask) {
  int best = 0;
  float bd = CUDART_INF_F;
  for (int nd = 0; nd < n_nodes; ++nd) {
    if (!mask[nd]) continue;
    float s = 0.f;
    for (int i = 0; i < d; ++i) {
      const float u = x[i] - cent[nd * d + i];
      s = fmaf(u, u, s);
    }
    if (s < bd) {
      bd = s;
      best = nd;
    }
  }
  return best;
}

// a4-a7 for the calling thread's walker (threads of warps that hold a walker
// call it; lanes past m take part in the warp votes only).  Kept out of line
// so that its registers are allocated apart from the rest of the run kernel.
template <int DMAX>
__device__ __noinline__ void walker_phase(const RunDesc& R, const LikParams& P, const SliceCfg& SC,
                                          const float* s_W, const int* s_seed, const float* s_chol, float* s_slots,
                                          long long& ev, int& fl, long long& cyc_draw, long long& cyc_walk) {
  const int tid = threadIdx.x, m = R.m, d = R.d;
  const bool act = tid < m;
  const int i = act ? tid : 0;
  const int sd = s_seed[i];
  const float thr_out = (R.correction == 3) ? s_W[m - 1] : s_W[0];
  const float thr_in = (R.correction == 3) ? s_W[m - 1] : s_W[i];
  WalkerOut O;
  O.new_x = R.new_x + (size_t)i * d;
  O.new_l = R.new_l + i;
  O.hist_l = R.hist_l + (size_t)i * R.t_max;
  O.hist_x = R.hist_x + (size_t)i * R.t_max * d;
  O.hist_len = R.hist_len + i;
  float* my_dirs = R.dirs + (size_t)i * R.n_steps * dir_row(DMAX);
  const long long c1 = clock64();
  long long e = 0;
  int f = 0;
  slice_walker<DMAX>(P, SC, i, act, R.live_x + sd, R.n_pad, R.live_l[sd], my_dirs, s_slots + (size_t)tid * dir_row(DMAX),
                     thr_out, thr_in, O, e, f);
  ev = act ? e : 0;
  fl = act ? f : 0;
  cyc_draw = 0;  // the draws happen before, block-wide (k_run)
  cyc_walk = clock64() - c1;
}

// a4-a7 with one walker per warp (RunDesc::walker_warp): warp w takes the
// walkers w, w + n_warps, ... in turn.  On return lane 0 of each warp holds
// in ev its walkers' likelihood evaluations and in fl how many of them hit a
// step-out or shrink cap (other lanes 0).  Called by every thread.
template <int DMAX>
__device__ __noinline__ void walker_phase_warp(const RunDesc& R, const LikParams& P, const SliceCfg& SC,
                                               const float* s_W, const int* s_seed, long long& ev, int& fl) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5, m = R.m, d = R.d;
  LaneLik<DMAX> Q;
  lane_lik<DMAX>(P, Q);
  const float thr_out = (R.correction == 3) ? s_W[m - 1] : s_W[0];
  long long e_sum = 0;
  int n_cap = 0;
  for (int i = wid; i < m; i += nw) {
    const int sd = s_seed[i];
    const float thr_in = (R.correction == 3) ? s_W[m - 1] : s_W[i];
    WalkerOut O;
    O.new_x = R.new_x + (size_t)i * d;
    O.new_l = R.new_l + i;
    O.hist_l = R.hist_l + (size_t)i * R.t_max;
    O.hist_x = R.hist_x + (size_t)i * R.t_max * d;
    O.hist_len = R.hist_len + i;
    long long e = 0;
    int f = 0;
    slice_walker_warp<DMAX>(P, Q, SC, i, R.live_x + sd, R.n_pad, R.live_l[sd],
                            R.dirs + (size_t)i * R.n_steps * dir_row(DMAX), thr_out, thr_in, O, e, f);
    if (lane == 0 && R.wk_evals) {
      R.wk_evals[i] = (int)e;
      R.wk_flags[i] = f;
    }
    e_sum += e;
    n_cap += (f != 0) ? 1 : 0;
  }
  ev = (lane == 0) ? e_sum : 0;
  fl = (lane == 0) ? n_cap : 0;
}

// a4-a7 for MLP runs: the walkers advance in lock step, one round at a time;
// each round the block evaluates every walker's pending candidates as one
// batch (on the tensor cores in BF16, or on the CUDA cores in FP32).  In
// BF16 mode a candidate whose log L falls within reeval_margin +
// reeval_rel |threshold| of the threshold it is compared with is
// re-evaluated in FP32 before the decision; each walker's final point and
// its history samples are re-evaluated in FP32 afterwards, so every log L
// that is stored (dead points, Algorithm 2) is an FP32 value.
//
// Candidate rows of the block's staging buffer xbuf: walker w's left
// stepping-out end (or its shrink candidate) in row w, its right end in row
// m + w, FP32 staging rows after the 2m; rows are mlp_xs(d) floats apart.
static __device__ __noinline__ bool mlp_batch_f32(const RunDesc& R, const float* xs, int xstride, int n, float* ls, float* act,
                                     const int* rows = nullptr) {
  for (int b0 = 0; b0 < n; b0 += kMlpF32NbWide) {
    if (rows)
      mlp_eval_f32<kMlpF32NbWide>(*R.mlp_desc, R.mlp_f32, xs, xstride, min(kMlpF32NbWide, n - b0), ls, act,
                                  rows + b0);
    else
      mlp_eval_f32<kMlpF32NbWide>(*R.mlp_desc, R.mlp_f32, xs + (size_t)b0 * xstride, xstride,
                                  min(kMlpF32NbWide, n - b0), ls + b0, act);
  }
  return true;
}

constexpr int kRunSplitNb = 32;  // candidates per FP32-accurate (three-plane) tensor-core call
constexpr int kRunX2Nb = 64;     // candidates per 16-bit (two-plane) tensor-core call

// One tensor-core evaluation by the run's whole cluster (this block is its
// CTA 0; the followers wait in mlp_follower): post the command, evaluate
// this CTA's share (CTA 0 builds the layer-0 operand from xs / rows and
// copies it into the followers), gather the partial chi^2.  Every thread of
// the block.
template <int NB, int P>
inline __device__ bool mlp_pass_cl(const RunDesc& R, const float* xs, int xstride, int n, float* ls, char* tsm,
                                   MlpCtx* ctx, ClusterMail* mail, unsigned C, const int* rows) {
  if (threadIdx.x == 0) {
    mail->op = P;  // kClOpBf16, kClOpX2 or kClOpFp32
    mail->n = n;
  }
  cl_sync();
  const XIn X{nullptr, xs, rows, xstride};
  mlp_eval_bf16_cl<NB, kRunMlpStages, P>(*R.mlp_desc, R.mlp_tiles, R.mlp_f32, X, n, tsm, ctx, mail, C, 0u);
  cl_sync();
  const bool ok = mlp_cl_collect(mail, C, n, ls, rows);
  if (!ok && threadIdx.x == 0) ctx_set_err(ctx);
  __syncthreads();
  return ok;
}

// A follower CTA of an MLP run's cluster: evaluates its share of every
// tensor-core pass CTA 0 posts, until CTA 0 posts the exit.  Every thread of
// the block.
inline __device__ void mlp_follower(const RunDesc& R, MlpCtx* ctx, ClusterMail* mail, char* tsm, unsigned C,
                                    unsigned rank) {
  const bool tc = R.precision != 0;
  if (tc) mlp_ctx_init(ctx);
  const unsigned m0 = cl_map(smem_u32(mail), 0);
  for (;;) {
    cl_sync();
    const int op = cl_ld_s32(m0 + (unsigned)offsetof(ClusterMail, op));
    if (op == kClOpExit || !tc) {
      if (tc) mlp_cl_drain(ctx);
      cl_sync();
      break;
    }
    const int n = cl_ld_s32(m0 + (unsigned)offsetof(ClusterMail, n));
    const XIn X{nullptr, nullptr, nullptr, 0};  // the layer-0 operand comes from CTA 0
    if (op == kClOpBf16)
      mlp_eval_bf16_cl<kMlpNbMax, kRunMlpStages, 1>(*R.mlp_desc, R.mlp_tiles, R.mlp_f32, X, n, tsm, ctx, mail, C,
                                                    rank);
    else if (op == kClOpX2)
      mlp_eval_bf16_cl<kRunX2Nb, kRunMlpStages, 2>(*R.mlp_desc, R.mlp_tiles, R.mlp_f32, X, n, tsm, ctx, mail, C,
                                                   rank);
    else
      mlp_eval_bf16_cl<kRunSplitNb, kRunMlpStages, 3>(*R.mlp_desc, R.mlp_tiles, R.mlp_f32, X, n, tsm, ctx, mail,
                                                      C, rank);
    cl_sync();
  }
  if (tc) mlp_ctx_free(ctx);
}

// CTA 0 of an MLP run's cluster, before it exits: posts the exit, waits for
// the followers to read it.
inline __device__ void mlp_leader_exit(MlpCtx* ctx, ClusterMail* mail, bool tc) {
  if (threadIdx.x == 0) mail->op = kClOpExit;
  cl_sync();
  if (tc) mlp_cl_drain(ctx);
  cl_sync();
}

// rows: the n rows of xs (and ls) to evaluate, or null for rows 0..n-1.
// With a cluster of C > 1 CTAs, every call is split over the cluster.
static __device__ __noinline__ bool mlp_batch_bf16(const RunDesc& R, const float* xs, int xstride, int n, float* ls, char* tsm,
                                      MlpCtx* ctx, ClusterMail* mail, unsigned C, const int* rows = nullptr) {
  // equal calls of at most kMlpNbMax candidates (each call streams every weight tile once)
  const int calls = (n + kMlpNbMax - 1) / kMlpNbMax;
  const int per = (n + calls - 1) / calls;
  bool ok = true;
  for (int b0 = 0; b0 < n && ok; b0 += per) {
    const int nb = min(per, n - b0);
    if (C > 1)
      ok = rows ? mlp_pass_cl<kMlpNbMax, 1>(R, xs, xstride, nb, ls, tsm, ctx, mail, C, rows + b0)
                : mlp_pass_cl<kMlpNbMax, 1>(R, xs + (size_t)b0 * xstride, xstride, nb, ls + b0, tsm, ctx, mail, C,
                                            nullptr);
    else
      ok = rows ? mlp_eval_bf16<kMlpNbMax, kRunMlpStages>(*R.mlp_desc, R.mlp_tiles, R.mlp_f32, xs, xstride, nb, ls,
                                                          tsm, ctx, rows + b0)
                : mlp_eval_bf16<kMlpNbMax, kRunMlpStages>(*R.mlp_desc, R.mlp_tiles, R.mlp_f32,
                                                          xs + (size_t)b0 * xstride, xstride, nb, ls + b0, tsm, ctx);
  }
  return ok;
}

// FP32-accurate evaluation on the tensor cores (three BF16 planes, for
// networks whose weights are BF16 values) of the listed rows of xs, into ls.
static __device__ __noinline__ bool mlp_reeval_tc(const RunDesc& R, const float* xs, int xstride, float* ls, const int* list,
                                     int n, char* tsm, MlpCtx* ctx, ClusterMail* mail, unsigned C) {
  bool ok = true;
  for (int b0 = 0; b0 < n && ok; b0 += kRunSplitNb) {
    const int nb = min(kRunSplitNb, n - b0);
    ok = (C > 1) ? mlp_pass_cl<kRunSplitNb, 3>(R, xs, xstride, nb, ls, tsm, ctx, mail, C, list + b0)
                 : mlp_eval_bf16<kRunSplitNb, kRunMlpStages, 3>(*R.mlp_desc, R.mlp_tiles, R.mlp_f32, xs, xstride, nb,
                                                                ls, tsm, ctx, list + b0);
  }
  return ok;
}

// 16-bit evaluation on the tensor cores (two BF16 planes: activations and
// inputs to a relative 2^-17, weights exact when they are BF16 values) of
// the listed rows of xs, into ls.
static __device__ __noinline__ bool mlp_eval_x2(const RunDesc& R, const float* xs, int xstride, float* ls,
                                                const int* list, int n, char* tsm, MlpCtx* ctx, ClusterMail* mail,
                                                unsigned C) {
  bool ok = true;
  for (int b0 = 0; b0 < n && ok; b0 += kRunX2Nb) {
    const int nb = min(kRunX2Nb, n - b0);
    ok = (C > 1) ? mlp_pass_cl<kRunX2Nb, 2>(R, xs, xstride, nb, ls, tsm, ctx, mail, C, list + b0)
                 : mlp_eval_bf16<kRunX2Nb, kRunMlpStages, 2>(*R.mlp_desc, R.mlp_tiles, R.mlp_f32, xs, xstride, nb, ls,
                                                             tsm, ctx, list + b0);
  }
  return ok;
}

// FP32 re-evaluation of the listed rows of xbuf (indices in list[0..n)),
// written back into lbuf; xg/lg: kMlpF32Nb staging rows.
static __device__ __noinline__ void mlp_reeval(const RunDesc& R, float* xbuf, int xstride, float* lbuf, const int* list, int n,
                                  float* xg, float* lg, float* act) {
  for (int g0 = 0; g0 < n; g0 += kMlpF32Nb) {
    const int ng = min(kMlpF32Nb, n - g0);
    for (int q = threadIdx.x; q < ng * xstride; q += blockDim.x)
      xg[q] = xbuf[(size_t)list[g0 + q / xstride] * xstride + q % xstride];
    __syncthreads();
    mlp_eval_f32<kMlpF32Nb>(*R.mlp_desc, R.mlp_f32, xg, xstride, ng, lg, act);
    for (int q = threadIdx.x; q < ng; q += blockDim.x) lbuf[list[g0 + q]] = lg[q];
    __syncthreads();
  }
}

template <int DMAX>
__device__ __noinline__ void walker_phase_mlp(const RunDesc& R, const SliceCfg& S_ref, const float* s_W, const int* s_seed,
                                              const float* s_chol, float* xbuf, float* lbuf, int* rlist, char* msm,
                                              MlpCtx* ctx, ClusterMail* mail, int* mvlist, BlockScratch& BS,
                                              long long& ev_out, int& fl_out, long long& re_out, int& err_out,
                                              long long& cyc_eval, long long& cyc_reeval, long long* count) {
  constexpr int RW = dir_row(DMAX);
  const SliceCfg S = S_ref;  // in registers: the loop's stores would make every read a reload
  const int tid = threadIdx.x, m = R.m, d = S.d;
  const int XS = mlp_xs(d);
  const unsigned C = cl_size();
  const bool bf16 = (R.precision == 1);
  // precision 2: every evaluation FP32-accurate on the tensor cores (the
  // FP32 path for networks whose weights are BF16 values)
  const bool tcfp = (R.precision == 2);
  // FP32 re-evaluations on the tensor cores when the weights are BF16 values
  const bool tc32 = bf16 && R.mlp_desc->w_bf16;
  // a 16-bit (two-plane) stage between the BF16 value and the FP32 one
  const bool two = tc32 && R.two_plane != 0;
  char* tsm = align1024_shared(msm);
  float* act = reinterpret_cast<float*>(msm);
  float* xg = xbuf + (size_t)2 * m * XS;  // kMlpF32Nb staging rows after the 2m candidate rows
  float* lg = lbuf + 2 * m;
  const bool mine = tid < m;
  const int i = mine ? tid : 0;
  const int sd = s_seed[i];
  const float thr_out = (R.correction == 3) ? s_W[m - 1] : s_W[0];
  const float thr_in = (R.correction == 3) ? s_W[m - 1] : s_W[i];
  const float* dirs = R.dirs + (size_t)i * S.n_steps * RW;
  draw_directions_block<DMAX>(S, 0, m, [&](int w) { return s_chol + (size_t)R.live_cid[s_seed[w]] * d * d; },
                              R.dirs);
  const uint32_t n0 = shrink_draw0(d);
  float x[DMAX], v[DMAX], pre[kPreShrink];
  float l = mine ? R.live_l[sd] : 0.f;
#pragma unroll
  for (int k = 0; k < DMAX; ++k) x[k] = (mine && k < d) ? R.live_x[(size_t)k * R.n_pad + sd] : 0.f;
  // phase 0: stepping out, both ends at once (their sequences of points do
  // not depend on each other, so the decisions are the sequential
  // sampler's, left end then right end); phase 2: shrinkage
  int step = 0, phase = 0, nexp0 = 0, nexp1 = 0, done = 0, nsh = 0, hlen = 0, flags = 0;
  long long evals = 0, reevals = 0;
  float a = 0.f, b = 0.f;
  auto load_step = [&](int s_) {
    const float* row = dirs + (size_t)s_ * RW;
#pragma unroll
    for (int k = 0; k < DMAX; ++k) v[k] = row[k];
    const float r = row[DMAX];
#pragma unroll
    for (int j = 0; j < kPreShrink; ++j) pre[j] = row[DMAX + 1 + j];
    a = -r * S.width;
    b = (1.f - r) * S.width;
  };
  bool active = mine && S.n_steps > 0;
  if (active) load_step(0);
  int err = 0;
  long long ce = 0, cr = 0;  // thread 0: cycles in the batch evaluations and the FP32 re-evaluations
  // Two candidate slots per walker (bit s of the masks): slot 0 = the left
  // end (phase 0) or the shrink candidate (phase 2), slot 1 = the right end.
  // has: the slot holds an in-box candidate in its xbuf row (to evaluate,
  // held back by the round cap, or pending); pend: its BF16 log L was near
  // the threshold and it waits for its FP32 value (the pending candidates
  // are re-evaluated together once kMlpF32Nb of them wait, one has waited
  // reeval_defer rounds, or no walker can move; a decision is only
  // delayed, never changed); hold: left out of the last round's weight pass
  // by the round cap (it goes first in the next round).
  int has = 0, pend = 0, pend2 = 0, hold = 0;  // pend2: waits for its 16-bit value (then pend: FP32)
  float tp0 = 0.f, tp1 = 0.f;  // the slots' positions on the line
  int age = 0, age2 = 0;       // rounds the oldest pending candidate has waited, per stage (uniform)
  const int cap = bf16 ? R.mlp_round_cap : 0;
  auto row_of = [&](int s) { return s ? m + tid : tid; };
  // (register arrays are indexed by compile-time constants only, so they stay in registers)
  auto put = [&](int s, const float (&u)[DMAX]) {
    float* dst = xbuf + (size_t)row_of(s) * XS;
#pragma unroll
    for (int k = 0; k < DMAX; ++k)
      if (k < d) dst[k] = u[k];
  };
  // stepping out on side s with the outcome of its end
  auto decide_out = [&](int s, bool in, float lp) {
    if (in) ++evals;
    const bool ok = in && (lp > thr_out);
    const int ne = s ? nexp1 : nexp0;
    const bool expand = ok && (ne < S.e_max);
    if (s == 0) {
      a = expand ? a - S.width : a;
      nexp0 = expand ? ne + 1 : 0;
    } else {
      b = expand ? b + S.width : b;
      nexp1 = expand ? ne + 1 : 0;
    }
    flags |= (ok && !expand) ? 1 : 0;
    if (!expand) done |= 1 << s;
  };
  // shrinkage with the outcome of the candidate at tp
  auto decide_shrink = [&](bool in, float lp, float tp) {
    if (in) ++evals;
    const bool ok = in && (lp > thr_in);
    if (step == S.n_steps - 1) {
      int hs = -1;
      if (nsh < S.t_max - 1) {
        hs = nsh;
        hlen = nsh + 1;
      } else if (ok) {
        hs = S.t_max - 1;
        hlen = S.t_max;
      }
      if (hs >= 0) {
        float u[DMAX];
        candidate<DMAX>(x, v, tp, u);
        R.hist_l[(size_t)i * S.t_max + hs] = lp;
#pragma unroll
        for (int k = 0; k < DMAX; ++k)
          if (k < d) R.hist_x[((size_t)i * S.t_max + hs) * d + k] = u[k];
      }
    }
    bool advance = ok;
    if (ok) {
      float u[DMAX];
      candidate<DMAX>(x, v, tp, u);
#pragma unroll
      for (int k = 0; k < DMAX; ++k) x[k] = u[k];
      l = lp;
    } else {
      if (tp < 0.f) a = tp;
      else b = tp;
      if (++nsh >= S.s_max) {
        flags |= 2;
        advance = true;
      }
    }
    if (advance) {
      ++step;
      if (step < S.n_steps) {
        load_step(step);
        phase = 0;
        nsh = 0;
        nexp0 = nexp1 = 0;
        done = 0;
      } else {
        active = false;
      }
    }
  };
  // the outcome of slot s's candidate (evaluated, in the box)
  auto decide = [&](int s, float lp) {
    has &= ~(1 << s);
    hold &= ~(1 << s);
    if (phase == 2) decide_shrink(true, lp, tp0);
    else decide_out(s, true, lp);
  };
  // Fills the walker's empty slots with its next in-box candidates;
  // proposals outside the unit cube need no likelihood and are settled here
  // (a rejection, in the walker's own order of draws).
  auto fill = [&]() {
    // terminates: every pass fills a slot or settles a proposal (at most s_max per step)
    for (int guard = 0, gmax = (S.s_max + 2) * (S.n_steps + 1); guard < gmax; ++guard) {
      if (!active) return;
      if (phase == 0) {
#pragma unroll
        for (int s = 0; s < 2; ++s) {
          if ((done >> s) & 1 || (has >> s) & 1) continue;
          const float tp = s ? b : a;
          float u[DMAX];
          if (candidate<DMAX>(x, v, tp, u)) {
            has |= 1 << s;
            if (s) tp1 = tp;
            else tp0 = tp;
            put(s, u);
          } else {
            decide_out(s, false, -CUDART_INF_F);
          }
        }
        if (has) return;
        phase = 2;  // both ends are outside the slice
      } else {
        if (has & 1) return;
        float uu = pre[0];
        if (nsh < kPreShrink) {
#pragma unroll
          for (int j = 1; j < kPreShrink; ++j)
            if (nsh == j) uu = pre[j];
        } else {  // later shrinks (rare): straight from the step's stream
          uu = u24(draw_at(S.k0, S.k1, S.t, (uint32_t)i, (uint32_t)step, n0 + (uint32_t)nsh));
        }
        const float tp = fmaf(uu, b - a, a);
        float u[DMAX];
        if (candidate<DMAX>(x, v, tp, u)) {
          has |= 1;
          tp0 = tp;
          put(0, u);
          return;
        }
        decide_shrink(false, -CUDART_INF_F, tp);
      }
    }
  };
  for (;;) {
    if (!__syncthreads_or(active ? 1 : 0)) break;
    fill();
    const int req = active ? (has & ~(pend | pend2)) : 0;  // slots whose candidate is evaluated this round (or held)
    // every walker finished while settling its proposals: no batch to evaluate
    if (!__syncthreads_or((req | pend | pend2) ? 1 : 0)) break;
    // this round's candidates (row indices), in thread order, left slot first;
    // with a cap, the held ones first, then the new ones, up to the cap
    const int n_old_me = __popc(req & hold), n_new_me = __popc(req & ~hold);
    int n_old, n_new;
    const int p_old = block_exclusive_scan(n_old_me, BS, &n_old);
    const int p_new = block_exclusive_scan(n_new_me, BS, &n_new);
    const int n_all = n_old + n_new;
    const int n_mv = (cap > 0) ? min(cap, n_all) : n_all;
    int take = 0;
    {
      int po = p_old, pn = n_old + p_new;
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        if (!((req >> s) & 1)) continue;
        const int pos = ((hold >> s) & 1) ? po++ : pn++;
        if (pos < n_mv) {
          mvlist[pos] = row_of(s);
          take |= 1 << s;
        }
      }
      hold = req & ~take;
    }
    __syncthreads();
    if (tid == 0) {  // rounds; passes and their candidates (thread 0 keeps the run's counters)
      count[0] += 1;
      const int per = bf16 ? kMlpNbMax : (tcfp ? kRunSplitNb : kMlpF32NbWide);
      count[bf16 ? 1 : 3] += (n_mv + per - 1) / per;
      count[bf16 ? 2 : 4] += n_mv;
    }
    long long c0 = clock64();
    if (bf16) {
      if (n_mv > 0 && !mlp_batch_bf16(R, xbuf, XS, n_mv, lbuf, tsm, ctx, mail, C, mvlist)) err = 1;
      long long c1 = clock64();
      ce += c1 - c0;
      c0 = c1;
      // candidates close to their threshold wait for a more precise value:
      // the 16-bit one (two), then, if that is close too, the FP32 one
      const float thr = (phase == 2) ? thr_in : thr_out;
      const float margin = fmaf(R.reeval_rel, fabsf(thr), R.reeval_margin);
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        if (!((take >> s) & 1)) continue;
        const float lv = lbuf[row_of(s)];
        if (margin > 0.f && fabsf(lv - thr) < margin) {
          if (two) pend2 |= 1 << s;
          else pend |= 1 << s;
        } else {
          decide(s, lv);
        }
      }
      // can this walker move next round: a live slot that is not pending
      const int live = (phase == 0) ? (~done & 3) : 1;
      if (two) {
        int cnt2;
        const int pos2 = block_exclusive_scan(__popc(pend2), BS, &cnt2);
        const int still2 = __syncthreads_or((active && (live & ~(pend | pend2))) ? 1 : 0);
        age2 = (cnt2 > 0) ? age2 + 1 : 0;
        if (cnt2 > 0 && (cnt2 >= kRunX2Nb || !still2 || age2 > R.reeval_defer)) {
          {
            int p = pos2;
#pragma unroll
            for (int s = 0; s < 2; ++s)
              if ((pend2 >> s) & 1) rlist[p++] = row_of(s);
          }
          __syncthreads();
          if (tid == 0) {
            count[5] += (cnt2 + kRunX2Nb - 1) / kRunX2Nb;
            count[6] += cnt2;
          }
          if (!mlp_eval_x2(R, xbuf, XS, lbuf, rlist, cnt2, tsm, ctx, mail, C)) err = 1;
          const float margin2 = fmaf(R.reeval2_rel, fabsf(thr), R.reeval2_margin);
          const int pd = pend2;
          pend2 = 0;
#pragma unroll
          for (int s = 0; s < 2; ++s) {
            if (!((pd >> s) & 1)) continue;
            const float lv = lbuf[row_of(s)];
            if (fabsf(lv - thr) < margin2) pend |= 1 << s;
            else decide(s, lv);
          }
          age2 = 0;
        }
      }
      int cnt;
      const int pos = block_exclusive_scan(__popc(pend), BS, &cnt);
      const int still = __syncthreads_or((active && (live & ~(pend | pend2))) ? 1 : 0);
      age = (cnt > 0) ? age + 1 : 0;
      if (cnt > 0 && (cnt >= (tc32 ? kRunSplitNb : kMlpF32Nb) || !still || age > R.reeval_defer)) {
        {
          int p = pos;
#pragma unroll
          for (int s = 0; s < 2; ++s)
            if ((pend >> s) & 1) rlist[p++] = row_of(s);
        }
        __syncthreads();
        if (tid == 0) {
          count[3] += (cnt + (tc32 ? kRunSplitNb : kMlpF32Nb) - 1) / (tc32 ? kRunSplitNb : kMlpF32Nb);
          count[4] += cnt;
        }
        if (tc32) {
          if (!mlp_reeval_tc(R, xbuf, XS, lbuf, rlist, cnt, tsm, ctx, mail, C)) err = 1;
        } else {
          mlp_reeval(R, xbuf, XS, lbuf, rlist, cnt, xg, lg, act);
        }
        reevals += (tid == 0) ? cnt : 0;
        const int pd = pend;
        pend = 0;
#pragma unroll
        for (int s = 0; s < 2; ++s)
          if ((pd >> s) & 1) decide(s, lbuf[row_of(s)]);
        age = 0;
      }
      cr += clock64() - c0;
    } else {
      if (n_mv > 0) {
        if (tcfp) {
          if (!mlp_reeval_tc(R, xbuf, XS, lbuf, mvlist, n_mv, tsm, ctx, mail, C)) err = 1;
        } else {
          mlp_batch_f32(R, xbuf, XS, n_mv, lbuf, act, mvlist);
        }
      }
      ce += clock64() - c0;
      __syncthreads();
#pragma unroll
      for (int s = 0; s < 2; ++s)
        if ((take >> s) & 1) decide(s, lbuf[row_of(s)]);
    }
    if (__syncthreads_or(err)) {
      err = 1;
      break;
    }
  }
  __syncthreads();
  // stored values in FP32: each walker's final point, then its history
  // samples (rows of xbuf in order: the wide FP32 evaluator)
  const long long c_end = clock64();
  if (bf16 && !err) {
    if (mine) {
#pragma unroll
      for (int k = 0; k < DMAX; ++k)
        if (k < d) xbuf[(size_t)tid * XS + k] = x[k];
    }
    if (tid < m) rlist[tid] = tid;
    __syncthreads();
    if (tid == 0) {
      count[3] += (m + (tc32 ? kRunSplitNb : kMlpF32NbWide) - 1) / (tc32 ? kRunSplitNb : kMlpF32NbWide);
      count[4] += m;
    }
    if (tc32) {
      if (!mlp_reeval_tc(R, xbuf, XS, lbuf, rlist, m, tsm, ctx, mail, C)) err = 1;
    } else {
      mlp_batch_f32(R, xbuf, XS, m, lbuf, act);
    }
    if (mine) l = lbuf[tid];
    reevals += (tid == 0) ? m : 0;
    // history samples: only Algorithm 2 (the history correction) reads them,
    // and it takes a sample only above a relaxed threshold, which lies above
    // W[0]; the samples within the margin of W[0] or above get their FP32
    // value, the others are never read
    const float thr0 = s_W[0];
    const float lim = thr0 - fmaf(R.reeval_rel, fabsf(thr0), R.reeval_margin);
    uint64_t want = 0ull;
    int nh = 0;
    if (mine && R.correction == 2)
      for (int h = 0; h < hlen; ++h)
        if (R.hist_l[(size_t)i * S.t_max + h] >= lim) {
          want |= 1ull << h;
          ++nh;
        }
    int tot;
    const int base = block_exclusive_scan(nh, BS, &tot);
    const int per_pass = 2 * m;
    for (int h0 = 0; h0 < tot; h0 += per_pass) {
      // stage up to 2m history samples per pass in xbuf
      const int nb = min(per_pass, tot - h0);
      for (int h = 0, j = 0; h < hlen; ++h) {
        if (!((want >> h) & 1ull)) continue;
        const int gidx = base + j++ - h0;
        if (gidx >= 0 && gidx < nb) {
          const float* hx = R.hist_x + ((size_t)i * S.t_max + h) * d;
          for (int k = 0; k < d; ++k) xbuf[(size_t)gidx * XS + k] = hx[k];
        }
      }
      for (int q = tid; q < nb; q += blockDim.x) rlist[q] = q;
      __syncthreads();
      if (tid == 0) {
        count[3] += (nb + (tc32 ? kRunSplitNb : kMlpF32NbWide) - 1) / (tc32 ? kRunSplitNb : kMlpF32NbWide);
        count[4] += nb;
      }
      if (tc32) {
        if (!mlp_reeval_tc(R, xbuf, XS, lbuf, rlist, nb, tsm, ctx, mail, C)) err = 1;
      } else {
        mlp_batch_f32(R, xbuf, XS, nb, lbuf, act);
      }
      for (int h = 0, j = 0; h < hlen; ++h) {
        if (!((want >> h) & 1ull)) continue;
        const int gidx = base + j++ - h0;
        if (gidx >= 0 && gidx < nb) R.hist_l[(size_t)i * S.t_max + h] = lbuf[gidx];
      }
      __syncthreads();
      reevals += (tid == 0) ? nb : 0;
    }
  }
  if (mine) {
#pragma unroll
    for (int k = 0; k < DMAX; ++k)
      if (k < d) R.new_x[(size_t)i * d + k] = x[k];
    R.new_l[i] = l;
    R.hist_len[i] = hlen;
    if (R.wk_evals) {
      R.wk_evals[i] = (int)evals;
      R.wk_flags[i] = flags;
    }
  }
  cr += clock64() - c_end;
  ev_out = mine ? evals : 0;
  fl_out = mine ? flags : 0;
  re_out = reevals;
  err_out = err;
  cyc_eval = ce;
  cyc_reeval = cr;
}

// Initial live points of an MLP run, evaluated in FP32.
template <int DMAX>
inline __device__ void init_live_mlp(const RunDesc& R, float* xbuf, float* lbuf, int* rlist, char* msm) {
  const int d = R.d, XS = mlp_xs(d);
  float* act = reinterpret_cast<float*>(msm);
  for (int j0 = 0; j0 < R.N; j0 += R.m) {
    const int nb = min(R.m, R.N - j0);
    for (int q = threadIdx.x; q < nb * d; q += blockDim.x) {
      const int j = j0 + q / d, k = q % d;
      const float xv = u24(draw_at(R.k0, R.k1, kTInit, (uint32_t)j, 0u, (uint32_t)k));
      R.live_x[(size_t)k * R.n_pad + j] = xv;
      xbuf[(size_t)(q / d) * XS + k] = xv;
    }
    for (int q = threadIdx.x; q < nb; q += blockDim.x) rlist[q] = q;
    __syncthreads();
    mlp_reeval(R, xbuf, XS, lbuf, rlist, nb, xbuf + (size_t)2 * R.m * XS, lbuf + 2 * R.m, act);
    for (int q = threadIdx.x; q < nb; q += blockDim.x) {
      R.live_l[j0 + q] = lbuf[q];
      R.live_cid[j0 + q] = 0;
    }
    __syncthreads();
  }
}

// Blocks of up to 256 threads.  For the small register classes two such
// blocks per SM cap the registers at 128 per thread (more runs resident per
// SM hide the walkers' latency); the wide classes keep the full register
// file.  NS_RUN_MINB overrides the choice at build time.
#ifdef NS_RUN_MINB
#define NS_MINB(D) NS_RUN_MINB
#else
#define NS_MINB(D) ((D) <= 12 ? 2 : 1)
#endif
// NS_RUN_MAXNREG (build time) caps the analytic run kernels' registers per
// thread directly instead (finer than whole blocks per SM).
#ifdef NS_RUN_MAXNREG
#define NS_RUN_BOUNDS(MLP, D) __launch_bounds__((MLP ? kMlpThreads : 256)) __maxnreg__(MLP ? 200 : NS_RUN_MAXNREG)
#else
#define NS_RUN_BOUNDS(MLP, D) __launch_bounds__((MLP ? kMlpThreads : 256), (MLP ? 1 : NS_MINB(D)))
#endif
template <int DMAX, bool MLP = false>
__global__ void NS_RUN_BOUNDS(MLP, DMAX) k_run(const RunDesc* __restrict__ runs, const int* __restrict__ ids, int chunk) {
  extern __shared__ __align__(16) char sm[];
  __shared__ RunDesc R;
  __shared__ RunState RS;
  __shared__ EvidState E;
  __shared__ int flag_any;
  __shared__ MlpCtx mlp_ctx;
  const int tid = threadIdx.x, B = blockDim.x;
  // MLP runs may be launched as clusters of C CTAs per run (CTA 0 runs the
  // sampler, the others share its tensor-core evaluations)
  unsigned C = 1, rank = 0;
  ClusterMail* mail = nullptr;
  if constexpr (MLP) {
    __shared__ ClusterMail cl_mail;
    mail = &cl_mail;
    C = cl_size();
    rank = cl_rank();
  }
  if (tid == 0) {
    R = runs[ids[blockIdx.x / C]];
    RS = *R.st;
    E.logz = RS.logz;
    E.info = RS.info;
    E.k = RS.k;
  }
  __syncthreads();
  const int d = R.d, N = R.N, m = R.m;
  const Carve cv = make_carve(d, m, R.n_nodes, DMAX, MLP, R.spill != 0);
  if constexpr (MLP) {
    if (rank > 0) {
      mlp_follower(R, &mlp_ctx, mail, align1024_shared(sm + cv.mlp), C, rank);
      return;
    }
  }
  if (RS.stopped || RS.status != 0) {
    if constexpr (MLP) {
      if (C > 1) mlp_leader_exit(&mlp_ctx, mail, false);
    }
    return;
  }
  if constexpr (MLP) {
    if (R.precision != 0) mlp_ctx_init(&mlp_ctx);
  }
  float* s_slots = reinterpret_cast<float*>(sm + cv.slots);
  float* s_xbuf = reinterpret_cast<float*>(sm + cv.xbuf);
  float* s_lbuf = reinterpret_cast<float*>(sm + cv.lbuf);
  int* s_rlist = reinterpret_cast<int*>(sm + cv.rlist);
  char* s_mlp = sm + cv.mlp;
  LikParams& P = *reinterpret_cast<LikParams*>(sm + cv.lik);
  BlockScratch& S = *reinterpret_cast<BlockScratch*>(sm + cv.scr);
  SelectScratch& X = *reinterpret_cast<SelectScratch*>(sm + cv.sel);
  float* s_chol = cv.chol_global ? R.chol : reinterpret_cast<float*>(sm + cv.chol);
  float* s_cent = reinterpret_cast<float*>(sm + cv.cent);
  int* s_mask = reinterpret_cast<int*>(sm + cv.mask);
  int* s_worst = reinterpret_cast<int*>(sm + cv.worst);
  float* s_W = reinterpret_cast<float*>(sm + cv.W);
  int* s_seed = reinterpret_cast<int*>(sm + cv.seed);
  int* s_sel_slot = reinterpret_cast<int*>(sm + cv.sel_slot);
  uint32_t* s_sel_key = reinterpret_cast<uint32_t*>(sm + cv.sel_key);
  const Cand A = cand_at(sm + cv.candA, m);
  const Cand Bf = cand_at(sm + cv.candB, m);
  const Cand Tm = cand_at(sm + cv.candT, m);
  int* s_list = reinterpret_cast<int*>(sm + cv.list);
  float* s_vals = reinterpret_cast<float*>(sm + cv.vals);
  int* s_ctr = reinterpret_cast<int*>(sm + cv.ctr);
  int* s_stage_cid = reinterpret_cast<int*>(sm + cv.stage_cid);

  if constexpr (!MLP) {  // likelihood parameters into shared memory
    const int* src = reinterpret_cast<const int*>(R.lik);
    int* dst = reinterpret_cast<int*>(&P);
    for (int i = tid; i < (int)(sizeof(LikParams) / 4); i += B) dst[i] = src[i];
  }
  __syncthreads();
  if (!RS.initialized) {
    if constexpr (MLP) init_live_mlp<DMAX>(R, s_xbuf, s_lbuf, s_rlist, s_mlp);
    else init_live<DMAX>(R, P);
    __syncthreads();
    if (tid == 0) {
      RS.n_evals += N;
      RS.initialized = 1;
      E.logz = -CUDART_INF;  // Z = 0 before the first death
      E.info = 0.0;
      E.k = 0;
    }
  }
  if (RS.t > 0) {  // cluster tables of the last re-clustering
    if (!cv.chol_global)
      for (int i = tid; i < R.n_nodes * d * d; i += B) s_chol[i] = R.chol[i];
    for (int i = tid; i < R.n_nodes * d; i += B) s_cent[i] = R.centres[i];
    for (int i = tid; i < R.n_nodes; i += B) s_mask[i] = R.mask[i];
  }
  __syncthreads();

  const double Nd = (double)N;
  SliceCfg SC;
  SC.d = d;
  SC.n_steps = R.n_steps;
  SC.e_max = R.e_max;
  SC.s_max = R.s_max;
  SC.t_max = R.t_max;
  SC.width = R.width;
  SC.k0 = R.k0;
  SC.k1 = R.k1;

  for (int it = 0; it < chunk; ++it) {
    if (RS.stopped || RS.status != 0) break;
    const uint32_t t = (uint32_t)RS.t;
    if (RS.n_dead + m + N > R.dead_cap) {
      if (tid == 0) RS.status = NS_ERR_BUDGET;
      __syncthreads();
      break;
    }
    long long c_prev = clock64();
    auto tick = [&](int ph) {
      if (tid == 0) {
        const long long c = clock64();
        RS.cycles[ph] += c - c_prev;
        c_prev = c;
      }
    };
    // a3: clustering
    if (R.recluster_every > 0 && (t % (uint32_t)R.recluster_every) == 0) cluster_phase(R, t, sm, cv, S);
    tick(kPhCluster);
    // a1-a2: selection
    select_worst(R.live_l, N, m, R.k0, R.k1, t, s_sel_slot, s_sel_key, s_worst, s_W, s_seed, X, S);
    tick(kPhSelect);
    // a4-a7: slice-sampling walkers
    long long ev = 0, re = 0, cyc_eval = 0, cyc_reeval = 0;
    int fl = 0, werr = 0;
    SC.t = t;
    if constexpr (MLP) {
      walker_phase_mlp<DMAX>(R, SC, s_W, s_seed, s_chol, s_xbuf, s_lbuf, s_rlist, s_mlp, &mlp_ctx, mail, s_list, S, ev,
                             fl, re, werr, cyc_eval, cyc_reeval, RS.mlp_count);
    } else {
      // every walker's rows of the iteration, spread over the whole block;
      // the walkers' cluster-factor offsets first (the update phase's
      // scratch), so that a row reads no global memory before its factor
      const long long cd = clock64();
      for (int w = tid; w < m; w += B) s_stage_cid[w] = R.live_cid[s_seed[w]] * d * d;
      __syncthreads();
      draw_directions_block<DMAX>(SC, 0, m, [&](int w) { return s_chol + s_stage_cid[w]; }, R.dirs);
      const long long cd1 = clock64();
      if (R.walker_warp) {
        walker_phase_warp<DMAX>(R, P, SC, s_W, s_seed, ev, fl);
        cyc_reeval = clock64() - cd1;
      } else if ((tid & ~31) < m) {
        walker_phase<DMAX>(R, P, SC, s_W, s_seed, s_chol, s_slots, ev, fl, cyc_eval, cyc_reeval);
        if (R.wk_evals && tid < m) {
          R.wk_evals[tid] = (int)ev;
          R.wk_flags[tid] = fl;
        }
        fl = fl ? 1 : 0;
      }
      if (tid == 0) {
        RS.cycles[6] += cd1 - cd;
        RS.cycles[7] += cyc_reeval;
      }
    }
    __syncthreads();
    tick(kPhSlice);
    if constexpr (MLP) {
      const long long re_sum = block_sum_ll(re, S);
      if (tid == 0) {
        RS.n_reeval += re_sum;
        RS.cycles[6] += cyc_eval;
        RS.cycles[7] += cyc_reeval;
      }
      if (__syncthreads_or(werr)) {
        if (tid == 0) RS.status = NS_ERR_BUDGET;
        __syncthreads();
        break;
      }
    }
    const long long ev_sum = block_sum_ll(ev, S);
    const long long capped = block_sum_ll(MLP ? (fl ? 1 : 0) : fl, S);  // walkers that hit a cap
    // a8-a9: Algorithms 1 and 2
    const int rel = batch_correct(m, R.K, R.correction, s_W, R.new_l, R.hist_l, R.hist_len, R.t_max, A, Bf, Tm,
                                  s_list, s_vals, s_ctr, S);
    tick(kPhCorrect);
    // a10: dead append (rejected, ascending) and live update (accepted into
    // S_W's slots).  The run's arrays are read into registers first: through
    // R, every field would be loaded again after each store.
    const long long nd0 = RS.n_dead;
    {
      float* const live_x = R.live_x;
      const float* const new_x = R.new_x;
      const float* const hist_x = R.hist_x;
      float* const dead_x = R.dead_x;
      float* const stage_x = R.stage_x;
      float* const live_l = R.live_l;
      int* const live_cid = R.live_cid;
      const int n_pad = R.n_pad, t_max = R.t_max, n_nodes = R.n_nodes;
      for (int q = tid; q < m * d; q += B) {
        const int j = q / d, i = q - j * d;
        {
          const int src = A.src[j], hp = A.hp[j];
          float val;
          if (src < m) val = live_x[(size_t)i * n_pad + s_worst[src]];
          else if (hp < 0) val = new_x[(size_t)(src - m) * d + i];
          else val = hist_x[((size_t)(src - m) * t_max + hp) * d + i];
          dead_x[(size_t)(nd0 + j) * d + i] = val;
        }
        {
          const int src = A.src[m + j], hp = A.hp[m + j];
          float val;
          if (src < m) val = live_x[(size_t)i * n_pad + s_worst[src]];
          else if (hp < 0) val = new_x[(size_t)(src - m) * d + i];
          else val = hist_x[((size_t)(src - m) * t_max + hp) * d + i];
          stage_x[(size_t)j * d + i] = val;
        }
      }
      for (int j = tid; j < m; j += B) {
        R.dead_l[nd0 + j] = A.l[j];
        const int src = A.src[m + j];
        s_stage_cid[j] = (src < m) ? live_cid[s_worst[src]] : -1;
      }
      __syncthreads();
      for (int q = tid; q < m * d; q += B) {
        const int j = q / d, i = q - j * d;
        live_x[(size_t)i * n_pad + s_worst[j]] = stage_x[(size_t)j * d + i];
      }
      for (int j = tid; j < m; j += B) {
        const int slot = s_worst[j];
        live_l[slot] = A.l[m + j];
        int c = s_stage_cid[j];
        if (c < 0) c = (n_nodes > 1) ? nearest_leaf(stage_x + (size_t)j * d, d, n_nodes, s_cent, s_mask) : 0;
        live_cid[slot] = c;
      }
    }
    __syncthreads();
    tick(kPhUpdate);
    // a11: evidence (FP64)
    evidence_add(E, N, m, A.l, R.dead_logw + nd0, false, S);
    float lm = -CUDART_INF_F;
    for (int j = tid; j < N; j += B) lm = fmaxf(lm, R.live_l[j]);
    const float lmax = block_max_f(lm, S);
    tick(kPhEvidence);
    if (tid == 0) {
      RS.n_dead = nd0 + m;
      RS.n_evals += ev_sum;
      RS.n_capped += capped;
      RS.n_relaxed += rel;
      RS.t = (int)t + 1;
      RS.n_iter += 1;
      const bool stop = (E.logz > -CUDART_INF) && ((double)lmax - (double)E.k / Nd - E.logz < R.log_stop);
      flag_any = stop ? 1 : ((RS.n_iter >= R.max_iter) ? 2 : 0);
    }
    __syncthreads();
    if (flag_any) {
      // final live tail, slot order: each point carries X_K / N
      const long long nd1 = RS.n_dead;
      evidence_add(E, N, N, R.live_l, R.dead_logw + nd1, true, S);
      for (int q = tid; q < N * d; q += B) {
        const int j = q / d, i = q - j * d;
        R.dead_x[(size_t)(nd1 + j) * d + i] = R.live_x[(size_t)i * R.n_pad + j];
      }
      for (int j = tid; j < N; j += B) R.dead_l[nd1 + j] = R.live_l[j];
      __syncthreads();
      if (tid == 0) {
        RS.n_dead = nd1 + N;
        RS.stopped = 1;
        if (flag_any == 2) RS.status = NS_ERR_BUDGET;
      }
      __syncthreads();
      break;
    }
  }
  __syncthreads();
  if constexpr (MLP) {
    if (C > 1) mlp_leader_exit(&mlp_ctx, mail, R.precision != 0);
    if (R.precision != 0) mlp_ctx_free(&mlp_ctx);
  }
  if (tid == 0) {
    RS.logz = E.logz;
    RS.info = E.info;
    RS.k = E.k;
    *R.st = RS;
  }
}

template <int DMAX>
__global__ void k_loglike(const LikParams P, int n, const float* __restrict__ x, float* __restrict__ out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  float xr[DMAX];
#pragma unroll
  for (int i = 0; i < DMAX; ++i) xr[i] = (i < P.d) ? x[(size_t)j * P.d + i] : 0.f;
  out[j] = loglike_u<DMAX>(P, xr);
}

// Step-level slice kernel: dir_scratch holds the walkers' per-step tables,
// [m][n_steps][dir_row(DMAX)].
template <int DMAX>
__global__ void k_slice(const LikParams P, SliceCfg SC, int m, int n_pad, int correction,
                        const float* __restrict__ live_x, const float* __restrict__ live_l,
                        const int* __restrict__ seed_slot, const float* __restrict__ W,
                        const float* __restrict__ chol, const int* __restrict__ cid, float* new_x,
                        float* new_l, float* hist_l, float* hist_x, int* hist_len, long long* evals,
                        int* flags, float* dir_scratch) {
  extern __shared__ __align__(16) char sm[];
  const int i0 = blockIdx.x * blockDim.x + threadIdx.x;
  const bool act = i0 < m;
  const int i = act ? i0 : 0;
  const int d = SC.d;
  const int sd = seed_slot[i];
  const float thr_out = (correction == 3) ? W[m - 1] : W[0];
  const float thr_in = (correction == 3) ? W[m - 1] : W[i];
  WalkerOut O;
  O.new_x = new_x + (size_t)i * d;
  O.new_l = new_l + i;
  O.hist_l = hist_l + (size_t)i * SC.t_max;
  O.hist_x = hist_x + (size_t)i * SC.t_max * d;
  O.hist_len = hist_len + i;
  float* my_dirs = dir_scratch + (size_t)i * SC.n_steps * dir_row(DMAX);
  {  // this block's walkers' rows, spread over the block
    const int w0 = blockIdx.x * blockDim.x, w1 = min(m, w0 + (int)blockDim.x);
    if (w0 < w1)
      draw_directions_block<DMAX>(SC, w0, w1, [&](int w) { return chol + (size_t)cid[seed_slot[w]] * d * d; },
                                  dir_scratch);
  }
  long long ev = 0;
  int fl = 0;
  float* slot = reinterpret_cast<float*>(sm) + (size_t)threadIdx.x * dir_row(DMAX);
  slice_walker<DMAX>(P, SC, i, act, live_x + sd, n_pad, live_l[sd], my_dirs, slot, thr_out, thr_in, O, ev, fl);
  if (act) {
    evals[i] = ev;
    flags[i] = fl;
  }
}

// Step-level slice kernel with one walker per warp (walker w on warp w of
// the grid); same tables and outputs as k_slice.
template <int DMAX>
__global__ void k_slice_warp(const LikParams P, SliceCfg SC, int m, int n_pad, int correction,
                             const float* __restrict__ live_x, const float* __restrict__ live_l,
                             const int* __restrict__ seed_slot, const float* __restrict__ W,
                             const float* __restrict__ chol, const int* __restrict__ cid, float* new_x,
                             float* new_l, float* hist_l, float* hist_x, int* hist_len, long long* evals,
                             int* flags, float* dir_scratch) {
  const int nw = blockDim.x >> 5, lane = threadIdx.x & 31, d = SC.d;
  const int w0 = blockIdx.x * nw, w1 = min(m, w0 + nw);
  if (w0 < w1)
    draw_directions_block<DMAX>(SC, w0, w1, [&](int w) { return chol + (size_t)cid[seed_slot[w]] * d * d; },
                                dir_scratch);
  const int i = w0 + (int)(threadIdx.x >> 5);
  if (i >= m) return;
  LaneLik<DMAX> Q;
  lane_lik<DMAX>(P, Q);
  const int sd = seed_slot[i];
  const float thr_out = (correction == 3) ? W[m - 1] : W[0];
  const float thr_in = (correction == 3) ? W[m - 1] : W[i];
  WalkerOut O;
  O.new_x = new_x + (size_t)i * d;
  O.new_l = new_l + i;
  O.hist_l = hist_l + (size_t)i * SC.t_max;
  O.hist_x = hist_x + (size_t)i * SC.t_max * d;
  O.hist_len = hist_len + i;
  long long ev = 0;
  int fl = 0;
  slice_walker_warp<DMAX>(P, Q, SC, i, live_x + sd, n_pad, live_l[sd],
                          dir_scratch + (size_t)i * SC.n_steps * dir_row(DMAX), thr_out, thr_in, O, ev, fl);
  if (lane == 0) {
    evals[i] = ev;
    flags[i] = fl;
  }
}

// Register classes: a run of dimension d uses the smallest class >= d.
#define NS_FOR_EACH_CLASS(X) X(2) X(4) X(6) X(8) X(10) X(12) X(16) X(20) X(24) X(28) X(32)

// Launchers, one set per class (defined in ns_inst.cu).
#define NS_DECLARE_LAUNCHERS(D)                                                                          \
  cudaError_t launch_run_##D(const RunDesc* runs, const int* ids, int n, int block, size_t smem, int chunk, \
                             cudaStream_t s);                                                            \
  cudaError_t launch_loglike_##D(const LikParams& P, int n, const float* x, float* out, cudaStream_t s);  \
  cudaError_t launch_slice_##D(const LikParams& P, const SliceCfg& SC, int m, int n_pad, int correction,   \
                               const float* live_x, const float* live_l, const int* seed_slot,           \
                               const float* W, const float* chol, const int* cid, float* new_x,          \
                               float* new_l, float* hist_l, float* hist_x, int* hist_len, long long* evals, \
                               int* flags, float* dir_scratch, int warp, cudaStream_t s);                  \
  cudaError_t occupancy_run_##D(int block, size_t smem, int* blocks_per_sm);
NS_FOR_EACH_CLASS(NS_DECLARE_LAUNCHERS)
cudaError_t launch_run_mlp(const RunDesc* runs, const int* ids, int n, int block, size_t smem, int chunk, int cluster,
                           cudaStream_t s);

}  // namespace nsd
