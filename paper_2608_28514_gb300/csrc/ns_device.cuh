// ns_device.cuh -- device building blocks of the batched nested sampler
// (arXiv 2608.28514) for sm_103a.  Every step of one iteration is a
// __device__ function operating on one run with one thread block; the
// persistent run kernel chains them, and the step-level kernels call them one
// at a time on caller buffers, so both paths execute the same code.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>
#include <math_constants.h>

namespace nsd {

constexpr int kMaxDim = 32;
constexpr int kMaxModes = 8;
constexpr int kMaxDepth = 6;
constexpr int kMaxNodes = 127;
constexpr int kMaxHistory = 64;
constexpr uint32_t kPurposeSeed = 0x10000u;
constexpr uint32_t kPurposeKmeans = 0x20000u;
constexpr uint32_t kTInit = 0xFFFFFFFFu;
constexpr unsigned kFull = 0xFFFFFFFFu;

enum LikKind { kIso = 0, kCorr = 1, kRosen = 2, kMix = 3, kMlp = 4, kGmm = 5, kShell = 6 };
constexpr int kMaxGmmModes = 64;
constexpr int kGmmCap = 512;  // GMM modes x DMAX

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two
// 32x32->64 multiplications, key bumped by the Weyl constants each round.
// ---------------------------------------------------------------------------
struct U4 {
  uint32_t x, y, z, w;
};

__device__ __forceinline__ U4 philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                     uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hi0 = __umulhi(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
    const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return U4{c0, c1, c2, c3};
}

// Draw n of stream (t, walker, purpose) = word n%4 of block (n/4, purpose,
// walker, t); the last block is cached.
struct Stream {
  uint32_t k0, k1, t, walker, purpose, n, blk;
  uint32_t c0, c1, c2, c3;
  __device__ __forceinline__ void init(uint32_t key0, uint32_t key1, uint32_t tt, uint32_t w,
                                       uint32_t p) {
    k0 = key0;
    k1 = key1;
    t = tt;
    walker = w;
    purpose = p;
    n = 0;
    blk = 0xFFFFFFFFu;
  }
  __device__ __forceinline__ uint32_t next() {
    const uint32_t b = n >> 2;
    if (b != blk) {
      const U4 r = philox(b, purpose, walker, t, k0, k1);
      c0 = r.x;
      c1 = r.y;
      c2 = r.z;
      c3 = r.w;
      blk = b;
    }
    const uint32_t q = n & 3u;
    ++n;
    return q == 0 ? c0 : (q == 1 ? c1 : (q == 2 ? c2 : c3));
  }
};

__device__ __forceinline__ uint32_t draw_at(uint32_t k0, uint32_t k1, uint32_t t, uint32_t w,
                                            uint32_t purpose, uint32_t n) {
  const U4 r = philox(n >> 2, purpose, w, t, k0, k1);
  const uint32_t q = n & 3u;
  return q == 0 ? r.x : (q == 1 ? r.y : (q == 2 ? r.z : r.w));
}

// 24-bit uniforms, exact in FP32.
__device__ __forceinline__ float u24(uint32_t w) { return (float)(w >> 8) * 5.9604644775390625e-8f; }
__device__ __forceinline__ float u24_open0(uint32_t w) {
  return (float)((w >> 8) + 1u) * 5.9604644775390625e-8f;
}
// Uniform integer in [0, n).
__device__ __forceinline__ int u_index(uint32_t w, int n) { return (int)__umulhi(w, (uint32_t)n); }

// ---------------------------------------------------------------------------
// Likelihoods (FP32).  theta_i = lo_i + span_i * u_i with u the unit-cube
// point; constants are folded so that each coordinate costs one FMA:
// c_i = lo_i - mean_i (Gaussians), cm_ki = lo_i - centre_ki (mixture).
// Every array is zero beyond d and every matrix has the fixed stride
// kMaxDim, so a register class DMAX >= d needs no bounds tests: padded
// coordinates are 0 and contribute 0.
// ---------------------------------------------------------------------------
struct LikParams {
  int kind, d, n_modes, pad0;
  float inv2s2;   // 1 / (2 sigma^2)
  float a, b;     // Rosenbrock
  float log_k;    // log n_modes
  float lo[kMaxDim];
  float span[kMaxDim];
  float c[kMaxDim];
  float rw[kMaxDim];               // Rosenbrock: 1 for the d-1 chain links, else 0
  float2 LpP[(kMaxDim / 2) * kMaxDim];  // [jp*kMaxDim + i] = (L[i][2jp], L[i][2jp+1]), L L^T = inverse covariance
  float cm[kMaxModes * kMaxDim];   // [k*kMaxDim + i]
  // GMM, rows of DMAX floats (the run's register class), zero-padded:
  float gm[kGmmCap];               // lo_i - mu_ki
  float giv[kGmmCap];              // 1 / (2 s_ki^2), 0 beyond d
  float glw[kMaxGmmModes];         // log w_k
};

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 ld2(const float* p) { return *reinterpret_cast<const float2*>(p); }

// u = x + tp v (two coordinates per packed FMA) and whether u is in the unit
// cube.
template <int DMAX>
__device__ __forceinline__ bool candidate(const float (&x)[DMAX], const float (&v)[DMAX], float tp,
                                          float (&u)[DMAX]) {
  const float2 t2 = f2(tp, tp);
#pragma unroll
  for (int i = 0; i < DMAX; i += 2) {
    const float2 r = __ffma2_rn(t2, f2(v[i], v[i + 1]), f2(x[i], x[i + 1]));
    u[i] = r.x;
    u[i + 1] = r.y;
  }
  float mn = u[0], mx = u[0];
#pragma unroll
  for (int i = 1; i < DMAX; ++i) {
    mn = fminf(mn, u[i]);
    mx = fmaxf(mx, u[i]);
  }
  return (mn >= 0.f) && (mx <= 1.f);
}

// logL at the unit-cube point u (zero beyond d).  Pairs of coordinates (and
// pairs of rows of L^T) go through one packed FMA each.
template <int DMAX>
__device__ __forceinline__ float loglike_u(const LikParams& P, const float (&u)[DMAX]) {
  float ll;
  switch (P.kind) {
    case kIso: {
      float2 acc = f2(0.f, 0.f);
#pragma unroll
      for (int i = 0; i < DMAX; i += 2) {
        const float2 y = __ffma2_rn(ld2(P.span + i), f2(u[i], u[i + 1]), ld2(P.c + i));
        acc = __ffma2_rn(y, y, acc);
      }
      ll = -(acc.x + acc.y) * P.inv2s2;
      break;
    }
    case kCorr: {
      float y[DMAX];
#pragma unroll
      for (int i = 0; i < DMAX; i += 2) {
        const float2 q = __ffma2_rn(ld2(P.span + i), f2(u[i], u[i + 1]), ld2(P.c + i));
        y[i] = q.x;
        y[i + 1] = q.y;
      }
      float2 acc = f2(0.f, 0.f);
#pragma unroll
      for (int jp = 0; jp < DMAX / 2; ++jp) {
        // (z_{2jp}, z_{2jp+1}) = sum_{i >= 2jp} (L[i][2jp], L[i][2jp+1]) y_i
        float2 z = f2(0.f, 0.f);
#pragma unroll
        for (int i = 2 * jp; i < DMAX; ++i) z = __ffma2_rn(P.LpP[jp * kMaxDim + i], f2(y[i], y[i]), z);
        acc = __ffma2_rn(z, z, acc);
      }
      ll = -0.5f * (acc.x + acc.y);
      break;
    }
    case kRosen: {
      float th[DMAX];
#pragma unroll
      for (int i = 0; i < DMAX; i += 2) {
        const float2 q = __ffma2_rn(ld2(P.span + i), f2(u[i], u[i + 1]), ld2(P.lo + i));
        th[i] = q.x;
        th[i + 1] = q.y;
      }
      float s = 0.f;
#pragma unroll
      for (int i = 0; i + 1 < DMAX; ++i) {
        const float p = P.a - th[i];
        const float q = fmaf(-th[i], th[i], th[i + 1]);
        s = fmaf(P.rw[i], fmaf(p, p, P.b * q * q), s);
      }
      ll = -s;
      break;
    }
    case kMix: {
      float e[kMaxModes];
      float emax = -CUDART_INF_F;
#pragma unroll
      for (int k = 0; k < kMaxModes; ++k) {
        e[k] = -CUDART_INF_F;
        if (k < P.n_modes) {
          float2 acc = f2(0.f, 0.f);
#pragma unroll
          for (int i = 0; i < DMAX; i += 2) {
            const float2 y = __ffma2_rn(ld2(P.span + i), f2(u[i], u[i + 1]), ld2(P.cm + k * kMaxDim + i));
            acc = __ffma2_rn(y, y, acc);
          }
          e[k] = -(acc.x + acc.y) * P.inv2s2;
          emax = fmaxf(emax, e[k]);
        }
      }
      float acc = 0.f;
#pragma unroll
      for (int k = 0; k < kMaxModes; ++k)
        if (k < P.n_modes) acc += expf(e[k] - emax);
      ll = emax + logf(acc) - P.log_k;
      break;
    }
    case kGmm: {
      // log sum_k w_k exp(-sum_i (theta_i - mu_ki)^2 / (2 s_ki^2)), online
      // max-shifted sum over the modes
      float mx = -CUDART_INF_F, acc = 0.f;
      for (int k = 0; k < P.n_modes; ++k) {
        const float* g = P.gm + k * DMAX;
        const float* w = P.giv + k * DMAX;
        float2 s = f2(0.f, 0.f);
#pragma unroll
        for (int i = 0; i < DMAX; i += 2) {
          const float2 y = __ffma2_rn(ld2(P.span + i), f2(u[i], u[i + 1]), ld2(g + i));
          s = __ffma2_rn(__fmul2_rn(y, ld2(w + i)), y, s);
        }
        const float e = P.glw[k] - (s.x + s.y);
        if (e > mx) {
          acc = fmaf(acc, expf(mx - e), 1.f);
          mx = e;
        } else {
          acc += expf(e - mx);
        }
      }
      ll = mx + logf(acc);
      break;
    }
    case kShell: {
      float2 acc = f2(0.f, 0.f);
#pragma unroll
      for (int i = 0; i < DMAX; i += 2) {
        const float2 y = __ffma2_rn(ld2(P.span + i), f2(u[i], u[i + 1]), ld2(P.c + i));
        acc = __ffma2_rn(y, y, acc);
      }
      const float z = sqrtf(acc.x + acc.y) - P.a;
      ll = -z * z * P.inv2s2;
      break;
    }
    default:
      ll = -CUDART_INF_F;
  }
  return (ll != ll) ? -CUDART_INF_F : ll;
}

// ---------------------------------------------------------------------------
// Block helpers (blockDim.x a multiple of 32, <= 1024)
// ---------------------------------------------------------------------------
struct BlockScratch {
  int iw[33];
  double dw[33];
  float fw[33];
  long long lw[33];
};

// Exclusive prefix sum of v over threads in thread order; *total = sum.
__device__ __forceinline__ int block_exclusive_scan(int v, BlockScratch& S, int* total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(kFull, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) S.iw[wid] = x;
  __syncthreads();
  if (wid == 0) {
    int w = lane < nw ? S.iw[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(kFull, w, o);
      if (lane >= o) w += y;
    }
    if (lane < nw) S.iw[lane] = w;  // inclusive warp totals
  }
  __syncthreads();
  const int base = wid > 0 ? S.iw[wid - 1] : 0;
  const int tot = S.iw[nw - 1];
  __syncthreads();
  *total = tot;
  return base + x - v;
}

__device__ __forceinline__ double block_sum_d(double v, BlockScratch& S) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(kFull, v, o);
  if (lane == 0) S.dw[wid] = v;
  __syncthreads();
  if (wid == 0) {
    double w = lane < nw ? S.dw[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) w += __shfl_down_sync(kFull, w, o);
    if (lane == 0) S.dw[32] = w;
  }
  __syncthreads();
  const double r = S.dw[32];
  __syncthreads();
  return r;
}

__device__ __forceinline__ double block_max_d(double v, BlockScratch& S) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(kFull, v, o));
  if (lane == 0) S.dw[wid] = v;
  __syncthreads();
  if (wid == 0) {
    double w = lane < nw ? S.dw[lane] : -CUDART_INF;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) w = fmax(w, __shfl_down_sync(kFull, w, o));
    if (lane == 0) S.dw[32] = w;
  }
  __syncthreads();
  const double r = S.dw[32];
  __syncthreads();
  return r;
}

__device__ __forceinline__ float block_max_f(float v, BlockScratch& S) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_down_sync(kFull, v, o));
  if (lane == 0) S.fw[wid] = v;
  __syncthreads();
  if (wid == 0) {
    float w = lane < nw ? S.fw[lane] : -CUDART_INF_F;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) w = fmaxf(w, __shfl_down_sync(kFull, w, o));
    if (lane == 0) S.fw[32] = w;
  }
  __syncthreads();
  const float r = S.fw[32];
  __syncthreads();
  return r;
}

__device__ __forceinline__ long long block_sum_ll(long long v, BlockScratch& S) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(kFull, v, o);
  if (lane == 0) S.lw[wid] = v;
  __syncthreads();
  if (wid == 0) {
    long long w = lane < nw ? S.lw[lane] : 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) w += __shfl_down_sync(kFull, w, o);
    if (lane == 0) S.lw[32] = w;
  }
  __syncthreads();
  const long long r = S.lw[32];
  __syncthreads();
  return r;
}

// ---------------------------------------------------------------------------
// a1-a2: the m worst live points (radix select on an order-preserving key,
// ties by slot) and the walkers' start slots.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t order_key(float f) {
  const uint32_t b = __float_as_uint(f);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

struct SelectScratch {
  unsigned hist[256];
  int found[4];
};

// sel_slot/sel_key: smem [m] scratch.  Outputs (any address space): worst[m]
// ascending by (logL, slot), W[m], seed_slot[m].
inline __device__ void select_worst(const float* __restrict__ logl, int N, int m, uint32_t k0, uint32_t k1,
                             uint32_t t, int* sel_slot, uint32_t* sel_key, int* worst, float* W,
                             int* seed_slot, SelectScratch& X, BlockScratch& S) {
  const int tid = threadIdx.x, B = blockDim.x;
  uint32_t prefix = 0, pmask = 0;
  int k = m;  // rank (1-based) still to find among keys matching the prefix
  for (int pass = 0; pass < 4; ++pass) {
    const int shift = 24 - 8 * pass;
    for (int i = tid; i < 256; i += B) X.hist[i] = 0;
    __syncthreads();
    for (int j = tid; j < N; j += B) {
      const uint32_t key = order_key(logl[j]);
      if ((key & pmask) == prefix) atomicAdd(&X.hist[(key >> shift) & 255u], 1u);
    }
    __syncthreads();
    if (tid < 32) {
      unsigned c[8];
      unsigned loc = 0;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        c[q] = X.hist[tid * 8 + q];
        loc += c[q];
      }
      unsigned incl = loc;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(kFull, incl, o);
        if (tid >= o) incl += y;
      }
      const unsigned excl = incl - loc;
      // the lane whose range holds the k-th key
      if (excl < (unsigned)k && incl >= (unsigned)k) {
        unsigned run = excl;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          if (run < (unsigned)k && run + c[q] >= (unsigned)k) {
            X.found[0] = tid * 8 + q;
            X.found[1] = (int)run;
          }
          run += c[q];
        }
      }
    }
    __syncthreads();
    const int digit = X.found[0];
    k -= X.found[1];
    prefix |= (uint32_t)digit << shift;
    pmask |= 255u << shift;
    __syncthreads();
  }
  const uint32_t T = prefix;  // key of the m-th smallest; k of the equal keys are taken
  // ordered compaction over slot chunks
  const int C = (N + B - 1) / B;
  const int j0 = min(N, tid * C), j1 = min(N, j0 + C);
  int n_eq = 0;
  for (int j = j0; j < j1; ++j) n_eq += (order_key(logl[j]) == T);
  int tot;
  int eq_base = block_exclusive_scan(n_eq, S, &tot);
  int n_sel = 0;
  {
    int e = eq_base;
    for (int j = j0; j < j1; ++j) {
      const uint32_t key = order_key(logl[j]);
      if (key < T || (key == T && e < k)) ++n_sel;
      if (key == T) ++e;
    }
  }
  int sel_base = block_exclusive_scan(n_sel, S, &tot);
  {
    int e = eq_base, p = sel_base;
    for (int j = j0; j < j1; ++j) {
      const uint32_t key = order_key(logl[j]);
      if (key < T || (key == T && e < k)) {
        sel_slot[p] = j;
        sel_key[p] = key;
        ++p;
      }
      if (key == T) ++e;
    }
  }
  __syncthreads();
  // sort the m selected by (key, slot): rank by counting
  for (int e = tid; e < m; e += B) {
    const uint32_t ke = sel_key[e];
    const int se = sel_slot[e];
    int r = 0;
    for (int q = 0; q < m; ++q) {
      const uint32_t kq = sel_key[q];
      r += (kq < ke) || (kq == ke && sel_slot[q] < se);
    }
    worst[r] = se;
    W[r] = logl[se];
  }
  // start slots: the idx-th survivor in ascending slot order; sel_slot is in
  // ascending slot order, so skip every selected slot at or below the index.
  for (int i = tid; i < m; i += B) {
    int s = u_index(draw_at(k0, k1, t, (uint32_t)i, kPurposeSeed, 0), N - m);
    for (int q = 0; q < m; ++q) {
      if (sel_slot[q] <= s) ++s;
      else break;
    }
    seed_slot[i] = s;
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// a4-a7: slice sampling, one walker per thread (section 2.2), with the
// expansion threshold thr_out (= W[0]) and the acceptance threshold thr_in
// (= W[i]) of section 3.1.
//
// Each iteration first draws, for every walker and every slice step, the
// direction v = L_c z/|z| (z: Box-Muller normals from the step's stream) and
// the bracket offset r, all threads of the block in step (draw_directions_block).  The walk then
// runs as a state machine in which a round evaluates one candidate per
// active walker: expansion to the left, expansion to the right, shrinkage;
// after the direction draws a step's stream continues with the shrink draws.
// ---------------------------------------------------------------------------
struct SliceCfg {
  int d, n_steps, e_max, s_max, t_max;
  float width;
  uint32_t k0, k1, t;
};

// First stream draw of a step after the direction and r (2 ceil(d/2) + 1).
__host__ __device__ __forceinline__ uint32_t shrink_draw0(int d) { return 2u * (uint32_t)((d + 1) / 2) + 1u; }

// Shrink draws of a step that are drawn ahead with its direction.
constexpr int kPreShrink = 3;

// Row of the per-step table: v[0..DMAX), r, kPreShrink shrink uniforms,
// padded to a multiple of 4 floats (16-byte rows).
__host__ __device__ constexpr int dir_row(int dmax) { return ((dmax + 1 + kPreShrink) + 3) & ~3; }

// One row of the per-step table: walker `walker`'s step s, from the step's
// stream; chol: the walker's cluster factor, [d][d] row-major lower; out:
// dir_row(DMAX) floats (zero beyond d).
template <int DMAX>
__device__ __forceinline__ void draw_row(const SliceCfg& S, int walker, int s, const float* __restrict__ chol,
                                         float* __restrict__ out) {
  constexpr int RW = dir_row(DMAX);
  const int d = S.d;
  // every Philox block the row needs, computed up front: the blocks are
  // independent, so their rounds overlap (drawn one after another, each
  // waited for the last).  Words 0 .. 2 ceil(d/2) - 1 feed the normals, then
  // come r and the shrink draws.
  constexpr int NP = (DMAX + 1) / 2, NB = (2 * NP + 1 + kPreShrink + 3) / 4;
  uint32_t w[4 * NB];
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    const U4 q = philox((uint32_t)b, (uint32_t)s, (uint32_t)walker, S.t, S.k0, S.k1);
    w[4 * b] = q.x;
    w[4 * b + 1] = q.y;
    w[4 * b + 2] = q.z;
    w[4 * b + 3] = q.w;
  }
  float z[DMAX];
#pragma unroll
  for (int i = 0; i < DMAX; ++i) z[i] = 0.f;
#pragma unroll
  for (int p = 0; p < NP; ++p)
    if (2 * p < d) {
      const float u1 = u24_open0(w[2 * p]);
      const float u2 = u24(w[2 * p + 1]);
      // Box-Muller; the angle on the special-function unit: 2 pi u2 - pi
      // stays in [-pi, pi), where the intrinsics are accurate to ~1e-6
      // absolute, and (cos, sin)(2 pi u2) = -(cos, sin)(2 pi u2 - pi).  The
      // radius keeps the accurate logarithm (relative accuracy near u1 = 1).
      const float rho = sqrtf(-2.f * logf(u1));
      const float th = fmaf(u2, 6.28318530717958648f, -3.14159265358979324f);
      z[2 * p] = -rho * __cosf(th);
      if (2 * p + 1 < DMAX && 2 * p + 1 < d) z[2 * p + 1] = -rho * __sinf(th);
    }
  float nz = 0.f;
#pragma unroll
  for (int i = 0; i < DMAX; ++i) nz = fmaf(z[i], z[i], nz);
  if (nz > 0.f) {
    const float inv = rsqrtf(nz);
#pragma unroll
    for (int i = 0; i < DMAX; ++i) z[i] *= inv;
  } else {
#pragma unroll
    for (int i = 0; i < DMAX; ++i) z[i] = (i == 0) ? 1.f : 0.f;
  }
  float row[RW];
#pragma unroll
  for (int i = 0; i < RW; ++i) row[i] = 0.f;
#pragma unroll
  for (int i = 0; i < DMAX; ++i) {
    float acc = 0.f;
    if (i < d) {
#pragma unroll
      for (int k = 0; k <= i; ++k) acc = fmaf(chol[i * d + k], z[k], acc);
    }
    row[i] = acc;
  }
  {
    const int nr = 2 * ((d + 1) / 2);  // the word of r (a select chain keeps w in registers)
#pragma unroll
    for (int k = 0; k <= 2 * NP; k += 2)
      if (k == nr) {
        row[DMAX] = u24(w[k]);
#pragma unroll
        for (int j = 0; j < kPreShrink; ++j) row[DMAX + 1 + j] = u24(w[k + 1 + j]);
      }
  }
#pragma unroll
  for (int i = 0; i < RW; i += 4)
    *reinterpret_cast<float4*>(out + i) = make_float4(row[i], row[i + 1], row[i + 2], row[i + 3]);
}

// The rows of walkers [w0, w1) (every step), spread over all threads of the
// block: consecutive threads take consecutive steps of a walker (so a warp
// mostly reads one cluster factor).  dirs: [walkers][n_steps][dir_row(DMAX)];
// chol_of(i): walker i's cluster factor.  Called by every thread; ends with a
// block barrier.
template <int DMAX, typename CholOf>
__device__ __forceinline__ void draw_directions_block(const SliceCfg& S_ref, int w0, int w1, CholOf chol_of,
                                                      float* __restrict__ dirs) {
  constexpr int RW = dir_row(DMAX);
  const SliceCfg S = S_ref;  // in registers across the rows' stores
  const int rows = (w1 - w0) * S.n_steps;
  for (int q = threadIdx.x; q < rows; q += blockDim.x) {
    const int i = w0 + q / S.n_steps, s = q - (i - w0) * S.n_steps;
    draw_row<DMAX>(S, i, s, chol_of(i), dirs + ((size_t)i * S.n_steps + s) * RW);
  }
  __syncthreads();
}

struct WalkerOut {
  float* new_x;      // [d]
  float* new_l;      // [1]
  float* hist_l;     // [t_max]
  float* hist_x;     // [t_max][d]
  int* hist_len;     // [1]
};

// Asynchronous global -> shared copies (cp.async, 16 bytes each); a thread
// waits only for the copies it issued.
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gmem_src) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// Starts copying one step's row (dir_row(DMAX) floats, 16-byte aligned) into
// this walker's shared-memory slot.
template <int DMAX>
__device__ __forceinline__ void prefetch_row(float* slot, const float* __restrict__ src) {
  constexpr int RW = dir_row(DMAX);
#pragma unroll
  for (int i = 0; i < RW; i += 4) cp_async16(slot + i, src + i);
  cp_async_commit();
}

// Waits for the walker's prefetched row and unpacks it.
template <int DMAX>
__device__ __forceinline__ void take_row(const float* slot, float (&v)[DMAX], float& r, float (&pre)[kPreShrink]) {
  cp_async_wait_all();
#pragma unroll
  for (int i = 0; i < DMAX; i += 2) {
    const float2 q = *reinterpret_cast<const float2*>(slot + i);
    v[i] = q.x;
    v[i + 1] = q.y;
  }
  r = slot[DMAX];
#pragma unroll
  for (int j = 0; j < kPreShrink; ++j) pre[j] = slot[DMAX + 1 + j];
}

// All lanes of a warp must call it.  dirs: this walker's table from
// draw_directions_block; slot: dir_row(DMAX) floats of shared memory (16-byte
// aligned) private to this walker, used to prefetch the next step's row.
// The step configuration is copied into registers first: read through the
// reference, every field would be loaded again after each store the loop
// makes (the history), which cost 14 % of the 10-D run kernel's time.
template <int DMAX>
inline __device__ void slice_walker(const LikParams& P, const SliceCfg& S, int walker, bool active,
                                    const float* __restrict__ x0, int x0_stride, float l0,
                                    const float* __restrict__ dirs, float* slot, float thr_out, float thr_in,
                                    const WalkerOut& O, long long& evals_out, int& flags_out) {
  constexpr int RW = dir_row(DMAX);
  const int d = S.d, n_steps = S.n_steps, e_max = S.e_max, s_max = S.s_max, t_max = S.t_max;
  const float width = S.width;
  const uint32_t k0 = S.k0, k1 = S.k1, t = S.t;
  const uint32_t n0 = shrink_draw0(d);
  float x[DMAX], v[DMAX];
  float pre[kPreShrink];
  float l = l0;
#pragma unroll
  for (int i = 0; i < DMAX; ++i) {
    x[i] = (active && i < d) ? x0[(size_t)i * x0_stride] : 0.f;
    v[i] = 0.f;
  }
#pragma unroll
  for (int j = 0; j < kPreShrink; ++j) pre[j] = 0.f;
  const bool was_active = active;
  int step = 0, phase = 0, nexp = 0, nsh = 0, hlen = 0, flags = 0;
  long long evals = 0;
  float a = 0.f, b = 0.f;
  if (n_steps <= 0) active = false;
  if (active) {
    prefetch_row<DMAX>(slot, dirs);
    float r;
    take_row<DMAX>(slot, v, r, pre);
    a = -r * width;
    b = (1.f - r) * width;
    if (n_steps > 1) prefetch_row<DMAX>(slot, dirs + RW);
  }
  while (__any_sync(kFull, active)) {
    if (active) {
      float tp = (phase == 0) ? a : b;
      if (phase == 2) {
        float uu;
        if (nsh < kPreShrink) {
          uu = pre[0];
#pragma unroll
          for (int j = 1; j < kPreShrink; ++j)
            if (nsh == j) uu = pre[j];
        } else {  // later shrinks (rare): straight from the step's stream
          uu = u24(draw_at(k0, k1, t, (uint32_t)walker, (uint32_t)step, n0 + (uint32_t)nsh));
        }
        tp = fmaf(uu, b - a, a);
      }
      float lp = -CUDART_INF_F;
      bool in;
      {
        float u[DMAX];
        in = candidate<DMAX>(x, v, tp, u);
        if (in) {
          lp = loglike_u<DMAX>(P, u);
          ++evals;
        }
      }
      const bool ok = in && (lp > ((phase == 2) ? thr_in : thr_out));
      if (phase < 2) {
        // expansion: predicated updates, no branches
        const bool expand = ok && (nexp < e_max);
        a = (expand && phase == 0) ? a - width : a;
        b = (expand && phase == 1) ? b + width : b;
        flags |= (ok && !expand) ? 1 : 0;
        nexp = expand ? nexp + 1 : 0;
        phase = expand ? phase : phase + 1;
      } else {
        if (step == n_steps - 1) {
          int hs = -1;
          if (nsh < t_max - 1) {
            hs = nsh;
            hlen = nsh + 1;
          } else if (ok) {
            hs = t_max - 1;
            hlen = t_max;
          }
          if (hs >= 0) {
            float u[DMAX];
            candidate<DMAX>(x, v, tp, u);
            O.hist_l[hs] = lp;
#pragma unroll
            for (int i = 0; i < DMAX; ++i)
              if (i < d) O.hist_x[(size_t)hs * d + i] = u[i];
          }
        }
        bool advance = ok;
        if (ok) {
          float u[DMAX];
          candidate<DMAX>(x, v, tp, u);  // the accepted point, bit for bit
#pragma unroll
          for (int i = 0; i < DMAX; ++i) x[i] = u[i];
          l = lp;
        } else {
          if (tp < 0.f) a = tp;
          else b = tp;
          if (++nsh >= s_max) {
            flags |= 2;
            advance = true;
          }
        }
        if (advance) {
          ++step;
          if (step < n_steps) {
            float r;
            take_row<DMAX>(slot, v, r, pre);
            a = -r * width;
            b = (1.f - r) * width;
            if (step + 1 < n_steps) prefetch_row<DMAX>(slot, dirs + (size_t)(step + 1) * RW);
            phase = 0;
            nsh = 0;
            nexp = 0;
          } else {
            active = false;
          }
        }
      }
    }
  }
  evals_out = evals;
  flags_out = flags;
  if (was_active) {
#pragma unroll
    for (int i = 0; i < DMAX; ++i)
      if (i < d) O.new_x[i] = x[i];
    O.new_l[0] = l;
    O.hist_len[0] = hlen;
  }
}

// ---------------------------------------------------------------------------
// a5-a7 with one walker per warp: the 32 lanes of a warp carry one walker,
// lane i its coordinate i (d <= 32).  The decisions, draws and history are
// those of slice_walker; only the order of the FP32 sums inside the
// likelihood differs (warp butterflies).  A butterfly leaves the same sum in
// every lane (each step adds the same two values, in either order), so every
// lane holds the same log L and the walker's control flow is warp-uniform.
// This suits runs with few walkers (m = 1 is the sequential sampler), where a
// thread per walker leaves most of a block idle.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float warp_sum_all(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

// The likelihood constants of one lane's coordinate; for the correlated
// Gaussian the lane's column of L (L L^T = inverse covariance): col[k] =
// L[k][lane] for k >= lane, else 0.
template <int DMAX>
struct LaneLik {
  float span, c, lo, rw;
  float col[DMAX];
};

template <int DMAX>
__device__ __forceinline__ void lane_lik(const LikParams& P, LaneLik<DMAX>& Q) {
  const int lane = threadIdx.x & 31;
  Q.span = P.span[lane];
  Q.c = P.c[lane];
  Q.lo = P.lo[lane];
  Q.rw = P.rw[lane];
#pragma unroll
  for (int k = 0; k < DMAX; ++k) {
    float v = 0.f;
    if (P.kind == kCorr && k >= lane) {
      const float2 q = P.LpP[(lane >> 1) * kMaxDim + k];
      v = (lane & 1) ? q.y : q.x;
    }
    Q.col[k] = v;
  }
}

// log L at the unit-cube point whose coordinate `lane` is u (0 beyond d);
// the same value in every lane.
template <int DMAX>
__device__ __forceinline__ float loglike_lane(const LikParams& P, const LaneLik<DMAX>& Q, float u) {
  const int lane = threadIdx.x & 31;
  switch (P.kind) {
    case kIso: {
      const float y = fmaf(Q.span, u, Q.c);
      return -warp_sum_all(y * y) * P.inv2s2;
    }
    case kCorr: {
      // z_lane = sum_{k >= lane} L[k][lane] y_k, then ||z||^2
      const float y = fmaf(Q.span, u, Q.c);
      float z = 0.f;
#pragma unroll
      for (int k = 0; k < DMAX; ++k) z = fmaf(Q.col[k], __shfl_sync(kFull, y, k), z);
      return -0.5f * warp_sum_all(z * z);
    }
    case kRosen: {
      const float th = fmaf(Q.span, u, Q.lo);
      const float nx = __shfl_down_sync(kFull, th, 1);
      const float p = P.a - th;
      const float q = fmaf(-th, th, nx);
      return -warp_sum_all(Q.rw * fmaf(p, p, P.b * q * q));
    }
    case kMix: {
      float e[kMaxModes];
      float emax = -CUDART_INF_F;
#pragma unroll
      for (int k = 0; k < kMaxModes; ++k) {
        e[k] = -CUDART_INF_F;
        if (k < P.n_modes) {
          const float y = fmaf(Q.span, u, P.cm[k * kMaxDim + lane]);
          e[k] = -warp_sum_all(y * y) * P.inv2s2;
          emax = fmaxf(emax, e[k]);
        }
      }
      float acc = 0.f;
#pragma unroll
      for (int k = 0; k < kMaxModes; ++k)
        if (k < P.n_modes) acc += expf(e[k] - emax);
      return emax + logf(acc) - P.log_k;
    }
    case kGmm: {
      float mx = -CUDART_INF_F, acc = 0.f;
      for (int k = 0; k < P.n_modes; ++k) {
        float t = 0.f;
        if (lane < DMAX) {
          const float y = fmaf(Q.span, u, P.gm[k * DMAX + lane]);
          t = (y * P.giv[k * DMAX + lane]) * y;
        }
        const float e = P.glw[k] - warp_sum_all(t);
        if (e > mx) {
          acc = fmaf(acc, expf(mx - e), 1.f);
          mx = e;
        } else {
          acc += expf(e - mx);
        }
      }
      return mx + logf(acc);
    }
    case kShell: {
      const float y = fmaf(Q.span, u, Q.c);
      const float z = sqrtf(warp_sum_all(y * y)) - P.a;
      return -z * z * P.inv2s2;
    }
    default:
      return -CUDART_INF_F;
  }
}

// One walker on the calling warp (every lane calls, with the same walker).
// x0: the seed point, coordinate i at x0[i * x0_stride]; dirs: the walker's
// per-step table [n_steps][dir_row(DMAX)].  Outputs as slice_walker.
template <int DMAX>
__device__ void slice_walker_warp(const LikParams& P, const LaneLik<DMAX>& Q, const SliceCfg& S, int walker,
                                  const float* __restrict__ x0, int x0_stride, float l0,
                                  const float* __restrict__ dirs, float thr_out, float thr_in, const WalkerOut& O,
                                  long long& evals_out, int& flags_out) {
  constexpr int RW = dir_row(DMAX);
  const int lane = threadIdx.x & 31, d = S.d;
  const int n_steps = S.n_steps, e_max = S.e_max, s_max = S.s_max, t_max = S.t_max;  // in registers
  const float width = S.width;
  const uint32_t k0 = S.k0, k1 = S.k1, t = S.t;
  const bool mine = lane < d;
  const uint32_t n0 = shrink_draw0(d);
  float x = mine ? x0[(size_t)lane * x0_stride] : 0.f;
  float l = l0;
  int step = 0, phase = 0, nexp = 0, nsh = 0, hlen = 0, flags = 0;
  long long evals = 0;
  float a = 0.f, b = 0.f, v = 0.f, pre0 = 0.f, pre1 = 0.f, pre2 = 0.f;
  auto load_step = [&](int s) {
    const float* row = dirs + (size_t)s * RW;
    v = (lane < DMAX) ? row[lane] : 0.f;
    const float r = row[DMAX];
    pre0 = row[DMAX + 1];
    pre1 = row[DMAX + 2];
    pre2 = row[DMAX + 3];
    a = -r * width;
    b = (1.f - r) * width;
  };
  if (n_steps > 0) load_step(0);
  while (step < n_steps) {
    float tp = (phase == 0) ? a : b;
    if (phase == 2) {
      const float uu =
          nsh == 0 ? pre0
                   : (nsh == 1 ? pre1
                               : (nsh == 2 ? pre2 : u24(draw_at(k0, k1, t, (uint32_t)walker, (uint32_t)step,
                                                                n0 + (uint32_t)nsh))));
      tp = fmaf(uu, b - a, a);
    }
    const float u = fmaf(tp, v, x);
    const bool in = __all_sync(kFull, u >= 0.f && u <= 1.f);
    float lp = -CUDART_INF_F;
    if (in) {
      lp = loglike_lane<DMAX>(P, Q, u);
      ++evals;
    }
    const bool ok = in && (lp > ((phase == 2) ? thr_in : thr_out));
    if (phase < 2) {
      const bool expand = ok && (nexp < e_max);
      a = (expand && phase == 0) ? a - width : a;
      b = (expand && phase == 1) ? b + width : b;
      flags |= (ok && !expand) ? 1 : 0;
      nexp = expand ? nexp + 1 : 0;
      phase = expand ? phase : phase + 1;
      continue;
    }
    if (step == n_steps - 1) {
      int hs = -1;
      if (nsh < t_max - 1) {
        hs = nsh;
        hlen = nsh + 1;
      } else if (ok) {
        hs = t_max - 1;
        hlen = t_max;
      }
      if (hs >= 0) {
        if (lane == 0) O.hist_l[hs] = lp;
        if (mine) O.hist_x[(size_t)hs * d + lane] = u;
      }
    }
    bool advance = ok;
    if (ok) {
      x = u;
      l = lp;
    } else {
      if (tp < 0.f) a = tp;
      else b = tp;
      if (++nsh >= s_max) {
        flags |= 2;
        advance = true;
      }
    }
    if (advance) {
      ++step;
      if (step < n_steps) {
        load_step(step);
        phase = 0;
        nsh = 0;
        nexp = 0;
      }
    }
  }
  evals_out = evals;
  flags_out = flags;
  if (mine) O.new_x[lane] = x;
  if (lane == 0) {
    O.new_l[0] = l;
    O.hist_len[0] = hlen;
  }
}

// ---------------------------------------------------------------------------
// a8-a9: Algorithm 1 (batch sorting) and Algorithm 2 (history correction).
// Candidates 0..m-1: removed points W; m..2m-1: walkers' new points.
// ---------------------------------------------------------------------------
struct Cand {
  float* l;
  float* P;
  int* src;
  int* H;
  int* hp;
};

__device__ __forceinline__ bool cand_less(float la, int sa, float lb, int sb) {
  return (la < lb) || (la == lb && sa < sb);
}

__device__ __forceinline__ void cand_copy(const Cand& from, int i, const Cand& to, int j) {
  to.l[j] = from.l[i];
  to.P[j] = from.P[i];
  to.src[j] = from.src[i];
  to.H[j] = from.H[i];
  to.hp[j] = from.hp[i];
}

// Sort the 2m entries of `in` by (l, src) into `out`: each half is ranked
// by counting within itself (skipped for a half already in order), then
// the halves are merged by binary search.  `tmp` holds the sorted halves.
__device__ __forceinline__ void cand_sort(const Cand& in, const Cand& tmp, const Cand& out, int m,
                                          bool first_half_sorted) {
  const int n = 2 * m;
  for (int e = threadIdx.x; e < n; e += blockDim.x) {
    const int h0 = (e < m) ? 0 : m;
    int r;
    if (h0 == 0 && first_half_sorted) {
      r = e;
    } else {
      const float le = in.l[e];
      const int se = in.src[e];
      r = 0;
      for (int q = h0; q < h0 + m; ++q) r += cand_less(in.l[q], in.src[q], le, se) ? 1 : 0;
    }
    cand_copy(in, e, tmp, h0 + r);
  }
  __syncthreads();
  for (int e = threadIdx.x; e < n; e += blockDim.x) {
    const int h0 = (e < m) ? 0 : m, o0 = m - h0;
    const float le = tmp.l[e];
    const int se = tmp.src[e];
    int lo = 0, hi = m;  // entries of the other half below e
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (cand_less(tmp.l[o0 + mid], tmp.src[o0 + mid], le, se)) lo = mid + 1;
      else hi = mid;
    }
    cand_copy(tmp, e, out, (e - h0) + lo);
  }
  __syncthreads();
}

// Ordered compaction of predicate over [0, n): out[rank] = index.
template <class Pred>
__device__ __forceinline__ int block_compact(int n, Pred pred, int* out, BlockScratch& S) {
  const int B = blockDim.x, tid = threadIdx.x;
  const int C = (n + B - 1) / B;
  const int j0 = min(n, tid * C), j1 = min(n, j0 + C);
  int cnt = 0;
  for (int j = j0; j < j1; ++j) cnt += pred(j) ? 1 : 0;
  int tot;
  int base = block_exclusive_scan(cnt, S, &tot);
  for (int j = j0; j < j1; ++j)
    if (pred(j)) out[base++] = j;
  __syncthreads();
  return tot;
}

// A, Bf, Tm: three candidate buffers of 2m entries each (smem).  On return
// the sorted candidates are in A: rejected A[0:m], accepted A[m:2m].
// list_f: smem int [2m]; vals: smem float [m].  Returns n_relaxed.
inline __device__ int batch_correct(int m, int K, int correction, const float* __restrict__ W,
                                    const float* __restrict__ new_l, const float* __restrict__ hist_l,
                                    const int* __restrict__ hist_len, int t_max, const Cand& A, const Cand& Bf,
                                    const Cand& Tm, int* list_f, float* vals, int* counter, BlockScratch& S) {
  const int tid = threadIdx.x, B = blockDim.x;
  // Bf holds the unsorted candidates: W (ascending, candidates 0..m-1), then
  // the walkers' new points (candidates m..2m-1)
  for (int i = tid; i < m; i += B) {
    Bf.l[i] = W[i];
    Bf.P[i] = -1.f;
    Bf.src[i] = i;
    Bf.H[i] = -1;
    Bf.hp[i] = -1;
    Bf.l[m + i] = new_l[i];
    Bf.P[m + i] = W[i];
    Bf.src[m + i] = m + i;
    Bf.H[m + i] = i;
    Bf.hp[m + i] = -1;
  }
  if (tid == 0) *counter = 0;
  __syncthreads();
  if (correction == 0 || correction == 3) {
    // the removed points die (already ascending), the new points go live
    for (int e = tid; e < m; e += B) {
      const float le = Bf.l[m + e];
      const int se = Bf.src[m + e];
      int r = 0;
      for (int q = m; q < 2 * m; ++q) r += cand_less(Bf.l[q], Bf.src[q], le, se) ? 1 : 0;
      cand_copy(Bf, e, A, e);
      cand_copy(Bf, m + e, A, m + r);
    }
    __syncthreads();
    return 0;
  }
  cand_sort(Bf, Tm, A, m, true);  // Alg1.sort
  if (correction == 2) {
    for (int k = 1; k <= K; ++k) {
      const Cand C = A;
      const float amin = C.l[m];
      const int nF = block_compact(
          m, [&](int j) { return C.H[m + j] >= 0 && C.P[m + j] >= amin; }, list_f, S);
      if (nF == 0) break;
      // instant deaths: rejected new points, ascending
      int* list_i = list_f + m;
      const int nI = block_compact(m, [&](int j) { return C.H[j] >= 0; }, list_i, S);
      const int np = min(nF, nI);
      for (int i = tid; i < np; i += B) vals[i] = C.l[list_i[i]];
      __syncthreads();
      for (int i = tid; i < np; i += B) {
        const int e = m + list_f[i];
        const int w = C.H[e];
        const float thr = vals[i];
        const int hl = min(hist_len[w], t_max);
        for (int h = 0; h < hl; ++h) {
          const float hv = hist_l[(size_t)w * t_max + h];
          if (hv > thr) {
            C.l[e] = hv;
            C.hp[e] = h;
            C.P[e] = thr;
            atomicAdd(counter, 1);
            break;
          }
        }
      }
      __syncthreads();
      // re-sort r and a: r is still in order, a may not be
      for (int e = tid; e < 2 * m; e += B) cand_copy(A, e, Bf, e);
      __syncthreads();
      cand_sort(Bf, Tm, A, m, true);
    }
  }
  const int rel = *counter;
  __syncthreads();
  return rel;
}

// ---------------------------------------------------------------------------
// a11: FP64 evidence.  X_k = exp(-k/N); a dead point k has weight
// L (X_{k-1} - X_k); the live tail shares X_K.  The batch of n points is
// added at once with the invariant Z (H + log Z) = sum w L.
// state: logz, info, k.  Returns per-point log weights in logw.
// ---------------------------------------------------------------------------
struct EvidState {
  double logz, info;
  long long k;
};

inline __device__ void evidence_add(EvidState& E, int N, int n, const float* __restrict__ l_in,
                             double* logw_out, bool live, BlockScratch& S) {
  const double Nd = (double)N;
  const double invN = 1.0 / Nd;
  const double cN = log(-expm1(-invN));
  const double live_off = -(double)E.k * invN - log(Nd);
  const int tid = threadIdx.x, B = blockDim.x;
  const long long k0 = E.k;
  double mx = E.logz;
  for (int j = tid; j < n; j += B) {
    const double l = (double)l_in[j];
    const double lw = live ? l + live_off : l - (double)(k0 + j) * invN + cN;
    if (logw_out) logw_out[j] = lw;
    mx = fmax(mx, lw);
  }
  mx = block_max_d(mx, S);
  if (mx == -CUDART_INF) {
    if (!live) E.k = k0 + n;
    return;
  }
  double sw = 0.0, swl = 0.0;
  for (int j = tid; j < n; j += B) {
    const double l = (double)l_in[j];
    const double lw = live ? l + live_off : l - (double)(k0 + j) * invN + cN;
    const double w = exp(lw - mx);
    sw += w;
    if (l > -CUDART_INF) swl += w * l;
  }
  sw = block_sum_d(sw, S);
  swl = block_sum_d(swl, S);
  if (tid == 0) {
    double Bs = sw, As = swl;
    if (E.logz > -CUDART_INF) {
      const double w0 = exp(E.logz - mx);
      Bs += w0;
      As += w0 * (E.info + E.logz);
    }
    const double lz = mx + log(Bs);
    S.dw[0] = lz;
    S.dw[1] = As / Bs - lz;
  }
  __syncthreads();
  E.logz = S.dw[0];
  E.info = S.dw[1];
  if (!live) E.k = k0 + n;
  __syncthreads();
}

// ---------------------------------------------------------------------------
// a3: clustering (section 2.1).  FP32 products accumulated per 64-point
// tile, FP64 across tiles; FP64 regularised Cholesky.
// ---------------------------------------------------------------------------
constexpr int kTile = 128;
constexpr int kTileS = kTile + 2;  // row stride of a moments tile: rows start on different banks

// One warp: L = chol(A) for a d x d FP64 matrix (smem, row-major; A is not
// changed).  Right-looking, in place in L: per column one reciprocal square
// root of the pivot, the column scaled by it, then the trailing lower
// triangle updated, one row per lane (d <= 32).  The chain of dependent FP64
// operations per column is the rsqrt and two more (FP64 latency bounds this
// on a part with few FP64 units; the left-looking form added a shuffle
// reduction, a square root, a dot-product chain and a divide per column).
// Returns false (uniformly) if a pivot is not positive.
inline __device__ bool warp_cholesky(int d, const double* A, double* L) {
  const int lane = threadIdx.x & 31;
  for (int q = lane; q < d * d; q += 32) L[q] = ((q % d) <= (q / d)) ? A[q] : 0.0;
  __syncwarp();
  for (int j = 0; j < d; ++j) {
    const double s = L[j * d + j];
    if (!(s > 0.0) || !isfinite(s)) return false;
    const double r = rsqrt(s);
    const int i = j + 1 + lane;
    double lij = 0.0;
    if (i < d) {
      lij = L[i * d + j] * r;
      L[i * d + j] = lij;
    }
    __syncwarp();
    if (lane == 0) L[j * d + j] = s * r;
    if (i < d)
      for (int k = j + 1; k <= i; ++k) L[i * d + k] -= lij * L[k * d + j];
    __syncwarp();
  }
  return true;
}

// Cyclic Jacobi eigendecomposition, one warp (the rare path of the
// regularised Cholesky: a covariance that is not numerically positive
// definite).  The rotations follow the serial cyclic order p < q; each
// rotation's column, row and eigenvector updates are spread over the lanes.
// Sweeps stop once the off-diagonal mass is below 1e-30 of the diagonal
// mass (converged to FP64 rounding).  A: d x d, destroyed; Q: eigenvectors
// in columns; lam: eigenvalues.  Every lane of the warp calls it.
inline __device__ void jacobi_eigen_warp(int d, double* A, double* Q, double* lam) {
  const int lane = threadIdx.x & 31;
  for (int i = lane; i < d * d; i += 32) Q[i] = ((i / d) == (i % d)) ? 1.0 : 0.0;
  __syncwarp();
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, dia = 0.0;
    for (int i = lane; i < d * d; i += 32) {
      const int a = i / d, b = i % d;
      const double v = A[i];
      if (b > a) off += v * v;
      else if (a == b) dia += v * v;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      off += __shfl_xor_sync(kFull, off, o);
      dia += __shfl_xor_sync(kFull, dia, o);
    }
    if (!(off > 1e-30 * dia)) break;
    for (int p = 0; p < d; ++p)
      for (int q = p + 1; q < d; ++q) {
        const double apq = A[p * d + q];
        if (apq == 0.0) continue;
        const double th = (A[q * d + q] - A[p * d + p]) / (2.0 * apq);
        const double tt = (th >= 0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
        const double c = 1.0 / sqrt(tt * tt + 1.0), s = tt * c;
        __syncwarp();
        for (int k = lane; k < d; k += 32) {
          const double akp = A[k * d + p], akq = A[k * d + q];
          A[k * d + p] = c * akp - s * akq;
          A[k * d + q] = s * akp + c * akq;
        }
        __syncwarp();
        for (int k = lane; k < d; k += 32) {
          const double apk = A[p * d + k], aqk = A[q * d + k];
          A[p * d + k] = c * apk - s * aqk;
          A[q * d + k] = s * apk + c * aqk;
          const double qkp = Q[k * d + p], qkq = Q[k * d + q];
          Q[k * d + p] = c * qkp - s * qkq;
          Q[k * d + q] = s * qkp + c * qkq;
        }
        __syncwarp();
      }
  }
  for (int i = lane; i < d; i += 32) lam[i] = A[i * d + i];
  __syncwarp();
}

// The eigen-clip of the regularised Cholesky, one warp: A <- Q diag(max(lam,
// 1e-10 lam_max)) Q^T + delta I from the covariance C.  work: [2 d d + d]
// FP64 (Q, lam), T: [d d] FP64 scratch.
inline __device__ void warp_eigen_clip(int d, const double* C, double delta, double* A, double* work, double* T) {
  const int lane = threadIdx.x & 31;
  double* Q = work;
  double* lam = work + d * d;
  for (int i = lane; i < d * d; i += 32) T[i] = C[i];
  __syncwarp();
  jacobi_eigen_warp(d, T, Q, lam);
  double lmax = 0.0;
  for (int i = 0; i < d; ++i) lmax = fmax(lmax, lam[i]);
  for (int q = lane; q < d * d; q += 32) {
    const int i = q / d, j = q % d;
    double s = 0.0;
    for (int k = 0; k < d; ++k) s += Q[i * d + k] * fmax(lam[k], 1e-10 * lmax) * Q[j * d + k];
    A[q] = s + (i == j ? delta : 0.0);
  }
  __syncwarp();
}

// Regularised Cholesky of the covariance in C (smem FP64, d x d):
// chol(C + delta I), delta = 1e-10 tr(C)/d; if that fails, eigenvalues are
// clipped at 1e-10 lambda_max first (section 2.1).  Work: smem FP64 [3 d d + d].
// Called by the whole block; the result lands in L (smem FP64).
inline __device__ void reg_cholesky(int d, double* C, double* L, double* work, BlockScratch& S) {
  const int tid = threadIdx.x;
  double* A = work;
  if (tid < 32) {  // the trace: a shuffle tree instead of a chain of d FP64 adds
    double part = 0.0;
    for (int i = tid; i < d; i += 32) part += C[i * d + i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(kFull, part, o);
    if (tid == 0) S.dw[0] = part;
  }
  __syncthreads();
  const double tr = S.dw[0];
  __syncthreads();
  if (!(tr > 0.0) || !isfinite(tr)) {
    for (int i = tid; i < d * d; i += blockDim.x) L[i] = ((i / d) == (i % d)) ? 1e-6 : 0.0;
    __syncthreads();
    return;
  }
  const double delta = 1e-10 * tr / d;
  for (int i = tid; i < d * d; i += blockDim.x) A[i] = C[i] + (((i / d) == (i % d)) ? delta : 0.0);
  __syncthreads();
  if (tid < 32) {
    const bool ok = warp_cholesky(d, A, L);
    if (tid == 0) S.iw[0] = ok ? 1 : 0;
  }
  __syncthreads();
  const int ok = S.iw[0];
  __syncthreads();
  if (ok) return;
  if (tid < 32) warp_eigen_clip(d, C, delta, A, work + d * d, work + 2 * d * d + d);
  __syncthreads();
  if (tid < 32) {
    const bool ok2 = warp_cholesky(d, A, L);
    if (tid == 0) S.iw[0] = ok2 ? 1 : 0;
  }
  __syncthreads();
  if (!S.iw[0] && tid == 0) {
    for (int i = 0; i < d * d; ++i) L[i] = 0.0;
    for (int i = 0; i < d; ++i) L[i * d + i] = sqrt(A[i * d + i] > 0 ? A[i * d + i] : 1e-12);
  }
  __syncthreads();
}

// Mean and covariance (1/n) of the points j in [0, N) with member(j) true
// (live_x [d][n_pad]), in one pass: coordinates are shifted by the first
// member x_ref (so that E[(x - x_ref)(x - x_ref)^T] - (mu - x_ref)(mu -
// x_ref)^T suffers no cancellation), products accumulate in FP32 within a
// tile of kTile points and in FP64 across tiles.  tile: smem float
// [d][kTileS] + d; acc: smem FP64 [d + d*d]; returns n.  Results: mean in
// acc[0:d], covariance in acc[d:d+d*d].
template <class Member>
inline __device__ int node_moments(const float* __restrict__ live_x, int n_pad, int N, int d, Member member,
                                   float* tile, double* acc, BlockScratch& S) {
  const int tid = threadIdx.x, B = blockDim.x;
  const int ne = d * (d + 1) / 2;
  float* ref = tile + d * kTileS;
  for (int i = tid; i < d + d * d; i += B) acc[i] = 0.0;
  if (tid == 0) {
    int j0 = 0;
    while (j0 < N && !member(j0)) ++j0;
    S.iw[0] = j0;
  }
  __syncthreads();
  const int jr = S.iw[0];
  for (int i = tid; i < d; i += B) ref[i] = (jr < N) ? live_x[(size_t)i * n_pad + jr] : 0.f;
  __syncthreads();
  int cnt = 0;
  for (int j0 = 0; j0 < N; j0 += kTile) {
    // eight loads in flight per thread before the first store (one at a
    // time, the tile's loads were most of the clustering phase)
    for (int q0 = tid; q0 < d * kTile; q0 += 8 * B) {
      float v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int q = q0 + u * B;
        const int i = q / kTile, jj = q % kTile, j = j0 + jj;
        v[u] = (q < d * kTile && j < N && member(j)) ? live_x[(size_t)i * n_pad + j] - ref[i] : 0.f;
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int q = q0 + u * B;
        if (q < d * kTile) tile[(q / kTile) * kTileS + q % kTile] = v[u];
      }
    }
    if (tid < kTile) cnt += (j0 + tid < N && member(j0 + tid)) ? 1 : 0;
    __syncthreads();
    for (int e = tid; e < ne + d; e += B) {
      if (e < ne) {
        int a = 0;
        while ((a + 1) * (a + 2) / 2 <= e) ++a;
        const int bcol = e - a * (a + 1) / 2;
        const float* ta = tile + a * kTileS;
        const float* tb = tile + bcol * kTileS;
        // four independent packed accumulators
        float2 s0 = f2(0.f, 0.f), s1 = s0, s2 = s0, s3 = s0;
#pragma unroll 4
        for (int jj = 0; jj < kTile; jj += 8) {
          s0 = __ffma2_rn(ld2(ta + jj), ld2(tb + jj), s0);
          s1 = __ffma2_rn(ld2(ta + jj + 2), ld2(tb + jj + 2), s1);
          s2 = __ffma2_rn(ld2(ta + jj + 4), ld2(tb + jj + 4), s2);
          s3 = __ffma2_rn(ld2(ta + jj + 6), ld2(tb + jj + 6), s3);
        }
        s0 = __fadd2_rn(__fadd2_rn(s0, s1), __fadd2_rn(s2, s3));
        acc[d + a * d + bcol] += (double)(s0.x + s0.y);
      } else {
        const float* ta = tile + (e - ne) * kTileS;
        float2 s0 = f2(0.f, 0.f), s1 = s0, s2 = s0, s3 = s0;
#pragma unroll 4
        for (int jj = 0; jj < kTile; jj += 8) {
          s0 = __fadd2_rn(ld2(ta + jj), s0);
          s1 = __fadd2_rn(ld2(ta + jj + 2), s1);
          s2 = __fadd2_rn(ld2(ta + jj + 4), s2);
          s3 = __fadd2_rn(ld2(ta + jj + 6), s3);
        }
        s0 = __fadd2_rn(__fadd2_rn(s0, s1), __fadd2_rn(s2, s3));
        acc[e - ne] += (double)(s0.x + s0.y);
      }
    }
    __syncthreads();
  }
  const int n = (int)block_sum_ll(cnt, S);
  const double inv = n > 0 ? 1.0 / n : 0.0;
  for (int e = tid; e < ne; e += B) {
    int a = 0;
    while ((a + 1) * (a + 2) / 2 <= e) ++a;
    const int bcol = e - a * (a + 1) / 2;
    const double v = acc[d + a * d + bcol] * inv - (acc[a] * inv) * (acc[bcol] * inv);
    acc[d + a * d + bcol] = v;
    acc[d + bcol * d + a] = v;
  }
  __syncthreads();
  for (int i = tid; i < d; i += B) acc[i] = acc[i] * inv + (double)ref[i];
  __syncthreads();
  return n;
}

}  // namespace nsd
