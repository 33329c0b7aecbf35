// ns_cluster.cuh -- the cluster tree of section 2.1 on one thread block:
// recursive 2-means splits to a fixed depth, per-node covariance and FP64
// regularised Cholesky, bounding-ellipsoid volumes, bottom-up pruning, leaf
// assignment.
//
// Layout: the points are the live set x [d][n_pad] (unit cube).  Splits work
// on the points whitened by the root node's Cholesky factor, stored in
// y [d][n_pad]; side[j] holds point j's child choices, bit k at level k.
// Nodes are in heap order (root 0, children 2n+1, 2n+2).
//
// Determinism: every sum has a fixed thread -> point assignment and a fixed
// reduction tree (warp shuffles, then warps in order); maxima use atomicMax
// on order-preserving keys, which do not depend on order.  A run is therefore
// reproducible bit for bit.
#pragma once

#include "ns_device.cuh"

namespace nsd {

constexpr int kMaxLeaves = 64;  // depth <= 6
constexpr int kRedW = 64;       // values per vector block reduction

// Scratch of one tree build; L = 2^depth leaves, n_nodes = 2 L - 1.
struct TreeScratch {
  float* c;           // [L][d]: the two centres of each node of the current level (slot 2q+s)
  float* red;         // [nwarps][kRedW] partial sums
  float* out;         // [kRedW] reduced sums
  unsigned long long* far;  // [L / 2] farthest-member keys of the current level
  int* cnt;           // [2 L]: members per node of the level, then per (node, side) slot
  int* misc;          // [8]
  double* leaf_mu;    // [L][d]
  double* node_mu;    // [n_nodes][d]
  double* node_M2;    // [n_nodes][d*d]   (d*d: full symmetric, for the Cholesky)
  int* node_n;        // [n_nodes]
  unsigned* node_m2;  // [n_nodes] bits of the largest squared Mahalanobis distance
  double* lv;         // [n_nodes] log volumes
  double* veff;       // [n_nodes] effective (pruned) log volumes
  int* spl;           // [n_nodes] accepted splits
  double* chol_work;  // per warp: [5 d d + d]
};

template <class F>
__host__ __device__ inline size_t tree_layout(int d, int n_nodes, int nwarps, int nw_chol, F&& take) {
  const int L = (n_nodes + 1) / 2;
  take(0, sizeof(float) * L * d);
  take(1, sizeof(float) * nwarps * kRedW);
  take(2, sizeof(float) * kRedW);
  take(3, sizeof(unsigned long long) * L);
  take(4, sizeof(int) * L * 2);
  take(5, sizeof(int) * 8);
  take(6, sizeof(double) * L * d);
  take(7, sizeof(double) * n_nodes * d);
  take(8, sizeof(double) * (size_t)n_nodes * d * d);
  take(9, sizeof(int) * n_nodes);
  take(10, sizeof(unsigned) * n_nodes);
  take(11, sizeof(double) * n_nodes);
  take(12, sizeof(double) * n_nodes);
  take(13, sizeof(int) * n_nodes);
  return take(14, sizeof(double) * nw_chol * (5 * d * d + d));
}

__host__ __device__ inline size_t tree_bytes(int d, int n_nodes, int nwarps, int nw_chol) {
  if (n_nodes <= 1) return 0;
  size_t b = 0;
  tree_layout(d, n_nodes, nwarps, nw_chol, [&](int, size_t x) {
    b += (x + 15) & ~(size_t)15;
    return b;
  });
  return b;
}

// Warps that factorise node covariances in parallel, bounded by a 48 KB
// budget of FP64 work space.
__host__ __device__ inline int tree_chol_warps(int d, int nwarps) {
  const int per = (int)(sizeof(double) * (5 * d * d + d));
  int w = (48 * 1024) / per;
  if (w < 1) w = 1;
  return w < nwarps ? w : nwarps;
}

__device__ inline TreeScratch tree_carve(char* base, int d, int n_nodes, int nwarps, int nw_chol) {
  char* p[15];
  size_t o = 0;
  tree_layout(d, n_nodes, nwarps, nw_chol, [&](int k, size_t x) {
    p[k] = base + o;
    o += (x + 15) & ~(size_t)15;
    return o;
  });
  TreeScratch T;
  T.c = reinterpret_cast<float*>(p[0]);
  T.red = reinterpret_cast<float*>(p[1]);
  T.out = reinterpret_cast<float*>(p[2]);
  T.far = reinterpret_cast<unsigned long long*>(p[3]);
  T.cnt = reinterpret_cast<int*>(p[4]);
  T.misc = reinterpret_cast<int*>(p[5]);
  T.leaf_mu = reinterpret_cast<double*>(p[6]);
  T.node_mu = reinterpret_cast<double*>(p[7]);
  T.node_M2 = reinterpret_cast<double*>(p[8]);
  T.node_n = reinterpret_cast<int*>(p[9]);
  T.node_m2 = reinterpret_cast<unsigned*>(p[10]);
  T.lv = reinterpret_cast<double*>(p[11]);
  T.veff = reinterpret_cast<double*>(p[12]);
  T.spl = reinterpret_cast<int*>(p[13]);
  T.chol_work = reinterpret_cast<double*>(p[14]);
  return T;
}

// Deterministic block sum of kRedW values per thread (unused entries 0).
__device__ inline void block_sum_vec(float (&v)[kRedW], const TreeScratch& T) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < kRedW; ++k) {
    float x = v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(kFull, x, o);
    if (lane == 0) T.red[wid * kRedW + k] = x;
  }
  __syncthreads();
  for (int k = threadIdx.x; k < kRedW; k += blockDim.x) {
    float s = 0.f;
    for (int w = 0; w < nw; ++w) s += T.red[w * kRedW + k];
    T.out[k] = s;
  }
  __syncthreads();
}

// node of point with side bits `bits` at level `lev`
__device__ __forceinline__ int node_at(int bits, int lev) {
  int n = 0;
  for (int k = 0; k < lev; ++k) n = 2 * n + 1 + ((bits >> k) & 1);
  return n;
}

__device__ __forceinline__ int depth_of(int nd) {
  int dep = 0;
  for (int k = nd; k > 0; k = (k - 1) / 2) ++dep;
  return dep;
}

// One warp: regularised Cholesky (section 2.1) of C (d x d FP64) into L;
// work: [3 d d + d] FP64.  Same rule as reg_cholesky (eigen-clip fallback
// by warp_eigen_clip).
__device__ inline void warp_reg_cholesky(int d, const double* C, double* L, double* work) {
  const int lane = threadIdx.x & 31;
  double tr = 0.0;
  for (int i = lane; i < d; i += 32) tr += C[i * d + i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) tr += __shfl_xor_sync(kFull, tr, o);
  if (!(tr > 0.0) || !isfinite(tr)) {
    for (int i = lane; i < d * d; i += 32) L[i] = ((i / d) == (i % d)) ? 1e-6 : 0.0;
    __syncwarp();
    return;
  }
  const double delta = 1e-10 * tr / d;
  double* A = work;
  for (int i = lane; i < d * d; i += 32) A[i] = C[i] + (((i / d) == (i % d)) ? delta : 0.0);
  __syncwarp();
  if (warp_cholesky(d, A, L)) return;
  warp_eigen_clip(d, C, delta, A, work + d * d, work + 2 * d * d + d);
  if (!warp_cholesky(d, A, L)) {
    if (lane == 0) {
      for (int i = 0; i < d * d; ++i) L[i] = 0.0;
      for (int i = 0; i < d; ++i) L[i * d + i] = sqrt(A[i * d + i] > 0 ? A[i * d + i] : 1e-12);
    }
    __syncwarp();
  }
}

__device__ __forceinline__ double logaddexp_d(double a, double b) {
  if (a == -CUDART_INF) return b;
  if (b == -CUDART_INF) return a;
  const double mx = fmax(a, b);
  return mx + log1p(exp(-fabs(a - b)));
}

// The tree for depth D >= 1.  Inputs: x, the root's mean mu0 (float [d])
// and FP32 Cholesky L0 (float [d][d]); the root's FP64 statistics are
// already in node_mu[0] / node_M2[0] / node_n[0] (filled by the caller).
// Outputs: per node centre (float), chol (float + FP64), logvol, count,
// split, mask; cid[j] = accepted leaf of point j.
struct TreeIO {
  const float* x;
  float* y;
  int* side;
  int N, n_pad, d, depth, n_min, kmeans_iters;
  float vol_frac;
  uint32_t k0, k1, t;
  float* centres;   // global [n_nodes][d]
  float* chol;      // global [n_nodes][d][d]
  double* chol64;   // global
  float* logvol;    // global
  int* count;       // global
  int* split;       // global
  int* mask;        // global
  int* cid;         // global [N]
  float* s_chol;    // smem [n_nodes][d][d]
  float* s_cent;    // smem [n_nodes][d]
  int* s_mask;      // smem [n_nodes]
  int bracket;      // 1: the FP32 factors (the directions') scaled by each node's bounding radius
};

// This thread's largest squared Mahalanobis distance, over the live points
// j = tid, tid + blockDim.x, ... < N (live_x [d][n_pad]), from the centre mu
// in the units of the FP32 factor L (forward substitution), as the bits of a
// non-negative float (ordered like the values, for atomicMax).
static __device__ __noinline__ unsigned max_mahalanobis2(const float* __restrict__ live_x, int n_pad, int N, int d,
                                            const float* L, const float* mu) {
  float best = 0.f;
  for (int j = threadIdx.x; j < N; j += blockDim.x) {
    float r[kMaxDim];
    float s2 = 0.f;
    for (int i = 0; i < d; ++i) {
      float s = live_x[(size_t)i * n_pad + j] - mu[i];
      for (int k = 0; k < i; ++k) s = fmaf(-L[i * d + k], r[k], s);
      r[i] = s / L[i * d + i];
      s2 = fmaf(r[i], r[i], s2);
    }
    best = fmaxf(best, s2);
  }
  return __float_as_uint(best);
}

inline __device__ __noinline__ void cluster_tree(const TreeIO& io, const TreeScratch& T, BlockScratch& S, int nw_chol) {
  const int tid = threadIdx.x, B = blockDim.x, lane = tid & 31, wid = tid >> 5;
  const int d = io.d, N = io.N, D = io.depth, n_nodes = (1 << (D + 1)) - 1;
  const int n_leaves = 1 << D;
  // ---- whiten by the root factor: y = L0^{-1} (x - mu0) ------------------
  for (int j = tid; j < N; j += B) {
    float r[kMaxDim];
    for (int i = 0; i < d; ++i) {
      float s = io.x[(size_t)i * io.n_pad + j] - io.s_cent[i];
      for (int k = 0; k < i; ++k) s = fmaf(-io.s_chol[i * d + k], r[k], s);
      r[i] = s / io.s_chol[i * d + i];
      io.y[(size_t)i * io.n_pad + j] = r[i];
    }
    io.side[j] = 0;
  }
  __syncthreads();
  // ---- 2-means splits, level by level -------------------------------------
  for (int lev = 0; lev < D; ++lev) {
    const int first = (1 << lev) - 1, nlev = 1 << lev;
    // members per node of this level
    for (int q = tid; q < 2 * n_leaves; q += B) T.cnt[q] = 0;
    __syncthreads();
    for (int j = tid; j < N; j += B) atomicAdd(&T.cnt[node_at(io.side[j], lev) - first], 1);
    __syncthreads();
    // first centre: the Philox-chosen member (ascending slot order)
    const int C = (N + B - 1) / B;
    const int j0 = min(N, tid * C), j1 = min(N, j0 + C);
    for (int q = 0; q < nlev; ++q) {
      const int nd = first + q;
      const int n_mem = T.cnt[q];
      int mine = 0;
      for (int j = j0; j < j1; ++j) mine += (node_at(io.side[j], lev) == nd);
      int tot;
      const int base = block_exclusive_scan(mine, S, &tot);
      if (n_mem >= 2) {
        const int p = u_index(draw_at(io.k0, io.k1, io.t, (uint32_t)nd, kPurposeKmeans, 0), n_mem);
        if (p >= base && p < base + mine) {
          int r = base;
          for (int j = j0; j < j1; ++j)
            if (node_at(io.side[j], lev) == nd) {
              if (r == p) {
                for (int i = 0; i < d; ++i) T.c[(2 * q) * d + i] = io.y[(size_t)i * io.n_pad + j];
              }
              ++r;
            }
        }
      }
      __syncthreads();
    }
    // second centre: the member farthest from the first (ties: lowest slot)
    for (int q = tid; q < nlev; q += B) T.far[q] = 0ull;
    __syncthreads();
    for (int jb = 0; jb < N; jb += B) {
      const int j = jb + tid;
      int q = -1;
      unsigned long long key = 0ull;
      if (j < N) {
        q = node_at(io.side[j], lev) - first;
        if (T.cnt[q] >= 2) {
          float s = 0.f;
          for (int i = 0; i < d; ++i) {
            const float u = io.y[(size_t)i * io.n_pad + j] - T.c[(2 * q) * d + i];
            s = fmaf(u, u, s);
          }
          key = ((unsigned long long)__float_as_uint(s) << 32) | (unsigned long long)(0xFFFFFFFFu - (unsigned)j);
        } else {
          q = -1;
        }
      }
      if (q >= 0) atomicMax(&T.far[q], key);
    }
    __syncthreads();
    for (int q = 0; q < nlev; ++q) {
      if (T.cnt[q] < 2) continue;
      const int jf = (int)(0xFFFFFFFFu - (unsigned)(T.far[q] & 0xFFFFFFFFull));
      for (int i = tid; i < d; i += B) T.c[(2 * q + 1) * d + i] = io.y[(size_t)i * io.n_pad + jf];
    }
    __syncthreads();
    // Lloyd iterations: assign, then move the centres; stop at a fixed point
    for (int it = 0; it < io.kmeans_iters; ++it) {
      int changed = 0;
      for (int j = tid; j < N; j += B) {
        const int nd = node_at(io.side[j], lev);
        const int q = nd - first;
        if (T.cnt[q] < 2) continue;
        float s0 = 0.f, s1 = 0.f;
        for (int i = 0; i < d; ++i) {
          const float yi = io.y[(size_t)i * io.n_pad + j];
          const float u0 = yi - T.c[(2 * q) * d + i];
          const float u1 = yi - T.c[(2 * q + 1) * d + i];
          s0 = fmaf(u0, u0, s0);
          s1 = fmaf(u1, u1, s1);
        }
        const int sd = (s1 < s0) ? 1 : 0;
        const int old = (io.side[j] >> lev) & 1;
        if (it == 0 || sd != old) {
          changed = 1;
          io.side[j] = (io.side[j] & ~(1 << lev)) | (sd << lev);
        }
      }
      const int any = __syncthreads_or(changed);
      if (!any) break;
      // exact member counts of the (node, side) slots
      const int slots = 2 * nlev;
      int* scount = T.cnt + n_leaves;
      for (int q = tid; q < slots; q += B) scount[q] = 0;
      __syncthreads();
      for (int j = tid; j < N; j += B) {
        const int bits = io.side[j];
        const int q = node_at(bits, lev) - first;
        if (T.cnt[q] >= 2) atomicAdd(&scount[2 * q + ((bits >> lev) & 1)], 1);
      }
      __syncthreads();
      // centre sums per slot, 16 slots x four dimensions at a time; a slot
      // left empty keeps its centre
      constexpr int kSl = kRedW / 4;
      for (int s0 = 0; s0 < slots; s0 += kSl) {
        for (int c0 = 0; c0 < d; c0 += 4) {
          float acc[kRedW];
#pragma unroll
          for (int k = 0; k < kRedW; ++k) acc[k] = 0.f;
          for (int j = tid; j < N; j += B) {
            const int bits = io.side[j];
            const int slot = 2 * (node_at(bits, lev) - first) + ((bits >> lev) & 1) - s0;
            float v4[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) v4[k] = (c0 + k < d) ? io.y[(size_t)(c0 + k) * io.n_pad + j] : 0.f;
#pragma unroll
            for (int sl = 0; sl < kSl; ++sl)
              if (sl == slot) {
#pragma unroll
                for (int k = 0; k < 4; ++k) acc[sl * 4 + k] += v4[k];
              }
          }
          block_sum_vec(acc, T);
          for (int sl = tid; sl < kSl && s0 + sl < slots; sl += B) {
            const int gs = s0 + sl;
            if (T.cnt[gs / 2] < 2 || scount[gs] == 0) continue;
            for (int k = 0; k < 4 && c0 + k < d; ++k) T.c[gs * d + c0 + k] = T.out[sl * 4 + k] / (float)scount[gs];
          }
          __syncthreads();
        }
      }
    }
    // nodes with fewer than two members keep every member in the first child
    __syncthreads();
  }
  // ---- node statistics: leaf means, leaf centred products, pairwise merge ---
  const int last_first = n_leaves - 1;
  const int ne = d * (d + 1) / 2;
  // counts per leaf
  for (int q = tid; q < 2 * n_leaves; q += B) T.cnt[q] = 0;
  __syncthreads();
  for (int j = tid; j < N; j += B) atomicAdd(&T.cnt[node_at(io.side[j], D) - last_first], 1);
  __syncthreads();
  // leaf means (sums relative to the root mean, FP32 per thread, FP64 after),
  // eight leaves x eight dimensions at a time
  constexpr int kLf = kRedW / 8;
  for (int l0 = 0; l0 < n_leaves; l0 += kLf) {
    for (int c0 = 0; c0 < d; c0 += 8) {
      float acc[kRedW];
#pragma unroll
      for (int k = 0; k < kRedW; ++k) acc[k] = 0.f;
      for (int j = tid; j < N; j += B) {
        const int lf = node_at(io.side[j], D) - last_first - l0;
        float v8[8];
#pragma unroll
        for (int k = 0; k < 8; ++k)
          v8[k] = (c0 + k < d) ? io.x[(size_t)(c0 + k) * io.n_pad + j] - io.s_cent[c0 + k] : 0.f;
#pragma unroll
        for (int l = 0; l < kLf; ++l)
          if (l == lf) {
#pragma unroll
            for (int k = 0; k < 8; ++k) acc[l * 8 + k] += v8[k];
          }
      }
      block_sum_vec(acc, T);
      for (int q = tid; q < kLf * 8; q += B) {
        const int l = q / 8, k = q % 8;
        if (l0 + l < n_leaves && c0 + k < d) {
          const int n = T.cnt[l0 + l];
          T.leaf_mu[(l0 + l) * d + c0 + k] =
              n > 0 ? (double)T.out[l * 8 + k] / n + (double)io.s_cent[c0 + k] : 0.0;
        }
      }
      __syncthreads();
    }
  }
  // leaf centred products, eight leaves x eight entries at a time
  for (int l0 = 0; l0 < n_leaves; l0 += kLf) {
    for (int e0 = 0; e0 < ne; e0 += 8) {
      float acc[kRedW];
#pragma unroll
      for (int k = 0; k < kRedW; ++k) acc[k] = 0.f;
      int ea[8], eb[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        int e = e0 + k, a = 0;
        if (e >= ne) e = 0;
        while ((a + 1) * (a + 2) / 2 <= e) ++a;
        ea[k] = a;
        eb[k] = e - a * (a + 1) / 2;
      }
      for (int j = tid; j < N; j += B) {
        const int lf = node_at(io.side[j], D) - last_first - l0;
        if (lf < 0 || lf >= kLf) continue;
        float p8[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const float ua = io.x[(size_t)ea[k] * io.n_pad + j] - (float)T.leaf_mu[(l0 + lf) * d + ea[k]];
          const float ub = io.x[(size_t)eb[k] * io.n_pad + j] - (float)T.leaf_mu[(l0 + lf) * d + eb[k]];
          p8[k] = (e0 + k < ne) ? ua * ub : 0.f;
        }
#pragma unroll
        for (int l = 0; l < kLf; ++l)
          if (l == lf) {
#pragma unroll
            for (int k = 0; k < 8; ++k) acc[l * 8 + k] += p8[k];
          }
      }
      block_sum_vec(acc, T);
      for (int q = tid; q < kLf * 8; q += B) {
        const int l = q / 8, k = q % 8;
        if (l0 + l < n_leaves && e0 + k < ne) {
          const int nd = last_first + l0 + l;
          const double v = (double)T.out[l * 8 + k];
          T.node_M2[(size_t)nd * d * d + ea[k] * d + eb[k]] = v;
          T.node_M2[(size_t)nd * d * d + eb[k] * d + ea[k]] = v;
        }
      }
      __syncthreads();
    }
  }
  for (int q = tid; q < n_leaves; q += B) {
    const int nd = last_first + q;
    T.node_n[nd] = T.cnt[q];
    for (int i = 0; i < d; ++i) T.node_mu[nd * d + i] = T.leaf_mu[q * d + i];
  }
  __syncthreads();
  // internal nodes below the root: merge the children (Chan et al.)
  for (int nd = last_first - 1; nd >= 1; --nd) {
    const int c1 = 2 * nd + 1, c2 = 2 * nd + 2;
    const int n1 = T.node_n[c1], n2 = T.node_n[c2], n = n1 + n2;
    for (int q = tid; q < d * d; q += B) {
      const int a = q / d, b = q % d;
      double v = T.node_M2[c1 * d * d + q] + T.node_M2[c2 * d * d + q];
      if (n1 > 0 && n2 > 0) {
        const double da = T.node_mu[c1 * d + a] - T.node_mu[c2 * d + a];
        const double db = T.node_mu[c1 * d + b] - T.node_mu[c2 * d + b];
        v += da * db * ((double)n1 * n2 / n);
      }
      T.node_M2[nd * d * d + q] = v;
    }
    for (int i = tid; i < d; i += B)
      T.node_mu[nd * d + i] =
          n > 0 ? (T.node_mu[c1 * d + i] * n1 + T.node_mu[c2 * d + i] * n2) / n : 0.0;
    if (tid == 0) T.node_n[nd] = n;
    __syncthreads();
  }
  // ---- Cholesky of every node below the root, nw_chol warps in parallel -------
  if (wid < nw_chol) {
    for (int nd = 1 + wid; nd < n_nodes; nd += nw_chol) {
      double* W = T.chol_work + (size_t)wid * (5 * d * d + d);
      double* Cv = W;
      double* Lv = W + d * d;
      const int n = T.node_n[nd];
      const double inv = n > 0 ? 1.0 / n : 0.0;
      for (int q = lane; q < d * d; q += 32) Cv[q] = T.node_M2[nd * d * d + q] * inv;
      __syncwarp();
      warp_reg_cholesky(d, Cv, Lv, W + 2 * d * d);
      for (int q = lane; q < d * d; q += 32) {
        io.chol64[(size_t)nd * d * d + q] = Lv[q];
        const float f = (float)Lv[q];
        io.chol[(size_t)nd * d * d + q] = f;
        io.s_chol[nd * d * d + q] = f;
      }
      for (int i = lane; i < d; i += 32) {
        const float c = (float)T.node_mu[nd * d + i];
        io.centres[nd * d + i] = c;
        io.s_cent[nd * d + i] = c;
      }
      __syncwarp();
    }
  }
  __syncthreads();
  // ---- bounding ellipsoids: largest squared Mahalanobis distance per node ---
  for (int q = tid; q < n_nodes; q += B) T.node_m2[q] = 0u;
  __syncthreads();
  for (int j = tid; j < N; j += B) {
    const int bits = io.side[j];
    for (int lev = 0; lev <= D; ++lev) {
      const int nd = node_at(bits, lev);
      const float* Lf = io.s_chol + nd * d * d;
      const float* mu = io.s_cent + nd * d;
      float r[kMaxDim];
      float s2 = 0.f;
      for (int i = 0; i < d; ++i) {
        float s = io.x[(size_t)i * io.n_pad + j] - mu[i];
        for (int k = 0; k < i; ++k) s = fmaf(-Lf[i * d + k], r[k], s);
        r[i] = s / Lf[i * d + i];
        s2 = fmaf(r[i], r[i], s2);
      }
      atomicMax(&T.node_m2[nd], __float_as_uint(s2));
    }
  }
  __syncthreads();
  // ---- volumes, pruning bottom-up, accepted leaves --------------------------
  for (int nd = tid; nd < n_nodes; nd += B) {
    const int n = T.node_n[nd];
    double l = 0.0;
    for (int i = 0; i < d; ++i) l += log((double)io.s_chol[(size_t)nd * d * d + i * d + i]);
    const double m2 = (double)__uint_as_float(T.node_m2[nd]);
    T.lv[nd] = (n > 0) ? l + 0.5 * d * log(m2) : -CUDART_INF;
  }
  __syncthreads();
  if (tid == 0) {
    for (int nd = n_nodes - 1; nd >= 0; --nd) {
      const int c1 = 2 * nd + 1, c2 = 2 * nd + 2;
      if (c1 >= n_nodes) {
        T.spl[nd] = 0;
        T.veff[nd] = T.lv[nd];
        continue;
      }
      const double vc = logaddexp_d(T.veff[c1], T.veff[c2]);
      const int ok =
          T.node_n[c1] > io.n_min && T.node_n[c2] > io.n_min && vc < log(1.0 - (double)io.vol_frac) + T.lv[nd];
      T.spl[nd] = ok;
      T.veff[nd] = ok ? vc : T.lv[nd];
    }
  }
  __syncthreads();
  for (int nd = tid; nd < n_nodes; nd += B) {
    int act = 1;  // every ancestor split
    for (int k = nd; k > 0; k = (k - 1) / 2) act &= T.spl[(k - 1) / 2];
    const int mk = act && !T.spl[nd];
    io.s_mask[nd] = mk;
    io.mask[nd] = mk;
    io.split[nd] = T.spl[nd];
    io.count[nd] = T.node_n[nd];
    io.logvol[nd] = (float)T.lv[nd];
  }
  __syncthreads();
  // ---- second bracket reading: each direction factor times its node's radius
  if (io.bracket == 1) {
    for (int q = tid; q < n_nodes * d * d; q += B) {
      const float rad = sqrtf(__uint_as_float(T.node_m2[q / (d * d)]));
      if (rad > 0.f && isfinite(rad)) {
        io.s_chol[q] *= rad;
        io.chol[q] = io.s_chol[q];
      }
    }
    __syncthreads();
  }
  // ---- each point's accepted leaf --------------------------------------------
  for (int j = tid; j < N; j += B) {
    const int bits = io.side[j];
    int nd = 0, lev = 0;
    while (lev < D && T.spl[nd]) {
      nd = 2 * nd + 1 + ((bits >> lev) & 1);
      ++lev;
    }
    io.cid[j] = nd;
  }
  __syncthreads();
}

}  // namespace nsd
