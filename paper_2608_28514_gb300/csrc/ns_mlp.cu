// ns_mlp.cu -- batched evaluation of the MLP (emulator-style) likelihood:
// the packed weight image, the BF16 tensor-core evaluator (tcgen05, TMA bulk
// copies, tensor memory) and the FP32 CUDA-core evaluator, behind the C ABI.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include "../../include/ns_gb300.h"
#include "ns_mlp.cuh"
#include "ns_mlp_cluster.cuh"

using namespace nsd;

namespace {

// Persistent: each block sets up its tensor memory and barriers once and
// evaluates batches of kMlpNbMax candidates, grid-strided.
constexpr int kMlpStandaloneStages = 4;
using MlpSmemStandalone = MlpSmem<kMlpNbMax, kMlpStandaloneStages>;

__global__ void __launch_bounds__(kMlpThreads, 1)
    k_mlp_bf16(const MlpDesc M, const uint8_t* __restrict__ tiles, const float* __restrict__ f32,
               const float* __restrict__ x, int n, float* __restrict__ out) {
  extern __shared__ __align__(1024) char sm_raw[];
  __shared__ MlpCtx ctx;
  char* sm = align1024_shared(sm_raw);
  mlp_ctx_init(&ctx);
  const int n_batches = (n + kMlpNbMax - 1) / kMlpNbMax;
  for (int b = blockIdx.x; b < n_batches; b += gridDim.x) {
    const int b0 = b * kMlpNbMax;
    const int nb = min(kMlpNbMax, n - b0);
    if (!mlp_eval_bf16<kMlpNbMax, kMlpStandaloneStages>(M, tiles, f32, x + (size_t)b0 * M.d, M.d, nb, out + b0,
                                                         sm, &ctx))
      for (int r = threadIdx.x; r < nb; r += blockDim.x) out[b0 + r] = __int_as_float(0x7fffffff);
  }
  mlp_ctx_free(&ctx);
}

// The FP32-accurate tensor-core variant (three BF16 planes), batches of 32.
constexpr int kMlpSplitNb = 32;
using MlpSmemSplit = MlpSmem<kMlpSplitNb, kMlpStandaloneStages, 3>;

__global__ void __launch_bounds__(kMlpThreads, 1)
    k_mlp_split3(const MlpDesc M, const uint8_t* __restrict__ tiles, const float* __restrict__ f32,
                 const float* __restrict__ x, int n, float* __restrict__ out) {
  extern __shared__ __align__(1024) char sm_raw[];
  __shared__ MlpCtx ctx;
  char* sm = align1024_shared(sm_raw);
  mlp_ctx_init(&ctx);
  const int n_batches = (n + kMlpSplitNb - 1) / kMlpSplitNb;
  for (int b = blockIdx.x; b < n_batches; b += gridDim.x) {
    const int b0 = b * kMlpSplitNb;
    const int nb = min(kMlpSplitNb, n - b0);
    if (!mlp_eval_bf16<kMlpSplitNb, kMlpStandaloneStages, 3>(M, tiles, f32, x + (size_t)b0 * M.d, M.d, nb,
                                                              out + b0, sm, &ctx))
      for (int r = threadIdx.x; r < nb; r += blockDim.x) out[b0 + r] = __int_as_float(0x7fffffff);
  }
  mlp_ctx_free(&ctx);
}

// The evaluators split over a cluster of C CTAs (ns_mlp_cluster.cuh): each
// cluster evaluates batches of NB candidates, grid-strided over clusters;
// CTA 0 sums the partial chi^2.
template <int NB, int P>
__global__ void __launch_bounds__(kMlpThreads, 1)
    k_mlp_cl(const MlpDesc M, const uint8_t* __restrict__ tiles, const float* __restrict__ f32,
             const float* __restrict__ x, int n, float* __restrict__ out) {
  extern __shared__ __align__(1024) char sm_raw[];
  __shared__ MlpCtx ctx;
  __shared__ ClusterMail mail;
  char* sm = align1024_shared(sm_raw);
  const unsigned C = cl_size(), rank = cl_rank();
  mlp_ctx_init(&ctx);
  cl_sync();  // every CTA's barriers are set up before any remote arrive
  const int n_clusters = (int)(gridDim.x / C), cid = (int)(blockIdx.x / C);
  const int n_batches = (n + NB - 1) / NB;
  for (int b = cid; b < n_batches; b += n_clusters) {
    const int b0 = b * NB;
    const int nb = min(NB, n - b0);
    const XIn X{x + (size_t)b0 * M.d, nullptr, nullptr, M.d};
    mlp_eval_bf16_cl<NB, kMlpStandaloneStages, P>(M, tiles, f32, X, nb, sm, &ctx, &mail, C, rank);
    cl_sync();
    if (rank == 0 && !mlp_cl_collect(&mail, C, nb, out + b0, nullptr))
      for (int r = threadIdx.x; r < nb; r += blockDim.x) out[b0 + r] = __int_as_float(0x7fffffff);
    cl_sync();  // the mailbox is free for the next batch
  }
  mlp_cl_drain(&ctx);
  cl_sync();
  mlp_ctx_free(&ctx);
}

// The 16-bit variant (two BF16 planes), batches of 64.
constexpr int kMlpX2Nb = 64;
using MlpSmemX2 = MlpSmem<kMlpX2Nb, kMlpStandaloneStages, 2>;

__global__ void __launch_bounds__(kMlpThreads, 1)
    k_mlp_x2(const MlpDesc M, const uint8_t* __restrict__ tiles, const float* __restrict__ f32,
             const float* __restrict__ x, int n, float* __restrict__ out) {
  extern __shared__ __align__(1024) char sm_raw[];
  __shared__ MlpCtx ctx;
  char* sm = align1024_shared(sm_raw);
  mlp_ctx_init(&ctx);
  const int n_batches = (n + kMlpX2Nb - 1) / kMlpX2Nb;
  for (int b = blockIdx.x; b < n_batches; b += gridDim.x) {
    const int b0 = b * kMlpX2Nb;
    const int nb = min(kMlpX2Nb, n - b0);
    if (!mlp_eval_bf16<kMlpX2Nb, kMlpStandaloneStages, 2>(M, tiles, f32, x + (size_t)b0 * M.d, M.d, nb, out + b0, sm,
                                                           &ctx))
      for (int r = threadIdx.x; r < nb; r += blockDim.x) out[b0 + r] = __int_as_float(0x7fffffff);
  }
  mlp_ctx_free(&ctx);
}

__global__ void __launch_bounds__(256, 1)
    k_mlp_f32(const MlpDesc M, const float* __restrict__ f32, const float* __restrict__ x, int n,
              float* __restrict__ out) {
  extern __shared__ __align__(16) float act[];
  const int b0 = blockIdx.x * kMlpF32NbWide;
  const int nb = min(kMlpF32NbWide, n - b0);
  mlp_eval_f32<kMlpF32NbWide>(M, f32, x + (size_t)b0 * M.d, M.d, nb, out + b0, act);
}

int round_up(int v, int q) { return (v + q - 1) / q * q; }

// Host description of the image; false (with a message) if the network does
// not fit the evaluators.
bool make_desc(const ns_likelihood& L, const double* lo, const double* hi, int d, MlpDesc* M, std::string* msg) {
  std::memset(M, 0, sizeof(*M));
  if (L.kind != NS_LIK_MLP || L.n_layers < 1 || L.n_layers > kMlpMaxLayers || !L.widths || !L.weights ||
      !L.biases || !L.data || !L.sigma_out) {
    *msg = "MLP likelihood needs 1..8 layers with widths, weights, biases, data and sigma_out";
    return false;
  }
  if (L.widths[0] != d || d > kMaxDim) {
    *msg = "MLP widths[0] must equal d (<= 32)";
    return false;
  }
  M->n_layers = L.n_layers;
  M->d = d;
  for (int i = 0; i < d; ++i) {
    M->lo[i] = (float)lo[i];
    M->span[i] = (float)(hi[i] - lo[i]);
  }
  int tiles = 0;
  long long f = 0;
  for (int l = 0; l < L.n_layers; ++l) {
    const int in = L.widths[l], out = L.widths[l + 1];
    if (in < 1 || out < 1 || out > 65536) {
      *msg = "MLP widths must be positive (and <= 65536)";
      return false;
    }
    M->in[l] = in;
    M->out[l] = out;
    M->kpad[l] = round_up(in, 64);
    M->mpad[l] = round_up(out, 128);
    if (M->kpad[l] > kMlpMaxK || (l + 1 < L.n_layers && M->mpad[l] > kMlpMaxK)) {
      *msg = "MLP layers wider than 512 are supported only as the output layer";
      return false;
    }
    M->tile0[l] = tiles;
    tiles += (M->mpad[l] / 128) * (M->kpad[l] / 64);
    M->bias0[l] = f;
    f += M->mpad[l];
  }
  const int last = L.n_layers - 1;
  M->data0 = f;
  f += M->mpad[last];
  M->isig0 = f;
  f += M->mpad[last];
  // FP32 weights stored as BF16 when every weight is a BF16 value (low 16 bits zero)
  long long n_w = 0;
  for (int l = 0; l < L.n_layers; ++l) n_w += (long long)M->in[l] * M->out[l];
  M->w_bf16 = 1;
  for (long long i = 0; i < n_w && M->w_bf16; ++i) {
    uint32_t u;
    std::memcpy(&u, L.weights + i, 4);
    if ((u & 0xFFFFu) != 0u || !std::isfinite(L.weights[i])) M->w_bf16 = 0;
  }
  for (int l = 0; l < L.n_layers; ++l) {
    M->w32_0[l] = f;
    const long long cnt = (long long)M->in[l] * M->out[l];
    f += M->w_bf16 ? (cnt + 1) / 2 : cnt;
  }
  M->n_tiles = tiles;
  M->tile_bytes = (long long)tiles * kMlpTileBytes;
  M->f32_floats = f;
  for (int k = 0; k < L.widths[last + 1]; ++k)
    if (!(L.sigma_out[k] > 0.f) || !std::isfinite(L.sigma_out[k]) || !std::isfinite(L.data[k])) {
      *msg = "MLP sigma_out must be positive and data finite";
      return false;
    }
  return true;
}

uint16_t bf16_bits(float v) {
  uint32_t u;
  std::memcpy(&u, &v, 4);
  const uint32_t rounding = ((u >> 16) & 1u) + 0x7FFFu;
  return (uint16_t)((u + rounding) >> 16);
}

std::string g_mlp_err;

// Descriptions of the images packed by ns_mlp_pack, by image address: a batch
// evaluation then needs no pass over the weights on the host.
std::mutex g_desc_mu;
std::unordered_map<const void*, MlpDesc> g_desc;

bool same_widths(const ns_likelihood& L, const MlpDesc& M) {
  if (L.n_layers != M.n_layers || !L.widths) return false;
  for (int l = 0; l < M.n_layers; ++l)
    if (L.widths[l] != M.in[l] || L.widths[l + 1] != M.out[l]) return false;
  return true;
}

}  // namespace

// Shared with ns_lib.cu (validation of MLP runs).
bool ns_mlp_make_desc(const ns_likelihood& L, const double* lo, const double* hi, int d, MlpDesc* M,
                      std::string* msg) {
  return make_desc(L, lo, hi, d, M, msg);
}

void ns_mlp_pack_host(const ns_likelihood& L, const MlpDesc& M, std::vector<uint8_t>& img) {
  img.assign((size_t)M.tile_bytes + sizeof(float) * (size_t)M.f32_floats, 0);
  const float* W = L.weights;
  const float* Bv = L.biases;
  for (int l = 0; l < M.n_layers; ++l) {
    const int in = M.in[l], out = M.out[l], MT = M.mpad[l] / 128, KB = M.kpad[l] / 64;
    for (int t = 0; t < MT; ++t)
      for (int kb = 0; kb < KB; ++kb) {
        uint8_t* tile = img.data() + (size_t)(M.tile0[l] + t * KB + kb) * kMlpTileBytes;
        for (int r = 0; r < 128; ++r)
          for (int k = 0; k < 64; ++k) {
            const int f = t * 128 + r, i = kb * 64 + k;
            const float v = (f < out && i < in) ? W[(size_t)f * in + i] : 0.f;
            const uint16_t b = bf16_bits(v);
            std::memcpy(tile + sw128_offset(r, k), &b, 2);
          }
      }
    float* f32 = reinterpret_cast<float*>(img.data() + M.tile_bytes);
    for (int o = 0; o < out; ++o) f32[M.bias0[l] + o] = Bv[o];
    uint16_t* w16 = reinterpret_cast<uint16_t*>(f32 + M.w32_0[l]);
    for (int o = 0; o < out; ++o)  // transposed: [in][out]
      for (int i = 0; i < in; ++i) {
        const float w = W[(size_t)o * in + i];
        if (M.w_bf16) {
          uint32_t u;
          std::memcpy(&u, &w, 4);
          w16[(size_t)i * out + o] = (uint16_t)(u >> 16);
        } else {
          f32[M.w32_0[l] + (size_t)i * out + o] = w;
        }
      }
    W += (size_t)in * out;
    Bv += out;
  }
  float* f32 = reinterpret_cast<float*>(img.data() + M.tile_bytes);
  const int last = M.n_layers - 1;
  for (int k = 0; k < M.out[last]; ++k) {
    f32[M.data0 + k] = L.data[k];
    f32[M.isig0 + k] = 1.f / L.sigma_out[k];
  }
}

cudaError_t ns_mlp_launch(const MlpDesc& M, const void* image, int n, const float* x, float* logl, int precision,
                          cudaStream_t s) {
  const uint8_t* tiles = static_cast<const uint8_t*>(image);
  const float* f32 = reinterpret_cast<const float*>(tiles + M.tile_bytes);
  if (precision == 3) {
    const int smem = MlpSmemX2::kBytes + 1024;
    cudaError_t e = cudaFuncSetAttribute(k_mlp_x2, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    int dev = 0, n_sm = 1;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const int n_batches = (n + kMlpX2Nb - 1) / kMlpX2Nb;
    k_mlp_x2<<<std::min(n_batches, n_sm), kMlpThreads, smem, s>>>(M, tiles, f32, x, n, logl);
  } else if (precision == 2) {
    const int smem = MlpSmemSplit::kBytes + 1024;
    cudaError_t e = cudaFuncSetAttribute(k_mlp_split3, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    int dev = 0, n_sm = 1;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const int n_batches = (n + kMlpSplitNb - 1) / kMlpSplitNb;
    k_mlp_split3<<<std::min(n_batches, n_sm), kMlpThreads, smem, s>>>(M, tiles, f32, x, n, logl);
  } else if (precision == 1) {
    const int smem = MlpSmemStandalone::kBytes + 1024;
    cudaError_t e = cudaFuncSetAttribute(k_mlp_bf16, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    int dev = 0, n_sm = 1;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const int n_batches = (n + kMlpNbMax - 1) / kMlpNbMax;
    k_mlp_bf16<<<std::min(n_batches, n_sm), kMlpThreads, smem, s>>>(M, tiles, f32, x, n, logl);
  } else {
    const int smem = (int)mlp_f32_act_bytes(kMlpF32NbWide);
    cudaError_t e = cudaFuncSetAttribute(k_mlp_f32, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    k_mlp_f32<<<(n + kMlpF32NbWide - 1) / kMlpF32NbWide, 256, smem, s>>>(M, f32, x, n, logl);
  }
  return cudaGetLastError();
}

// The cluster-split evaluators: `cluster` CTAs per batch, at most one
// cluster per `cluster` SMs.
cudaError_t ns_mlp_launch_cluster(const MlpDesc& M, const void* image, int n, const float* x, float* logl,
                                  int precision, int cluster, cudaStream_t s) {
  const uint8_t* tiles = static_cast<const uint8_t*>(image);
  const float* f32 = reinterpret_cast<const float*>(tiles + M.tile_bytes);
  int dev = 0, n_sm = 1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int nb = precision == 2 ? kMlpSplitNb : kMlpNbMax;
  const int n_batches = (n + nb - 1) / nb;
  const int n_clusters = std::max(1, std::min(n_batches, n_sm / cluster));
  const int smem = (precision == 2 ? (int)MlpSmemSplit::kBytes : (int)MlpSmemStandalone::kBytes) + 1024;
  auto kern = precision == 2 ? k_mlp_cl<kMlpSplitNb, 3> : k_mlp_cl<kMlpNbMax, 1>;
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(n_clusters * cluster), 1, 1);
  cfg.blockDim = dim3(kMlpThreads, 1, 1);
  cfg.dynamicSmemBytes = (size_t)smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)cluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, M, tiles, f32, x, n, logl);
}

extern "C" {

size_t ns_mlp_image_bytes(const ns_likelihood* lik, int d) {
  if (!lik) return 0;
  MlpDesc M;
  std::string msg;
  std::vector<double> lo(d > 0 ? d : 1, 0.0), hi(d > 0 ? d : 1, 1.0);
  if (!make_desc(*lik, lo.data(), hi.data(), d, &M, &msg)) return 0;
  return (size_t)M.tile_bytes + sizeof(float) * (size_t)M.f32_floats;
}

ns_status ns_mlp_pack(const ns_likelihood* lik, int d, void* image, void* stream) {
  if (!lik || !image) return NS_ERR_ARG;
  MlpDesc M;
  std::string msg;
  std::vector<double> lo(d > 0 ? d : 1, 0.0), hi(d > 0 ? d : 1, 1.0);
  if (!make_desc(*lik, lo.data(), hi.data(), d, &M, &msg)) {
    g_mlp_err = msg;
    return NS_ERR_ARG;
  }
  if (reinterpret_cast<uintptr_t>(image) % 1024 != 0) {
    g_mlp_err = "ns_mlp_pack: image must be 1024-byte aligned";
    return NS_ERR_ARG;
  }
  std::vector<uint8_t> img;
  ns_mlp_pack_host(*lik, M, img);
  cudaError_t e = cudaMemcpyAsync(image, img.data(), img.size(), cudaMemcpyHostToDevice, (cudaStream_t)stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e == cudaSuccess) {
    std::lock_guard<std::mutex> lk(g_desc_mu);
    g_desc[image] = M;
  }
  return e == cudaSuccess ? NS_OK : NS_ERR_CUDA;
}

ns_status ns_mlp_loglike(const ns_likelihood* lik, const double* lo, const double* hi, int d, const void* image, int n,
                         const float* x, float* logl, int precision, void* stream) {
  if (!lik || !lo || !hi || !image || n < 0 || (n > 0 && (!x || !logl)) || precision < 0 || precision > 3)
    return NS_ERR_ARG;
  MlpDesc M;
  bool cached = false;
  {
    std::lock_guard<std::mutex> lk(g_desc_mu);
    auto it = g_desc.find(image);
    if (it != g_desc.end() && it->second.d == d && same_widths(*lik, it->second)) {
      M = it->second;
      cached = true;
    }
  }
  if (cached) {
    for (int i = 0; i < d; ++i) {
      if (!(lo[i] < hi[i]) || !std::isfinite(lo[i]) || !std::isfinite(hi[i])) return NS_ERR_ARG;
      M.lo[i] = (float)lo[i];
      M.span[i] = (float)(hi[i] - lo[i]);
    }
  } else {
    std::string msg;
    if (!make_desc(*lik, lo, hi, d, &M, &msg)) {
      g_mlp_err = msg;
      return NS_ERR_ARG;
    }
  }
  if (precision >= 2 && !M.w_bf16) {
    g_mlp_err = "ns_mlp_loglike: precision 2 and 3 need weights that are BF16 values";
    return NS_ERR_ARG;
  }
  if (n == 0) return NS_OK;
  return ns_mlp_launch(M, image, n, x, logl, precision, (cudaStream_t)stream) == cudaSuccess ? NS_OK
                                                                                           : NS_ERR_CUDA;
}

ns_status ns_mlp_loglike_cluster(const ns_likelihood* lik, const double* lo, const double* hi, int d,
                                 const void* image, int n, const float* x, float* logl, int precision, int cluster,
                                 void* stream) {
  if (!lik || !lo || !hi || !image || n < 0 || (n > 0 && (!x || !logl)) || precision < 1 || precision > 2 ||
      (cluster != 2 && cluster != 4))
    return NS_ERR_ARG;
  MlpDesc M;
  std::string msg;
  if (!make_desc(*lik, lo, hi, d, &M, &msg)) {
    g_mlp_err = msg;
    return NS_ERR_ARG;
  }
  if (precision == 2 && !M.w_bf16) {
    g_mlp_err = "ns_mlp_loglike_cluster: precision 2 needs weights that are BF16 values";
    return NS_ERR_ARG;
  }
  if (!mlp_cluster_fits(M, cluster)) {
    g_mlp_err = "ns_mlp_loglike_cluster: every layer's 128-row tile count must be a multiple of the cluster size";
    return NS_ERR_ARG;
  }
  if (n == 0) return NS_OK;
  return ns_mlp_launch_cluster(M, image, n, x, logl, precision, cluster, (cudaStream_t)stream) == cudaSuccess
             ? NS_OK
             : NS_ERR_CUDA;
}

}  // extern "C"
