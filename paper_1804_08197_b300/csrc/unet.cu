// Learned reconstruction: a 3-level residual U-Net (32 / 64 / 128 channels,
// 3x3 convolutions, BF16 weights and activations, FP32 accumulation) that
// turns a half-resolution, coarser-step render into a full-resolution image:
// out = bilinear_2x(in) + pixel_shuffle_2x(head(unet(in))). Trained on the
// GPU with the project's own forward and backward kernels (Adam, MSE), used
// with the plain full-rate render as fallback and yardstick (PSNR).
//
// Layers (h x w = half-resolution size, multiple of 4):
//   c1a 16->32, c1b 32->32 (= e1)               at h x w      (input: RGBA + 12 zero channels)
//   pool, c2a 32->64, c2b 64->64 (= e2)          at h/2 x w/2
//   pool, c3a 64->128, c3b 128->128              at h/4 x w/4
//   up, concat [up 128 | e2 64], d2a 192->64, d2b 64->64   at h/2 x w/2
//   up, concat [up 64 | e1 32],  d1a 96->32,  d1b 32->32   at h x w
//   head 32->16 (no ReLU, FP32) -> pixel shuffle -> 4 channels at 2h x 2w
#include <math.h>
#include <algorithm>
#include <string.h>

#include <string>
#include <vector>

#include "internal.h"
#include "unet_gemm.cuh"
#include "unet_tc.cuh"
#include "unet_ws.cuh"
#include "unet_wgrad_tc.cuh"

using namespace sg;
using namespace sg::nn;

namespace {

constexpr int kLayers = 11;
enum { C1A, C1B, C2A, C2B, C3A, C3B, D2A, D2B, D1A, D1B, HEAD };
const int kCin[kLayers] = {16, 32, 32, 64, 64, 128, 192, 64, 96, 32, 32};
const int kCout[kLayers] = {32, 32, 64, 64, 128, 128, 64, 64, 32, 32, 16};
constexpr int kWgradSplits = 32;      // pixel splits of the mma.sync weight gradient
constexpr int kWgradMaxSplits = 128;  // pixel splits of the tcgen05 one (partials permitting)

// ------------------------------------------------------------------ elementwise kernels

template <typename F>
__global__ void k_each(int64_t n, F f) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) f(i);
}

unsigned blocks_for(int64_t n) {
  int64_t b = (n + 255) / 256;
  if (b > 148 * 64) b = 148 * 64;
  return (unsigned)(b < 1 ? 1 : b);
}

template <typename F>
cudaError_t each(int64_t n, cudaStream_t s, F f) {
  if (n <= 0) return cudaSuccess;
  k_each<<<blocks_for(n), 256, 0, s>>>(n, f);
  return cudaGetLastError();
}

// sum over i < n of f(i) into *out (+=): grid-stride with whole warps, then
// one atomic per warp
template <typename F>
__global__ void k_sum(int64_t n, F f, float* out) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t n_round = (n + 31) / 32 * 32;
  float v = 0.f;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_round; i += stride)
    if (i < n) v += f(i);
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(out, v);
}

template <typename F>
cudaError_t sum(int64_t n, float* out, cudaStream_t s, F f) {
  if (n <= 0) return cudaSuccess;
  k_sum<<<blocks_for(n), 256, 0, s>>>(n, f, out);
  return cudaGetLastError();
}

struct Crops {
  const float* ptr[64];  // per batch element, FP32 RGBA rows
  int64_t pitch;         // floats between rows
};

struct OutPtrs {
  float* p[64];
};
struct ConstOutPtrs {
  const float* p[64];
};

// per-item kernels with 32-bit indices (every count here is < 2^31), one
// item = one pixel or one pixel x 8-channel chunk, 16-byte accesses
template <typename F>
__global__ void k_each32(int n, F f) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) f(i);
}
template <typename F>
cudaError_t each32(int64_t n, cudaStream_t s, F f) {
  if (n <= 0) return cudaSuccess;
  k_each32<<<blocks_for(n), 256, 0, s>>>((int)n, f);
  return cudaGetLastError();
}

struct Pix {  // pixel index -> (n, y, x) of an N x H x W grid
  int n, y, x;
  __device__ Pix(int i, int H, int W) {
    const int hw = H * W;
    n = i / hw;
    const int r = i - n * hw;
    y = r / W;
    x = r - y * W;
  }
};

__device__ __forceinline__ void bf8_to_f(const uint4& v, float* f) {
  const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&v);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float2 t = __bfloat1622float2(h[i]);
    f[2 * i] = t.x;
    f[2 * i + 1] = t.y;
  }
}
__device__ __forceinline__ uint4 f_to_bf8(const float* f) {
  uint4 v;
  __nv_bfloat162* h = reinterpret_cast<__nv_bfloat162*>(&v);
#pragma unroll
  for (int i = 0; i < 4; ++i) h[i] = __floats2bfloat162_rn(f[2 * i], f[2 * i + 1]);
  return v;
}

// dst[q, doff + c] = mean of the 2x2 children of src (BF16, channels in chunks of 8)
cudaError_t pool_fwd(const bf16* src, int sstride, int soff, bf16* dst, int dstride, int doff, int C, int N, int h,
                     int w, cudaStream_t s) {
  const int h2 = h / 2, w2 = w / 2, nc = C / 8;
  return each32((int64_t)N * h2 * w2 * nc, s, [=] __device__(int i) {
    const int q = i / nc, c = (i - q * nc) * 8;
    const Pix P(q, h2, w2);
    float acc[8] = {0, 0, 0, 0, 0, 0, 0, 0}, f[8];
#pragma unroll
    for (int dy = 0; dy < 2; ++dy)
#pragma unroll
      for (int dx = 0; dx < 2; ++dx) {
        bf8_to_f(*reinterpret_cast<const uint4*>(src + ((size_t)(P.n * h + 2 * P.y + dy) * w + 2 * P.x + dx) * sstride +
                                                 soff + c),
                 f);
#pragma unroll
        for (int k = 0; k < 8; ++k) acc[k] += f[k];
      }
#pragma unroll
    for (int k = 0; k < 8; ++k) acc[k] *= 0.25f;
    *reinterpret_cast<uint4*>(dst + (size_t)q * dstride + doff + c) = f_to_bf8(acc);
  });
}

// dst (2h x 2w) [q, doff + c] = src (h x w) nearest
cudaError_t up_fwd(const bf16* src, int sstride, bf16* dst, int dstride, int doff, int C, int N, int h, int w,
                   cudaStream_t s) {
  const int H = 2 * h, W = 2 * w, nc = C / 8;
  return each32((int64_t)N * H * W * nc, s, [=] __device__(int i) {
    const int q = i / nc, c = (i - q * nc) * 8;
    const Pix P(q, H, W);
    *reinterpret_cast<uint4*>(dst + (size_t)q * dstride + doff + c) =
        *reinterpret_cast<const uint4*>(src + ((size_t)(P.n * h + P.y / 2) * w + P.x / 2) * sstride + c);
  });
}

// gradient of nearest upsampling: dst (h x w) += sum of the 4 children in src (2h x 2w, FP32)
cudaError_t up_bwd(const float* src, int sstride, float* dst, int dstride, int C, int N, int h, int w,
                   cudaStream_t s) {
  const int nc = C / 4;
  return each32((int64_t)N * h * w * nc, s, [=] __device__(int i) {
    const int q = i / nc, c = (i - q * nc) * 4;
    const Pix P(q, h, w);
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int dy = 0; dy < 2; ++dy)
#pragma unroll
      for (int dx = 0; dx < 2; ++dx) {
        const float4 v = *reinterpret_cast<const float4*>(
            src + ((size_t)(P.n * 2 * h + 2 * P.y + dy) * (2 * w) + 2 * P.x + dx) * sstride + c);
        acc.x += v.x; acc.y += v.y; acc.z += v.z; acc.w += v.w;
      }
    float4* o = reinterpret_cast<float4*>(dst + (size_t)q * dstride + c);
    float4 t = *o;
    t.x += acc.x; t.y += acc.y; t.z += acc.z; t.w += acc.w;
    *o = t;
  });
}

// gradient of 2x2 average pooling: dst (2h x 2w)[., doff + c] += src (h x w) / 4 (FP32)
cudaError_t pool_bwd(const float* src, int sstride, float* dst, int dstride, int doff, int C, int N, int h, int w,
                     cudaStream_t s) {
  const int H = 2 * h, W = 2 * w, nc = C / 4;
  return each32((int64_t)N * H * W * nc, s, [=] __device__(int i) {
    const int q = i / nc, c = (i - q * nc) * 4;
    const Pix P(q, H, W);
    const float4 v = *reinterpret_cast<const float4*>(src + ((size_t)(P.n * h + P.y / 2) * w + P.x / 2) * sstride + c);
    float4* o = reinterpret_cast<float4*>(dst + (size_t)q * dstride + doff + c);
    float4 t = *o;
    t.x += 0.25f * v.x; t.y += 0.25f * v.y; t.z += 0.25f * v.z; t.w += 0.25f * v.w;
    *o = t;
  });
}

}  // namespace

struct sg_unet {
  int max_n = 0, max_h = 0, max_w = 0;
  int tc = 4;                 // convolutions: 4 persistent tcgen05, 3/2 tcgen05 halo reuse, 1 implicit GEMM, 0 mma.sync
  uint32_t* d_err = nullptr;  // set by a tcgen05 kernel whose bounded wait gave up
  int n = 0, h = 0, w = 0;  // shape of the last forward
  int64_t nparam = 0;
  int64_t woff[kLayers], boff[kLayers];
  float* d_param = nullptr;   // FP32 master weights + biases
  float* d_grad = nullptr;
  float* d_m = nullptr;
  float* d_v = nullptr;
  bf16* d_w = nullptr;        // BF16 copy of the weights [Cout][9][Cin]
  bf16* d_wt = nullptr;       // flipped / transposed for the input gradient [Cin][9][Cout]
  int64_t step = 0;
  // activations (BF16) and their gradients (FP32), NHWC
  bf16 *in16 = nullptr, *a1 = nullptr, *cat1 = nullptr, *p1 = nullptr, *a2 = nullptr, *cat2 = nullptr,
       *p2 = nullptr, *a3 = nullptr, *b3 = nullptr, *a4 = nullptr, *d2 = nullptr, *a5 = nullptr, *d1 = nullptr;
  float* head = nullptr;      // [N][h][w][16] FP32
  float *g_a1 = nullptr, *g_cat1 = nullptr, *g_p1 = nullptr, *g_a2 = nullptr, *g_cat2 = nullptr, *g_p2 = nullptr,
        *g_a3 = nullptr, *g_b3 = nullptr, *g_a4 = nullptr, *g_d2 = nullptr, *g_a5 = nullptr, *g_d1 = nullptr,
        *g_head = nullptr;
  bf16* dz = nullptr;         // masked gradient staging (largest layer)
  float* dw_part = nullptr;   // [S][9][Cout][Cin], room for kWgradSplits x 9 x 128 x 192
  float* db_part = nullptr;   // [S][Cout], room for kWgradMaxSplits x 128
  // tcgen05 weight gradients: transposed operands, grown on demand
  uint16_t* wg_dzT = nullptr;
  bool dzT_ready = false;  // wg_dzT holds the current layer's masked gradient
  uint16_t* wg_xT3 = nullptr;
  size_t wg_dzT_bytes = 0, wg_xT3_bytes = 0;
  float* d_loss = nullptr;    // [2]
  // sg_render_learned: the reduced render of both eyes and (judging) the
  // full-rate render, grown on demand; squared-error sums of the judge
  float* lrn_half = nullptr;
  float* lrn_full = nullptr;
  size_t lrn_half_bytes = 0, lrn_full_bytes = 0;
  float* lrn_acc = nullptr;   // [2]
  Crops in_crops;
  std::vector<void*> allocs;
};

namespace {

cudaError_t alloc(sg_unet* u, void** p, size_t bytes) {
  cudaError_t e = cudaMalloc(p, bytes < 16 ? 16 : bytes);
  if (e == cudaSuccess) u->allocs.push_back(*p);
  return e;
}

void free_unet(sg_unet* u) {
  for (void* p : u->allocs) cudaFree(p);
  cudaFree(u->wg_dzT);
  cudaFree(u->wg_xT3);
  cudaFree(u->lrn_half);
  cudaFree(u->lrn_full);
  cudaFree(u->lrn_acc);
  delete u;
}

// ---- conv launch helpers

template <int BN>
cudaError_t conv_bn(const ConvArgs& a, cudaStream_t s) {
  const int64_t M = (int64_t)a.N * a.H * a.W;
  dim3 grid((unsigned)((M + kConvBM - 1) / kConvBM), a.Cout / BN);
  if (a.Cin % 32 == 0)
    k_conv3x3<BN, 2><<<grid, 128, 0, s>>>(a);
  else
    k_conv3x3<BN, 1><<<grid, 128, 0, s>>>(a);
  return cudaGetLastError();
}

template <int BN>
cudaError_t conv_tc(const ConvArgs& a, uint32_t* err, cudaStream_t s) {
  const int64_t M = (int64_t)a.N * a.H * a.W;
  const int smem = kTcStages * (kTcBM + BN) * kTcBK * 2;
  static bool configured = false;  // per template instance, set once on first use
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(k_conv3x3_tc<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  dim3 grid((unsigned)((M + kTcBM - 1) / kTcBM), a.Cout / BN);
  k_conv3x3_tc<BN><<<grid, 128, smem, s>>>(a, err);
  return cudaGetLastError();
}

#ifndef SG_HALO_ROWS
#define SG_HALO_ROWS 4
#endif

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// against the driver library); looked up once
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_tiled() {
  static EncodeTiledFn fn = nullptr;
  static bool looked = false;
  if (!looked) {
    looked = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

// Tensor map of a convolution input (NHWC BF16, in_stride channels per
// pixel): boxes of cw channels x 130 pixels x `rows` rows of one image,
// written to shared memory with the given swizzle.
cudaError_t input_tensor_map(const ConvArgs& a, CUtensorMap* m, int rows = 1, int cw = 8,
                             CUtensorMapSwizzle swz = CU_TENSOR_MAP_SWIZZLE_NONE) {
  EncodeTiledFn fn = encode_tiled();
  if (!fn) return cudaErrorNotSupported;
  if ((reinterpret_cast<uintptr_t>(a.in) & 15) || (a.in_stride % 8) || (a.in_off % 8)) return cudaErrorInvalidValue;
  const cuuint64_t dims[4] = {(cuuint64_t)a.in_stride, (cuuint64_t)a.W, (cuuint64_t)a.H, (cuuint64_t)a.N};
  const cuuint64_t strides[3] = {(cuuint64_t)a.in_stride * 2, (cuuint64_t)a.W * a.in_stride * 2,
                                 (cuuint64_t)a.H * a.W * a.in_stride * 2};
  const cuuint32_t box[4] = {(cuuint32_t)cw, 130, (cuuint32_t)rows, 1}, estr[4] = {1, 1, 1, 1};
  const CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<bf16*>(a.in), dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, swz, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// Tensor map of convolution weights ([Cout][9 Cin] BF16): boxes of cw input
// channels of one tap x bn output channels, written with the given swizzle.
cudaError_t weight_tensor_map(const ConvArgs& a, int bn, int cw, CUtensorMapSwizzle swz, CUtensorMap* m) {
  EncodeTiledFn fn = encode_tiled();
  if (!fn) return cudaErrorNotSupported;
  if ((reinterpret_cast<uintptr_t>(a.wt) & 15) || (a.Cin % 8) || bn > 256) return cudaErrorInvalidValue;
  const cuuint64_t dims[2] = {(cuuint64_t)9 * a.Cin, (cuuint64_t)a.Cout};
  const cuuint64_t strides[1] = {(cuuint64_t)9 * a.Cin * 2};
  const cuuint32_t box[2] = {(cuuint32_t)cw, (cuuint32_t)bn}, estr[2] = {1, 1};
  const CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<bf16*>(a.wt), dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, swz, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// streaming multiprocessors of the current device (queried once per device)
int sm_count() {
  static int n[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 1;
  if (!n[dev] && cudaDeviceGetAttribute(&n[dev], cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) n[dev] = 0;
  return n[dev] > 0 ? n[dev] : 1;
}

// persistent warp-specialised convolution: one CTA per SM, as many ring
// stages as fit in about 220 KB of shared memory
template <int BN, int R, int CW>
cudaError_t conv_ws(const ConvArgs& a, uint32_t* err, cudaStream_t s, const HeadOut* head_out = nullptr) {
  using S = WsShape<BN, R, CW>;
  // pooling needs whole 2 x 2 windows in every row pair a warp takes
  if (a.pool_out && (R % 4 || a.H % 2 || a.W % 2)) return cudaErrorInvalidValue;
  if (a.Cout > kWsMaxCout) return cudaErrorInvalidValue;
  // shared memory: the ring of stages, [the resident weights,] the eight
  // epilogue warps' staging rows, and room to align the ring to 1024 bytes.
  // With one output-channel block every tile multiplies the same weights:
  // they stay resident when the ring still gets two input stages.
  const int avail = 220 * 1024 - 1024 - 8 * S::kOut;
  const int wbytes = (a.Cin / CW * 9 * S::kBlk + 1023) / 1024 * 1024;
  const int wres = (a.Cout == BN && (avail - wbytes) / S::kA >= 2) ? 1 : 0;
  const int stages = wres ? std::min(kWsMaxStages, (avail - wbytes) / S::kA) : std::min(kWsMaxStages, avail / S::kStage);
  const int smem = (wres ? stages * S::kA + wbytes : stages * S::kStage) + 8 * S::kOut + 1024;
  // (the kernel's static shared memory, the bias, barriers and flags, takes the last 2 KB)
  if (stages < 1 || smem > 225 * 1024) return cudaErrorInvalidValue;
  static int configured = 0;  // per template instance: the largest dynamic size allowed so far
  if (smem > configured) {
    cudaError_t e = cudaFuncSetAttribute(k_conv3x3_ws<BN, R, CW>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    configured = smem;
  }
  const CUtensorMapSwizzle swz = CW == 32 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_32B;
  CUtensorMap tin, twt;
  memset(&tin, 0, sizeof tin);
  memset(&twt, 0, sizeof twt);
  cudaError_t e = input_tensor_map(a, &tin, R + 2, CW, swz);
  if (e == cudaSuccess) e = weight_tensor_map(a, BN, CW, swz, &twt);
  if (e != cudaSuccess) return e;
  const int64_t nt = (int64_t)a.N * ((a.H + R - 1) / R) * ((a.W + 127) / 128) * (a.Cout / BN);
  const int grid = (int)std::min<int64_t>(nt, sm_count());
  if (grid < 1) return cudaSuccess;
  HeadOut ho;
  memset(&ho, 0, sizeof ho);
  if (head_out) ho = *head_out;
  k_conv3x3_ws<BN, R, CW><<<grid, kWsThreads, smem, s>>>(a, stages, wres, err, tin, twt, ho);
  return cudaGetLastError();
}

template <int BN, int R, int CC, bool TMA = false>
cudaError_t conv_halo(const ConvArgs& a, uint32_t* err, cudaStream_t s) {
  // two stages only where two CTAs still fit on an SM
  constexpr int kOne = halo_stage_bytes<BN, R, CC>();
#ifndef SG_HALO_STAGE2_LIMIT
#define SG_HALO_STAGE2_LIMIT (110 * 1024)
#endif
  const int stages = (a.Cin / CC > 1 && 2 * kOne <= SG_HALO_STAGE2_LIMIT) ? 2 : 1;
  const int smem = stages * kOne;
  static bool configured = false;  // per template instance, set once on first use
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(k_conv3x3_halo<BN, R, CC, TMA>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * kOne);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  CUtensorMap tmap;
  memset(&tmap, 0, sizeof tmap);
  if (TMA) {
    cudaError_t e = input_tensor_map(a, &tmap);
    if (e != cudaSuccess) return e;
  }
  dim3 grid((a.W + 127) / 128, a.N * ((a.H + R - 1) / R), a.Cout / BN);
  k_conv3x3_halo<BN, R, CC, TMA><<<grid, 128, smem, s>>>(a, stages, err, tmap);
  return cudaGetLastError();
}

template <int BN, bool TMA>
cudaError_t conv_halo_cc(const ConvArgs& a, uint32_t* err, cudaStream_t s) {
#ifndef SG_HALO_CC16_ONLY
  if (a.Cin % 32 == 0) return conv_halo<BN, SG_HALO_ROWS, 32, TMA>(a, err, s);
#endif
  return conv_halo<BN, SG_HALO_ROWS, 16, TMA>(a, err, s);
}

// mode: 0 mma.sync, 1 tcgen05 implicit GEMM, 2 tcgen05 with halo reuse,
// 3 the same with the input row segments staged by TMA, 4 persistent
// warp-specialised halo reuse (TMA ring, two TMEM accumulators)
cudaError_t conv(const ConvArgs& a, cudaStream_t s, uint32_t* tc_err = nullptr, int mode = 2,
                 const HeadOut* head_out = nullptr) {
  // pooled and upsampled copies come from the persistent kernel's epilogue only
  if ((a.pool_out || a.up_out) && !(tc_err && mode == 4 && a.Cin % 16 == 0 && a.Cout % 16 == 0 && !head_out))
    return cudaErrorInvalidValue;
  if (head_out) {
    // the network's output from the head's epilogue: persistent path, 16 channels
    if (!tc_err || mode != 4 || a.Cout != 16 || a.Cin % 16 || a.out || a.out_f32) return cudaErrorInvalidValue;
    return a.Cin % 32 == 0 ? conv_ws<16, 8, 32>(a, tc_err, s, head_out) : conv_ws<16, 8, 16>(a, tc_err, s, head_out);
  }
  if (tc_err && mode == 4 && a.Cin % 16 == 0 && a.Cout % 16 == 0) {
    if (a.Cin % 32 == 0) {
      if (a.Cout % 64 == 0) return conv_ws<64, 4, 32>(a, tc_err, s);
      if (a.Cout % 32 == 0) return conv_ws<32, 8, 32>(a, tc_err, s);
      return conv_ws<16, 8, 32>(a, tc_err, s);
    }
    if (a.Cout % 64 == 0) return conv_ws<64, 4, 16>(a, tc_err, s);
    if (a.Cout % 32 == 0) return conv_ws<32, 8, 16>(a, tc_err, s);
    return conv_ws<16, 8, 16>(a, tc_err, s);
  }
  if (tc_err && mode == 3 && a.Cin % 16 == 0) {
    if (a.Cout % 64 == 0) return conv_halo_cc<64, true>(a, tc_err, s);
    if (a.Cout % 32 == 0) return conv_halo_cc<32, true>(a, tc_err, s);
    return conv_halo_cc<16, true>(a, tc_err, s);
  }
  if (tc_err && mode >= 2 && a.Cin % 16 == 0) {
    if (a.Cout % 64 == 0) return conv_halo_cc<64, false>(a, tc_err, s);
    if (a.Cout % 32 == 0) return conv_halo_cc<32, false>(a, tc_err, s);
    return conv_halo_cc<16, false>(a, tc_err, s);
  }
  if (tc_err) {
    if (a.Cout % 128 == 0) return conv_tc<128>(a, tc_err, s);
    if (a.Cout % 64 == 0) return conv_tc<64>(a, tc_err, s);
    if (a.Cout % 32 == 0) return conv_tc<32>(a, tc_err, s);
    return conv_tc<16>(a, tc_err, s);
  }
  if (a.Cout % 128 == 0) return conv_bn<128>(a, s);
  if (a.Cout % 64 == 0) return conv_bn<64>(a, s);
  if (a.Cout % 32 == 0) return conv_bn<32>(a, s);
  return conv_bn<16>(a, s);
}

// dW[co][tap][ci] += sum over the S splits of part[k][tap][co][ci] (elements
// e < 9 Cout Cin, e = (co 9 + tap) Cin + ci), db[co] += sum of bpart[k][co]
// (the next Cout elements). Thread (x, y) of a block sums the splits k = y,
// y + 8, ... of element 32 blockIdx + x in order; the eight partial sums are
// then added in order of y: a fixed order, the same on every run.
__global__ void k_wgrad_reduce(const float* __restrict__ part, const float* __restrict__ bpart, int S, int Cout,
                               int Cin, float* __restrict__ gw, float* __restrict__ gb) {
  __shared__ float sum[8][33];
  const int nw = 9 * Cout * Cin;
  const int e = blockIdx.x * 32 + threadIdx.x, g = threadIdx.y;
  float acc = 0.f;
  if (e < nw) {
    const int ci = e % Cin, tap = (e / Cin) % 9, co = e / (9 * Cin);
    const size_t base = ((size_t)tap * Cout + co) * Cin + ci, stride = (size_t)nw;
#pragma unroll 4
    for (int k = g; k < S; k += 8) acc += part[k * stride + base];
  } else if (e < nw + Cout) {
#pragma unroll 4
    for (int k = g; k < S; k += 8) acc += bpart[(size_t)k * Cout + (e - nw)];
  }
  sum[g][threadIdx.x] = acc;
  __syncthreads();
  if (g == 0) {
    float t = sum[0][threadIdx.x];
#pragma unroll
    for (int i = 1; i < 8; ++i) t += sum[i][threadIdx.x];
    if (e < nw)
      gw[e] += t;
    else if (e < nw + Cout)
      gb[e - nw] += t;
  }
}

// the shapes the tcgen05 weight gradient takes (others: mma.sync)
bool wgrad_tc_shape(const sg_unet* u, int L, int N, int H, int W) {
  const int Cin = kCin[L], Cout = kCout[L];
  (void)N;
  return u->tc == 4 && W % 8 == 0 && (H * W) % 32 == 0 && Cin % 16 == 0 && Cout % 16 == 0 && Cout <= 128 &&
         encode_tiled() != nullptr;
}

// scratch of at least `bytes` (contents not kept when it grows)
cudaError_t grow(uint16_t** p, size_t* have, size_t bytes) {
  if (*have >= bytes) return cudaSuccess;
  cudaFree(*p);
  *p = nullptr;
  *have = 0;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e == cudaSuccess) *have = bytes;
  return e;
}

template <int NB>
cudaError_t wgrad_tc_launch(const WgradTcArgs& a, int S, uint32_t* err, const CUtensorMap& tA,
                            const CUtensorMap& tB, cudaStream_t s) {
  using Sh = WgradTcShape<NB>;
  const int stages = Sh::kMaxStages;
  const int smem = stages * Sh::kStage + 2048;  // + the ones tile and room to align to 1024
  static bool configured = false;                // per template instance, set once on first use
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(k_wgrad_tc<NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  k_wgrad_tc<NB><<<dim3(a.Cin / NB, S), 128, smem, s>>>(a, stages, err, tA, tB);
  return cudaGetLastError();
}

// tcgen05 weight gradient into dw_part / db_part; returns the number of
// splits, 0 when the shape needs the mma.sync kernel instead
int wgrad_tc(sg_unet* u, int L, const bf16* dz, int dz_stride, const bf16* in, int in_stride, int in_off, int N,
             int H, int W, cudaStream_t s, cudaError_t* err) {
  const int Cin = kCin[L], Cout = kCout[L];
  *err = cudaSuccess;
  const bool dzT_ready = u->dzT_ready;
  u->dzT_ready = false;
  if (!wgrad_tc_shape(u, L, N, H, W) || dz_stride != Cout || (reinterpret_cast<uintptr_t>(in) & 15)) return 0;
  EncodeTiledFn fn = encode_tiled();
  const int64_t P = (int64_t)N * H * W, plane = (int64_t)N * (H + 2) * W;
  cudaError_t e = grow(&u->wg_dzT, &u->wg_dzT_bytes, (size_t)Cout * P * 2);
  if (e == cudaSuccess) e = grow(&u->wg_xT3, &u->wg_xT3_bytes, (size_t)3 * Cin * plane * 2);
  if (e != cudaSuccess) {
    *err = e;
    return 0;
  }
  if (!dzT_ready)
    k_transpose_dz<<<dim3((unsigned)((P + 63) / 64), (Cout + 31) / 32), dim3(32, 8), 0, s>>>(
        reinterpret_cast<const uint16_t*>(dz), dz_stride, Cout, P, u->wg_dzT);
  k_shift_transpose<<<dim3((W + 63) / 64, H + 2, N * ((Cin + 31) / 32)), dim3(32, 8), 0, s>>>(
      reinterpret_cast<const uint16_t*>(in), in_stride, in_off, Cin, N, H, W, u->wg_xT3);
  if ((e = cudaGetLastError()) != cudaSuccess) {
    *err = e;
    return 0;
  }
  const int NB = Cin % 32 == 0 ? 32 : 16;
  CUtensorMap tA, tB;
  memset(&tA, 0, sizeof tA);
  memset(&tB, 0, sizeof tB);
  const cuuint32_t one[4] = {1, 1, 1, 1};
  {
    const cuuint64_t dims[2] = {(cuuint64_t)P, (cuuint64_t)Cout};
    const cuuint64_t strides[1] = {(cuuint64_t)P * 2};
    const cuuint32_t box[2] = {32, (cuuint32_t)Cout};
    if (fn(&tA, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, u->wg_dzT, dims, strides, box, one, CU_TENSOR_MAP_INTERLEAVE_NONE,
           CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS) {
      *err = cudaErrorInvalidValue;
      return 0;
    }
  }
  {
    const cuuint64_t dims[4] = {(cuuint64_t)(H + 2) * W, (cuuint64_t)N, (cuuint64_t)Cin, 3};
    const cuuint64_t strides[3] = {(cuuint64_t)(H + 2) * W * 2, (cuuint64_t)plane * 2, (cuuint64_t)Cin * plane * 2};
    const cuuint32_t box[4] = {32, 1, (cuuint32_t)NB, 1};
    if (fn(&tB, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, u->wg_xT3, dims, strides, box, one, CU_TENSOR_MAP_INTERLEAVE_NONE,
           CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS) {
      *err = cudaErrorInvalidValue;
      return 0;
    }
  }
  // splits: about two CTAs per SM, within the partial buffers and the chunks
  const int64_t chunks = P / 32;
  const int nci = Cin / NB;
  int64_t S = (2 * sm_count() + nci - 1) / nci;
  S = std::min<int64_t>(S, kWgradMaxSplits);
  S = std::min<int64_t>(S, (int64_t)kWgradSplits * 9 * 128 * 192 / (9 * Cout * Cin));
  S = std::max<int64_t>(1, std::min<int64_t>(S, chunks));
  WgradTcArgs a;
  a.Cin = Cin;
  a.Cout = Cout;
  a.N = N;
  a.H = H;
  a.W = W;
  a.chunks = chunks;
  a.per = (chunks + S - 1) / S;
  S = (chunks + a.per - 1) / a.per;  // no split without pixels
  a.dw_part = u->dw_part;
  a.db_part = u->db_part;
  e = NB == 32 ? wgrad_tc_launch<32>(a, (int)S, u->d_err, tA, tB, s) : wgrad_tc_launch<16>(a, (int)S, u->d_err, tA, tB, s);
  if (e != cudaSuccess) {
    *err = e;
    return 0;
  }
  return (int)S;
}

cudaError_t wgrad(sg_unet* u, int L, const bf16* dz, int dz_stride, const bf16* in, int in_stride, int in_off,
                  int N, int H, int W, cudaStream_t s) {
  WgradArgs a;
  a.dz = dz;
  a.dz_stride = dz_stride;
  a.dz_off = 0;
  a.in = in;
  a.in_stride = in_stride;
  a.in_off = in_off;
  a.dw_part = u->dw_part;
  a.db_part = u->db_part;
  a.N = N;
  a.H = H;
  a.W = W;
  a.Cin = kCin[L];
  a.Cout = kCout[L];
  cudaError_t e;
  int S = wgrad_tc(u, L, dz, dz_stride, in, in_stride, in_off, N, H, W, s, &e);
  if (e != cudaSuccess) return e;
  if (S == 0) {
    S = a.S = kWgradSplits;
    const int TM = a.Cout % 32 == 0 ? 32 : 16, TN = a.Cin % 32 == 0 ? 32 : 16;
    dim3 grid(a.Cout / TM, a.Cin / TN, 9 * a.S);
    if (TM == 32 && TN == 32) k_wgrad<32, 32><<<grid, 128, 0, s>>>(a);
    else if (TM == 32) k_wgrad<32, 16><<<grid, 128, 0, s>>>(a);
    else if (TN == 32) k_wgrad<16, 32><<<grid, 128, 0, s>>>(a);
    else k_wgrad<16, 16><<<grid, 128, 0, s>>>(a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  // sum the splits into the gradient: dW[co][tap][ci] (+=), db[co] (+=)
  const int nw = 9 * a.Cout * a.Cin;
  k_wgrad_reduce<<<(nw + a.Cout + 31) / 32, dim3(32, 8), 0, s>>>(u->dw_part, u->db_part, S, a.Cout, a.Cin,
                                                                 u->d_grad + u->woff[L], u->d_grad + u->boff[L]);
  return cudaGetLastError();
}

ConvArgs conv_args(sg_unet* u, int L, const bf16* in, int in_stride, int in_off, int N, int H, int W) {
  ConvArgs a;
  memset(&a, 0, sizeof a);
  a.in = in;
  a.in_stride = in_stride;
  a.in_off = in_off;
  a.wt = u->d_w + u->woff[L];
  a.bias = u->d_param + u->boff[L];
  a.N = N;
  a.H = H;
  a.W = W;
  a.Cin = kCin[L];
  a.Cout = kCout[L];
  a.relu = L != HEAD;
  return a;
}

// masked gradient: dz = bf16(dy * (y > 0)) (no mask for the head), 8 channels per item
cudaError_t relu_bwd(const float* dy, int dy_stride, int dy_off, const bf16* y, int y_stride, int y_off, int C,
                     int64_t P, bf16* dz, cudaStream_t s) {
  const int nc = C / 8;
  return each32(P * nc, s, [=] __device__(int i) {
    const int p = i / nc, c = (i - p * nc) * 8;
    const float4* g = reinterpret_cast<const float4*>(dy + (size_t)p * dy_stride + dy_off + c);
    const float4 g0 = g[0], g1 = g[1];
    float f[8] = {g0.x, g0.y, g0.z, g0.w, g1.x, g1.y, g1.z, g1.w};
    if (y) {
      float yv[8];
      bf8_to_f(*reinterpret_cast<const uint4*>(y + (size_t)p * y_stride + y_off + c), yv);
#pragma unroll
      for (int k = 0; k < 8; ++k)
        if (!(yv[k] > 0.f)) f[k] = 0.f;
    }
    *reinterpret_cast<uint4*>(dz + (size_t)p * C + c) = f_to_bf8(f);
  });
}

// the masked output gradient of layer L (as relu_bwd), written transposed as
// well when the layer's weight gradient runs on tcgen05
cudaError_t masked_grad(sg_unet* u, int L, const float* dy, int dy_stride, int dy_off, const bf16* y, int y_stride,
                        int y_off, int N, int H, int W, bf16* dz, cudaStream_t s) {
  const int C = kCout[L];
  const int64_t P = (int64_t)N * H * W;
  u->dzT_ready = false;
  if (!wgrad_tc_shape(u, L, N, H, W)) return relu_bwd(dy, dy_stride, dy_off, y, y_stride, y_off, C, P, dz, s);
  cudaError_t e = grow(&u->wg_dzT, &u->wg_dzT_bytes, (size_t)C * P * 2);
  if (e != cudaSuccess) return e;
  k_relu_bwd_t<<<dim3((unsigned)((P + 63) / 64), (C + 31) / 32), dim3(32, 8), 0, s>>>(
      dy, dy_stride, dy_off, reinterpret_cast<const uint16_t*>(y), y_stride, y_off, C, P,
      reinterpret_cast<uint16_t*>(dz), u->wg_dzT);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  u->dzT_ready = true;
  return cudaSuccess;
}

// input gradient of a conv: dx[:, off..off+Cin) += conv(dz, flipped weights)
cudaError_t dgrad(sg_unet* u, int L, const bf16* dz, float* dx, int dx_stride, int dx_off, int N, int H, int W,
                  cudaStream_t s) {
  ConvArgs a;
  memset(&a, 0, sizeof a);
  a.in = dz;
  a.in_stride = kCout[L];
  a.in_off = 0;
  a.wt = u->d_wt + u->woff[L];
  a.N = N;
  a.H = H;
  a.W = W;
  a.Cin = kCout[L];
  a.Cout = kCin[L];
  a.out_f32 = dx;
  a.f32_stride = dx_stride;
  a.f32_off = dx_off;
  a.f32_accumulate = 1;
  return conv(a, s, u->tc ? u->d_err : nullptr, u->tc);
}

// He-normal initial weights (counter-based Box-Muller), zero biases, zero head
__global__ void k_init(float* p, int64_t n, float stdv, uint64_t seed, int64_t base) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t z = seed * 0x9E3779B97F4A7C15ull + (uint64_t)(base + i) * 0xD1B54A32D192ED03ull;
    z ^= z >> 31; z *= 0xBF58476D1CE4E5B9ull; z ^= z >> 29; z *= 0x94D049BB133111EBull; z ^= z >> 32;
    const float u1 = ((z >> 40) + 1) * (1.0f / 16777217.0f), u2 = ((z & 0xFFFFFF)) * (1.0f / 16777216.0f);
    p[i] = stdv * sqrtf(-2.0f * logf(u1)) * cospif(2.0f * u2);
  }
}

// per layer: the weights' offset in the parameter vector and the shape
// (by value into the Adam kernel)
struct LayerTable {
  int64_t woff[kLayers];
  int cin[kLayers], cout[kLayers];
};

cudaError_t refresh_bf16(sg_unet* u, cudaStream_t s) {
  // BF16 weights and the flipped/transposed copy used by the input gradient
  for (int L = 0; L < kLayers; ++L) {
    const int Cin = kCin[L], Cout = kCout[L];
    const float* w = u->d_param + u->woff[L];
    bf16* wb = u->d_w + u->woff[L];
    bf16* wt = u->d_wt + u->woff[L];
    cudaError_t e = each((int64_t)Cout * 9 * Cin, s, [=] __device__(int64_t i) {
      const int ci = (int)(i % Cin), tap = (int)((i / Cin) % 9), co = (int)(i / (9 * Cin));
      const bf16 v = __float2bfloat16_rn(w[i]);
      wb[i] = v;
      wt[((size_t)ci * 9 + (8 - tap)) * Cout + co] = v;
    });
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// ---- forward / backward schedule

cudaError_t forward(sg_unet* u, const Crops& c, int N, int h, int w, float* out, int64_t out_pitch,
                    float* const* out_ptrs, cudaStream_t s) {
  cudaError_t e;
  const int h2 = h / 2, w2 = w / 2, h4 = h / 4, w4 = w / 4;
  const int64_t P1 = (int64_t)N * h * w;
  // input: RGBA -> 16 BF16 channels (4 + 12 zero), one pixel per item
  bf16* in16 = u->in16;
  const Crops cc = c;
  e = each32(P1, s, [=] __device__(int i) {
    const Pix P(i, h, w);
    const float4 v = *reinterpret_cast<const float4*>(cc.ptr[P.n] + (int64_t)P.y * cc.pitch + P.x * 4);
    const float f[8] = {v.x, v.y, v.z, v.w, 0.f, 0.f, 0.f, 0.f}, zero[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    uint4* o = reinterpret_cast<uint4*>(in16 + (size_t)i * 16);
    o[0] = f_to_bf8(f);
    o[1] = f_to_bf8(zero);
  });
  if (e) return e;
  ConvArgs a;
  a = conv_args(u, C1A, u->in16, 16, 0, N, h, w); a.out = u->a1; a.out_stride = 32; a.out_off = 0;
  if ((e = conv(a, s, u->tc ? u->d_err : nullptr, u->tc))) return e;
  // e1 lives in cat1 at channel offset 64 (after the 64 upsampled channels)
  // the persistent path writes the pooled and upsampled copies from the
  // producing convolution's epilogue; the others run them as separate passes
  const bool fused = u->tc == 4;
  a = conv_args(u, C1B, u->a1, 32, 0, N, h, w); a.out = u->cat1; a.out_stride = 96; a.out_off = 64;
  if (fused) { a.pool_out = u->p1; a.pool_stride = 32; a.pool_off = 0; }  // pool e1 -> p1
  if ((e = conv(a, s, u->tc ? u->d_err : nullptr, u->tc))) return e;
  if (!fused && (e = pool_fwd(u->cat1, 96, 64, u->p1, 32, 0, 32, N, h, w, s))) return e;
  a = conv_args(u, C2A, u->p1, 32, 0, N, h2, w2); a.out = u->a2; a.out_stride = 64; a.out_off = 0;
  if ((e = conv(a, s, u->tc ? u->d_err : nullptr, u->tc))) return e;
  a = conv_args(u, C2B, u->a2, 64, 0, N, h2, w2); a.out = u->cat2; a.out_stride = 192; a.out_off = 128;
  if (fused) { a.pool_out = u->p2; a.pool_stride = 64; a.pool_off = 0; }  // pool e2 -> p2
  if ((e = conv(a, s, u->tc ? u->d_err : nullptr, u->tc))) return e;
  if (!fused && (e = pool_fwd(u->cat2, 192, 128, u->p2, 64, 0, 64, N, h2, w2, s))) return e;
  a = conv_args(u, C3A, u->p2, 64, 0, N, h4, w4); a.out = u->a3; a.out_stride = 128; a.out_off = 0;
  if ((e = conv(a, s, u->tc ? u->d_err : nullptr, u->tc))) return e;
  a = conv_args(u, C3B, u->a3, 128, 0, N, h4, w4); a.out = u->b3; a.out_stride = 128; a.out_off = 0;
  if (fused) { a.up_out = u->cat2; a.up_stride = 192; a.up_off = 0; }  // up b3 -> cat2[:, 0..128)
  if ((e = conv(a, s, u->tc ? u->d_err : nullptr, u->tc))) return e;
  if (!fused && (e = up_fwd(u->b3, 128, u->cat2, 192, 0, 128, N, h4, w4, s))) return e;
  a = conv_args(u, D2A, u->cat2, 192, 0, N, h2, w2); a.out = u->a4; a.out_stride = 64; a.out_off = 0;
  if ((e = conv(a, s, u->tc ? u->d_err : nullptr, u->tc))) return e;
  a = conv_args(u, D2B, u->a4, 64, 0, N, h2, w2); a.out = u->d2; a.out_stride = 64; a.out_off = 0;
  if (fused) { a.up_out = u->cat1; a.up_stride = 96; a.up_off = 0; }  // up d2 -> cat1[:, 0..64)
  if ((e = conv(a, s, u->tc ? u->d_err : nullptr, u->tc))) return e;
  if (!fused && (e = up_fwd(u->d2, 64, u->cat1, 96, 0, 64, N, h2, w2, s))) return e;
  a = conv_args(u, D1A, u->cat1, 96, 0, N, h, w); a.out = u->a5; a.out_stride = 32; a.out_off = 0;
  if ((e = conv(a, s, u->tc ? u->d_err : nullptr, u->tc))) return e;
  a = conv_args(u, D1B, u->a5, 32, 0, N, h, w); a.out = u->d1; a.out_stride = 32; a.out_off = 0;
  if ((e = conv(a, s, u->tc ? u->d_err : nullptr, u->tc))) return e;
  a = conv_args(u, HEAD, u->d1, 32, 0, N, h, w);
  if (u->tc == 4) {
    // the persistent path writes the output from the head's epilogue
    HeadOut ho;
    memset(&ho, 0, sizeof ho);
    for (int n = 0; n < N; ++n) {
      ho.in[n] = c.ptr[n];
      ho.out[n] = out_ptrs ? out_ptrs[n] : out + (size_t)n * 2 * h * out_pitch;
    }
    ho.in_pitch = c.pitch;
    ho.out_pitch = out_pitch;
    ho.on = 1;
    if ((e = conv(a, s, u->d_err, 4, &ho))) return e;
  } else {
    a.out_f32 = u->head; a.f32_stride = 16; a.f32_off = 0;
    if ((e = conv(a, s, u->tc ? u->d_err : nullptr, u->tc))) return e;
  }
  // out = bilinear 2x (half-pixel centres, clamp) of the input + pixel shuffle of the head
  if (u->tc != 4) {
    const float* head = u->head;
    const int H2 = 2 * h, W2 = 2 * w;
    OutPtrs op;
    for (int n = 0; n < N; ++n) op.p[n] = out_ptrs ? out_ptrs[n] : out + (size_t)n * H2 * out_pitch;
    const int64_t opitch = out_pitch;
    e = each32((int64_t)N * H2 * W2, s, [=] __device__(int i) {
      const Pix P(i, H2, W2);
      const float ux = 0.5f * P.x - 0.25f, uy = 0.5f * P.y - 0.25f;
      const float fx0 = floorf(ux), fy0 = floorf(uy);
      const float fx = ux - fx0, fy = uy - fy0;
      const int x0 = min(max((int)fx0, 0), w - 1), x1 = min(max((int)fx0 + 1, 0), w - 1);
      const int y0 = min(max((int)fy0, 0), h - 1), y1 = min(max((int)fy0 + 1, 0), h - 1);
      const float* src = cc.ptr[P.n];
      const float4 v00 = *reinterpret_cast<const float4*>(src + y0 * cc.pitch + x0 * 4);
      const float4 v01 = *reinterpret_cast<const float4*>(src + y0 * cc.pitch + x1 * 4);
      const float4 v10 = *reinterpret_cast<const float4*>(src + y1 * cc.pitch + x0 * 4);
      const float4 v11 = *reinterpret_cast<const float4*>(src + y1 * cc.pitch + x1 * 4);
      const float a00 = (1.f - fy) * (1.f - fx), a01 = (1.f - fy) * fx, a10 = fy * (1.f - fx), a11 = fy * fx;
      const float* hp = head + ((size_t)(P.n * h + P.y / 2) * w + P.x / 2) * 16 + (P.y & 1) * 2 + (P.x & 1);
      float4 o;
      o.x = a00 * v00.x + a01 * v01.x + a10 * v10.x + a11 * v11.x + hp[0];
      o.y = a00 * v00.y + a01 * v01.y + a10 * v10.y + a11 * v11.y + hp[4];
      o.z = a00 * v00.z + a01 * v01.z + a10 * v10.z + a11 * v11.z + hp[8];
      o.w = a00 * v00.w + a01 * v01.w + a10 * v10.w + a11 * v11.w + hp[12];
      *reinterpret_cast<float4*>(op.p[P.n] + (int64_t)P.y * opitch + P.x * 4) = o;
    });
    if (e) return e;
  }
  u->n = N;
  u->h = h;
  u->w = w;
  u->in_crops = c;
  return cudaSuccess;
}

cudaError_t backward(sg_unet* u, const Crops& tgt, const float* out, int64_t out_pitch, float* const* out_ptrs,
                     cudaStream_t s) {
  cudaError_t e;
  const int N = u->n, h = u->h, w = u->w, h2 = h / 2, w2 = w / 2, h4 = h / 4, w4 = w / 4;
  const int64_t P1 = (int64_t)N * h * w, P2 = P1 / 4, P3 = P1 / 16;
  const int H2 = 2 * h, W2 = 2 * w;
  const int64_t count = (int64_t)N * H2 * W2 * 4;
  // zero gradients of parameters and activations
  if ((e = cudaMemsetAsync(u->d_grad, 0, u->nparam * sizeof(float), s))) return e;
  const size_t f = sizeof(float);
  if ((e = cudaMemsetAsync(u->g_cat1, 0, P1 * 96 * f, s)) || (e = cudaMemsetAsync(u->g_a1, 0, P1 * 32 * f, s)) ||
      (e = cudaMemsetAsync(u->g_p1, 0, P2 * 32 * f, s)) || (e = cudaMemsetAsync(u->g_a2, 0, P2 * 64 * f, s)) ||
      (e = cudaMemsetAsync(u->g_cat2, 0, P2 * 192 * f, s)) || (e = cudaMemsetAsync(u->g_p2, 0, P3 * 64 * f, s)) ||
      (e = cudaMemsetAsync(u->g_a3, 0, P3 * 128 * f, s)) || (e = cudaMemsetAsync(u->g_b3, 0, P3 * 128 * f, s)) ||
      (e = cudaMemsetAsync(u->g_a4, 0, P2 * 64 * f, s)) || (e = cudaMemsetAsync(u->g_d2, 0, P2 * 64 * f, s)) ||
      (e = cudaMemsetAsync(u->g_a5, 0, P1 * 32 * f, s)) || (e = cudaMemsetAsync(u->g_d1, 0, P1 * 32 * f, s)) ||
      (e = cudaMemsetAsync(u->d_loss, 0, 2 * f, s)))
    return e;
  // MSE over all outputs; d out = 2 (out - target) / count, routed to the head by the pixel shuffle
  {
    ConstOutPtrs op;
    for (int n = 0; n < N; ++n) op.p[n] = out_ptrs ? out_ptrs[n] : out + (size_t)n * H2 * out_pitch;
    float* gh = u->g_head;
    float* loss = u->d_loss;
    const Crops t = tgt;
    const int64_t opitch = out_pitch;
    const float scale = 1.0f / (float)count;
    const int64_t npix = (int64_t)N * H2 * W2;
    e = each32(npix, s, [=] __device__(int i) {
      const Pix P(i, H2, W2);
      const float4 o = *reinterpret_cast<const float4*>(op.p[P.n] + (int64_t)P.y * opitch + P.x * 4);
      const float4 g = *reinterpret_cast<const float4*>(t.ptr[P.n] + (int64_t)P.y * t.pitch + P.x * 4);
      float* hp = gh + ((size_t)(P.n * h + P.y / 2) * w + P.x / 2) * 16 + (P.y & 1) * 2 + (P.x & 1);
      hp[0] = 2.0f * (o.x - g.x) * scale;
      hp[4] = 2.0f * (o.y - g.y) * scale;
      hp[8] = 2.0f * (o.z - g.z) * scale;
      hp[12] = 2.0f * (o.w - g.w) * scale;
    });
    if (e) return e;
    e = sum(npix, loss, s, [=] __device__(int64_t i) {
      const Pix P((int)i, H2, W2);
      const float4 o = *reinterpret_cast<const float4*>(op.p[P.n] + (int64_t)P.y * opitch + P.x * 4);
      const float4 g = *reinterpret_cast<const float4*>(t.ptr[P.n] + (int64_t)P.y * t.pitch + P.x * 4);
      const float dx = o.x - g.x, dy = o.y - g.y, dz = o.z - g.z, dw = o.w - g.w;
      return (dx * dx + dy * dy + dz * dz + dw * dw) * scale;
    });
    if (e) return e;
  }
  bf16* dz = u->dz;
  // head (no ReLU)
  if ((e = masked_grad(u, HEAD, u->g_head, 16, 0, nullptr, 0, 0, N, h, w, dz, s))) return e;
  if ((e = wgrad(u, HEAD, dz, 16, u->d1, 32, 0, N, h, w, s))) return e;
  if ((e = dgrad(u, HEAD, dz, u->g_d1, 32, 0, N, h, w, s))) return e;
  // d1b: y = d1, x = a5
  if ((e = masked_grad(u, D1B, u->g_d1, 32, 0, u->d1, 32, 0, N, h, w, dz, s))) return e;
  if ((e = wgrad(u, D1B, dz, 32, u->a5, 32, 0, N, h, w, s))) return e;
  if ((e = dgrad(u, D1B, dz, u->g_a5, 32, 0, N, h, w, s))) return e;
  // d1a: y = a5, x = cat1 (96)
  if ((e = masked_grad(u, D1A, u->g_a5, 32, 0, u->a5, 32, 0, N, h, w, dz, s))) return e;
  if ((e = wgrad(u, D1A, dz, 32, u->cat1, 96, 0, N, h, w, s))) return e;
  if ((e = dgrad(u, D1A, dz, u->g_cat1, 96, 0, N, h, w, s))) return e;
  if ((e = up_bwd(u->g_cat1, 96, u->g_d2, 64, 64, N, h2, w2, s))) return e;  // up: g_d2 += children
  // d2b: y = d2, x = a4
  if ((e = masked_grad(u, D2B, u->g_d2, 64, 0, u->d2, 64, 0, N, h2, w2, dz, s))) return e;
  if ((e = wgrad(u, D2B, dz, 64, u->a4, 64, 0, N, h2, w2, s))) return e;
  if ((e = dgrad(u, D2B, dz, u->g_a4, 64, 0, N, h2, w2, s))) return e;
  // d2a: y = a4, x = cat2 (192)
  if ((e = masked_grad(u, D2A, u->g_a4, 64, 0, u->a4, 64, 0, N, h2, w2, dz, s))) return e;
  if ((e = wgrad(u, D2A, dz, 64, u->cat2, 192, 0, N, h2, w2, s))) return e;
  if ((e = dgrad(u, D2A, dz, u->g_cat2, 192, 0, N, h2, w2, s))) return e;
  if ((e = up_bwd(u->g_cat2, 192, u->g_b3, 128, 128, N, h4, w4, s))) return e;  // up: g_b3 += children
  // c3b: y = b3, x = a3
  if ((e = masked_grad(u, C3B, u->g_b3, 128, 0, u->b3, 128, 0, N, h4, w4, dz, s))) return e;
  if ((e = wgrad(u, C3B, dz, 128, u->a3, 128, 0, N, h4, w4, s))) return e;
  if ((e = dgrad(u, C3B, dz, u->g_a3, 128, 0, N, h4, w4, s))) return e;
  // c3a: y = a3, x = p2
  if ((e = masked_grad(u, C3A, u->g_a3, 128, 0, u->a3, 128, 0, N, h4, w4, dz, s))) return e;
  if ((e = wgrad(u, C3A, dz, 128, u->p2, 64, 0, N, h4, w4, s))) return e;
  if ((e = dgrad(u, C3A, dz, u->g_p2, 64, 0, N, h4, w4, s))) return e;
  // pool: g_cat2[:, 128..192) += g_p2 / 4 (e2's gradient lives at its place in cat2)
  if ((e = pool_bwd(u->g_p2, 64, u->g_cat2, 192, 128, 64, N, h4, w4, s))) return e;
  // c2b: y = e2 = cat2[:, 128..), x = a2
  if ((e = masked_grad(u, C2B, u->g_cat2, 192, 128, u->cat2, 192, 128, N, h2, w2, dz, s))) return e;
  if ((e = wgrad(u, C2B, dz, 64, u->a2, 64, 0, N, h2, w2, s))) return e;
  if ((e = dgrad(u, C2B, dz, u->g_a2, 64, 0, N, h2, w2, s))) return e;
  // c2a: y = a2, x = p1
  if ((e = masked_grad(u, C2A, u->g_a2, 64, 0, u->a2, 64, 0, N, h2, w2, dz, s))) return e;
  if ((e = wgrad(u, C2A, dz, 64, u->p1, 32, 0, N, h2, w2, s))) return e;
  if ((e = dgrad(u, C2A, dz, u->g_p1, 32, 0, N, h2, w2, s))) return e;
  if ((e = pool_bwd(u->g_p1, 32, u->g_cat1, 96, 64, 32, N, h2, w2, s))) return e;  // pool: e1's gradient
  // c1b: y = e1 = cat1[:, 64..), x = a1
  if ((e = masked_grad(u, C1B, u->g_cat1, 96, 64, u->cat1, 96, 64, N, h, w, dz, s))) return e;
  if ((e = wgrad(u, C1B, dz, 32, u->a1, 32, 0, N, h, w, s))) return e;
  if ((e = dgrad(u, C1B, dz, u->g_a1, 32, 0, N, h, w, s))) return e;
  // c1a: y = a1, x = in16 (no input gradient)
  if ((e = masked_grad(u, C1A, u->g_a1, 32, 0, u->a1, 32, 0, N, h, w, dz, s))) return e;
  if ((e = wgrad(u, C1A, dz, 32, u->in16, 16, 0, N, h, w, s))) return e;
  return cudaSuccess;
}

sg_status check_shape(const sg_unet* u, int n, int h, int w) {
  if (n < 1 || n > u->max_n || n > 64 || h < 4 || w < 4 || h % 4 || w % 4 || (int64_t)h * w > (int64_t)u->max_h * u->max_w) {
    set_error("unet: batch 1..max_batch (<= 64), h and w multiples of 4 with h*w <= max_h*max_w");
    return SG_ERR_INVALID_ARG;
  }
  return SG_OK;
}

}  // namespace

namespace sg {
namespace nn {
// Failure-detection self-test: the bounded wait of the tensor-core kernels
// on an mbarrier that expects one arrival which never comes. No copy, MMA
// or TMEM allocation is in flight; after `limit` polls the wait gives up and
// the kernel raises the error word as a stalled convolution would.
__global__ void k_wait_selftest(uint32_t* err, uint32_t limit) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&bar)));
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0 && !mbar_wait_limit(smem_u32(&bar), 0, limit)) atomicExch(err, 1u);
}
}  // namespace nn
}  // namespace sg

extern "C" {

sg_status sg_unet_create(int max_batch, int max_h, int max_w, uint64_t seed, sg_unet** out) {
  return sg::guarded("sg_unet_create", [&]() -> sg_status {
    if (!out || max_batch < 1 || max_batch > 64 || max_h < 4 || max_w < 4 || max_h % 4 || max_w % 4) {
      set_error("sg_unet_create: max_batch 1..64, max_h and max_w multiples of 4");
      return SG_ERR_INVALID_ARG;
    }
    sg_unet* u = new sg_unet();
    u->max_n = max_batch;
    u->max_h = max_h;
    u->max_w = max_w;
    int64_t off = 0;
    for (int L = 0; L < kLayers; ++L) {
      u->woff[L] = off;
      off += (int64_t)kCout[L] * 9 * kCin[L];
      u->boff[L] = off;
      off += kCout[L];
    }
    u->nparam = off;
    const int64_t P1 = (int64_t)max_batch * max_h * max_w, P2 = P1 / 4, P3 = P1 / 16;
    const size_t b = sizeof(bf16), f = sizeof(float);
    cudaError_t e = cudaSuccess;
    void** p;
  #define A_(ptr, bytes) \
    if (e == cudaSuccess) { p = reinterpret_cast<void**>(&(ptr)); e = alloc(u, p, (bytes)); }
    A_(u->d_param, off * f) A_(u->d_grad, off * f) A_(u->d_m, off * f) A_(u->d_v, off * f)
    A_(u->d_w, off * b) A_(u->d_wt, off * b)
    A_(u->in16, P1 * 16 * b) A_(u->a1, P1 * 32 * b) A_(u->cat1, P1 * 96 * b) A_(u->p1, P2 * 32 * b)
    A_(u->a2, P2 * 64 * b) A_(u->cat2, P2 * 192 * b) A_(u->p2, P3 * 64 * b) A_(u->a3, P3 * 128 * b)
    A_(u->b3, P3 * 128 * b) A_(u->a4, P2 * 64 * b) A_(u->d2, P2 * 64 * b) A_(u->a5, P1 * 32 * b) A_(u->d1, P1 * 32 * b)
    A_(u->head, P1 * 16 * f)
    A_(u->g_a1, P1 * 32 * f) A_(u->g_cat1, P1 * 96 * f) A_(u->g_p1, P2 * 32 * f) A_(u->g_a2, P2 * 64 * f)
    A_(u->g_cat2, P2 * 192 * f) A_(u->g_p2, P3 * 64 * f) A_(u->g_a3, P3 * 128 * f) A_(u->g_b3, P3 * 128 * f)
    A_(u->g_a4, P2 * 64 * f) A_(u->g_d2, P2 * 64 * f) A_(u->g_a5, P1 * 32 * f) A_(u->g_d1, P1 * 32 * f)
    A_(u->g_head, P1 * 16 * f) A_(u->dz, P1 * 32 * b)
    A_(u->dw_part, (size_t)kWgradSplits * 9 * 128 * 192 * f) A_(u->db_part, (size_t)kWgradMaxSplits * 128 * f)
    A_(u->d_loss, 2 * f)
    A_(u->d_err, 16)
  #undef A_
    if (e != cudaSuccess) {
      free_unet(u);
      set_error(std::string("sg_unet_create: ") + cudaGetErrorString(e));
      return SG_ERR_OOM;
    }
    // He-normal weights, zero biases; the head starts at zero so the untrained
    // network is exactly the bilinear upsampling of its input
    cudaMemset(u->d_param, 0, off * f);
    cudaMemset(u->d_err, 0, 16);
    cudaMemset(u->d_m, 0, off * f);
    cudaMemset(u->d_v, 0, off * f);
    for (int L = 0; L < HEAD; ++L) {
      const int64_t n = (int64_t)kCout[L] * 9 * kCin[L];
      const int fan_in = 9 * (L == C1A ? 4 : kCin[L]);
      k_init<<<blocks_for(n), 256>>>(u->d_param + u->woff[L], n, sqrtf(2.0f / fan_in), seed, u->woff[L]);
    }
    e = cudaGetLastError();
    if (e == cudaSuccess) {
      // input channels 4..15 of c1a are padding: their weights stay zero
      float* w = u->d_param + u->woff[C1A];
      e = each((int64_t)kCout[C1A] * 9 * 16, 0, [=] __device__(int64_t i) {
        if (i % 16 >= 4) w[i] = 0.f;
      });
    }
    if (e == cudaSuccess) e = refresh_bf16(u, 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
      free_unet(u);
      return cuda_fail(e, "sg_unet_create");
    }
    *out = u;
    return SG_OK;
  });
}

sg_status sg_unet_set_tensor_path(sg_unet* u, int tcgen05) {
  if (!u || tcgen05 < 0 || tcgen05 > 4) {
    set_error("sg_unet_set_tensor_path: NULL or mode not 0..4");
    return SG_ERR_INVALID_ARG;
  }
  u->tc = tcgen05;
  return SG_OK;
}

sg_status sg_unet_check(sg_unet* u) {
  if (!u) {
    set_error("sg_unet_check: NULL");
    return SG_ERR_INVALID_ARG;
  }
  uint32_t e = 0;
  cudaError_t ce = cudaMemcpy(&e, u->d_err, sizeof e, cudaMemcpyDeviceToHost);
  if (ce != cudaSuccess) return cuda_fail(ce, "sg_unet_check");
  if (e) {
    cudaMemset(u->d_err, 0, sizeof e);
    set_error("sg_unet: a tensor-core wait timed out (results of the affected launches are invalid)");
    return SG_ERR_TIMEOUT;
  }
  return SG_OK;
}

sg_status sg_unet_wait_selftest(sg_unet* u, uint32_t polls, void* stream) {
  if (!u || polls == 0 || polls > kTcSpinLimit) {
    set_error("sg_unet_wait_selftest: NULL network or polls outside [1, 2^24]");
    return SG_ERR_INVALID_ARG;
  }
  nn::k_wait_selftest<<<1, 32, 0, (cudaStream_t)stream>>>(u->d_err, polls);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "sg_unet_wait_selftest");
  return SG_OK;
}

sg_status sg_unet_destroy(sg_unet* u) {
  if (!u) return SG_OK;
  cudaDeviceSynchronize();
  free_unet(u);
  return SG_OK;
}

sg_status sg_unet_param_count(sg_unet* u, int64_t* n) {
  if (!u || !n) {
    set_error("sg_unet_param_count: NULL argument");
    return SG_ERR_INVALID_ARG;
  }
  *n = u->nparam;
  return SG_OK;
}

sg_status sg_unet_get_params(sg_unet* u, float* host, int64_t n, int which) {
  if (!u || !host || n < u->nparam || which < 0 || which > 1) {
    set_error("sg_unet_get_params: NULL, too small, or which not 0/1");
    return SG_ERR_INVALID_ARG;
  }
  cudaError_t e = cudaMemcpy(host, which ? u->d_grad : u->d_param, u->nparam * sizeof(float), cudaMemcpyDeviceToHost);
  return e == cudaSuccess ? SG_OK : cuda_fail(e, "sg_unet_get_params");
}

sg_status sg_unet_set_params(sg_unet* u, const float* host, int64_t n) {
  if (!u || !host || n != u->nparam) {
    set_error("sg_unet_set_params: NULL or wrong count");
    return SG_ERR_INVALID_ARG;
  }
  cudaError_t e = cudaMemcpy(u->d_param, host, n * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = refresh_bf16(u, 0);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  return e == cudaSuccess ? SG_OK : cuda_fail(e, "sg_unet_set_params");
}

sg_status sg_unet_forward(sg_unet* u, const float* const* in, int64_t in_pitch, int n, int h, int w, float* const* out,
                          int64_t out_pitch, void* stream) {
  sg::NvtxRange nvtx_range("sg_unet_forward");
  if (!u || !in || !out) {
    set_error("sg_unet_forward: NULL argument");
    return SG_ERR_INVALID_ARG;
  }
  sg_status st = check_shape(u, n, h, w);
  if (st != SG_OK) return st;
  if (in_pitch < 4 * w || out_pitch < 8 * w) {
    set_error("sg_unet_forward: pitch smaller than a row");
    return SG_ERR_INVALID_ARG;
  }
  Crops c;
  for (int i = 0; i < n; ++i) {
    if (!in[i] || !out[i]) {
      set_error("sg_unet_forward: NULL image pointer");
      return SG_ERR_INVALID_ARG;
    }
    c.ptr[i] = in[i];
  }
  c.pitch = in_pitch;
  cudaError_t e = forward(u, c, n, h, w, nullptr, out_pitch, out, (cudaStream_t)stream);
  return e == cudaSuccess ? SG_OK : cuda_fail(e, "sg_unet_forward");
}

sg_status sg_unet_backward(sg_unet* u, const float* const* target, int64_t target_pitch, const float* const* out,
                           int64_t out_pitch, float* loss, void* stream) {
  sg::NvtxRange nvtx_range("sg_unet_backward");
  if (!u || !target || !out || u->n == 0) {
    set_error("sg_unet_backward: NULL argument or no forward pass before");
    return SG_ERR_INVALID_ARG;
  }
  Crops t;
  for (int i = 0; i < u->n; ++i) t.ptr[i] = target[i];
  t.pitch = target_pitch;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = backward(u, t, nullptr, out_pitch, const_cast<float* const*>(out), s);
  if (e == cudaSuccess && loss) e = cudaMemcpyAsync(loss, u->d_loss, sizeof(float), cudaMemcpyDeviceToDevice, s);
  return e == cudaSuccess ? SG_OK : cuda_fail(e, "sg_unet_backward");
}

sg_status sg_unet_adam_step(sg_unet* u, float lr, float beta1, float beta2, float eps, void* stream) {
  if (!u || !(lr > 0.f) || !(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f) || !(eps > 0.f)) {
    set_error("sg_unet_adam_step: bad hyper-parameters");
    return SG_ERR_INVALID_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  ++u->step;
  const float c1 = 1.0f - powf(beta1, (float)u->step), c2 = 1.0f - powf(beta2, (float)u->step);
  float *p = u->d_param, *g = u->d_grad, *m = u->d_m, *v = u->d_v;
  bf16 *wb = u->d_w, *wt = u->d_wt;
  const int64_t pad_lo = u->woff[C1A], pad_n = (int64_t)kCout[C1A] * 9 * 16;
  LayerTable lt;
  for (int L = 0; L < kLayers; ++L) {
    lt.woff[L] = u->woff[L];
    lt.cin[L] = kCin[L];
    lt.cout[L] = kCout[L];
  }
  // one pass: the update, then (for a weight) its BF16 copy and the
  // flipped / transposed one the input gradient reads, as refresh_bf16 does
  cudaError_t e = each(u->nparam, s, [=] __device__(int64_t i) {
    // the padding input channels of the first layer stay zero
    if (i >= pad_lo && i < pad_lo + pad_n && (i - pad_lo) % 16 >= 4) return;
    const float gi = g[i];
    const float mi = beta1 * m[i] + (1.f - beta1) * gi, vi = beta2 * v[i] + (1.f - beta2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float pn = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    p[i] = pn;
    int L = kLayers - 1;
    while (L > 0 && i < lt.woff[L]) --L;
    const int64_t r = i - lt.woff[L];
    const int Cin = lt.cin[L], Cout = lt.cout[L];
    if (r < (int64_t)Cout * 9 * Cin) {
      const int ci = (int)(r % Cin), tap = (int)((r / Cin) % 9), co = (int)(r / (9 * Cin));
      const bf16 b16 = __float2bfloat16_rn(pn);
      wb[i] = b16;
      wt[lt.woff[L] + ((int64_t)ci * 9 + (8 - tap)) * Cout + co] = b16;
    }
  });
  return e == cudaSuccess ? SG_OK : cuda_fail(e, "sg_unet_adam_step");
}

// PSNR of a against b over count floats (values in [0, 1]): 10 log10(1 / MSE)
sg_status sg_psnr(const float* a, const float* b, int64_t count, float* out_db, void* stream) {
  if (!a || !b || !out_db || count <= 0) {
    set_error("sg_psnr: NULL argument or empty");
    return SG_ERR_INVALID_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  float* acc = out_db;  // accumulate the squared error sum in the output, then convert
  cudaError_t e = cudaMemsetAsync(acc, 0, sizeof(float), s);
  if (e == cudaSuccess)
    e = sum(count, acc, s, [=] __device__(int64_t i) {
      const float d = a[i] - b[i];
      return d * d;
    });
  if (e == cudaSuccess)
    e = each(1, s, [=] __device__(int64_t) {
      const float mse = acc[0] / (float)count;
      acc[0] = mse > 0.f ? 10.0f * log10f(1.0f / mse) : 1000.0f;
    });
  return e == cudaSuccess ? SG_OK : cuda_fail(e, "sg_psnr");
}

// ---------------------------------------------------------------- checkpoints

namespace {
constexpr uint32_t kCkptMagic = 0x4e554753u;  // "SGUN"
constexpr uint32_t kCkptVersion = 1;
struct CkptHeader {
  uint32_t magic, version;
  int64_t nparam, step;
};
}  // namespace

sg_status sg_unet_save(sg_unet* u, const char* path) {
  return sg::guarded("sg_unet_save", [&]() -> sg_status {
    if (!u || !path) {
      set_error("sg_unet_save: NULL argument");
      return SG_ERR_INVALID_ARG;
    }
    std::vector<float> host((size_t)u->nparam * 3);
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(host.data(), u->d_param, u->nparam * sizeof(float), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess)
      e = cudaMemcpy(host.data() + u->nparam, u->d_m, u->nparam * sizeof(float), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess)
      e = cudaMemcpy(host.data() + 2 * u->nparam, u->d_v, u->nparam * sizeof(float), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "sg_unet_save");
    FILE* f = fopen(path, "wb");
    if (!f) {
      set_error(std::string("sg_unet_save: cannot open ") + path);
      return SG_ERR_IO;
    }
    const CkptHeader h{kCkptMagic, kCkptVersion, u->nparam, u->step};
    const bool ok = fwrite(&h, sizeof h, 1, f) == 1 && fwrite(host.data(), sizeof(float), host.size(), f) == host.size();
    if (fclose(f) != 0 || !ok) {
      set_error(std::string("sg_unet_save: write failed: ") + path);
      return SG_ERR_IO;
    }
    return SG_OK;
  });
}

sg_status sg_unet_load(sg_unet* u, const char* path) {
  return sg::guarded("sg_unet_load", [&]() -> sg_status {
    if (!u || !path) {
      set_error("sg_unet_load: NULL argument");
      return SG_ERR_INVALID_ARG;
    }
    FILE* f = fopen(path, "rb");
    if (!f) {
      set_error(std::string("sg_unet_load: cannot open ") + path);
      return SG_ERR_IO;
    }
    CkptHeader h;
    std::vector<float> host((size_t)u->nparam * 3);
    const bool ok = fread(&h, sizeof h, 1, f) == 1 && h.magic == kCkptMagic && h.version == kCkptVersion &&
                    h.nparam == u->nparam && h.step >= 0 &&
                    fread(host.data(), sizeof(float), host.size(), f) == host.size();
    fclose(f);
    if (!ok) {
      set_error(std::string("sg_unet_load: not a checkpoint of this network (or truncated): ") + path);
      return SG_ERR_IO;
    }
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(u->d_param, host.data(), u->nparam * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
      e = cudaMemcpy(u->d_m, host.data() + u->nparam, u->nparam * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
      e = cudaMemcpy(u->d_v, host.data() + 2 * u->nparam, u->nparam * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = refresh_bf16(u, nullptr);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "sg_unet_load");
    u->step = h.step;
    return SG_OK;
  });
}

// ---------------------------------------------------------------- a learned frame

sg_status sg_render_learned(sg_volume* vol, sg_unet* u, const sg_pose* pose, const sg_learned_params* prm,
                            float* out_rgba[2], float* psnr_db, int32_t* fell_back, void* stream) {
  sg::NvtxRange nvtx_range("sg_render_learned");
  if (!vol || !u || !pose || !prm || !out_rgba || !out_rgba[0] || !out_rgba[1]) {
    set_error("sg_render_learned: NULL argument");
    return SG_ERR_INVALID_ARG;
  }
  const int W = pose->width, H = pose->height, w = W / 2, h = H / 2;
  if (W % 8 || H % 8 || W < 8 || H < 8 || (int64_t)h * w > (int64_t)u->max_h * u->max_w || u->max_n < 2) {
    set_error("sg_render_learned: width and height must be multiples of 8, the half-resolution image within the "
              "network's max_h x max_w pixels, and the network must take batches of 2");
    return SG_ERR_INVALID_ARG;
  }
  if (prm->judge && (!psnr_db || !fell_back)) {
    set_error("sg_render_learned: judging needs psnr_db and fell_back");
    return SG_ERR_INVALID_ARG;
  }
  if (prm->half_slot < 0 || prm->half_slot >= 256 || prm->half_slot == pose->slot || !(prm->step > 0.0f)) {
    set_error("sg_render_learned: half_slot in [0, 255] other than pose->slot, and step > 0");
    return SG_ERR_INVALID_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  auto grow = [](float** p, size_t* have, size_t bytes) {
    if (*have >= bytes) return cudaSuccess;
    cudaFree(*p);
    *p = nullptr;
    *have = 0;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaSuccess) *have = bytes;
    return e;
  };
  const size_t half_px = (size_t)w * h, full_px = (size_t)W * H;
  cudaError_t e = grow(&u->lrn_half, &u->lrn_half_bytes, 2 * half_px * 4 * sizeof(float));
  if (e == cudaSuccess && prm->judge) e = grow(&u->lrn_full, &u->lrn_full_bytes, 2 * full_px * 4 * sizeof(float));
  if (e == cudaSuccess && !u->lrn_acc) e = cudaMalloc(&u->lrn_acc, 2 * sizeof(float));
  if (e != cudaSuccess) {
    set_error(std::string("sg_render_learned: buffers: ") + cudaGetErrorString(e));
    return SG_ERR_OOM;
  }
  // the reduced render: half resolution, twice the step, at the level of
  // detail of the full-resolution image (its pixels are twice as large)
  sg_pose hp = *pose;
  hp.width = w;
  hp.height = h;
  hp.pixel_error = prm->pixel_error_half > 0.0f ? prm->pixel_error_half : 0.5f * pose->pixel_error;
  hp.slot = prm->half_slot;
  sg_render_config keep;
  sg_status st = sg_get_render_config(vol, &keep);
  if (st != SG_OK) return st;
  auto render = [&](const sg_pose* p, float step, const sg_render_config& cfg, float* outs[2]) -> sg_status {
    sg_status r = sg_select_lod_batch(vol, p, 1, stream);
    if (r != SG_OK) return r;
    if (cfg.tile_w || cfg.persistent) {
      r = sg_set_render_config(vol, &cfg);
      if (r != SG_OK) return r;
    }
    sg_render_params rp;
    memset(&rp, 0, sizeof rp);
    rp.step = step;
    rp.term_alpha = prm->term_alpha > 0.0f ? prm->term_alpha : 0.99f;
    rp.empty_skip = 1;
    rp.mode = SG_MODE_EMISSION_ABSORPTION;
    r = sg_render(vol, p, &rp, outs, stream);
    sg_set_render_config(vol, &keep);
    return r;
  };
  float* half[2] = {u->lrn_half, u->lrn_half + half_px * 4};
  if ((st = render(&hp, 2.0f * prm->step, prm->half_config, half)) != SG_OK) return st;
  const float* hin[2] = {half[0], half[1]};
  if ((st = sg_unet_forward(u, hin, (int64_t)w * 4, 2, h, w, out_rgba, (int64_t)W * 4, stream)) != SG_OK) return st;
  if (!prm->judge) return SG_OK;
  // the yardstick: the plain full-rate render, the stereo PSNR
  // 10 log10(1 / mean of the eyes' MSE) on the device, and the fallback
  float* full[2] = {u->lrn_full, u->lrn_full + full_px * 4};
  if ((st = render(pose, prm->step, prm->full_config, full)) != SG_OK) return st;
  float* acc = u->lrn_acc;
  const int64_t cnt = (int64_t)full_px * 4;
  const float* o0 = out_rgba[0];
  const float* o1 = out_rgba[1];
  const float* f0 = full[0];
  const float* f1 = full[1];
  e = cudaMemsetAsync(acc, 0, 2 * sizeof(float), s);
  if (e == cudaSuccess)
    e = sum(cnt, acc, s, [=] __device__(int64_t i) {
      const float d = o0[i] - f0[i];
      return d * d;
    });
  if (e == cudaSuccess)
    e = sum(cnt, acc + 1, s, [=] __device__(int64_t i) {
      const float d = o1[i] - f1[i];
      return d * d;
    });
  const float thr = prm->threshold_db;
  if (e == cudaSuccess)
    e = each(1, s, [=] __device__(int64_t) {
      const float m0 = acc[0] / (float)cnt, m1 = acc[1] / (float)cnt, m = 0.5f * (m0 + m1);
      psnr_db[0] = m0 > 0.f ? 10.0f * log10f(1.0f / m0) : 1000.0f;
      psnr_db[1] = m1 > 0.f ? 10.0f * log10f(1.0f / m1) : 1000.0f;
      psnr_db[2] = m > 0.f ? 10.0f * log10f(1.0f / m) : 1000.0f;
      *fell_back = psnr_db[2] < thr ? 1 : 0;
    });
  // a frame below the threshold shows the full-rate render
  float* d0 = out_rgba[0];
  float* d1 = out_rgba[1];
  const int32_t* fb = fell_back;
  if (e == cudaSuccess)
    e = each(cnt / 4, s, [=] __device__(int64_t i) {
      if (!*fb) return;
      reinterpret_cast<float4*>(d0)[i] = reinterpret_cast<const float4*>(f0)[i];
      reinterpret_cast<float4*>(d1)[i] = reinterpret_cast<const float4*>(f1)[i];
    });
  return e == cudaSuccess ? SG_OK : cuda_fail(e, "sg_render_learned");
}

}  // extern "C"
