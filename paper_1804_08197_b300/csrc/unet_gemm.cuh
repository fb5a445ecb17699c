// Tensor-core GEMM kernels of the learned reconstruction network (BF16 in,
// FP32 accumulate): a 3x3 implicit-GEMM convolution (forward, and the input
// gradient with flipped / transposed weights) and the weight-gradient GEMM.
// Activations are NHWC: element (n, y, x, c) of a tensor with channel stride
// `stride` and channel offset `off` sits at ((n H + y) W + x) stride + off + c,
// so a concatenation is two tensors sharing one buffer at different offsets.
#pragma once
#include <cuda_bf16.h>
#include <stdint.h>

namespace sg {
namespace nn {

typedef __nv_bfloat16 bf16;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// 16-byte asynchronous global -> shared copy; src_bytes = 0 fills zeros
__device__ __forceinline__ void cp_async16(void* dst, const void* src, int src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_u32(dst)), "l"(src), "r"(src_bytes));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

__device__ __forceinline__ void ldsm_x4(uint32_t* r, const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(smem_u32(p)));
}
__device__ __forceinline__ void ldsm_x4_t(uint32_t* r, const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(smem_u32(p)));
}
__device__ __forceinline__ void ldsm_x2_t(uint32_t* r, const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0,%1}, [%2];\n"
               : "=r"(r[0]), "=r"(r[1])
               : "r"(smem_u32(p)));
}

// D(16x8, f32) += A(16x16, bf16, row) * B(16x8, bf16, col)
__device__ __forceinline__ void mma_bf16(float* d, const uint32_t* a, const uint32_t* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

struct ConvArgs {
  const bf16* in;
  int in_stride, in_off;   // input channels [in_off, in_off + Cin)
  const bf16* wt;          // [Cout][9][Cin], tap = 3 (dy+1) + (dx+1)
  const float* bias;       // [Cout] or NULL
  bf16* out;               // BF16 output (NULL: none)
  int out_stride, out_off;
  float* out_f32;          // FP32 output (NULL: none)
  int f32_stride, f32_off;
  int f32_accumulate;      // 1: out_f32 += result
  int N, H, W, Cin, Cout;
  int relu;
  // persistent tcgen05 kernel only (the others reject them): the BF16 output
  // also written 2x2-mean pooled (H/2 x W/2 grid) and nearest-2x upsampled
  // (2H x 2W grid), each at its own pixel stride and channel offset
  bf16* pool_out;
  int pool_stride, pool_off;
  bf16* up_out;
  int up_stride, up_off;
};

constexpr int kConvBM = 128;

// out[p][co] = act(bias[co] + sum_{tap, ci} in[p + tap][ci] * wt[co][tap][ci]),
// zero padding. CTA: 128 pixels x BN output channels, 4 warps of 32 pixels;
// K runs over (tap, 16*KC-channel chunk), double-buffered with cp.async.
template <int BN, int KC>
__global__ void __launch_bounds__(128) k_conv3x3(ConvArgs a) {
  constexpr int BK = 16 * KC;
  constexpr int LD = BK + 8;  // padded row (bf16) so ldmatrix rows hit distinct banks
  __shared__ __align__(16) bf16 sA[2][kConvBM][LD];
  __shared__ __align__(16) bf16 sB[2][BN][LD];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t M = (int64_t)a.N * a.H * a.W;
  const int64_t m0 = (int64_t)blockIdx.x * kConvBM;
  const int n0 = blockIdx.y * BN;
  const int cchunks = a.Cin / BK;
  const int nchunk = 9 * cchunks;

  auto load = [&](int chunk, int st) {
    const int tap = chunk / cchunks, c0 = (chunk % cchunks) * BK;
    const int dy = tap / 3 - 1, dx = tap % 3 - 1;
    constexpr int PPR = BK / 8;  // 16-byte pieces per row
    for (int id = tid; id < kConvBM * PPR; id += 128) {
      const int r = id / PPR, part = id % PPR;
      const int64_t p = m0 + r;
      const bf16* src = a.in;
      int bytes = 0;
      if (p < M) {
        const int x = (int)(p % a.W), y = (int)((p / a.W) % a.H);
        const int64_t n = p / ((int64_t)a.W * a.H);
        const int yy = y + dy, xx = x + dx;
        if (yy >= 0 && yy < a.H && xx >= 0 && xx < a.W) {
          src = a.in + (((n * a.H + yy) * a.W + xx) * a.in_stride + a.in_off + c0 + part * 8);
          bytes = 16;
        }
      }
      cp_async16(&sA[st][r][part * 8], src, bytes);
    }
    for (int id = tid; id < BN * PPR; id += 128) {
      const int r = id / PPR, part = id % PPR;
      const bf16* src = a.wt + ((size_t)(n0 + r) * 9 + tap) * a.Cin + c0 + part * 8;
      cp_async16(&sB[st][r][part * 8], src, 16);
    }
  };

  float acc[2][BN / 8][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < BN / 8; ++j)
#pragma unroll
      for (int k = 0; k < 4; ++k) acc[i][j][k] = 0.f;

  load(0, 0);
  cp_async_commit();
  for (int c = 0; c < nchunk; ++c) {
    if (c + 1 < nchunk) {
      load(c + 1, (c + 1) & 1);
      cp_async_commit();
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    const int st = c & 1;
#pragma unroll
    for (int kk = 0; kk < KC; ++kk) {
      uint32_t af[2][4];
#pragma unroll
      for (int mt = 0; mt < 2; ++mt)
        ldsm_x4(af[mt], &sA[st][warp * 32 + mt * 16 + (lane & 15)][kk * 16 + (lane >> 4) * 8]);
#pragma unroll
      for (int j = 0; j < BN / 16; ++j) {
        uint32_t bfr[4];
        ldsm_x4(bfr, &sB[st][j * 16 + (lane & 7) + (lane >> 4) * 8][kk * 16 + ((lane >> 3) & 1) * 8]);
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
          mma_bf16(acc[mt][2 * j], af[mt], &bfr[0]);
          mma_bf16(acc[mt][2 * j + 1], af[mt], &bfr[2]);
        }
      }
    }
    __syncthreads();
  }

  // epilogue: fragment (row g / g+8, cols 2 tig, 2 tig + 1)
  const int g = lane >> 2, tig = lane & 3;
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int64_t p = m0 + warp * 32 + mt * 16 + g + h * 8;
      if (p >= M) continue;
#pragma unroll
      for (int nt = 0; nt < BN / 8; ++nt) {
        const int co = n0 + nt * 8 + 2 * tig;
        float v0 = acc[mt][nt][2 * h], v1 = acc[mt][nt][2 * h + 1];
        if (a.bias) {
          v0 += a.bias[co];
          v1 += a.bias[co + 1];
        }
        if (a.relu) {
          v0 = fmaxf(v0, 0.f);
          v1 = fmaxf(v1, 0.f);
        }
        if (a.out) {
          *reinterpret_cast<__nv_bfloat162*>(a.out + p * a.out_stride + a.out_off + co) = __floats2bfloat162_rn(v0, v1);
        }
        if (a.out_f32) {
          float2* o = reinterpret_cast<float2*>(a.out_f32 + p * a.f32_stride + a.f32_off + co);
          if (a.f32_accumulate) {
            float2 q = *o;
            q.x += v0;
            q.y += v1;
            *o = q;
          } else {
            *o = make_float2(v0, v1);
          }
        }
      }
    }
}

struct WgradArgs {
  const bf16* dz;  // gradient w.r.t. the conv output (pre-activation), [P][Cout] at dz_stride/dz_off
  int dz_stride, dz_off;
  const bf16* in;  // conv input, [P][Cin] at in_stride/in_off
  int in_stride, in_off;
  float* dw_part;  // [S][9][Cout][Cin]
  float* db_part;  // [S][Cout]
  int N, H, W, Cin, Cout, S;
};

// dW[tap][co][ci] = sum_p dz[p][co] in[p + tap][ci] over split s of the
// pixels: an M = Cout tile (TM), N = Cin tile (TN), K = pixels GEMM. Each of
// the 4 warps takes 32-pixel chunks in turn; partial tiles are summed in
// shared memory and stored (no atomics); a second kernel sums the splits.
template <int TM, int TN>
__global__ void __launch_bounds__(128) k_wgrad(WgradArgs a) {
  constexpr int LDZ = TM + 8, LDX = TN + 8;
  __shared__ __align__(16) bf16 sZ[4][32][LDZ];
  __shared__ __align__(16) bf16 sX[4][32][LDX];
  __shared__ float sRed[TM * TN];
  __shared__ float sBias[4][TM];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int m0 = blockIdx.x * TM, n0 = blockIdx.y * TN;
  const int tap = blockIdx.z / a.S, s = blockIdx.z % a.S;
  const int dy = tap / 3 - 1, dx = tap % 3 - 1;
  const int64_t P = (int64_t)a.N * a.H * a.W;
  const int64_t per = (P + a.S - 1) / a.S;
  const int64_t p_begin = s * per, p_end = min(P, p_begin + per);
  const bool do_bias = (tap == 4 && blockIdx.y == 0);

  float acc[TM / 16][TN / 8][4];
#pragma unroll
  for (int i = 0; i < TM / 16; ++i)
#pragma unroll
    for (int j = 0; j < TN / 8; ++j)
#pragma unroll
      for (int k = 0; k < 4; ++k) acc[i][j][k] = 0.f;
  float bsum = 0.f;  // lane co = lane (< TM)

  for (int64_t pc = p_begin + warp * 32; pc < p_end; pc += 4 * 32) {
    // each lane stages one pixel row of dz (TM channels) and of the shifted input (TN channels)
    const int64_t p = pc + lane;
    {
      uint4* dzr = reinterpret_cast<uint4*>(&sZ[warp][lane][0]);
      uint4* xr = reinterpret_cast<uint4*>(&sX[warp][lane][0]);
      const uint4 zero = make_uint4(0, 0, 0, 0);
      if (p < p_end) {
        const uint4* zs = reinterpret_cast<const uint4*>(a.dz + p * a.dz_stride + a.dz_off + m0);
#pragma unroll
        for (int q = 0; q < TM / 8; ++q) dzr[q] = zs[q];
        const int x = (int)(p % a.W), y = (int)((p / a.W) % a.H);
        const int64_t n = p / ((int64_t)a.W * a.H);
        const int yy = y + dy, xx = x + dx;
        if (yy >= 0 && yy < a.H && xx >= 0 && xx < a.W) {
          const uint4* xs =
              reinterpret_cast<const uint4*>(a.in + ((n * a.H + yy) * a.W + xx) * a.in_stride + a.in_off + n0);
#pragma unroll
          for (int q = 0; q < TN / 8; ++q) xr[q] = xs[q];
        } else {
#pragma unroll
          for (int q = 0; q < TN / 8; ++q) xr[q] = zero;
        }
      } else {
#pragma unroll
        for (int q = 0; q < TM / 8; ++q) dzr[q] = zero;
#pragma unroll
        for (int q = 0; q < TN / 8; ++q) xr[q] = zero;
      }
    }
    __syncwarp();
    if (do_bias && lane < TM)
      for (int k = 0; k < 32; ++k) bsum += __bfloat162float(sZ[warp][k][lane]);
#pragma unroll
    for (int kk = 0; kk < 2; ++kk) {  // two k16 steps over the 32 pixels
      uint32_t af[TM / 16][4];
#pragma unroll
      for (int mt = 0; mt < TM / 16; ++mt)
        ldsm_x4_t(af[mt], &sZ[warp][kk * 16 + (lane >> 4) * 8 + (lane & 7)][mt * 16 + ((lane >> 3) & 1) * 8]);
#pragma unroll
      for (int j = 0; j < TN / 16; ++j) {
        uint32_t bfr[4];
        ldsm_x4_t(bfr, &sX[warp][kk * 16 + ((lane >> 3) & 1) * 8 + (lane & 7)][j * 16 + (lane >> 4) * 8]);
#pragma unroll
        for (int mt = 0; mt < TM / 16; ++mt) {
          mma_bf16(acc[mt][2 * j], af[mt], &bfr[0]);
          mma_bf16(acc[mt][2 * j + 1], af[mt], &bfr[2]);
        }
      }
    }
    __syncwarp();
  }
  // reduce the four warps' tiles
  for (int i = tid; i < TM * TN; i += 128) sRed[i] = 0.f;
  if (lane < TM) sBias[warp][lane] = bsum;
  __syncthreads();
  const int g = lane >> 2, tig = lane & 3;
#pragma unroll
  for (int mt = 0; mt < TM / 16; ++mt)
#pragma unroll
    for (int nt = 0; nt < TN / 8; ++nt)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int r = mt * 16 + g + h * 8, cidx = nt * 8 + 2 * tig;
        atomicAdd(&sRed[r * TN + cidx], acc[mt][nt][2 * h]);
        atomicAdd(&sRed[r * TN + cidx + 1], acc[mt][nt][2 * h + 1]);
      }
  __syncthreads();
  float* dst = a.dw_part + (((size_t)s * 9 + tap) * a.Cout + m0) * a.Cin + n0;
  for (int i = tid; i < TM * TN; i += 128) dst[(size_t)(i / TN) * a.Cin + i % TN] = sRed[i];
  if (do_bias && tid < TM)
    a.db_part[(size_t)s * a.Cout + m0 + tid] = sBias[0][tid] + sBias[1][tid] + sBias[2][tid] + sBias[3][tid];
}

}  // namespace nn
}  // namespace sg
