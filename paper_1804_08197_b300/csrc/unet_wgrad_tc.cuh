// Weight and bias gradients of a 3x3 convolution on tcgen05.
//
//   dW[co][tap][ci] = sum_p dz[p][co] x[p + tap][ci],   db[co] = sum_p dz[p][co]
//
// over the pixels p of N images (x zero outside each image). The pixel
// dimension is the contraction (K), so both operands are made K-major:
//   dzT  [Cout][P]                       the gradient, channel-major;
//   xT3  [3 dx][Cin][N][H + 2][W]        the input, channel-major, one copy per
//                                        horizontal shift dx (zero where x + dx
//                                        leaves the row) with a zero row above
//                                        and below each image.
// For a chunk of 32 consecutive pixels of one image (k0 .. k0 + 31), tap
// (dy, dx) then reads the 32 contiguous elements of xT3[dx][ci][n] starting
// at (1 + dy) W + k0: a TMA box of 32 pixels (64 bytes, 64-byte swizzle) per
// channel row, aligned whenever W is a multiple of 8.
//
// k_wgrad_tc: CTA (ci chunk of NB channels, pixel split s). A TMA producer
// thread stages per chunk one box of dzT (Cout rows; the MMA's rows past
// Cout only feed accumulator rows that are never stored) and nine boxes of
// xT3 (NB rows each). One thread issues per chunk, tap and 16-pixel step a
// tcgen05.mma M = 128 (co) x N = NB (ci) x K = 16 into that tap's TMEM
// accumulator, and (ci chunk 0 only) one against a 16-row tile of ones,
// whose accumulator holds db. The accumulators are stored as the split's
// partial sums, summed by a second kernel in a fixed order (deterministic).
#pragma once
#include <cuda.h>
#include <stdint.h>

#include "unet_ws.cuh"

namespace sg {
namespace nn {

// 16 TMEM columns of this warp's 32 lanes -> registers (the caller waits)
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t* v) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
        "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(taddr));
}

// dzT[c][p] = dz[p * stride + c] (BF16 bits); tiles of 64 pixels x 32
// channels through shared memory, written as pixel pairs (P is even)
__global__ void k_transpose_dz(const uint16_t* __restrict__ dz, int stride, int C, int64_t P,
                               uint16_t* __restrict__ dzT) {
  __shared__ uint16_t t[32][66];
  const int64_t p0 = (int64_t)blockIdx.x * 64;
  const int c0 = blockIdx.y * 32, tx = threadIdx.x;
  for (int r = threadIdx.y; r < 64; r += 8) {
    const int64_t p = p0 + r;
    const int c = c0 + tx;
    t[tx][r] = (p < P && c < C) ? dz[p * stride + c] : (uint16_t)0;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int c = c0 + r;
    const int64_t p = p0 + 2 * tx;
    if (c < C && p < P)
      *reinterpret_cast<uint32_t*>(dzT + (int64_t)c * P + p) = (uint32_t)t[r][2 * tx] | ((uint32_t)t[r][2 * tx + 1] << 16);
  }
}

// The masked output gradient of a layer, in both layouts the backward pass
// uses: dz[p][c] = bf16(dy[p][c] if y[p][c] > 0 (or no y) else 0) for the
// input gradient, and dzT[c][p] for the weight gradient; tiles of 64 pixels x
// 32 channels, the transpose through shared memory
__global__ void k_relu_bwd_t(const float* __restrict__ dy, int dy_stride, int dy_off, const uint16_t* __restrict__ y,
                             int y_stride, int y_off, int C, int64_t P, uint16_t* __restrict__ dz,
                             uint16_t* __restrict__ dzT) {
  __shared__ uint16_t t[32][66];
  const int64_t p0 = (int64_t)blockIdx.x * 64;
  const int c0 = blockIdx.y * 32, tx = threadIdx.x;
  for (int r = threadIdx.y; r < 64; r += 8) {
    const int64_t p = p0 + r;
    const int c = c0 + tx;
    uint16_t v = 0;
    if (p < P && c < C) {
      float f = dy[p * dy_stride + dy_off + c];
      if (y && !(__bfloat162float(__ushort_as_bfloat16(y[p * y_stride + y_off + c])) > 0.f)) f = 0.f;
      v = __bfloat16_as_ushort(__float2bfloat16_rn(f));
      dz[p * C + c] = v;
    }
    t[tx][r] = v;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int c = c0 + r;
    const int64_t p = p0 + 2 * tx;
    if (c < C && p < P)
      *reinterpret_cast<uint32_t*>(dzT + (int64_t)c * P + p) = (uint32_t)t[r][2 * tx] | ((uint32_t)t[r][2 * tx + 1] << 16);
  }
}

// xT3[d][c][n][yp][x] = x[n][yp - 1][x + d - 1][c] (zero outside the image),
// yp in [0, H + 2); block: 64 pixels of one padded row x 32 channels, written
// as pixel pairs (W is even)
__global__ void k_shift_transpose(const uint16_t* __restrict__ x, int stride, int off, int Cin, int N, int H, int W,
                                  uint16_t* __restrict__ xT3) {
  __shared__ uint16_t t[32][67];
  const int nct = (Cin + 31) / 32;
  const int x0 = blockIdx.x * 64, yp = blockIdx.y, n = blockIdx.z / nct, c0 = (blockIdx.z % nct) * 32;
  const int tx = threadIdx.x, y = yp - 1;
  const bool row_in = y >= 0 && y < H;
  for (int j = threadIdx.y; j < 66; j += 8) {
    const int xx = x0 - 1 + j, c = c0 + tx;
    uint16_t v = 0;
    if (row_in && xx >= 0 && xx < W && c < Cin) v = x[(((int64_t)n * H + y) * W + xx) * stride + off + c];
    t[tx][j] = v;
  }
  __syncthreads();
  const int64_t plane = (int64_t)N * (H + 2) * W;
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int c = c0 + r, xo = x0 + 2 * tx;
    if (c >= Cin || xo >= W) continue;
    const int64_t o = (int64_t)c * plane + ((int64_t)n * (H + 2) + yp) * W + xo;
#pragma unroll
    for (int d = 0; d < 3; ++d)
      *reinterpret_cast<uint32_t*>(xT3 + (int64_t)d * Cin * plane + o) =
          (uint32_t)t[r][2 * tx + d] | ((uint32_t)t[r][2 * tx + 1 + d] << 16);
  }
}

struct WgradTcArgs {
  int Cin, Cout, N, H, W;
  int64_t chunks;  // 32-pixel chunks over all images
  int64_t per;     // chunks per split
  float* dw_part;  // [S][9][Cout][Cin]
  float* db_part;  // [S][Cout]
};

template <int NB>
struct WgradTcShape {
  static constexpr int kA = 128 * 64;  // room for the dzT box: up to 128 rows x 32 pixels
  static constexpr int kTap = NB * 64;  // xT3 box of one tap: NB rows x 32 pixels
  static constexpr int kStage = (kA + 9 * kTap + 1023) / 1024 * 1024;
  static constexpr int kMaxStages = 6;
};

template <int NB>
__global__ void __launch_bounds__(128, 1)
    k_wgrad_tc(WgradTcArgs a, int stages, uint32_t* err, const __grid_constant__ CUtensorMap tA,
               const __grid_constant__ CUtensorMap tB) {
  using S = WgradTcShape<NB>;
  constexpr int kBias = 9 * NB;  // TMEM column of the bias accumulator
  constexpr int kCols = kBias + 16 <= 256 ? 256 : 512;
  static_assert(NB == 16 || NB == 32, "channel chunk");
  extern __shared__ uint8_t smem_raw[];
  __shared__ uint64_t full[S::kMaxStages], empty[S::kMaxStages], done_bar;
  __shared__ uint32_t tmem_base_s;
  __shared__ volatile int abort_s;
  __shared__ int skip_s, produced_s, consumed_s, issued_s;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // 64-byte swizzle patterns repeat every 512 bytes: the ones tile and the
  // stages start on 1024
  const uint32_t ones = (smem_u32(smem_raw) + 1023u) & ~1023u;
  const uint32_t ring = ones + 1024;

  if (tid == 0) skip_s = *reinterpret_cast<volatile uint32_t*>(err) != 0;
  __syncthreads();
  if (skip_s) return;

  const int ci0 = blockIdx.x * NB, split = blockIdx.y;
  const bool bias = blockIdx.x == 0;
  const int64_t c_begin = (int64_t)split * a.per;
  const int64_t c_end = c_begin + a.per < a.chunks ? c_begin + a.per : a.chunks;
  const int nck = c_end > c_begin ? (int)(c_end - c_begin) : 0;
  const int cpi = a.H * a.W / 32;  // chunks per image
  const uint32_t tx = (uint32_t)(64 * a.Cout + 9 * S::kTap);  // bytes the copies of one chunk deliver

  // the ones tile: 16 rows x 32 pixels of BF16 1.0 (equal values: the swizzle is moot)
  for (int i = tid; i < 16 * 64 / 4; i += 128)
    asm volatile("st.shared.u32 [%0], %1;\n" ::"r"(ones + 4 * i), "r"(0x3F803F80u) : "memory");
  if (tid == 0) {
    for (int s = 0; s < stages; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&full[s])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&empty[s])));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&done_bar)));
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    abort_s = 0;
    produced_s = consumed_s = issued_s = 0;
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&tmem_base_s)),
                 "r"(kCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  // the ones tile is read by the tensor core (async proxy)
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = tmem_base_s;

  if (warp == 0 && lane == 0) {
    // ---- producer
    int j = 0;
    for (; j < nck; ++j) {
      const int st = j % stages, use = j / stages;
      if (use > 0 && !ws_wait(smem_u32(&empty[st]), (use - 1) & 1, &abort_s)) break;
      const int64_t c = c_begin + j;
      const int n = (int)(c / cpi), k0 = (int)(c % cpi) * 32;
      const uint32_t base = ring + st * S::kStage, fb = smem_u32(&full[st]);
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(fb), "r"(tx) : "memory");
      asm volatile(
          "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n" ::"r"(
              base),
          "l"(reinterpret_cast<uint64_t>(&tA)), "r"((int)((int64_t)n * a.H * a.W + k0)), "r"(0), "r"(fb)
          : "memory");
#pragma unroll
      for (int tap = 0; tap < 9; ++tap) {
        const int dy = tap / 3 - 1, dx = tap % 3 - 1;
        asm volatile(
            "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
            "[%6];\n" ::"r"(base + S::kA + tap * S::kTap),
            "l"(reinterpret_cast<uint64_t>(&tB)), "r"(k0 + (1 + dy) * a.W), "r"(n), "r"(ci0), "r"(dx + 1), "r"(fb)
            : "memory");
      }
    }
    produced_s = j;
    if (j < nck) abort_s = 1;
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer
    constexpr uint32_t idN = tc_idesc(128, NB), id16 = tc_idesc(128, 16);
    int j = 0;
    for (; j < nck; ++j) {
      const int st = j % stages, use = j / stages;
      if (!ws_wait(smem_u32(&full[st]), use & 1, &abort_s)) break;
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      const uint32_t base = ring + st * S::kStage;
#pragma unroll
      for (int kk = 0; kk < 2; ++kk) {
        const uint32_t accum = (j > 0 || kk > 0) ? 1u : 0u;
        const uint64_t da = ws_desc(base + kk * 32, 512, 4);
#pragma unroll
        for (int tap = 0; tap < 9; ++tap) {
          const uint64_t db = ws_desc(base + S::kA + tap * S::kTap + kk * 32, 512, 4);
          asm volatile(
              "{\n\t.reg .pred p;\n\t"
              "setp.ne.b32 p, %4, 0;\n\t"
              "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem + tap * NB),
              "l"(da), "l"(db), "r"(idN), "r"(accum));
        }
        if (bias) {
          const uint64_t db = ws_desc(ones + kk * 32, 512, 4);
          asm volatile(
              "{\n\t.reg .pred p;\n\t"
              "setp.ne.b32 p, %4, 0;\n\t"
              "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem + kBias),
              "l"(da), "l"(db), "r"(id16), "r"(accum));
        }
      }
      issued_s = 1;
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                       smem_u32(&empty[st]))
                   : "memory");
    }
    consumed_s = j;
    if (j < nck) abort_s = 1;
    // every MMA of this CTA is done when done_bar completes
    if (issued_s)
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                       smem_u32(&done_bar))
                   : "memory");
  }
  __syncthreads();
  bool ok = abort_s == 0;
  if (issued_s) ok = __all_sync(0xffffffffu, ws_wait(smem_u32(&done_bar), 0, nullptr)) && ok;
  if (!ok) {
    // after a give-up: wait (bounded) for this CTA's copies in flight
    if (warp == 0 && lane == 0) {
      const int p = produced_s;
      for (int g = consumed_s > p - stages ? consumed_s : p - stages; g < p; ++g)
        ws_wait(smem_u32(&full[g % stages]), (g / stages) & 1, nullptr);
      atomicExch(err, 1u);
    }
  } else {
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    // epilogue: lane = output channel co (warp w: TMEM lanes 32 w .. 32 w + 31)
    const int co = warp * 32 + lane;
    const uint32_t lb = tmem + ((uint32_t)(warp * 32) << 16);
    float* dst = a.dw_part + (int64_t)split * 9 * a.Cout * a.Cin;
#pragma unroll 1
    for (int tap = 0; tap < 9; ++tap)
#pragma unroll
      for (int c = 0; c < NB; c += 16) {
        uint32_t v[16];
        if (nck > 0) {
          tmem_ld16(lb + tap * NB + c, v);
          asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
        } else {
#pragma unroll
          for (int i = 0; i < 16; ++i) v[i] = 0u;
        }
        if (co < a.Cout) {
          float4* o = reinterpret_cast<float4*>(dst + ((int64_t)tap * a.Cout + co) * a.Cin + ci0 + c);
#pragma unroll
          for (int i = 0; i < 4; ++i)
            o[i] = make_float4(__uint_as_float(v[4 * i]), __uint_as_float(v[4 * i + 1]), __uint_as_float(v[4 * i + 2]),
                               __uint_as_float(v[4 * i + 3]));
        }
      }
    if (bias) {
      uint32_t v[16];
      if (nck > 0) {
        tmem_ld16(lb + kBias, v);
        asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
      } else {
        v[0] = 0u;
      }
      if (co < a.Cout) a.db_part[(int64_t)split * a.Cout + co] = __uint_as_float(v[0]);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 1) {
    __syncwarp();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kCols));
  }
}

}  // namespace nn
}  // namespace sg
