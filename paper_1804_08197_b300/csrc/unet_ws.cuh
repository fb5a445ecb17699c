// Persistent, warp-specialised 3x3 convolution on tcgen05 (the halo-reuse
// scheme of k_conv3x3_halo, pipelined across channel chunks and tiles).
//
// A tile is R output rows x 128 pixels x BN output channels of one image;
// the grid holds one CTA per SM and each CTA walks tiles t = blockIdx.x,
// blockIdx.x + gridDim.x, ... Three roles run side by side:
//   warp 0 (one thread)   producer: per CW-channel chunk of a tile, one TMA
//                         tensor copy of the R + 2 input row segments (130
//                         pixels with the halo, zero outside the image) and
//                         one per tap of the chunk's weights, into one stage
//                         of a shared-memory ring;
//   warp 1 (one thread)   MMA issuer: 3 (R + 2) CW / 16 tcgen05.mma
//                         (M = 128 pixels, K = 16) per chunk into one of two
//                         TMEM accumulators; tcgen05.commit frees the stage
//                         and, after a tile's last chunk, hands the
//                         accumulator to
//   warps 2-9             epilogue: tcgen05.ld, bias, ReLU, BF16/FP32 stores,
//                         zeroing of what was read (tcgen05.st), then release
//                         of the accumulator to the MMA issuer; two warps per
//                         TMEM lane quarter (32 pixels), each taking every
//                         other output row.
// So the loads of chunk c + 1 overlap the MMAs of chunk c, and the epilogue
// of one tile overlaps the MMAs of the next.
//
// Copies: a pixel's CW channels are one 2 CW-byte row of the TMA box (64 B
// for CW = 32), and the operands use the matching swizzled K-major layout
// (64-byte swizzle for CW = 32, 32-byte for CW = 16): a TMA box row of 16
// bytes costs about as much as one of 64, so wide rows move a chunk with a
// quarter of the requests of one 8-channel plane per copy.
//
// One MMA per input row i, horizontal shift dx and 16-channel step serves
// the (up to) three output rows that row feeds: its B operand is the
// weights of taps dy = +1, 0, -1 side by side (N = 3 BN; 2 BN or BN at the
// band's edge rows) and its D the accumulators of output rows i - 2, i - 1,
// i, side by side in TMEM. So the tensor core fetches each input row segment
// 3 times per chunk instead of 9. Such an MMA adds to rows that earlier MMAs
// already hold and to rows not yet touched, so the accumulators start at
// zero instead of being overwritten by a first MMA.
//
// Shared-memory stage (1024-byte aligned): the input [R + 2 rows][130 px]
// [2 CW bytes], then the weights [3 dx][3 dy: +1, 0, -1][BN rows][2 CW
// bytes], both swizzled by the TMA. A of input row i, shift dx starts
// (130 i + dx) rows in; B of shift dx starts at its weights; both advance 32
// bytes per 16-channel step; 8-row groups are 16 CW bytes apart.
//
// Every wait is bounded (about a second) and gives up early once another
// role has given up; the CTA then drains its own copies and MMAs in flight
// (again bounded), raises the error word and frees its TMEM.
#pragma once
#include <cuda.h>
#include <stdint.h>

#include "unet_tc.cuh"

namespace sg {
namespace nn {

constexpr int kWsMaxStages = 6;
constexpr int kWsThreads = 320;  // producer warp, MMA warp, 8 epilogue warps

template <int BN, int R, int CW>
struct WsShape {
  static constexpr int kRowPitch = 2 * CW;                                  // bytes of one pixel's chunk
  static constexpr int kRow = 130 * kRowPitch;                              // one input row segment
  static constexpr int kA = ((R + 2) * kRow + 1023) / 1024 * 1024;          // input part of a stage
  static constexpr int kBlk = BN * kRowPitch;                               // one tap's weights
  static constexpr int kDx = 3 * kBlk;                                      // the weights of one dx
  static constexpr int kStage = (kA + 9 * kBlk + 1023) / 1024 * 1024;
  static constexpr uint32_t kTx = (uint32_t)((R + 2) * kRow + 9 * kBlk);  // bytes one chunk's copies deliver
};

// bounded wait that also returns (false) once *abort is set
__device__ __forceinline__ bool ws_wait(uint32_t bar, uint32_t parity, volatile int* abort) {
  for (uint32_t i = 0; i < kTcSpinLimit; ++i) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
    if (i >= 32) {
      if (abort && *abort) return false;
      __nanosleep(64);
    }
  }
  return false;
}

// zeroes 16 TMEM columns of this warp's 32 lanes
__device__ __forceinline__ void tmem_zero16(uint32_t taddr) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1};\n" ::"r"(taddr),
      "r"(0u)
      : "memory");
}

// Shared-memory descriptor of a swizzled K-major operand: start address,
// stride byte offset between 8-row groups and the swizzle mode (bits 61-63:
// 4 = 64-byte, 6 = 32-byte); the leading byte offset is unused (one MMA's 16
// channels lie inside one swizzled row). The swizzle follows the address
// bits, like the TMA's, so an operand may start any number of rows into a
// pattern with base offset 0 (a start shifted by dx pixels reads what the
// copy wrote there; parity against the unswizzled paths checks this).
__device__ __forceinline__ uint64_t ws_desc(uint32_t addr, uint32_t sbo, uint32_t mode) {
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)1 << 16) | ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) |
         (1ull << 46) | ((uint64_t)mode << 61);
}

// The network's output written by the head convolution's epilogue (its 16
// channels per half-rate pixel): out = bilinear 2x upsampling of the RGBA
// input (half-pixel centres, edges clamped) + pixel shuffle of the head.
struct HeadOut {
  const float* in[64];          // per image: RGBA input rows, in_pitch floats apart
  float* out[64];               // per image: RGBA output rows (2H x 2W), out_pitch floats apart
  int64_t in_pitch, out_pitch;
  int on;                       // 0: the convolution writes out / out_f32 as usual
};

// output pixels (2y + sy, 2x + sx) of image n from the head's 16 values v
__device__ __forceinline__ void ws_head_out(const HeadOut& ho, int n, int y, int x, int H, int W, const float* v) {
  const float* src = ho.in[n];
  float4 nb[3][3];  // the clamped 3 x 3 neighbourhood of the input pixel
#pragma unroll
  for (int dy = 0; dy < 3; ++dy)
#pragma unroll
    for (int dx = 0; dx < 3; ++dx) {
      const int yy = min(max(y + dy - 1, 0), H - 1), xx = min(max(x + dx - 1, 0), W - 1);
      nb[dy][dx] = *reinterpret_cast<const float4*>(src + (int64_t)yy * ho.in_pitch + xx * 4);
    }
#pragma unroll
  for (int sy = 0; sy < 2; ++sy)
#pragma unroll
    for (int sx = 0; sx < 2; ++sx) {
      const int Y = 2 * y + sy, X = 2 * x + sx;
      const float ux = 0.5f * X - 0.25f, uy = 0.5f * Y - 0.25f;
      const float fx0 = floorf(ux), fy0 = floorf(uy);
      const float fx = ux - fx0, fy = uy - fy0;
      const int x0 = min(max((int)fx0, 0), W - 1) - x + 1, x1 = min(max((int)fx0 + 1, 0), W - 1) - x + 1;
      const int y0 = min(max((int)fy0, 0), H - 1) - y + 1, y1 = min(max((int)fy0 + 1, 0), H - 1) - y + 1;
      const float4 v00 = nb[y0][x0], v01 = nb[y0][x1], v10 = nb[y1][x0], v11 = nb[y1][x1];
      const float a00 = (1.f - fy) * (1.f - fx), a01 = (1.f - fy) * fx, a10 = fy * (1.f - fx), a11 = fy * fx;
      const int sh = sy * 2 + sx;
      float4 o;
      o.x = a00 * v00.x + a01 * v01.x + a10 * v10.x + a11 * v11.x + v[sh];
      o.y = a00 * v00.y + a01 * v01.y + a10 * v10.y + a11 * v11.y + v[sh + 4];
      o.z = a00 * v00.z + a01 * v01.z + a10 * v10.z + a11 * v11.z + v[sh + 8];
      o.w = a00 * v00.w + a01 * v01.w + a10 * v10.w + a11 * v11.w + v[sh + 12];
      *reinterpret_cast<float4*>(ho.out[n] + (int64_t)Y * ho.out_pitch + X * 4) = o;
    }
}

template <int BN, int R, int CW>
__global__ void __launch_bounds__(kWsThreads, 1)
    k_conv3x3_ws(ConvArgs a, int stages, uint32_t* err, const __grid_constant__ CUtensorMap tin,
                 const __grid_constant__ CUtensorMap twt, const __grid_constant__ HeadOut ho) {
  using S = WsShape<BN, R, CW>;
  constexpr int kAcc = R * BN;  // TMEM columns of one accumulator
  constexpr int kCols =
      2 * kAcc <= 32 ? 32 : (2 * kAcc <= 64 ? 64 : (2 * kAcc <= 128 ? 128 : (2 * kAcc <= 256 ? 256 : 512)));
  constexpr uint32_t kMode = CW == 32 ? 4u : 6u;  // 64-byte / 32-byte swizzle
  constexpr uint32_t kSbo = 8 * S::kRowPitch;
  static_assert(2 * kAcc <= 512, "two accumulators must fit in TMEM");
  static_assert(BN % 16 == 0 && 3 * BN <= 256 && R >= 2, "N of the MMA, rows per tile");
  static_assert(CW == 16 || CW == 32, "chunk width");
  static_assert(S::kBlk % 512 == 0, "weight blocks aligned to the swizzle pattern");
  extern __shared__ uint8_t smem_raw[];
  __shared__ uint64_t full[kWsMaxStages], empty[kWsMaxStages], tfull[2], tempty[2], done_bar;
  __shared__ uint32_t tmem_base_s;
  __shared__ volatile int abort_s;
  __shared__ int skip_s, produced_s, consumed_s, issued_s;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // the swizzle patterns repeat every 256 / 512 bytes: stages start on 1024
  const uint32_t smem0 = (smem_u32(smem_raw) + 1023u) & ~1023u;

  // an earlier CTA gave up on a wait: the outputs are invalid anyway
  if (tid == 0) skip_s = *reinterpret_cast<volatile uint32_t*>(err) != 0;
  __syncthreads();
  if (skip_s) return;

  const int tiles_x = (a.W + 127) / 128, bands = (a.H + R - 1) / R, nz = a.Cout / BN;
  const int nt = a.N * bands * tiles_x * nz, nch = a.Cin / CW;
  if (tid == 0) {
    for (int s = 0; s < stages; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&full[s])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&empty[s])));
    }
    for (int b = 0; b < 2; ++b) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&tfull[b])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 8;\n" ::"r"(smem_u32(&tempty[b])));
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
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = tmem_base_s;

  // tile t -> (image n, first row y0, first pixel x0, output-channel block z);
  // the channel blocks of one pixel tile are neighbours (shared input in L2)
  auto decode = [&](int t, int& n, int& y0, int& x0, int& z) {
    z = t % nz;
    int q = t / nz;
    x0 = (q % tiles_x) * 128;
    q /= tiles_x;
    y0 = (q % bands) * R;
    n = q / bands;
  };

  if (warp == 0) {
    if (lane == 0) {
      // ---- producer
      int f = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < nt && ok; t += gridDim.x) {
        int n, y0, x0, z;
        decode(t, n, y0, x0, z);
        for (int ch = 0; ch < nch; ++ch) {
          const int st = f % stages, use = f / stages;
          if (use > 0 && !ws_wait(smem_u32(&empty[st]), (use - 1) & 1, &abort_s)) {
            ok = false;
            break;
          }
          const uint32_t base = smem0 + st * S::kStage, fb = smem_u32(&full[st]);
          asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(fb), "r"(S::kTx) : "memory");
          asm volatile(
              "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
              "%5}], [%6];\n" ::"r"(base),
              "l"(reinterpret_cast<uint64_t>(&tin)), "r"(a.in_off + ch * CW), "r"(x0 - 1), "r"(y0 - 1), "r"(n),
              "r"(fb)
              : "memory");
#pragma unroll
          for (int tap = 0; tap < 9; ++tap)
            asm volatile(
                "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
                "[%4];\n" ::"r"(base + S::kA + (tap % 3) * S::kDx + (2 - tap / 3) * S::kBlk),
                "l"(reinterpret_cast<uint64_t>(&twt)), "r"(tap * a.Cin + ch * CW), "r"(z * BN), "r"(fb)
                : "memory");
          ++f;
        }
      }
      produced_s = f;
      if (!ok) abort_s = 1;
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---- MMA issuer
      constexpr uint32_t id1 = tc_idesc(128, BN), id2 = tc_idesc(128, 2 * BN), id3 = tc_idesc(128, 3 * BN);
      int f = 0, j = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < nt && ok; t += gridDim.x, ++j) {
        const int b = j & 1, u = j >> 1;
        // phase u of tempty[b]: the accumulator is zero (set up, or read and cleared)
        if (!ws_wait(smem_u32(&tempty[b]), u & 1, &abort_s)) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        for (int ch = 0; ch < nch; ++ch) {
          const int st = f % stages, use = f / stages;
          if (!ws_wait(smem_u32(&full[st]), use & 1, &abort_s)) {
            ok = false;
            break;
          }
          ++f;
          asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
          const uint32_t base = smem0 + st * S::kStage;
#pragma unroll
          for (int i = 0; i < R + 2; ++i) {
            // output rows r_lo .. r_hi take input row i (through dy = i - 1 - r)
            const int r_lo = i - 2 > 0 ? i - 2 : 0, r_hi = i < R - 1 ? i : R - 1;
            const int nb = r_hi - r_lo + 1, blk0 = r_lo - i + 2;
            const uint32_t idesc = nb == 1 ? id1 : (nb == 2 ? id2 : id3);
#pragma unroll
            for (int dx = 0; dx < 3; ++dx)
#pragma unroll
              for (int kk = 0; kk < CW / 16; ++kk) {
                const uint32_t aaddr = base + (i * 130 + dx) * S::kRowPitch + kk * 32;
                const uint64_t da = ws_desc(aaddr, kSbo, kMode);
                const uint64_t db = ws_desc(base + S::kA + dx * S::kDx + blk0 * S::kBlk + kk * 32, kSbo, kMode);
                asm volatile(
                    "{\n\t.reg .pred p;\n\t"
                    "setp.ne.b32 p, %4, 0;\n\t"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem + b * kAcc + r_lo * BN),
                    "l"(da), "l"(db), "r"(idesc), "r"(1u));
              }
          }
          issued_s = 1;
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                           smem_u32(&empty[st]))
                       : "memory");
        }
        if (!ok) break;
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                         smem_u32(&tfull[b]))
                     : "memory");
      }
      consumed_s = f;
      if (!ok) abort_s = 1;
    }
  } else {
    // ---- epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31, rows eh, eh + 2, ...
    const int eq = warp & 3, eh = (warp - 2) >> 2;
    const uint32_t lane_base = tmem + ((uint32_t)(eq * 32) << 16);
    // both accumulators start at zero (phase 0 of tempty)
#pragma unroll 1
    for (int bb = 0; bb < 2; ++bb)
#pragma unroll 1
      for (int r = eh; r < R; r += 2)
#pragma unroll
        for (int c0 = 0; c0 < BN; c0 += 16) tmem_zero16(lane_base + bb * kAcc + r * BN + c0);
    asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncwarp();
    if (lane == 0) {
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(&tempty[0])) : "memory");
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(&tempty[1])) : "memory");
    }
    int j = 0;
    for (int t = blockIdx.x; t < nt; t += gridDim.x, ++j) {
      const int b = j & 1, u = j >> 1;
      const bool ok = __all_sync(0xffffffffu, ws_wait(smem_u32(&tfull[b]), u & 1, &abort_s));
      if (!ok) {
        if (lane == 0) abort_s = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      int n, y0, x0, z;
      decode(t, n, y0, x0, z);
      const int x = x0 + eq * 32 + lane, n0 = z * BN;
#pragma unroll
      for (int c0 = 0; c0 < BN; c0 += 16) {
        float bias[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) bias[i] = a.bias ? __ldg(a.bias + n0 + c0 + i) : 0.f;
#pragma unroll 1
        for (int r = eh; r < R; r += 2) {
          const int y = y0 + r;
          uint32_t v32[16];
          const uint32_t taddr = lane_base + b * kAcc + r * BN + c0;
          asm volatile(
              "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
              : "=r"(v32[0]), "=r"(v32[1]), "=r"(v32[2]), "=r"(v32[3]), "=r"(v32[4]), "=r"(v32[5]), "=r"(v32[6]),
                "=r"(v32[7]), "=r"(v32[8]), "=r"(v32[9]), "=r"(v32[10]), "=r"(v32[11]), "=r"(v32[12]), "=r"(v32[13]),
                "=r"(v32[14]), "=r"(v32[15])
              : "r"(taddr));
          asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
          tmem_zero16(taddr);  // ready for the tile after next
          if (x < a.W && y < a.H) {
            const int64_t pr = ((int64_t)n * a.H + y) * a.W + x;
            float v[16];
#pragma unroll
            for (int i = 0; i < 16; ++i) {
              v[i] = __uint_as_float(v32[i]) + bias[i];
              if (a.relu) v[i] = fmaxf(v[i], 0.f);
            }
            if (a.out) {
              uint32_t packed[8];
#pragma unroll
              for (int i = 0; i < 8; ++i) {
                __nv_bfloat162 h2 = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
                packed[i] = *reinterpret_cast<uint32_t*>(&h2);
              }
              uint4* o = reinterpret_cast<uint4*>(a.out + pr * a.out_stride + a.out_off + n0 + c0);
              o[0] = make_uint4(packed[0], packed[1], packed[2], packed[3]);
              o[1] = make_uint4(packed[4], packed[5], packed[6], packed[7]);
            }
            if (BN == 16 && ho.on) ws_head_out(ho, n, y, x, a.H, a.W, v);
            if (a.out_f32) {
              float4* o = reinterpret_cast<float4*>(a.out_f32 + pr * a.f32_stride + a.f32_off + n0 + c0);
#pragma unroll
              for (int i = 0; i < 4; ++i) {
                float4 q = make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
                if (a.f32_accumulate) {
                  const float4 o0 = o[i];
                  q.x += o0.x; q.y += o0.y; q.z += o0.z; q.w += o0.w;
                }
                o[i] = q;
              }
            }
          }
        }
      }
      // the accumulator is read and zero again: hand it back to the MMA issuer
      asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory");
      asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(&tempty[b])) : "memory");
    }
  }
  __syncthreads();
  // after a give-up: wait (bounded) for this CTA's own copies and MMAs in flight
  if (abort_s) {
    if (warp == 0 && lane == 0) {
      const int p = produced_s;
      for (int g = consumed_s > p - stages ? consumed_s : p - stages; g < p; ++g)
        ws_wait(smem_u32(&full[g % stages]), (g / stages) & 1, nullptr);
    }
    if (warp == 1 && lane == 0 && issued_s) {
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                       smem_u32(&done_bar))
                   : "memory");
      ws_wait(smem_u32(&done_bar), 0, nullptr);
    }
    if (tid == 0) atomicExch(err, 1u);
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
