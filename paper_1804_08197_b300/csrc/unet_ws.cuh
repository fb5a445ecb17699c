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
//   warps 2-9             epilogue: tcgen05.ld, ReLU, BF16/FP32 stores
//                         (optionally also 2x2-pooled or nearest-2x
//                         upsampled copies of the BF16 output), the next
//                         tile's bias written over what was read
//                         (tcgen05.st), then release of the accumulator to
//                         the MMA issuer; two warps per TMEM lane quarter
//                         (32 pixels), each taking every other output row
//                         (every other row pair when pooling).
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
// the bias (written by the epilogue) instead of being overwritten by a first
// MMA.
//
// After the ring, each epilogue warp has a staging row of 32 pixels x BN
// BF16 channels: its TMEM reads land there one pixel per lane and leave as
// 16-byte chunks with the lanes of a pixel side by side, so a store covers
// whole pixel rows instead of one 32-byte piece per lane.
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
constexpr int kWsMaxCout = 256;  // output channels of a layer

template <int BN, int R, int CW>
struct WsShape {
  static constexpr int kRowPitch = 2 * CW;                                  // bytes of one pixel's chunk
  static constexpr int kRow = 130 * kRowPitch;                              // one input row segment
  static constexpr int kA = ((R + 2) * kRow + 1023) / 1024 * 1024;          // input part of a stage
  static constexpr int kBlk = BN * kRowPitch;                               // one tap's weights
  static constexpr int kDx = 3 * kBlk;                                      // the weights of one dx
  static constexpr int kStage = (kA + 9 * kBlk + 1023) / 1024 * 1024;
  static constexpr uint32_t kTx = (uint32_t)((R + 2) * kRow + 9 * kBlk);  // bytes one chunk's copies deliver
  static constexpr int kCpp = BN / 8;                                       // 16-byte chunks of a pixel's BN channels
  static constexpr int kOut = 32 * BN * 2;                                  // one epilogue warp's row: 32 px x BN BF16
};

// 16-byte slot of chunk `sub` of pixel p in an epilogue warp's staging row:
// the chunk index is XOR-ed with a function of p so that any 8 lanes storing
// one chunk of 8 pixels, or loading the chunks of consecutive pixels, hit 8
// different 16-byte bank groups
template <int CPP>
__device__ __forceinline__ int ws_slot(int p, int sub) {
  return p * CPP + (sub ^ ((p / (8 / CPP)) % CPP));
}

// one 32-lane x N-column TMEM load (FP32 bit patterns, N = 16 or 32), waited for
template <int N>
__device__ __forceinline__ void ws_ld(uint32_t taddr, uint32_t (&v)[N]) {
  static_assert(N == 16 || N == 32, "columns per load");
  if constexpr (N == 16) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
          "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(taddr));
  } else {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,"
        "%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
          "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]),
          "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
          "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(taddr));
  }
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
}

// the same N columns of every lane of the warp set to bias[0..N) (shared
// memory, the same for each lane): an accumulator's starting value
template <int N>
__device__ __forceinline__ void ws_st_bias(uint32_t taddr, uint32_t bias_smem) {
  uint32_t v[N];
#pragma unroll
  for (int i = 0; i < N; i += 4)
    asm volatile("ld.shared.v4.b32 {%0, %1, %2, %3}, [%4];\n"
                 : "=r"(v[i]), "=r"(v[i + 1]), "=r"(v[i + 2]), "=r"(v[i + 3])
                 : "r"(bias_smem + 4u * i));
  if constexpr (N == 16) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};\n" ::"r"(
            taddr),
        "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]), "r"(v[9]),
        "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15])
        : "memory");
  } else {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,"
        "%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};\n" ::"r"(taddr),
        "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]), "r"(v[9]),
        "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15]), "r"(v[16]), "r"(v[17]), "r"(v[18]),
        "r"(v[19]), "r"(v[20]), "r"(v[21]), "r"(v[22]), "r"(v[23]), "r"(v[24]), "r"(v[25]), "r"(v[26]), "r"(v[27]),
        "r"(v[28]), "r"(v[29]), "r"(v[30]), "r"(v[31])
        : "memory");
  }
}

__device__ __forceinline__ float bf_lo(uint32_t p) { return __uint_as_float(p << 16); }
__device__ __forceinline__ float bf_hi(uint32_t p) { return __uint_as_float(p & 0xFFFF0000u); }

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

// output pixels (2y + sy, 2x + sx) of image n from the head's 16 values v.
// Output pixel X = 2x + sx samples the input at x - 1/4 (sx = 0) or x + 1/4
// (sx = 1): between columns x - 1 and x with weights 1/4, 3/4, or x and
// x + 1 with 3/4, 1/4; rows alike. Edges clamp the indices (the clamped
// 3 x 3 neighbourhood below), never the weights.
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
      // the interpolation's first row / column in the neighbourhood and the
      // weight of the second (fy, fx)
      const float fy = sy ? 0.25f : 0.75f, fx = sx ? 0.25f : 0.75f;
      const float4 v00 = nb[sy][sx], v01 = nb[sy][sx + 1], v10 = nb[sy + 1][sx], v11 = nb[sy + 1][sx + 1];
      const float a00 = (1.f - fy) * (1.f - fx), a01 = (1.f - fy) * fx, a10 = fy * (1.f - fx), a11 = fy * fx;
      const int sh = sy * 2 + sx;
      float4 o;
      o.x = a00 * v00.x + a01 * v01.x + a10 * v10.x + a11 * v11.x + v[sh];
      o.y = a00 * v00.y + a01 * v01.y + a10 * v10.y + a11 * v11.y + v[sh + 4];
      o.z = a00 * v00.z + a01 * v01.z + a10 * v10.z + a11 * v11.z + v[sh + 8];
      o.w = a00 * v00.w + a01 * v01.w + a10 * v10.w + a11 * v11.w + v[sh + 12];
      *reinterpret_cast<float4*>(ho.out[n] + (int64_t)(2 * y + sy) * ho.out_pitch + (2 * x + sx) * 4) = o;
    }
}

template <int BN, int R, int CW>
__global__ void __launch_bounds__(kWsThreads, 1)
    k_conv3x3_ws(ConvArgs a, int stages, int wres, uint32_t* err, const __grid_constant__ CUtensorMap tin,
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
  __shared__ uint64_t full[kWsMaxStages], empty[kWsMaxStages], tfull[2], tempty[2], done_bar, wfull;
  __shared__ uint32_t tmem_base_s;
  __shared__ volatile int abort_s;
  __shared__ int skip_s, produced_s, consumed_s, issued_s, wissued_s;
  __shared__ __align__(16) float bias_s[kWsMaxCout];  // the layer's bias (zero without one)
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // the swizzle patterns repeat every 256 / 512 bytes: stages start on 1024
  const uint32_t smem0 = (smem_u32(smem_raw) + 1023u) & ~1023u;

  // an earlier CTA gave up on a wait: the outputs are invalid anyway
  if (tid == 0) skip_s = *reinterpret_cast<volatile uint32_t*>(err) != 0;
  __syncthreads();
  if (skip_s) return;
  for (int i = tid; i < a.Cout; i += kWsThreads) bias_s[i] = a.bias ? __ldg(a.bias + i) : 0.f;

  const int tiles_x = (a.W + 127) / 128, bands = (a.H + R - 1) / R, nz = a.Cout / BN;
  const int nt = a.N * bands * tiles_x * nz, nch = a.Cin / CW;
  // resident weights (one output-channel block, wres = 1): the ring holds
  // only input, and every chunk's weights sit after it, loaded once
  const uint32_t sstride = wres ? (uint32_t)S::kA : (uint32_t)S::kStage;
  const uint32_t wbase = smem0 + (uint32_t)stages * sstride;
  const uint32_t wbytes = wres ? (uint32_t)((nch * 9 * S::kBlk + 1023) / 1024 * 1024) : 0u;
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
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&wfull)));
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    abort_s = 0;
    produced_s = consumed_s = issued_s = wissued_s = 0;
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
      if (wres) {
        const uint32_t wb = smem_u32(&wfull);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(wb),
                     "r"((uint32_t)(nch * 9 * S::kBlk))
                     : "memory");
        for (int ch = 0; ch < nch; ++ch)
#pragma unroll
          for (int tap = 0; tap < 9; ++tap)
            asm volatile(
                "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
                "[%4];\n" ::"r"(wbase + (uint32_t)(ch * 9 * S::kBlk + (tap % 3) * S::kDx + (2 - tap / 3) * S::kBlk)),
                "l"(reinterpret_cast<uint64_t>(&twt)), "r"(tap * a.Cin + ch * CW), "r"(0), "r"(wb)
                : "memory");
        wissued_s = 1;
      }
      for (int t = blockIdx.x; t < nt && ok; t += gridDim.x) {
        int n, y0, x0, z;
        decode(t, n, y0, x0, z);
        for (int ch = 0; ch < nch; ++ch) {
          const int st = f % stages, use = f / stages;
          if (use > 0 && !ws_wait(smem_u32(&empty[st]), (use - 1) & 1, &abort_s)) {
            ok = false;
            break;
          }
          const uint32_t base = smem0 + st * sstride, fb = smem_u32(&full[st]);
          const uint32_t tx = wres ? S::kTx - (uint32_t)(9 * S::kBlk) : S::kTx;
          asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(fb), "r"(tx) : "memory");
          asm volatile(
              "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
              "%5}], [%6];\n" ::"r"(base),
              "l"(reinterpret_cast<uint64_t>(&tin)), "r"(a.in_off + ch * CW), "r"(x0 - 1), "r"(y0 - 1), "r"(n),
              "r"(fb)
              : "memory");
          if (!wres)
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
      bool ok = !wres || ws_wait(smem_u32(&wfull), 0, &abort_s);
      for (int t = blockIdx.x; t < nt && ok; t += gridDim.x, ++j) {
        const int b = j & 1, u = j >> 1;
        // phase u of tempty[b]: the accumulator holds the bias (set up, or read and refilled)
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
          const uint32_t base = smem0 + st * sstride;
          const uint32_t wch = wres ? wbase + (uint32_t)(ch * 9 * S::kBlk) : base + (uint32_t)S::kA;
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
                const uint64_t db = ws_desc(wch + dx * S::kDx + blk0 * S::kBlk + kk * 32, kSbo, kMode);
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
    // ---- epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 (pixels), the
    // rows eh, eh + 2, ...; when pooling, the row pairs (2p, 2p + 1) for
    // p = eh, eh + 2, ..., so that a warp holds both rows of a window
    const int eq = warp & 3, eh = (warp - 2) >> 2;
    const uint32_t lane_base = tmem + ((uint32_t)(eq * 32) << 16);
    const bool pool = a.pool_out != nullptr;
    constexpr int kCh = BN < 32 ? BN : 32;  // TMEM columns per load
    auto row_of = [&](int q) { return pool ? 4 * (q >> 1) + 2 * eh + (q & 1) : eh + 2 * q; };
    const uint32_t bias0 = smem_u32(bias_s);
    // an accumulator starts at the bias of its tile's output-channel block,
    // so the MMAs add onto it: accumulators 0 and 1 for this CTA's first two tiles
#pragma unroll 1
    for (int bb = 0; bb < 2; ++bb) {
      const int t = blockIdx.x + bb * gridDim.x;
      if (t >= nt) break;
      const uint32_t bz = bias0 + 4u * (uint32_t)((t % nz) * BN);
#pragma unroll 1
      for (int q = 0; q < R / 2; ++q)
#pragma unroll
        for (int c = 0; c < BN; c += kCh)
          ws_st_bias<kCh>(lane_base + bb * kAcc + row_of(q) * BN + c, bz + 4u * c);
    }
    asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncwarp();
    if (lane == 0) {
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(&tempty[0])) : "memory");
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(&tempty[1])) : "memory");
    }
    // this warp's staging row (after the ring): 32 pixels x BN BF16 channels
    const uint32_t ostage = wbase + wbytes + (uint32_t)(warp - 2) * S::kOut;
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
      const int xw = x0 + eq * 32, x = xw + lane, n0 = z * BN;
      // the tile after next takes this accumulator over: its bias block
      const int tn = t + 2 * gridDim.x;
      const bool refill = tn < nt;
      const uint32_t bzn = bias0 + 4u * (uint32_t)((tn % nz) * BN);
      uint32_t held[BN / 2];  // the BF16 outputs of a pooling window's first row (pairs)
#pragma unroll 1
      for (int q = 0; q < R / 2; ++q) {
        const int r = row_of(q);
        const int y = y0 + r;
        const bool inside = x < a.W && y < a.H;
        const bool second = pool && (q & 1);
#pragma unroll
        for (int c = 0; c < BN; c += kCh) {
          uint32_t v[kCh];
          const uint32_t taddr = lane_base + b * kAcc + r * BN + c;
          ws_ld<kCh>(taddr, v);
          if (refill) ws_st_bias<kCh>(taddr, bzn + 4u * c);  // ready for the tile after next
          float f[kCh];
#pragma unroll
          for (int i = 0; i < kCh; ++i) f[i] = a.relu ? fmaxf(__uint_as_float(v[i]), 0.f) : __uint_as_float(v[i]);
          uint32_t pk[kCh / 2];
#pragma unroll
          for (int i = 0; i < kCh / 2; ++i) {
            __nv_bfloat162 h2 = __floats2bfloat162_rn(f[2 * i], f[2 * i + 1]);
            pk[i] = *reinterpret_cast<uint32_t*>(&h2);
          }
          if (pool) {
            if (!second) {
#pragma unroll
              for (int i = 0; i < kCh / 2; ++i) held[c / 2 + i] = pk[i];
            } else {
              // 2x2 mean of the BF16 values as stored, summed in the order
              // (y-1, x), (y-1, x+1), (y, x), (y, x+1). The even lane of a
              // pixel pair pools the chunk's first half of channels, the odd
              // lane the second: each trades the half it does not pool for
              // its neighbour's half of the one it does (x is even on even
              // lanes: tiles start at multiples of 128 pixels)
              const bool odd = lane & 1;
              constexpr int kH = kCh / 4;  // packed pairs in half a chunk
              float ps[2 * kH];
#pragma unroll
              for (int i = 0; i < kH; ++i) {
                const uint32_t a0 = held[c / 2 + i], a1 = held[c / 2 + kH + i];
                const uint32_t b0 = pk[i], b1 = pk[kH + i];
                // mine: the half this lane pools; theirs: the neighbour's copy of it
                const uint32_t m0 = odd ? a1 : a0, m1 = odd ? b1 : b0;
                const uint32_t t0 = __shfl_xor_sync(0xffffffffu, odd ? a0 : a1, 1);
                const uint32_t t1 = __shfl_xor_sync(0xffffffffu, odd ? b0 : b1, 1);
                // (y-1, x) + (y-1, x+1) + (y, x) + (y, x+1): x is the even pixel
                const uint32_t e0 = odd ? t0 : m0, o0 = odd ? m0 : t0, e1 = odd ? t1 : m1, o1 = odd ? m1 : t1;
                ps[2 * i] = ((bf_lo(e0) + bf_lo(o0)) + bf_lo(e1)) + bf_lo(o1);
                ps[2 * i + 1] = ((bf_hi(e0) + bf_hi(o0)) + bf_hi(e1)) + bf_hi(o1);
              }
              if (inside) {
                uint32_t po[kH];
#pragma unroll
                for (int i = 0; i < kH; ++i) {
                  __nv_bfloat162 h2 = __floats2bfloat162_rn(ps[2 * i] * 0.25f, ps[2 * i + 1] * 0.25f);
                  po[i] = *reinterpret_cast<uint32_t*>(&h2);
                }
                const int64_t pp = ((int64_t)n * (a.H >> 1) + (y >> 1)) * (a.W >> 1) + (x >> 1);
                uint4* o = reinterpret_cast<uint4*>(a.pool_out + pp * a.pool_stride + a.pool_off + n0 + c +
                                                    (odd ? kCh / 2 : 0));
#pragma unroll
                for (int i = 0; i < kH / 4; ++i) o[i] = make_uint4(po[4 * i], po[4 * i + 1], po[4 * i + 2], po[4 * i + 3]);
              }
            }
          }
          if (a.out) {
            // BF16 into the staging row (pixel = lane), written out below
#pragma unroll
            for (int hh = 0; hh < kCh / 8; ++hh)
              asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};\n" ::"r"(
                               ostage + 16u * ws_slot<S::kCpp>(lane, c / 8 + hh)),
                           "r"(pk[4 * hh]), "r"(pk[4 * hh + 1]), "r"(pk[4 * hh + 2]), "r"(pk[4 * hh + 3])
                           : "memory");
          }
          if (inside) {
            const int64_t pr = ((int64_t)n * a.H + y) * a.W + x;
            if constexpr (BN == 16) {
              if (ho.on) ws_head_out(ho, n, y, x, a.H, a.W, f);
            }
            if (a.out_f32) {
              float4* o = reinterpret_cast<float4*>(a.out_f32 + pr * a.f32_stride + a.f32_off + n0 + c);
#pragma unroll
              for (int i = 0; i < kCh / 4; ++i) {
                float4 q4 = make_float4(f[4 * i], f[4 * i + 1], f[4 * i + 2], f[4 * i + 3]);
                if (a.f32_accumulate) {
                  const float4 o0 = o[i];
                  q4.x += o0.x; q4.y += o0.y; q4.z += o0.z; q4.w += o0.w;
                }
                o[i] = q4;
              }
            }
          }
        }
        if (a.out) {
          // the row's 32 pixels x BN channels leave as 16-byte chunks, the
          // lanes of one pixel side by side (whole pixel rows per store)
          __syncwarp();
#pragma unroll
          for (int it = 0; it < S::kCpp; ++it) {
            const int g = it * 32 + lane, p = g / S::kCpp, sub = g % S::kCpp;
            uint4 val;
            asm volatile("ld.shared.v4.b32 {%0, %1, %2, %3}, [%4];\n"
                         : "=r"(val.x), "=r"(val.y), "=r"(val.z), "=r"(val.w)
                         : "r"(ostage + 16u * ws_slot<S::kCpp>(p, sub))
                         : "memory");
            const int xp = xw + p;
            if (xp < a.W && y < a.H) {
              const int64_t pr = ((int64_t)n * a.H + y) * a.W + xp;
              *reinterpret_cast<uint4*>(a.out + pr * a.out_stride + a.out_off + n0 + sub * 8) = val;
              if (a.up_out) {
                // nearest 2x: the four children (2y + sy, 2xp + sx) of a 2H x 2W grid
#pragma unroll
                for (int sy = 0; sy < 2; ++sy)
#pragma unroll
                  for (int sx = 0; sx < 2; ++sx) {
                    const int64_t pu = ((int64_t)n * 2 * a.H + 2 * y + sy) * (2 * a.W) + 2 * xp + sx;
                    *reinterpret_cast<uint4*>(a.up_out + pu * a.up_stride + a.up_off + n0 + sub * 8) = val;
                  }
              }
            }
          }
          __syncwarp();
        }
      }
      // the accumulator is read and holds the next tile's bias: hand it back to the MMA issuer
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
      if (wissued_s) ws_wait(smem_u32(&wfull), 0, nullptr);
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
