// 3x3 convolution as an implicit GEMM on the 5th-generation tensor cores
// (tcgen05, sm_100 family): BF16 operands in shared memory, FP32
// accumulator in tensor memory (TMEM), one thread issuing the MMAs.
//
// Tile: 128 output pixels (M) x BN output channels (N) per CTA; K = 9 Cin
// (tap-major, then channel) in blocks of 64, zero-padded to a multiple of 64.
// Operands are gathered with cp.async into the canonical K-major layout
// without swizzle: 8-row x 16-byte core matrices, 128 bytes each; along K
// core matrices are 128 B apart (leading byte offset), along M/N 8-row groups
// are 1024 B apart (stride byte offset). A 3-stage ring overlaps the gather
// of block k+2 with the MMAs of block k; tcgen05.commit arrives on the
// stage's mbarrier when its MMAs are done. Every wait is bounded: on timeout
// the CTA raises an error word and leaves (after freeing its TMEM).
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "unet_gemm.cuh"

namespace sg {
namespace nn {

constexpr int kTcBM = 128, kTcBK = 64, kTcStages = 3;
// Bounded waits: non-blocking polls, backing off with a short sleep after
// the first few, so the bound is also a time bound (about 1-2 s).
constexpr uint32_t kTcSpinLimit = 1u << 24;

__device__ __forceinline__ uint64_t tc_smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  // start address, leading / stride byte offsets (all >> 4), descriptor
  // version 1, no swizzle, base offset 0
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);
}

// kind::f16 instruction descriptor: D FP32, A and B BF16, both K-major, M x N
__host__ __device__ constexpr uint32_t tc_idesc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// polls the mbarrier phase with the given parity at most `limit` times
__device__ __forceinline__ bool mbar_wait_limit(uint32_t bar, uint32_t parity, uint32_t limit) {
  for (uint32_t i = 0; i < limit; ++i) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
    if (i >= 32) __nanosleep(64);
  }
  return false;
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  return mbar_wait_limit(bar, parity, kTcSpinLimit);
}

template <int BN>
__global__ void __launch_bounds__(128) k_conv3x3_tc(ConvArgs a, uint32_t* err) {
  constexpr int kTmemCols = BN < 32 ? 32 : BN;
  constexpr int kAStage = kTcBM * kTcBK * 2;  // bytes
  constexpr int kBStage = BN * kTcBK * 2;
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ uint64_t bars[kTcStages];
  __shared__ uint32_t tmem_base_s;
  __shared__ volatile int abort_s;
  uint8_t* sA = smem;
  uint8_t* sB = smem + kTcStages * kAStage;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t M = (int64_t)a.N * a.H * a.W;
  const int64_t m0 = (int64_t)blockIdx.x * kTcBM;
  const int n0 = blockIdx.y * BN;
  const int K = 9 * a.Cin;
  const int nkb = (K + kTcBK - 1) / kTcBK;

  if (tid == 0) {
    for (int s = 0; s < kTcStages; ++s)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&bars[s])));
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    abort_s = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&tmem_base_s)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = tmem_base_s;

  // this thread gathers row `tid` of A (pixel m0 + tid) and row `tid` of B (channel n0 + tid)
  const int64_t p = m0 + tid;
  const bool prow = p < M;
  int px = 0, py = 0;
  int64_t pn = 0;
  if (prow) {
    px = (int)(p % a.W);
    py = (int)((p / a.W) % a.H);
    pn = p / ((int64_t)a.W * a.H);
  }
  auto gather = [&](int kb, int st) {
    const uint32_t arow = smem_u32(sA + st * kAStage) + (tid >> 3) * 1024 + (tid & 7) * 16;
#pragma unroll
    for (int j = 0; j < kTcBK / 8; ++j) {
      const int k = kb * kTcBK + j * 8;
      const void* src = a.in;
      int bytes = 0;
      if (prow && k < K) {
        const int tap = k / a.Cin, c = k % a.Cin;
        const int yy = py + tap / 3 - 1, xx = px + tap % 3 - 1;
        if (yy >= 0 && yy < a.H && xx >= 0 && xx < a.W) {
          src = a.in + (((pn * a.H + yy) * a.W + xx) * a.in_stride + a.in_off + c);
          bytes = 16;
        }
      }
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(arow + j * 128), "l"(src), "r"(bytes));
    }
    if (tid < BN) {
      const uint32_t brow = smem_u32(sB + st * kBStage) + (tid >> 3) * 1024 + (tid & 7) * 16;
#pragma unroll
      for (int j = 0; j < kTcBK / 8; ++j) {
        const int k = kb * kTcBK + j * 8;
        const void* src = a.wt;
        int bytes = 0;
        if (k < K) {
          src = a.wt + (size_t)(n0 + tid) * K + k;
          bytes = 16;
        }
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(brow + j * 128), "l"(src), "r"(bytes));
      }
    }
  };

  // prologue: blocks 0 .. stages-2
#pragma unroll
  for (int s = 0; s < kTcStages - 1; ++s) {
    if (s < nkb) gather(s, s);
    cp_async_commit();
  }
  constexpr uint32_t idesc = tc_idesc(kTcBM, BN);
  // no thread ever leaves the loop early (every __syncthreads is reached by
  // all); after a timed-out wait the CTA only skips work and reports
  for (int kb = 0; kb < nkb; ++kb) {
    const int st = kb % kTcStages;
    cp_async_wait<kTcStages - 2>();
    // this thread's copies into stage st are complete; make them visible to the tensor core
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    __syncthreads();
    const bool aborted = abort_s != 0;
    if (tid == 0 && !aborted) {
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      const uint32_t a_base = smem_u32(sA + st * kAStage), b_base = smem_u32(sB + st * kBStage);
#pragma unroll
      for (int kk = 0; kk < kTcBK / 16; ++kk) {
        const uint64_t da = tc_smem_desc(a_base + kk * 256, 128, 1024);
        const uint64_t db = tc_smem_desc(b_base + kk * 256, 128, 1024);
        const uint32_t accum = (kb > 0 || kk > 0) ? 1u : 0u;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
            "l"(da), "l"(db), "r"(idesc), "r"(accum));
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                       smem_u32(&bars[st]))
                   : "memory");
    }
    // refill the stage used by block kb-1 with block kb+stages-1 once its MMAs are done
    const int nxt = kb + kTcStages - 1;
    if (nxt < nkb && !aborted) {
      const int sn = nxt % kTcStages;
      bool ready = true;
      if (nxt >= kTcStages) {
        const int use = (nxt - kTcStages) / kTcStages;  // completed use of stage sn
        ready = mbar_wait(smem_u32(&bars[sn]), use & 1);
        if (!ready) abort_s = 1;
      }
      if (ready) gather(nxt, sn);
    }
    cp_async_commit();
  }
  __syncthreads();
  // wait for the last block's MMAs
  if (abort_s == 0) {
    const int last = nkb - 1, st = last % kTcStages, use = last / kTcStages;
    if (!mbar_wait(smem_u32(&bars[st]), use & 1)) abort_s = 1;
  }
  cp_async_wait<0>();
  __syncthreads();
  if (abort_s) {
    if (tid == 0) atomicExch(err, 1u);
  } else {
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    // epilogue: warp w reads TMEM lanes 32w .. 32w+31 (pixel rows), 16 columns at a time
    const int64_t pr = m0 + warp * 32 + lane;
#pragma unroll
    for (int c0 = 0; c0 < BN; c0 += 16) {
      uint32_t r[16];
      const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
      if (pr < M) {
        float v[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          v[i] = __uint_as_float(r[i]);
          if (a.bias) v[i] += a.bias[n0 + c0 + i];
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
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kTmemCols));
}

}  // namespace nn
}  // namespace sg

namespace sg {
namespace nn {

// Halo-reuse variant for Cin a multiple of CC (16 or 32) and BN <= 64: a CTA
// computes R consecutive output rows x 128 pixels of one image row band and
// loads, per CC-channel chunk, the R + 2 input row segments it needs (130
// pixels with the left/right halo, zero outside the image) once. Each segment
// is stored K-major with a 16-byte row pitch ([CC/8 k-chunks][136 pixels][8
// channels]), so tap (dy, dx) of output row r is a descriptor starting dx + 1
// pixel rows into segment r + dy + 1: leading byte offset 2176 (next 8
// channels), stride byte offset 128 (next 8 pixels). Weights of the chunk for
// all 9 taps sit in the canonical layout ([tap][BN/8][CC/8][8 rows][16 B]).
// R accumulators of BN columns each live side by side in TMEM.
constexpr int kHaloPx = 136;  // 130 used + padding

template <int CC>
__host__ __device__ constexpr int halo_seg_bytes() {
  return (CC / 8) * kHaloPx * 16;
}

template <int BN, int R, int CC>
__host__ __device__ constexpr int halo_stage_bytes() {
  return (R + 2) * halo_seg_bytes<CC>() + 9 * BN * CC * 2;
}

// TMA: the input row segments arrive as tensor copies (one per segment and
// 8-channel group: a box of 8 channels x 130 pixels of the NHWC input, which
// lands as that group's [pixel][16 B] plane; pixels and rows outside the
// image read as zero), issued by one thread and completed on a per-stage
// mbarrier; the weights still come by cp.async. Without TMA every thread
// gathers both with cp.async.
template <int BN, int R, int CC, bool TMA>
__global__ void __launch_bounds__(128) k_conv3x3_halo(ConvArgs a, int stages, uint32_t* err,
                                                     const __grid_constant__ CUtensorMap tmap) {
  constexpr int kCols = R * BN < 32 ? 32 : (R * BN <= 64 ? 64 : (R * BN <= 128 ? 128 : 256));
  constexpr int kHaloSeg = halo_seg_bytes<CC>(), KC = CC / 8;
  constexpr int kA = (R + 2) * kHaloSeg, kStage = halo_stage_bytes<BN, R, CC>();
  constexpr uint32_t kTmaBytes = (R + 2) * KC * 130 * 16;  // bytes the copies of one chunk deliver
  extern __shared__ __align__(1024) uint8_t smem[];
  __shared__ uint64_t bars[2];
  __shared__ uint64_t tbars[2];
  __shared__ uint32_t tmem_base_s;
  __shared__ volatile int abort_s;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int x0 = blockIdx.x * 128;
  const int bands = (a.H + R - 1) / R;
  const int n = blockIdx.y / bands, y0 = (blockIdx.y % bands) * R;
  const int n0 = blockIdx.z * BN;
  const int K = 9 * a.Cin, nch = a.Cin / CC;
  // an earlier CTA gave up on a wait: the outputs are invalid anyway, leave
  // before allocating anything (one read, shared by the whole CTA)
  __shared__ int skip_s;
  if (tid == 0) skip_s = *reinterpret_cast<volatile uint32_t*>(err) != 0;
  __syncthreads();
  if (skip_s) return;

  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&bars[0])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&bars[1])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&tbars[0])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&tbars[1])));
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    abort_s = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&tmem_base_s)),
                 "r"(kCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = tmem_base_s;

  auto gather = [&](int ch, int st) {
    const uint32_t base = smem_u32(smem + st * kStage);
    if (TMA) {
      if (tid == 0) {
        const uint32_t tb = smem_u32(&tbars[st]);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(tb), "r"(kTmaBytes) : "memory");
#pragma unroll
        for (int seg = 0; seg < R + 2; ++seg)
#pragma unroll
          for (int kc = 0; kc < KC; ++kc)
            asm volatile(
                "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
                "[%6];\n" ::"r"(base + seg * kHaloSeg + kc * (kHaloPx * 16)),
                "l"(reinterpret_cast<uint64_t>(&tmap)), "r"(a.in_off + ch * CC + kc * 8), "r"(x0 - 1), "r"(y0 + seg - 1),
                "r"(n), "r"(tb)
                : "memory");
      }
    }
    // input segments: (R + 2) rows x 130 pixels x KC chunks of 8 channels
    constexpr int kItemsA = TMA ? 0 : (R + 2) * 130 * KC;
    for (int it = tid; it < kItemsA; it += 128) {
      const int seg = it / (130 * KC), rem = it - seg * (130 * KC), px = rem / KC, kc = rem % KC;
      const int yy = y0 + seg - 1, xx = x0 + px - 1;
      const void* src = a.in;
      int bytes = 0;
      if (yy >= 0 && yy < a.H && xx >= 0 && xx < a.W) {
        src = a.in + ((((int64_t)n * a.H + yy) * a.W + xx) * a.in_stride + a.in_off + ch * CC + kc * 8);
        bytes = 16;
      }
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(base + seg * kHaloSeg + kc * (kHaloPx * 16) +
                                                                               px * 16),
                   "l"(src), "r"(bytes));
    }
    // weights of this chunk, all taps
    constexpr int kItemsB = 9 * BN * KC;
    for (int it = tid; it < kItemsB; it += 128) {
      const int tap = it / (BN * KC), rem = it - tap * (BN * KC), r = rem / KC, kc = rem % KC;
      const bf16* src = a.wt + (size_t)(n0 + r) * K + tap * a.Cin + ch * CC + kc * 8;
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(base + kA + tap * (BN * CC * 2) +
                                                                          (r >> 3) * (KC * 128) + kc * 128 + (r & 7) * 16),
                   "l"(src));
    }
  };

  constexpr uint32_t idesc = tc_idesc(128, BN);
  gather(0, 0);
  cp_async_commit();
  for (int ch = 0; ch < nch; ++ch) {
    const int st = stages > 1 ? (ch & 1) : 0;
    cp_async_wait<0>();
    if (TMA && abort_s == 0) {
      // this chunk's tensor copies (the stage's use count gives the phase)
      const int use = stages > 1 ? ch >> 1 : ch;
      if (!mbar_wait(smem_u32(&tbars[st]), use & 1)) abort_s = 1;
    }
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    __syncthreads();
    const bool aborted = abort_s != 0;
    if (tid == 0 && !aborted) {
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      const uint32_t base = smem_u32(smem + st * kStage);
#pragma unroll
      for (int r = 0; r < R; ++r)
#pragma unroll
        for (int tap = 0; tap < 9; ++tap)
#pragma unroll
          for (int kk = 0; kk < CC / 16; ++kk) {
            const int dy = tap / 3 - 1, dx = tap % 3 - 1;
            const uint64_t da =
                tc_smem_desc(base + (r + dy + 1) * kHaloSeg + (dx + 1) * 16 + 2 * kk * (kHaloPx * 16), kHaloPx * 16, 128);
            const uint64_t db = tc_smem_desc(base + kA + tap * (BN * CC * 2) + 2 * kk * 128, 128, KC * 128);
            const uint32_t accum = (ch > 0 || tap > 0 || kk > 0) ? 1u : 0u;
            asm volatile(
                "{\n\t.reg .pred p;\n\t"
                "setp.ne.b32 p, %4, 0;\n\t"
                "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem + r * BN),
                "l"(da), "l"(db), "r"(idesc), "r"(accum));
          }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                       smem_u32(&bars[st]))
                   : "memory");
    }
    if (ch + 1 < nch && !aborted) {
      // the next chunk's buffer: with two stages it was used by chunk ch - 1,
      // with one stage by chunk ch (just issued); wait for those MMAs first
      const int sn = stages > 1 ? ((ch + 1) & 1) : 0;
      const int prev = stages > 1 ? ch - 1 : ch;
      bool ready = true;
      if (prev >= 0) {
        const int use = stages > 1 ? prev >> 1 : prev;
        ready = mbar_wait(smem_u32(&bars[sn]), use & 1);
        if (!ready) abort_s = 1;
      }
      if (ready) gather(ch + 1, sn);
    }
    cp_async_commit();
  }
  __syncthreads();
  if (abort_s == 0) {
    const int last = nch - 1;
    const int st = stages > 1 ? (last & 1) : 0, use = stages > 1 ? last >> 1 : last;
    if (!mbar_wait(smem_u32(&bars[st]), use & 1)) abort_s = 1;
  }
  cp_async_wait<0>();
  __syncthreads();
  if (abort_s) {
    if (tid == 0) atomicExch(err, 1u);
  } else {
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const int x = x0 + warp * 32 + lane;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int y = y0 + r;
#pragma unroll
      for (int c0 = 0; c0 < BN; c0 += 16) {
        uint32_t v32[16];
        const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + r * BN + c0;
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
            : "=r"(v32[0]), "=r"(v32[1]), "=r"(v32[2]), "=r"(v32[3]), "=r"(v32[4]), "=r"(v32[5]), "=r"(v32[6]),
              "=r"(v32[7]), "=r"(v32[8]), "=r"(v32[9]), "=r"(v32[10]), "=r"(v32[11]), "=r"(v32[12]), "=r"(v32[13]),
              "=r"(v32[14]), "=r"(v32[15])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
        if (x < a.W && y < a.H) {
          const int64_t pr = ((int64_t)n * a.H + y) * a.W + x;
          float v[16];
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            v[i] = __uint_as_float(v32[i]);
            if (a.bias) v[i] += a.bias[n0 + c0 + i];
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
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kCols));
}

}  // namespace nn
}  // namespace sg
