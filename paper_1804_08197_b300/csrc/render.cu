// Ray casting ("DVR Techniques"): one ray per pixel, sampled at a fixed step,
// trilinear interpolation, per-channel transfer function, emission-absorption
// compositing front to back with early termination. Blocks of the selected
// octree cut ("Octree Representation") are visited front to back along each
// ray in a single pass: the ray walks the level-0 block grid (leaf map), jumps
// a whole block of level L at once, and inside a block walks small cubic
// sub-blocks so that transparent ones cost no samples.
//
// Sample lattice: t0 + k step (k >= 0, t in level-0 voxels, t0 = volume
// entry). A block of level L takes every 2^L-th lattice point. Lattice points
// are assigned to blocks by exit distances only: a block owns the points
// before its exit that no earlier block owned, so every point is taken or
// skipped exactly once, whatever rounding does at faces.
#include <math.h>

#include "internal.h"

namespace sg {
namespace {

constexpr int kTileW = 16, kTileH = 8, kThreads = kTileW * kTileH;

#ifdef SG_RENDER_EVENT_STATS
// diagnostic build only: per-event counters of the ray loop
// [0] samples [1] sub-block jumps [2] rendered block entries [3] skipped block
// entries [4] warp loop trips [5] lane loop iterations [6] rays that hit
// [7] samples that changed the accumulated opacity (alpha > 0)
__device__ unsigned long long g_events[8];
#define SG_EV(i, n) ev[i] += (n)
#else
#define SG_EV(i, n) ((void)0)
#endif
// Register budget of the brick-edge specialised one-ray-per-thread kernels:
// 64 per thread, i.e. 32 resident warps per SM (on the 1024^3 bench 64
// registers without spills beat 72 registers at 28 warps; 48 registers spill
// and lose). The generic, two-rays-per-thread and EXT kernels would spill under
// it and keep the compiler's choice.
#ifndef SG_RENDER_WARPS_PER_SM
#define SG_RENDER_WARPS_PER_SM 32
#endif
constexpr int kWarpsPerSM = SG_RENDER_WARPS_PER_SM;
// Lattice points a sample iteration may take (the first after a sub-block
// lookup, the others without one while they stay in the block): fewer loop
// trips per sample and fewer iterations in which the warp also runs the jump
// and block-step paths for its other lanes. Three fit the one-channel
// kernels' 64 registers without spills (on the 1024^3 bench: 2 / 3 / 4 ->
// 482 / 494 / 481 stereo fps).
#ifndef SG_SAMPLES_PER_ITER
#define SG_SAMPLES_PER_ITER 3
#endif
constexpr int kSamplesPerIter = SG_SAMPLES_PER_ITER;
__host__ __device__ constexpr int min_blocks(int threads, int rpt, int bk, bool ext = false) {
  return (rpt == 1 && bk != 0 && !ext) ? kWarpsPerSM * 32 / threads : 1;
}


struct ImageJob {
  // ray direction (unnormalised) = dx * x_ndc + dy * y_ndc + d0, voxel space:
  // the homogeneous unprojection of NDC (x, y, 1) minus w times the eye,
  // folded on the host in FP64 so the kernel has no near/far cancellation
  float dx[3], dy[3], d0[3];
  float eye[3];    // voxel space
  int32_t W, H;
  int32_t tile_begin;  // first flat tile index of this image
  int32_t tiles_x;
  float4* out;
  uint32_t* cnt;
  const uint32_t* leaf;
  const float* depth;  // optional: world distance to an opaque surface per pixel
  // optional lens: NDC of a warped pixel -> the undistorted NDC it looks through
  int lens;
  float k1, k2, lscale, laspect, lcx, lcy;
};

template <int MAXI>
struct Jobs {
  ImageJob img[MAXI];
  int32_t n;
  int32_t total_tiles;
};

struct Args {
  const uint8_t* pool;
  size_t brick_bytes;
  const uint8_t* subdist;   // [slot][8 octants][nsub^3] transparent sub-blocks ahead
  const float4* lut;   // [nch][levels][kMaxTF]
  int nch, levels, B, nsub, sub_words, sub, sub_shift;
  int nb0[3];
  float dims0[3];
  int n[kMaxCh];
  float lo[kMaxCh], inv_w[kMaxCh];
  // a table input of channel c below vzero[c] reads two table entries of
  // alpha exactly 0 (at every level and in every optical model but MIP),
  // so the channel's sample adds exactly nothing; the plain
  // emission-absorption kernels skip such samples
  float vzero[kMaxCh];
  float step, inv_step, term;
  int empty_skip;
  int mip_skip;        // MIP may skip transparent space (every table transparent only at its low end)
  float inv_voxel;     // level-0 voxels per world unit (the model's uniform scale, inverted)
  float voxel;         // world units per level-0 voxel
  // "Visualization Enhancements" (kernels instantiated with EXT only)
  int grad[kMaxCh];    // the table reads the gradient magnitude
  int pal_m[kMaxCh];   // depth palette entries (0: the table's colour)
  float pal_near[kMaxCh], pal_inv[kMaxCh];
  const float4* palette;  // [nch][kMaxTF]
  unsigned long long* total_samples;
  uint8_t* touched;    // diagnostic kernels only: per slot, a sample was taken from the brick
};

// Exact integer <-> float conversions on the FMA/ALU pipes (the conversion
// unit runs at a fraction of the FMA rate, and the loop below needs several
// per sample): an integer 0 <= v < 2^23 is OR-ed into the mantissa of 2^23
// and 2^23 subtracted; floor/ceil of |x| < 2^22 is read from the mantissa of
// x + 1.5 * 2^23 added with round-down / round-up.
constexpr float kMagic = 12582912.0f;  // 1.5 * 2^23
constexpr int kMagicBits = 0x4B400000;
__device__ __forceinline__ float u2f(uint32_t v) { return __int_as_float(0x4B000000 | v) - 8388608.0f; }
__device__ __forceinline__ int floor_i(float x) { return __float_as_int(__fadd_rd(x, kMagic)) - kMagicBits; }
__device__ __forceinline__ int ceil_i(float x) { return __float_as_int(__fadd_ru(x, kMagic)) - kMagicBits; }
__device__ __forceinline__ float floor_f(float x) { return __fadd_rd(x, kMagic) - kMagic; }

// lattice point k: t0 + k step, the one FP32 expression every owner test uses
__device__ __forceinline__ float lattice_t(int k, float t0, const Args& a) { return fmaf(u2f((uint32_t)k), a.step, t0); }

// first lattice index k >= kmin with t_k >= t (exact: the ownership split
// between blocks uses it)
__device__ inline int first_k_at(float t, float t0, const Args& a, int kmin) {
  int k = max(ceil_i((t - t0) * a.inv_step), kmin);
  while (k > kmin && lattice_t(k - 1, t0, a) >= t) --k;
  while (lattice_t(k, t0, a) < t) ++k;
  return k;
}

// Trilinear interpolation at brick-local coordinate (lx, ly, lz) of a brick
// of edge B (BK: B as a compile-time constant, 0 = runtime). Voxels are
// turned into floats by OR-ing them into the mantissa of 2^23: differences of
// two such biased values are exact, and one subtraction of 2^23 per pair
// unbiases the base, so the result equals the plain FP32 formula.
template <typename T, int BK>
__device__ __forceinline__ float tri(const T* __restrict__ b, int Brt, float lx, float ly, float lz) {
  const int B = BK ? BK : Brt, R = B + 2, RR = R * R;
  const float rx = __fadd_rd(lx, kMagic), ry = __fadd_rd(ly, kMagic), rz = __fadd_rd(lz, kMagic);
  const float wx = lx - (rx - kMagic), wy = ly - (ry - kMagic), wz = lz - (rz - kMagic);
  const int ix = min(max(__float_as_int(rx) - kMagicBits, 0), B), iy = min(max(__float_as_int(ry) - kMagicBits, 0), B),
            iz = min(max(__float_as_int(rz) - kMagicBits, 0), B);
  const T* p = b + (iz * RR + iy * R + ix);
  auto bias = [](uint32_t v) { return __int_as_float(0x4B000000 | v); };
  const float b000 = bias(p[0]), b100 = bias(p[1]), b010 = bias(p[R]), b110 = bias(p[R + 1]);
  const float b001 = bias(p[RR]), b101 = bias(p[RR + 1]), b011 = bias(p[RR + R]), b111 = bias(p[RR + R + 1]);
  const float c00 = fmaf(wx, b100 - b000, b000 - 8388608.0f), c10 = fmaf(wx, b110 - b010, b010 - 8388608.0f);
  const float c01 = fmaf(wx, b101 - b001, b001 - 8388608.0f), c11 = fmaf(wx, b111 - b011, b011 - 8388608.0f);
  const float c0 = fmaf(wy, c10 - c00, c00), c1 = fmaf(wy, c11 - c01, c01);
  return fmaf(wz, c1 - c0, c0);
}

__device__ __forceinline__ float4 classify(const Args& a, int c, int L, float v) {
  const float x = fminf(fmaxf((v - a.lo[c]) * a.inv_w[c], 0.0f), 1.0f);
  const float q = x * (float)(a.n[c] - 1);
  const float fl = fminf(floor_f(q), (float)(a.n[c] - 2));  // entry index as an exact float
  const int i = __float_as_int(fl + kMagic) - kMagicBits;
  const float f = q - fl;
  const float4* t = a.lut + 2 * (((size_t)c * a.levels + L) * kMaxTF + i);
  const float4 e0 = __ldg(t), de = __ldg(t + 1);
  return make_float4(fmaf(f, de.x, e0.x), fmaf(f, de.y, e0.y), fmaf(f, de.z, e0.z), fmaf(f, de.w, e0.w));
}

// Gradient magnitude per level-0 voxel: central differences of the
// trilinear field at +-1/2 level-L voxel along each axis (the taps stay
// within the brick's apron), times 2^-L.
template <typename T, int BK>
__device__ __forceinline__ float grad_input(const T* __restrict__ br, int B, float lx, float ly, float lz, float sL) {
  const float gx = tri<T, BK>(br, B, lx + 0.5f, ly, lz) - tri<T, BK>(br, B, lx - 0.5f, ly, lz);
  const float gy = tri<T, BK>(br, B, lx, ly + 0.5f, lz) - tri<T, BK>(br, B, lx, ly - 0.5f, lz);
  const float gz = tri<T, BK>(br, B, lx, ly, lz + 0.5f) - tri<T, BK>(br, B, lx, ly, lz - 0.5f);
  return sqrtf(gx * gx + gy * gy + gz * gz) * sL;
}

// the table's input for channel c: the trilinear value, or (EXT kernels,
// gradient tables) the gradient magnitude
template <typename T, int BK, bool EXT>
__device__ __forceinline__ float table_input(const Args& a, const T* __restrict__ br, int c, float lx, float ly, float lz,
                                             float sL) {
  if (EXT && a.grad[c]) return grad_input<T, BK>(br, a.B, lx, ly, lz, sL);
  return tri<T, BK>(br, a.B, lx, ly, lz);
}

// depth palette colour of channel c at world distance d from the eye
__device__ __forceinline__ float3 palette_at(const Args& a, int c, float d) {
  const int m = a.pal_m[c];
  const float4* p = a.palette + (size_t)c * kMaxTF;
  if (m == 1) {
    const float4 e = __ldg(p);
    return make_float3(e.x, e.y, e.z);
  }
  const float x = fminf(fmaxf((d - a.pal_near[c]) * a.pal_inv[c], 0.0f), 1.0f);
  const float q = x * (float)(m - 1);
  const float fl = fminf(floorf(q), (float)(m - 2));
  const int i = (int)fl;
  const float f = q - fl;
  const float4 e0 = __ldg(p + i), e1 = __ldg(p + i + 1);
  return make_float3(fmaf(f, e1.x - e0.x, e0.x), fmaf(f, e1.y - e0.y, e0.y), fmaf(f, e1.z - e0.z, e0.z));
}

// classified sample of channel c (colour from the depth palette in EXT
// kernels when the channel has one); t = the sample's distance from the eye
// in level-0 voxels
template <typename T, int BK, bool EXT>
__device__ __forceinline__ float4 classify_sample(const Args& a, const T* __restrict__ br, int c, int L, float lx,
                                                  float ly, float lz, float sL, float t) {
  float4 e = classify(a, c, L, table_input<T, BK, EXT>(a, br, c, lx, ly, lz, sL));
  if (EXT && a.pal_m[c] > 0) {
    const float3 p = palette_at(a, c, t * a.voxel);
    e.x = p.x;
    e.y = p.y;
    e.z = p.z;
  }
  return e;
}

// Trilinear value + classification + front-to-back compositing of one sample
// at brick-local coordinate l (all channels, additive blend). Returns true
// when the ray is opaque enough to stop.
template <typename T, int BK, bool EXT, int NC = 0>
__device__ __forceinline__ bool composite_sample(const Args& a, const T* __restrict__ brick0, int L, float lx, float ly,
                                                 float lz, float sL, float t, float4& acc) {
  float sa, sr, sg, sb;
  if (NC == 1 || (NC == 0 && a.nch == 1)) {
    // one channel: alpha is an interpolation of table entries in [0, 1], so
    // the additive blend below never saturates
    float4 e;
    if (!EXT) {
      const float v = tri<T, BK>(brick0, a.B, lx, ly, lz);
      if (v < a.vzero[0]) return false;  // alpha 0: acc unchanged (and below term, or the ray had stopped)
      e = classify(a, 0, L, v);
    } else {
      e = classify_sample<T, BK, EXT>(a, brick0, 0, L, lx, ly, lz, sL, t);
    }
    sa = e.w;
    sr = e.w * e.x;
    sg = e.w * e.y;
    sb = e.w * e.z;
  } else {
    sa = 0.0f; sr = 0.0f; sg = 0.0f; sb = 0.0f;
    auto channel = [&](int c) {
      const T* br = reinterpret_cast<const T*>(reinterpret_cast<const uint8_t*>(brick0) + (size_t)c * a.brick_bytes);
      float4 e;
      if (!EXT) {
        const float v = tri<T, BK>(br, a.B, lx, ly, lz);
        if (v < a.vzero[c]) return;  // alpha 0: adds exactly nothing to the blend
        e = classify(a, c, L, v);
      } else {
        e = classify_sample<T, BK, EXT>(a, br, c, L, lx, ly, lz, sL, t);
      }
      sa += e.w;
      sr = fmaf(e.w, e.x, sr);
      sg = fmaf(e.w, e.y, sg);
      sb = fmaf(e.w, e.z, sb);
    };
    if (NC >= 2) {
#pragma unroll
      for (int c = 0; c < NC; ++c) channel(c);
    } else {
      for (int c = 0; c < a.nch; ++c) channel(c);
    }
    if (sa > 1.0f) {  // additive blend saturates: alpha 1, colour renormalised
      const float r = 1.0f / sa;
      sr *= r; sg *= r; sb *= r;
      sa = 1.0f;
    }
  }
  const float w = 1.0f - acc.w;
  acc.x = fmaf(w, sr, acc.x);
  acc.y = fmaf(w, sg, acc.y);
  acc.z = fmaf(w, sb, acc.z);
  acc.w = fmaf(w, sa, acc.w);
  return acc.w >= a.term;
}

// Emission-only sample: every channel adds its table colour times its
// emission weight (the table's alpha for this level is alpha * step 2^L /
// ref_step); no absorption, the ray never stops early.
template <typename T, int BK, bool EXT, int NC = 0>
__device__ __forceinline__ void emission_sample(const Args& a, const T* __restrict__ brick0, int L, float lx, float ly,
                                                float lz, float sL, float t, float4& acc) {
  const int nch = NC == 1 ? 1 : a.nch;
  for (int c = 0; c < nch; ++c) {
    const T* br = reinterpret_cast<const T*>(reinterpret_cast<const uint8_t*>(brick0) + (size_t)c * a.brick_bytes);
    float4 e;
    if (!EXT) {
      const float v = tri<T, BK>(br, a.B, lx, ly, lz);
      if (v < a.vzero[c]) continue;  // emission weight 0: adds exactly nothing
      e = classify(a, c, L, v);
    } else {
      e = classify_sample<T, BK, EXT>(a, br, c, L, lx, ly, lz, sL, t);
    }
    acc.x = fmaf(e.w, e.x, acc.x);
    acc.y = fmaf(e.w, e.y, acc.y);
    acc.z = fmaf(e.w, e.z, acc.z);
  }
}

// Maximum intensity projection sample: the running maximum of each
// channel's table input, with the distance of the first sample reaching it.
template <typename T, int BK, bool EXT, int NC = 0>
__device__ __forceinline__ void mip_sample(const Args& a, const T* __restrict__ brick0, float lx, float ly, float lz,
                                           float sL, float t, float (&vmax)[kMaxCh], float (&tat)[kMaxCh]) {
#pragma unroll
  for (int c = 0; c < kMaxCh; ++c) {
    if (c >= (NC == 1 ? 1 : a.nch)) break;
    const T* br = reinterpret_cast<const T*>(reinterpret_cast<const uint8_t*>(brick0) + (size_t)c * a.brick_bytes);
    const float v = table_input<T, BK, EXT>(a, br, c, lx, ly, lz, sL);
    if (v > vmax[c]) {
      vmax[c] = v;
      tat[c] = t;
    }
  }
}

// exit distance of a ray from a slab along one axis, given the bound it
// leaves through (the upper one for d > 0, the lower one for d < 0)
__device__ __forceinline__ float exit_through(float o, float d, float inv, float bnd) {
  return d != 0.0f ? (bnd - o) * inv : INFINITY;
}

__device__ inline int cell_of(float p, float invB, int lo, int hi) {
  return min(max(floor_i(p * invB), lo), hi);
}

// One ray: pixel (px, py) of image J; acc = premultiplied RGBA, cnt = samples
// composited. A single flat loop advances the ray by one event per
// iteration (take a sample, jump over transparent sub-blocks, or move to
// the next block), so the lanes of a warp stay in one loop instead of
// diverging across nested ones.
template <typename T, int BK, int MODE, bool EXT, bool TOUCH = false, int NC = 0>
__device__ __forceinline__ void trace_ray(const Args& a, const ImageJob& J, int px, int py, bool active, float4& acc,
                                          uint32_t& cnt) {
  acc = make_float4(0.f, 0.f, 0.f, 0.f);
  cnt = 0;
  float x = 2.0f * ((float)px + 0.5f) / (float)J.W - 1.0f;
  float y = 1.0f - 2.0f * ((float)py + 0.5f) / (float)J.H;
  if (J.lens) {
    const float ex = x - J.lcx, ey = y - J.lcy;
    const float r2 = (ex * J.laspect) * (ex * J.laspect) + ey * ey;
    const float f = (1.0f + r2 * (J.k1 + J.k2 * r2)) * J.lscale;
    x = fmaf(ex, f, J.lcx);
    y = fmaf(ey, f, J.lcy);
  }
  float3 d = make_float3(fmaf(J.dx[0], x, fmaf(J.dy[0], y, J.d0[0])), fmaf(J.dx[1], x, fmaf(J.dy[1], y, J.d0[1])),
                         fmaf(J.dx[2], x, fmaf(J.dy[2], y, J.d0[2])));
  const float dn = rsqrtf(d.x * d.x + d.y * d.y + d.z * d.z);
  d.x *= dn; d.y *= dn; d.z *= dn;
  const float3 o = make_float3(J.eye[0], J.eye[1], J.eye[2]);
  const float3 inv = make_float3(1.0f / d.x, 1.0f / d.y, 1.0f / d.z);

  // clip to [0,N]^3 (slab method); an axis-parallel ray outside a slab misses
  float tn = -INFINITY, tf = INFINITY;
  {
    const float oo[3] = {o.x, o.y, o.z}, dd[3] = {d.x, d.y, d.z}, ii[3] = {inv.x, inv.y, inv.z};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      if (dd[k] == 0.0f) {
        if (oo[k] < 0.0f || oo[k] > a.dims0[k]) tf = -INFINITY;
        continue;
      }
      const float t1 = (0.0f - oo[k]) * ii[k], t2 = (a.dims0[k] - oo[k]) * ii[k];
      tn = fmaxf(tn, fminf(t1, t2));
      tf = fminf(tf, fmaxf(t1, t2));
    }
  }
  const float t0 = fmaxf(tn, 0.0f);
  float t1 = tf;
  // an opaque surface from the scene's depth buffer ends the ray
  if (J.depth && active) t1 = fminf(t1, __ldg(J.depth + (size_t)py * J.W + px) * a.inv_voxel);
  // a degenerate matrix gives a NaN direction and an unbounded segment: no hit
  const bool hit = active && isfinite(t0) && isfinite(t1) && t1 > t0 && (t1 - t0) * a.inv_step < 4.0e6f &&
                   isfinite(d.x + d.y + d.z);
  if (!hit) return;
  // transparent space may be skipped unless a MIP maximum could lie there
  const bool skip = a.empty_skip && (MODE != SG_MODE_MIP || a.mip_skip);
  float vmax[kMaxCh], tat[kMaxCh];
#pragma unroll
  for (int c = 0; c < kMaxCh; ++c) {
    vmax[c] = -INFINITY;
    tat[c] = 0.0f;
  }
#ifdef SG_RENDER_EVENT_STATS
  unsigned long long ev[8] = {0, 0, 0, 0, 0, 0, 1, 0};
#endif

  const int B = BK ? BK : a.B;
  const float Bf = (float)B, invB = 1.0f / Bf;
  int cx = cell_of(fmaf(t0, d.x, o.x), invB, 0, a.nb0[0] - 1);
  int cy = cell_of(fmaf(t0, d.y, o.y), invB, 0, a.nb0[1] - 1);
  int cz = cell_of(fmaf(t0, d.z, o.z), invB, 0, a.nb0[2] - 1);
  int k = 0;            // next lattice point
  int kb = 0;           // first lattice point owned by the current block
  int L = 0, kstep = 1; // current block's level and lattice stride
  int ax = -1;          // axis through which the current block is left (-1: no block yet)
  float tend = -1.0f;   // exit of the current block (clipped to t1)
  float texit = -1.0f;  // unclipped exit
  uint32_t slot = 0;
  const T* brick0 = nullptr;               // the current block's brick (channel 0)
  const uint8_t* subd = nullptr;           // its sub-block distance map for this ray's octant
  const int oct = (d.x < 0.0f ? 1 : 0) | (d.y < 0.0f ? 2 : 0) | (d.z < 0.0f ? 4 : 0);
  const int nsub3 = a.nsub * a.nsub * a.nsub;
  float3 lo = make_float3(0.f, 0.f, 0.f);  // block origin, level-0 voxels
  float sL = 1.0f;                         // 2^-L
  bool render = false;
  const int nsm = a.nsub - 1;

  for (int guard = 0; guard < (1 << 25); ++guard) {
#ifdef SG_RENDER_EVENT_STATS
    {
      const unsigned am = __activemask();
      if ((am & ((1u << (threadIdx.x & 31)) - 1u)) == 0u) ++ev[4];
      ++ev[5];
    }
#endif
    const float t = lattice_t(k, t0, a);
    if (!render || !(t < tend)) {
      // ---- leave the current block and enter the next one
      if (ax >= 0) {
        if (texit >= t1) break;
        const int nl_x = (cx >> L) << L, nl_y = (cy >> L) << L, nl_z = (cz >> L) << L;
        const int nh_x = min(nl_x + (1 << L), a.nb0[0]), nh_y = min(nl_y + (1 << L), a.nb0[1]),
                  nh_z = min(nl_z + (1 << L), a.nb0[2]);
        // the neighbour across the exit face along axis ax; on the other two
        // axes the cell of the exit point, clamped to the block just left
        // (all three formed, the exit axis then replaced: no 3-way branch)
        const int c_ax = ax == 0 ? (d.x > 0.0f ? nh_x : nl_x - 1)
                                 : (ax == 1 ? (d.y > 0.0f ? nh_y : nl_y - 1) : (d.z > 0.0f ? nh_z : nl_z - 1));
        const int n_ax = ax == 0 ? a.nb0[0] : (ax == 1 ? a.nb0[1] : a.nb0[2]);
        if (c_ax < 0 || c_ax >= n_ax) break;
        const int ncx = cell_of(fmaf(texit, d.x, o.x), invB, nl_x, nh_x - 1);
        const int ncy = cell_of(fmaf(texit, d.y, o.y), invB, nl_y, nh_y - 1);
        const int ncz = cell_of(fmaf(texit, d.z, o.z), invB, nl_z, nh_z - 1);
        cx = ax == 0 ? c_ax : ncx;
        cy = ax == 1 ? c_ax : ncy;
        cz = ax == 2 ? c_ax : ncz;
        // lattice points before the exit belong to the block just left
        k = first_k_at(tend, t0, a, kb);
      }
      const uint32_t e = __ldg(J.leaf + ((size_t)cz * a.nb0[1] + cy) * a.nb0[0] + cx);
      L = e & 15;
      const int nl_x = (cx >> L) << L, nl_y = (cy >> L) << L, nl_z = (cz >> L) << L;
      lo = make_float3(u2f(nl_x) * Bf, u2f(nl_y) * Bf, u2f(nl_z) * Bf);
      const float span = u2f(B << L);
      const float ex = exit_through(o.x, d.x, inv.x, d.x > 0.0f ? fminf(lo.x + span, a.dims0[0]) : lo.x);
      const float ey = exit_through(o.y, d.y, inv.y, d.y > 0.0f ? fminf(lo.y + span, a.dims0[1]) : lo.y);
      const float ez = exit_through(o.z, d.z, inv.z, d.z > 0.0f ? fminf(lo.z + span, a.dims0[2]) : lo.z);
      ax = 0;
      texit = ex;
      if (ey < texit) { texit = ey; ax = 1; }
      if (ez < texit) { texit = ez; ax = 2; }
      tend = fminf(texit, t1);
      kb = k;
      render = !(e & kLeafNone) && !(skip && (e & 16u));
      SG_EV(render ? 2 : 3, 1);
      if (!render) continue;  // owns its lattice points without sampling them: leave at once
      kstep = 1 << L;
      k = (k + kstep - 1) & ~(kstep - 1);
      slot = (e & ~kLeafNone) >> 5;
      brick0 = reinterpret_cast<const T*>(a.pool + (size_t)slot * a.nch * a.brick_bytes);
      subd = a.subdist + ((size_t)slot * 8 + oct) * nsub3;
      sL = __int_as_float((127 - L) << 23);
      continue;
    }
    // ---- lattice point k lies in a rendered block of level L
    const float px0 = fmaf(t, d.x, o.x), py0 = fmaf(t, d.y, o.y), pz0 = fmaf(t, d.z, o.z);
    // brick-local coordinate: level-L position - block origin + 1 (apron) - 0.5 (voxel centre)
    const float lx = fmaf(px0 - lo.x, sL, 0.5f), ly = fmaf(py0 - lo.y, sL, 0.5f), lz = fmaf(pz0 - lo.z, sL, 0.5f);
    if (skip) {
      const int sx = min(max(floor_i(lx - 0.5f) >> a.sub_shift, 0), nsm);
      const int sy = min(max(floor_i(ly - 0.5f) >> a.sub_shift, 0), nsm);
      const int sz = min(max(floor_i(lz - 0.5f) >> a.sub_shift, 0), nsm);
      const int sid = (sz * a.nsub + sy) * a.nsub + sx;
      const int D = __ldg(subd + sid);
      if (D > 0) {
        // the box of D sub-blocks ahead of this one in the ray's octant is
        // transparent: jump to its exit through a far face (clipped to the
        // brick); the lattice points skipped have alpha exactly 0
        const float S = u2f(a.sub << L);
        const int ex_i = d.x > 0.0f ? min(sx + D, a.nsub) : max(sx - D + 1, 0);
        const int ey_i = d.y > 0.0f ? min(sy + D, a.nsub) : max(sy - D + 1, 0);
        const int ez_i = d.z > 0.0f ? min(sz + D, a.nsub) : max(sz - D + 1, 0);
        const float ts = fminf(fminf(exit_through(o.x, d.x, inv.x, fmaf(u2f(ex_i), S, lo.x)),
                                     exit_through(o.y, d.y, inv.y, fmaf(u2f(ey_i), S, lo.y))),
                               fminf(exit_through(o.z, d.z, inv.z, fmaf(u2f(ez_i), S, lo.z)), tend));
        // a rounded-up target may skip a point lying within rounding of the
        // exit: it is inside the cube's footprint margin, alpha 0, exact
        k = max(ceil_i((ts - t0) * a.inv_step), k + 1);
        k = (k + kstep - 1) & ~(kstep - 1);
        SG_EV(1, 1);
        continue;
      }
    }
    ++cnt;
    SG_EV(0, 1);
    if (TOUCH) a.touched[slot] = 1;
    bool stop = false;
    if (MODE == SG_MODE_EMISSION_ABSORPTION) {
#ifdef SG_RENDER_EVENT_STATS
      const float w_before = acc.w;
      stop = composite_sample<T, BK, EXT, NC>(a, brick0, L, lx, ly, lz, sL, t, acc);
      SG_EV(7, acc.w != w_before ? 1 : 0);
#else
      stop = composite_sample<T, BK, EXT, NC>(a, brick0, L, lx, ly, lz, sL, t, acc);
#endif
    } else if (MODE == SG_MODE_EMISSION) {
      emission_sample<T, BK, EXT, NC>(a, brick0, L, lx, ly, lz, sL, t, acc);
    } else {
      mip_sample<T, BK, EXT, NC>(a, brick0, lx, ly, lz, sL, t, vmax, tat);
    }
    if (stop) break;
    k += kstep;
    // the next lattice points of the same block, taken without a sub-block
    // lookup: a sample in a transparent sub-block adds exactly nothing (and
    // cannot raise a MIP maximum that matters), so taking it is always exact
#pragma unroll
    for (int u = 1; u < kSamplesPerIter; ++u) {
      const float t2 = lattice_t(k, t0, a);
      if (!(t2 < tend)) break;
      const float qx = fmaf(t2, d.x, o.x), qy = fmaf(t2, d.y, o.y), qz = fmaf(t2, d.z, o.z);
      const float mx = fmaf(qx - lo.x, sL, 0.5f), my = fmaf(qy - lo.y, sL, 0.5f), mz = fmaf(qz - lo.z, sL, 0.5f);
      ++cnt;
      SG_EV(0, 1);
      if (MODE == SG_MODE_EMISSION_ABSORPTION)
        stop = composite_sample<T, BK, EXT, NC>(a, brick0, L, mx, my, mz, sL, t2, acc);
      else if (MODE == SG_MODE_EMISSION)
        emission_sample<T, BK, EXT, NC>(a, brick0, L, mx, my, mz, sL, t2, acc);
      else
        mip_sample<T, BK, EXT, NC>(a, brick0, mx, my, mz, sL, t2, vmax, tat);
      if (stop) break;
      k += kstep;
    }
    if (stop) break;
  }
  if (MODE == SG_MODE_MIP && cnt > 0) {
    // classify each channel's maximum (the MIP tables hold the transfer
    // functions as given, the same for every level), blend the channels
    // additively with alpha capped at 1, premultiply
    float sa = 0.0f, sr = 0.0f, sg = 0.0f, sb = 0.0f;
#pragma unroll
    for (int c = 0; c < kMaxCh; ++c) {
      if (c >= (NC == 1 ? 1 : a.nch)) break;
      float4 e = classify(a, c, 0, vmax[c]);
      if (EXT && a.pal_m[c] > 0) {
        const float3 p = palette_at(a, c, tat[c] * a.voxel);
        e.x = p.x;
        e.y = p.y;
        e.z = p.z;
      }
      sa += e.w;
      sr = fmaf(e.w, e.x, sr);
      sg = fmaf(e.w, e.y, sg);
      sb = fmaf(e.w, e.z, sb);
    }
    if (sa > 1.0f) {
      const float r = 1.0f / sa;
      sr *= r; sg *= r; sb *= r;
      sa = 1.0f;
    }
    acc = make_float4(sr, sg, sb, sa);
  }
#ifdef SG_RENDER_EVENT_STATS
  for (int i = 0; i < 8; ++i)
    if (ev[i]) atomicAdd(&g_events[i], ev[i]);
#endif
}

template <typename T, int MAXI, int BK, int MODE, bool EXT, bool TOUCH = false, int NC = 0>
__global__ void __launch_bounds__(kThreads, min_blocks(kThreads, 1, BK, EXT)) k_render(Args a, Jobs<MAXI> jobs) {
  const int tile = blockIdx.x;
  int im = 0;
  while (im + 1 < jobs.n && tile >= jobs.img[im + 1].tile_begin) ++im;
  const ImageJob& J = jobs.img[im];
  const int lt = tile - J.tile_begin;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // warp = 8 x 4 pixels, CTA = 2 x 2 warps
  const int px = (lt % J.tiles_x) * kTileW + (warp & 1) * 8 + (lane & 7);
  const int py = (lt / J.tiles_x) * kTileH + (warp >> 1) * 4 + (lane >> 3);
  const bool active = px < J.W && py < J.H;

  float4 acc;
  uint32_t cnt;
  trace_ray<T, BK, MODE, EXT, TOUCH, NC>(a, J, px, py, active, acc, cnt);
  if (active) {
    const size_t pix = (size_t)py * J.W + px;
    J.out[pix] = acc;
    if (J.cnt) J.cnt[pix] = cnt;
  }
  if (a.total_samples) {
    __syncwarp();
    const unsigned c = __reduce_add_sync(0xffffffffu, cnt);
    if (lane == 0) atomicAdd(a.total_samples, (unsigned long long)c);
  }
}

// Tiles of TW x TH pixels (warps cover 8 x 4 sub-tiles), RPT rays per thread.
// PERSIST: a grid sized to the machine pulls tiles from a global counter
// (work queue over all images of the batch, whatever their sizes); else one
// CTA per tile.
template <typename T, int TW, int TH, int RPT, bool PERSIST, int BK, int NC>
__global__ void __launch_bounds__(TW * TH / RPT, min_blocks(TW * TH / RPT, RPT, BK))
    k_render_tiles(Args a, Jobs<128> jobs, int* __restrict__ counter) {
  constexpr int kN = TW * TH / RPT;
  constexpr int kSubX = TW / 8;
  __shared__ int s_tile;
  uint32_t total = 0;
  for (int it = 0;; ++it) {
    int tile;
    if (PERSIST) {
      if (threadIdx.x == 0) s_tile = atomicAdd(counter, 1);
      __syncthreads();
      tile = s_tile;
      __syncthreads();
    } else {
      if (it > 0) break;
      tile = blockIdx.x;
    }
    if (tile >= jobs.total_tiles) break;
    int im = 0;
    while (im + 1 < jobs.n && tile >= jobs.img[im + 1].tile_begin) ++im;
    const ImageJob& J = jobs.img[im];
    const int lt = tile - J.tile_begin;
    const int tx = lt % J.tiles_x, ty = lt / J.tiles_x;
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
      const int idx = threadIdx.x + r * kN;
      const int sub = idx >> 5, lane = idx & 31;
      const int px = tx * TW + (sub % kSubX) * 8 + (lane & 7);
      const int py = ty * TH + (sub / kSubX) * 4 + (lane >> 3);
      const bool active = px < J.W && py < J.H;
      float4 acc;
      uint32_t cnt;
      trace_ray<T, BK, SG_MODE_EMISSION_ABSORPTION, false, false, NC>(a, J, px, py, active, acc, cnt);
      if (active) {
        const size_t pix = (size_t)py * J.W + px;
        J.out[pix] = acc;
        if (J.cnt) J.cnt[pix] = cnt;
      }
      total += cnt;
    }
  }
  if (a.total_samples) {
    __syncwarp();
    const unsigned c = __reduce_add_sync(0xffffffffu, total);
    if ((threadIdx.x & 31) == 0) atomicAdd(a.total_samples, (unsigned long long)c);
  }
}

bool inv4(const double* m, double* out) {
  // Gauss-Jordan elimination with partial pivoting (column major in/out)
  double A[4][8];
  for (int r = 0; r < 4; ++r)
    for (int c = 0; c < 4; ++c) {
      A[r][c] = m[c * 4 + r];
      A[r][4 + c] = r == c ? 1.0 : 0.0;
    }
  for (int c = 0; c < 4; ++c) {
    int p = c;
    for (int r = c + 1; r < 4; ++r)
      if (fabs(A[r][c]) > fabs(A[p][c])) p = r;
    if (!(fabs(A[p][c]) > 1e-300)) return false;
    for (int k = 0; k < 8; ++k) { double tmp = A[c][k]; A[c][k] = A[p][k]; A[p][k] = tmp; }
    const double piv = A[c][c];
    for (int k = 0; k < 8; ++k) A[c][k] /= piv;
    for (int r = 0; r < 4; ++r) {
      if (r == c) continue;
      const double f = A[r][c];
      for (int k = 0; k < 8; ++k) A[r][k] -= f * A[c][k];
    }
  }
  for (int r = 0; r < 4; ++r)
    for (int c = 0; c < 4; ++c) out[c * 4 + r] = A[r][4 + c];
  return true;
}

void mul4(const double* a, const double* b, double* o) {
  double r[16];
  for (int c = 0; c < 4; ++c)
    for (int rr = 0; rr < 4; ++rr) {
      double s = 0.0;
      for (int k = 0; k < 4; ++k) s += a[k * 4 + rr] * b[c * 4 + k];
      r[c * 4 + rr] = s;
    }
  for (int i = 0; i < 16; ++i) o[i] = r[i];
}

bool setup_image(const sg_volume* v, const sg_pose* p, int e, ImageJob* J) {
  double M[16], V[16], P[16], VM[16], PVM[16], inv[16], vminv[16];
  for (int i = 0; i < 16; ++i) {
    M[i] = v->desc.model[i];
    V[i] = p->view[e][i];
    P[i] = p->proj[e][i];
  }
  mul4(V, M, VM);
  mul4(P, VM, PVM);
  if (!inv4(PVM, inv) || !inv4(VM, vminv)) return false;
  double eye[3];
  for (int k = 0; k < 3; ++k) eye[k] = vminv[12 + k] / vminv[15];
  // h(x, y) = inv (x, y, 1, 1); direction = h.xyz - h.w eye (the far point
  // seen from the eye, times h.w); oriented so that it points forward
  const double hw = inv[11] + inv[15];
  const double sgn = hw < 0.0 ? -1.0 : 1.0;
  for (int r = 0; r < 3; ++r) {
    J->dx[r] = (float)(sgn * (inv[0 + r] - eye[r] * inv[3]));
    J->dy[r] = (float)(sgn * (inv[4 + r] - eye[r] * inv[7]));
    J->d0[r] = (float)(sgn * ((inv[8 + r] + inv[12 + r]) - eye[r] * (inv[11] + inv[15])));
    J->eye[r] = (float)eye[r];
  }
  J->W = p->width;
  J->H = p->height;
  J->leaf = v->sel[p->slot].d_leaf;
  return true;
}

Args make_args(const sg_volume* v, const sg_render_params* prm) {
  Args a;
  a.pool = v->d_pool;
  a.brick_bytes = v->brick_bytes;
  a.subdist = v->d_subdist;
  a.lut = v->d_lut;
  a.nch = v->nch;
  a.levels = v->levels;
  a.B = v->B;
  a.nsub = v->nsub;
  a.sub_words = v->sub_words;
  a.sub = v->sub;
  a.sub_shift = v->sub_shift;
  for (int k = 0; k < 3; ++k) {
    a.nb0[k] = v->geom[0].nb[k];
    a.dims0[k] = (float)v->geom[0].dims[k];
  }
  for (int c = 0; c < kMaxCh; ++c) {
    a.n[c] = c < v->nch ? v->tf[c].n : 2;
    a.lo[c] = c < v->nch ? v->tf[c].lo : 0.f;
    a.inv_w[c] = c < v->nch ? 1.0f / (v->tf[c].hi - v->tf[c].lo) : 1.f;
  }
  for (int c = 0; c < kMaxCh; ++c) {
    a.vzero[c] = -INFINITY;
    if (c >= v->nch || v->tf[c].zero_run < 2) continue;
    // the table index the kernel's classify takes for input x, in the same
    // FP32 operations; monotone in x, so the inputs whose index is at most
    // zero_run - 2 (entries i and i + 1 both of alpha 0) lie below the
    // smallest input whose index reaches zero_run - 1, found by bisection
    // over the non-negative floats (trilinear inputs are never negative)
    const int n = a.n[c], need = v->tf[c].zero_run - 1;
    const float lo = a.lo[c], iw = a.inv_w[c];
    auto index_of = [&](float x) {
      const float u = std::fmin(std::fmax((x - lo) * iw, 0.0f), 1.0f);
      const float q = u * (float)(n - 1);
      return (int)std::fmin(std::floor(q), (float)(n - 2));
    };
    auto bits_f = [](uint32_t b) {
      float f;
      memcpy(&f, &b, 4);
      return f;
    };
    if (index_of(0.0f) < need) {
      uint32_t lo_b = 0, hi_b = 0x7F800000u;  // index(0) < need <= index(+inf)
      while (hi_b - lo_b > 1) {
        const uint32_t mid = lo_b + (hi_b - lo_b) / 2;
        if (index_of(bits_f(mid)) >= need) hi_b = mid; else lo_b = mid;
      }
      a.vzero[c] = bits_f(hi_b);
    }
  }
  a.step = prm->step;
  a.inv_step = 1.0f / prm->step;
  a.term = prm->term_alpha > 0.0f ? prm->term_alpha : 0.99f;
  a.empty_skip = prm->empty_skip;
  a.total_samples = prm->sample_total;
  a.touched = prm->touched;
  // voxels per world unit: the model's scale is uniform, so the length of
  // its first column is the voxel size
  const float* m = v->desc.model;
  a.inv_voxel = (float)(1.0 / sqrt((double)m[0] * m[0] + (double)m[1] * m[1] + (double)m[2] * m[2]));
  a.voxel = (float)sqrt((double)m[0] * m[0] + (double)m[1] * m[1] + (double)m[2] * m[2]);
  a.mip_skip = 1;
  for (int c = 0; c < v->nch; ++c) a.mip_skip &= v->tf[c].low_end_transparent ? 1 : 0;
  a.palette = v->d_palette;
  for (int c = 0; c < kMaxCh; ++c) {
    const bool on = c < v->nch;
    a.grad[c] = on ? v->tf[c].gradient : 0;
    a.pal_m[c] = on ? v->tf[c].pal_m : 0;
    a.pal_near[c] = on ? v->tf[c].pal_near : 0.0f;
    a.pal_inv[c] = on && v->tf[c].pal_m > 0 ? (float)(1.0 / ((double)v->tf[c].pal_far - v->tf[c].pal_near)) : 0.0f;
  }
  return a;
}

template <int MAXI>
bool make_jobs(const sg_volume* v, const sg_pose* poses, int n, const sg_render_params* prm, float* const* outs,
               int TW, int TH, Jobs<MAXI>* jobs) {
  int ni = 0, tiles = 0;
  for (int i = 0; i < n; ++i)
    for (int e = 0; e < 2; ++e) {
      ImageJob& J = jobs->img[ni];
      if (!setup_image(v, &poses[i], e, &J)) return false;
      J.out = reinterpret_cast<float4*>(outs[2 * i + e]);
      J.cnt = prm->sample_count[e] && n == 1 ? prm->sample_count[e] : nullptr;
      J.depth = n == 1 ? prm->depth[e] : nullptr;
      J.lens = 0;
      if (prm->lens && n == 1) {
        const sg_lens& Ls = *prm->lens;
        J.lens = 1;
        J.k1 = Ls.k1;
        J.k2 = Ls.k2;
        J.lscale = Ls.scale > 0.0f ? Ls.scale : 1.0f / (1.0f + Ls.k1 + Ls.k2);
        J.laspect = Ls.aspect > 0.0f ? Ls.aspect : (float)J.W / (float)J.H;
        J.lcx = Ls.centre[e][0];
        J.lcy = Ls.centre[e][1];
      }
      J.tiles_x = (J.W + TW - 1) / TW;
      J.tile_begin = tiles;
      tiles += J.tiles_x * ((J.H + TH - 1) / TH);
      ++ni;
    }
  jobs->n = ni;
  jobs->total_tiles = tiles;
  return true;
}

template <typename T, int TW, int TH, int RPT, int BK, int NC>
cudaError_t launch_tiles(sg_volume* v, const Args& a, const Jobs<128>& jobs, bool persist, cudaStream_t s) {
  constexpr int kN = TW * TH / RPT;
  if (!persist) {
    k_render_tiles<T, TW, TH, RPT, false, BK, NC><<<jobs.total_tiles, kN, 0, s>>>(a, jobs, nullptr);
    return cudaGetLastError();
  }
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_render_tiles<T, TW, TH, RPT, true, BK, NC>, kN, 0);
  if (per_sm < 1) per_sm = 1;
  int grid = sms * per_sm;
  if (grid > jobs.total_tiles) grid = jobs.total_tiles;
  // word 0 of the volume's device control block is the tile queue head
  cudaError_t e = cudaMemsetAsync(v->d_err, 0, sizeof(uint32_t), s);
  if (e != cudaSuccess) return e;
  k_render_tiles<T, TW, TH, RPT, true, BK, NC><<<grid, kN, 0, s>>>(a, jobs, reinterpret_cast<int*>(v->d_err));
  return cudaGetLastError();
}

template <typename T, int BK, int NC>
cudaError_t dispatch_tiles(sg_volume* v, const Args& a, const sg_pose* poses, int n, const sg_render_params* prm,
                           float* const* outs, const sg_render_config& c, cudaStream_t s) {
  Jobs<128> jobs;  // by-value kernel parameter block (about 13 KB)
  const bool p = c.persistent != 0;
#define SG_TILE(TW, TH, RPT)                                                              \
  if (c.tile_w == TW && c.tile_h == TH && c.rays_per_thread == RPT) {                     \
    if (!make_jobs<128>(v, poses, n, prm, outs, TW, TH, &jobs)) return cudaErrorInvalidValue; \
    return launch_tiles<T, TW, TH, RPT, BK, NC>(v, a, jobs, p, s);                        \
  }
  SG_TILE(16, 8, 1)
  SG_TILE(8, 16, 1)
  SG_TILE(32, 4, 1)
  SG_TILE(8, 8, 1)
  SG_TILE(16, 16, 2)
  SG_TILE(32, 8, 2)
#undef SG_TILE
  return cudaErrorInvalidValue;
}

template <int MAXI, int BK, int MODE, bool EXT = false, bool TOUCH = false, int NC = 0>
cudaError_t launch_impl(sg_volume* v, const sg_pose* poses, int n, const sg_render_params* prm, float* const* outs,
                        cudaStream_t s) {
  Args a = make_args(v, prm);
  Jobs<MAXI> jobs;
  if (!make_jobs<MAXI>(v, poses, n, prm, outs, kTileW, kTileH, &jobs)) return cudaErrorInvalidValue;
  if (v->esize == 1)
    k_render<uint8_t, MAXI, BK, MODE, EXT, TOUCH, NC><<<jobs.total_tiles, kThreads, 0, s>>>(a, jobs);
  else
    k_render<uint16_t, MAXI, BK, MODE, EXT, TOUCH, NC><<<jobs.total_tiles, kThreads, 0, s>>>(a, jobs);
  return cudaGetLastError();
}

// Brick edges with a specialised kernel (voxel offsets become immediates);
// any other edge runs the generic one.
template <int BK>
cudaError_t launch_b(sg_volume* v, const sg_pose* poses, int n, const sg_render_params* prm, float* const* outs,
                     cudaStream_t s) {
  // gradient tables or depth palettes: the EXT kernels (one CTA per 16x8 tile)
  bool ext = false;
  for (int c = 0; c < v->nch; ++c) ext |= v->tf[c].gradient || v->tf[c].pal_m > 0;
  if (prm->touched) {
    // the diagnostic of the bricks a frame reads: the default kernel with a
    // flag store per sample
    if (ext || prm->mode != SG_MODE_EMISSION_ABSORPTION || n != 1) return cudaErrorInvalidValue;
    return launch_impl<2, BK, SG_MODE_EMISSION_ABSORPTION, false, true>(v, poses, n, prm, outs, s);
  }
  if (ext) {
    if (prm->mode == SG_MODE_EMISSION) return launch_impl<128, BK, SG_MODE_EMISSION, true>(v, poses, n, prm, outs, s);
    if (prm->mode == SG_MODE_MIP) return launch_impl<128, BK, SG_MODE_MIP, true>(v, poses, n, prm, outs, s);
    return launch_impl<128, BK, SG_MODE_EMISSION_ABSORPTION, true>(v, poses, n, prm, outs, s);
  }
  // every plain kernel comes in two builds: one channel known at compile
  // time (no loop over channels in the code), and any channel count.
  // Emission-only and MIP run the one-CTA-per-16x8-tile kernel (the launch
  // shapes and the autotuner serve the emission-absorption model).
  const bool one = v->nch == 1, two = v->nch == 2;
  if (prm->mode == SG_MODE_EMISSION)
    return one ? launch_impl<128, BK, SG_MODE_EMISSION, false, false, 1>(v, poses, n, prm, outs, s)
               : launch_impl<128, BK, SG_MODE_EMISSION>(v, poses, n, prm, outs, s);
  if (prm->mode == SG_MODE_MIP)
    return one ? launch_impl<128, BK, SG_MODE_MIP, false, false, 1>(v, poses, n, prm, outs, s)
               : launch_impl<128, BK, SG_MODE_MIP>(v, poses, n, prm, outs, s);
  const sg_render_config& c = v->render_cfg;
  // (emission-absorption: one, two or any channels)
  if (c.tile_w == 0) {  // default: one 16 x 8 CTA per tile
    if (n == 1)
      return one ? launch_impl<2, BK, SG_MODE_EMISSION_ABSORPTION, false, false, 1>(v, poses, n, prm, outs, s)
           : two ? launch_impl<2, BK, SG_MODE_EMISSION_ABSORPTION, false, false, 2>(v, poses, n, prm, outs, s)
                 : launch_impl<2, BK, SG_MODE_EMISSION_ABSORPTION>(v, poses, n, prm, outs, s);
    return one ? launch_impl<128, BK, SG_MODE_EMISSION_ABSORPTION, false, false, 1>(v, poses, n, prm, outs, s)
         : two ? launch_impl<128, BK, SG_MODE_EMISSION_ABSORPTION, false, false, 2>(v, poses, n, prm, outs, s)
               : launch_impl<128, BK, SG_MODE_EMISSION_ABSORPTION>(v, poses, n, prm, outs, s);
  }
  Args a = make_args(v, prm);
  if (v->esize == 1)
    return one ? dispatch_tiles<uint8_t, BK, 1>(v, a, poses, n, prm, outs, c, s)
         : two ? dispatch_tiles<uint8_t, BK, 2>(v, a, poses, n, prm, outs, c, s)
               : dispatch_tiles<uint8_t, BK, 0>(v, a, poses, n, prm, outs, c, s);
  return one ? dispatch_tiles<uint16_t, BK, 1>(v, a, poses, n, prm, outs, c, s)
       : two ? dispatch_tiles<uint16_t, BK, 2>(v, a, poses, n, prm, outs, c, s)
             : dispatch_tiles<uint16_t, BK, 0>(v, a, poses, n, prm, outs, c, s);
}

}  // namespace

cudaError_t launch_render(sg_volume* v, const sg_pose* poses, int n, const sg_render_params* prm, float* const* outs,
                          cudaStream_t s) {
  if (n < 1 || n > 64) return cudaErrorInvalidValue;
  switch (v->B) {
    case 32: return launch_b<32>(v, poses, n, prm, outs, s);
    case 64: return launch_b<64>(v, poses, n, prm, outs, s);
    case 128: return launch_b<128>(v, poses, n, prm, outs, s);
    default: return launch_b<0>(v, poses, n, prm, outs, s);
  }
}

bool render_config_supported(const sg_render_config* c) {
  const int shapes[][3] = {{16, 8, 1}, {8, 16, 1}, {32, 4, 1}, {8, 8, 1}, {16, 16, 2}, {32, 8, 2}};
  if (c->tile_w == 0 && c->tile_h == 0) return true;
  for (auto& sh : shapes)
    if (c->tile_w == sh[0] && c->tile_h == sh[1] && c->rays_per_thread == sh[2]) return true;
  return false;
}

int render_config_candidates(sg_render_config* out, int cap) {
  const int shapes[][3] = {{16, 8, 1}, {8, 16, 1}, {32, 4, 1}, {8, 8, 1}, {16, 16, 2}, {32, 8, 2}};
  int k = 0;
  for (int p = 0; p < 2; ++p)
    for (auto& sh : shapes) {
      if (k >= cap) return k;
      sg_render_config c = {};
      c.persistent = p;
      c.tile_w = sh[0];
      c.tile_h = sh[1];
      c.rays_per_thread = sh[2];
      out[k++] = c;
    }
  return k;
}

}  // namespace sg

#ifdef SG_RENDER_EVENT_STATS
// diagnostic build only: reads and clears the ray-loop event counters
extern "C" int sg_debug_render_events(unsigned long long* out8) {
  if (cudaMemcpyFromSymbol(out8, sg::g_events, sizeof(sg::g_events)) != cudaSuccess) return 1;
  static const unsigned long long zero[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  return cudaMemcpyToSymbol(sg::g_events, zero, sizeof(zero)) == cudaSuccess ? 0 : 1;
}
#endif
