// Transfer-function preparation ("DVR Techniques": transfer functions tau
// and T; "Visualization Enhancements": one table per channel).
//  - which blocks and sub-blocks (skip_block^3 voxels) are transparent under the tables
//    (alpha exactly 0 over their whole value range), used to drop subtrees
//    during selection and to skip work while ray casting;
//  - per-level opacity-corrected tables for the current sample spacing.
#include "internal.h"

namespace sg {
namespace {

struct TFParams {
  int nch;
  int n[kMaxCh];
  int grad[kMaxCh];  // the table reads the gradient magnitude
  float lo[kMaxCh], hi[kMaxCh];
  const float* raw;  // [nch][kMaxTF][4]
};

// A value range is transparent when every table entry a value in it can
// touch has alpha 0. The index is decided in FP32, in this exact order:
// x = (v - lo) / (hi - lo) clamped to [0,1], q = x (n-1), entries
// floor(q(vmin)) - 1 .. floor(q(vmax)) + 2 (the one-entry margins absorb a
// one-ulp difference in how a sampler computes q). Unknown ranges
// (vmin > vmax) are never transparent.
__device__ bool range_empty(const TFParams& p, int c, uint32_t vmin, uint32_t vmax) {
  if (vmin > vmax) return false;
  const int n = p.n[c];
  // the table's input over the range: the values, or for gradient input
  // [0, sqrt(3) (vmax - vmin)] (each central difference of the trilinear
  // field spans at most vmax - vmin, and level-L gradients are divided by
  // 2^L >= 1)
  float in0 = __uint2float_rn(vmin), in1 = __uint2float_rn(vmax);
  if (p.grad[c]) {
    in0 = 0.0f;
    in1 = __fmul_rn(1.7320508f, __uint2float_rn(vmax - vmin));
  }
  const float width = __fsub_rn(p.hi[c], p.lo[c]);
  float x0 = __fdiv_rn(__fsub_rn(in0, p.lo[c]), width);
  float x1 = __fdiv_rn(__fsub_rn(in1, p.lo[c]), width);
  x0 = fminf(fmaxf(x0, 0.0f), 1.0f);
  x1 = fminf(fmaxf(x1, 0.0f), 1.0f);
  int ilo = (int)floorf(__fmul_rn(x0, (float)(n - 1))) - 1;
  int ihi = (int)floorf(__fmul_rn(x1, (float)(n - 1))) + 2;
  ilo = max(ilo, 0);
  ihi = min(ihi, n - 1);
  const float* a = p.raw + (size_t)c * kMaxTF * 4;
  for (int i = ilo; i <= ihi; ++i)
    if (a[4 * i + 3] != 0.0f) return false;
  return true;
}

__global__ void k_own_empty(TFParams p, const uint32_t* __restrict__ range, int64_t total, uint8_t* __restrict__ flags) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    bool e = true;
    for (int c = 0; c < p.nch && e; ++c) e = range_empty(p, c, range[(i * p.nch + c) * 2], range[(i * p.nch + c) * 2 + 1]);
    flags[i] = e ? kOwnEmpty : 0;
  }
}

// subtree-transparent = transparent itself and every existing child subtree-transparent
__global__ void k_subtree(uint8_t* __restrict__ flags, int64_t nodes, int T, int64_t off, int nbx, int nby, int nbz,
                          int64_t coff, int cbx, int cby, int cbz, int leaf_level) {
  const int64_t per = (int64_t)nbx * nby * nbz;
  const int64_t total = per * T;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    int64_t t = i / per, b = i % per;
    int bx = (int)(b % nbx), by = (int)((b / nbx) % nby), bz = (int)(b / ((int64_t)nbx * nby));
    uint8_t* f = flags + t * nodes + off + b;
    bool e = (*f & kOwnEmpty) != 0;
    if (!leaf_level)
      for (int k = 0; k < 8 && e; ++k) {
        int cx = 2 * bx + (k & 1), cy = 2 * by + ((k >> 1) & 1), cz = 2 * bz + ((k >> 2) & 1);
        if (cx >= cbx || cy >= cby || cz >= cbz) continue;
        e = (flags[t * nodes + coff + ((int64_t)cz * cby + cy) * cbx + cx] & kSubtreeEmpty) != 0;
      }
    if (e) *f |= kSubtreeEmpty;
  }
}

// one thread per 64-bit word of sub-block transparency bits of a slot
__global__ void k_sub_empty(TFParams p, const uint16_t* __restrict__ subrange, int64_t slots, int ns3, int words,
                            uint64_t* __restrict__ out, const int32_t* __restrict__ slot_list) {
  const int64_t total = slots * words;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t slot = slot_list ? slot_list[i / words] : i / words;
    int w = (int)(i % words);
    uint64_t bits = 0;
    for (int k = 0; k < 64; ++k) {
      int s = w * 64 + k;
      if (s >= ns3) break;
      bool e = true;
      for (int c = 0; c < p.nch && e; ++c) {
        const uint16_t* r = subrange + ((slot * ns3 + s) * p.nch + c) * 2;
        e = range_empty(p, c, r[0], r[1]);
      }
      if (e) bits |= 1ull << k;
    }
    out[slot * words + w] = bits;
  }
}

// Directional distance maps, one per octant of ray directions (signs of
// the direction's x, y, z; a zero component counts as positive): for
// sub-block c and octant s, D = the largest k such that the box of k
// sub-blocks ahead of c in the octant's directions (c itself included, k
// along each axis) holds only transparent sub-blocks, that is
// min over non-transparent q in the octant of max_axis (q - c) s. D = 0: c is
// not transparent; 255: nothing non-transparent ahead in this brick (the jump
// is clipped to the brick). A ray moving into that octant from inside c stays
// in the box until it leaves through one of its far faces, so it may cross
// the box without a sample; ignoring what lies behind the ray gives longer
// jumps than one symmetric distance. Exact, by the separable transform per
// octant: a one-sided 1-D distance along x, then along y and z the one-sided
// max-plus erosion g'(i) = min over j on the octant's side of i of
// max(|i - j|, g(j)), one column per thread in registers.
constexpr int kDistInf = 255;
// One column, in place in shared memory, entries taken in the scan order so
// that every read sees an input value. The scan of entry i stops once the
// distance |j - i| reaches the best value so far (no farther entry can lower
// it), and a column holding only "nothing ahead" (kDistInf) stays as it is:
// the same result as the full min over the side, at a fraction of the work.
__device__ __forceinline__ void erode_column(uint8_t* __restrict__ base, int stride, int n, int sgn) {
  bool all_inf = true;
  for (int j = 0; j < n && all_inf; ++j) all_inf = base[j * stride] == kDistInf;
  if (all_inf) return;
  if (sgn > 0) {
    for (int i = 0; i < n; ++i) {
      int best = kDistInf;
      for (int j = i; j < n && j - i < best; ++j) best = min(best, max(j - i, (int)base[j * stride]));
      base[i * stride] = (uint8_t)best;
    }
  } else {
    for (int i = n - 1; i >= 0; --i) {
      int best = kDistInf;
      for (int j = i; j >= 0 && i - j < best; --j) best = min(best, max(i - j, (int)base[j * stride]));
      base[i * stride] = (uint8_t)best;
    }
  }
}

__global__ void k_sub_dist(const uint64_t* __restrict__ bits, int nsub, int words, uint8_t* __restrict__ dist,
                           const int32_t* __restrict__ slot_list) {
  extern __shared__ uint64_t sdw[];
  const int64_t slot = slot_list ? slot_list[blockIdx.x] : blockIdx.x;
  const int n = nsub, n2 = nsub * nsub, ns3 = n2 * nsub;
  // the brick's transparency bits, then the distance map being built
  uint64_t* w = sdw;
  uint8_t* sd = reinterpret_cast<uint8_t*>(sdw + words);
  for (int i = threadIdx.x; i < words; i += blockDim.x) w[i] = bits[slot * words + i];
  __syncthreads();
  {
    const int oct = blockIdx.y;  // one octant of ray directions per CTA
    const int sx = (oct & 1) ? -1 : 1, sy = (oct & 2) ? -1 : 1, sz = (oct & 4) ? -1 : 1;
    // x: distance to the nearest non-transparent sub-block ahead in the row
    for (int r = threadIdx.x; r < n2; r += blockDim.x) {
      uint8_t* row = sd + r * n;
      int last = 2 * kDistInf * sx + (sx > 0 ? n : 0);
      for (int k = 0; k < n; ++k) {
        const int x = sx > 0 ? n - 1 - k : k;
        const int i = r * n + x;
        if (!((w[i >> 6] >> (i & 63)) & 1ull)) last = x;
        row[x] = (uint8_t)min((last - x) * sx, kDistInf);
      }
    }
    __syncthreads();
    for (int c = threadIdx.x; c < n2; c += blockDim.x)  // y columns: (x, z) = (c % n, c / n)
      erode_column(sd + (c / n) * n2 + (c % n), n, n, sy);
    __syncthreads();
    for (int c = threadIdx.x; c < n2; c += blockDim.x)  // z columns: (x, y) = (c % n, c / n)
      erode_column(sd + c, n2, n, sz);
    __syncthreads();
    uint8_t* out = dist + (slot * 8 + oct) * ns3;
    for (int i = threadIdx.x; i < ns3; i += blockDim.x) out[i] = sd[i];
    __syncthreads();
  }
}

// Opacity correction per level: a level-L sample stands for step 2^L
// level-0 voxels: alpha' = 1 - (1 - alpha)^(step 2^L / ref_step).
struct LutParams {
  int nch, levels, mode;
  int n[kMaxCh];
  float ref[kMaxCh];
};

// Table entry e of channel c for level L, per optical model: emission-
// absorption stores the opacity of one level-L sample (step 2^L level-0
// voxels), 1 - (1 - alpha)^(step 2^L / ref_step); emission-only stores the
// emission weight of that sample, alpha * step 2^L / ref_step; maximum
// intensity projection stores the table as given.
__device__ __forceinline__ float4 lut_entry(const float* __restrict__ raw, const LutParams& p, float step, int c,
                                            int L, int e) {
  const float* r = raw + ((size_t)c * kMaxTF + e) * 4;
  const float ex = step * (float)(1 << L) / p.ref[c];
  const float a = r[3];
  float ac;
  if (p.mode == SG_MODE_EMISSION)
    ac = a * ex;
  else if (p.mode == SG_MODE_MIP)
    ac = a;
  else
    ac = (a >= 1.0f) ? 1.0f : 1.0f - powf(1.0f - a, ex);
  return make_float4(r[0], r[1], r[2], ac);
}

// Opacity-corrected tables, one per (channel, level): entry e holds the pair
// (value_e, value_{e+1} - value_e), so that interpolation between entries e
// and e+1 is one FMA per component (the difference is the FP32 one the
// renderer would form itself; the last entry's difference is 0).
__global__ void k_lut(const float* __restrict__ raw, LutParams p, float step, float4* __restrict__ lut) {
  const int total = p.nch * p.levels * kMaxTF;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    int e = i % kMaxTF, L = (i / kMaxTF) % p.levels, c = i / (kMaxTF * p.levels);
    if (e >= p.n[c]) continue;
    const float4 v0 = lut_entry(raw, p, step, c, L, e);
    const float4 v1 = e + 1 < p.n[c] ? lut_entry(raw, p, step, c, L, e + 1) : v0;
    lut[2 * (size_t)i] = v0;
    lut[2 * (size_t)i + 1] = make_float4(v1.x - v0.x, v1.y - v0.y, v1.z - v0.z, v1.w - v0.w);
  }
}

TFParams make_params(const sg_volume* v) {
  TFParams p;
  p.nch = v->nch;
  for (int c = 0; c < kMaxCh; ++c) {
    p.n[c] = c < v->nch ? v->tf[c].n : 2;
    p.lo[c] = c < v->nch ? v->tf[c].lo : 0.0f;
    p.hi[c] = c < v->nch ? v->tf[c].hi : 1.0f;
    p.grad[c] = c < v->nch ? v->tf[c].gradient : 0;
  }
  p.raw = v->d_tf_raw;
  return p;
}

unsigned grid_for(int64_t total, int threads) {
  int64_t b = (total + threads - 1) / threads;
  if (b > 148 * 32) b = 148 * 32;
  if (b < 1) b = 1;
  return (unsigned)b;
}

}  // namespace

cudaError_t launch_tf_flags(sg_volume* v, cudaStream_t s, const int32_t* d_slots, int nslots) {
  TFParams p = make_params(v);
  int64_t total = v->nodes * v->T;
  k_own_empty<<<grid_for(total, 256), 256, 0, s>>>(p, v->d_range, total, v->d_nodeflags);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  for (int L = 0; L < v->levels; ++L) {
    const LevelGeom& g = v->geom[L];
    const LevelGeom& cg = v->geom[L > 0 ? L - 1 : 0];
    int64_t n = (int64_t)g.nb[0] * g.nb[1] * g.nb[2] * v->T;
    k_subtree<<<grid_for(n, 256), 256, 0, s>>>(v->d_nodeflags, v->nodes, v->T, g.off, g.nb[0], g.nb[1], g.nb[2],
                                               cg.off, cg.nb[0], cg.nb[1], cg.nb[2], L == 0);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  // sub-block bits and distances: every slot, or only the listed ones
  const int ns3 = v->nsub * v->nsub * v->nsub;
  const int64_t nsl = d_slots ? nslots : v->pool_slots;
  if (nsl <= 0) return cudaSuccess;
  const int64_t words = nsl * v->sub_words;
  k_sub_empty<<<grid_for(words, 128), 128, 0, s>>>(p, v->d_subrange, nsl, ns3, v->sub_words, v->d_subempty, d_slots);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_sub_dist<<<dim3((unsigned)nsl, 8), 256, ns3 + v->sub_words * sizeof(uint64_t), s>>>(
      v->d_subempty, v->nsub, v->sub_words, v->d_subdist, d_slots);
  return cudaGetLastError();
}

cudaError_t launch_lut(sg_volume* v, float step, int mode, cudaStream_t s) {
  LutParams p;
  p.nch = v->nch;
  p.levels = v->levels;
  p.mode = mode;
  for (int c = 0; c < kMaxCh; ++c) {
    p.n[c] = c < v->nch ? v->tf[c].n : 2;
    p.ref[c] = c < v->nch ? v->tf[c].ref_step : 1.0f;
  }
  int total = v->nch * v->levels * kMaxTF;
  k_lut<<<grid_for(total, 256), 256, 0, s>>>(v->d_tf_raw, p, step, v->d_lut);
  return cudaGetLastError();
}

}  // namespace sg
