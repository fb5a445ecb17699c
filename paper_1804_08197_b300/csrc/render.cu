// Ray casting ("DVR Techniques"): one ray per pixel, sampled at a fixed step,
// trilinear interpolation, per-channel transfer function, emission-absorption
// compositing front to back with early termination. Blocks of the selected
// octree cut ("Octree Representation") are visited front to back along each
// ray in a single pass: the ray walks the level-0 block grid (leaf map), jumps
// a whole block of level L at once, and inside a block walks 8^3-voxel
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
// minimum resident CTAs per SM requested from the register allocator
#ifndef SG_RENDER_MINB
#define SG_RENDER_MINB 1
#endif

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
  const uint64_t* subempty;
  const float4* lut;   // [nch][levels][kMaxTF]
  int nch, levels, B, nsub, sub_words;
  int nb0[3];
  float dims0[3];
  int n[kMaxCh];
  float lo[kMaxCh], inv_w[kMaxCh];
  float step, inv_step, term;
  int empty_skip;
  unsigned long long* total_samples;
};

// first lattice index k >= kmin with t0 + k step >= t (same FP32 expression
// as the sampling loop, so the split is consistent)
__device__ inline int first_k_at(float t, float t0, const Args& a, int kmin) {
  float kf = ceilf((t - t0) * a.inv_step);
  int k = kf > (float)kmin ? (int)fminf(kf, 1.0e9f) : kmin;
  while (k > kmin && fmaf((float)(k - 1), a.step, t0) >= t) --k;
  while (fmaf((float)k, a.step, t0) < t) ++k;
  return k;
}

template <typename T>
__device__ inline float tri(const T* __restrict__ b, int R, float lx, float ly, float lz, int B) {
  float fx = floorf(lx), fy = floorf(ly), fz = floorf(lz);
  int ix = min(max((int)fx, 0), B), iy = min(max((int)fy, 0), B), iz = min(max((int)fz, 0), B);
  float wx = lx - fx, wy = ly - fy, wz = lz - fz;
  const T* p = b + ((size_t)iz * R + iy) * R + ix;
  const size_t RR = (size_t)R * R;
  float v000 = p[0], v100 = p[1], v010 = p[R], v110 = p[R + 1];
  float v001 = p[RR], v101 = p[RR + 1], v011 = p[RR + R], v111 = p[RR + R + 1];
  float c00 = fmaf(wx, v100 - v000, v000), c10 = fmaf(wx, v110 - v010, v010);
  float c01 = fmaf(wx, v101 - v001, v001), c11 = fmaf(wx, v111 - v011, v011);
  float c0 = fmaf(wy, c10 - c00, c00), c1 = fmaf(wy, c11 - c01, c01);
  return fmaf(wz, c1 - c0, c0);
}

__device__ inline float4 classify(const Args& a, int c, int L, float v) {
  float x = fminf(fmaxf((v - a.lo[c]) * a.inv_w[c], 0.0f), 1.0f);
  float q = x * (float)(a.n[c] - 1);
  int i = min((int)q, a.n[c] - 2);
  float f = q - (float)i;
  const float4* t = a.lut + ((size_t)c * a.levels + L) * kMaxTF + i;
  float4 e0 = __ldg(t), e1 = __ldg(t + 1);
  return make_float4(fmaf(f, e1.x - e0.x, e0.x), fmaf(f, e1.y - e0.y, e0.y), fmaf(f, e1.z - e0.z, e0.z),
                     fmaf(f, e1.w - e0.w, e0.w));
}

// Samples lattice points k (multiples of 2^L, k >= kfirst) with t_k < t_end
// inside one block; returns true when the ray terminated.
template <typename T>
__device__ inline bool sample_run(const Args& a, const T* __restrict__ brick0, int L, float3 o, float3 d,
                                  float t0, float t_end, int kfirst, float3 nlo, float4& acc, uint32_t& cnt) {
  const int kstep = 1 << L;
  const float s = __int_as_float((127 - L) << 23);  // 2^-L
  const int R = a.B + 2;
  for (int k = (kfirst + kstep - 1) & ~(kstep - 1);; k += kstep) {
    const float t = fmaf((float)k, a.step, t0);
    if (!(t < t_end)) break;
    // brick-local coordinate: level-L position + 0.5 (apron) - 0.5 (voxel centre) - block origin
    const float lx = fmaf(fmaf(t, d.x, o.x), s, -nlo.x);
    const float ly = fmaf(fmaf(t, d.y, o.y), s, -nlo.y);
    const float lz = fmaf(fmaf(t, d.z, o.z), s, -nlo.z);
    float sa = 0.0f, sr = 0.0f, sg = 0.0f, sb = 0.0f;
    for (int c = 0; c < a.nch; ++c) {
      const T* br = reinterpret_cast<const T*>(reinterpret_cast<const uint8_t*>(brick0) + (size_t)c * a.brick_bytes);
      float v = tri<T>(br, R, lx, ly, lz, a.B);
      float4 e = classify(a, c, L, v);
      sa += e.w;
      sr = fmaf(e.w, e.x, sr);
      sg = fmaf(e.w, e.y, sg);
      sb = fmaf(e.w, e.z, sb);
    }
    if (sa > 1.0f) {  // additive blend saturates: alpha 1, colour renormalised
      float r = 1.0f / sa;
      sr *= r; sg *= r; sb *= r;
      sa = 1.0f;
    }
    const float w = 1.0f - acc.w;
    acc.x = fmaf(w, sr, acc.x);
    acc.y = fmaf(w, sg, acc.y);
    acc.z = fmaf(w, sb, acc.z);
    acc.w = fmaf(w, sa, acc.w);
    ++cnt;
    if (acc.w >= a.term) return true;
  }
  return false;
}

// exit distance of a ray from the slab [lo, hi] along one axis
__device__ inline float axis_exit(float o, float d, float inv, float lo, float hi) {
  return d > 0.0f ? (hi - o) * inv : (d < 0.0f ? (lo - o) * inv : INFINITY);
}

__device__ inline int cell_of(float p, float Bf, int lo, int hi) {
  return min(max((int)floorf(p / Bf), lo), hi);
}

template <typename T, int MAXI>
__global__ void __launch_bounds__(kThreads, SG_RENDER_MINB) k_render(Args a, Jobs<MAXI> jobs) {
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

  const float x = 2.0f * ((float)px + 0.5f) / (float)J.W - 1.0f;
  const float y = 1.0f - 2.0f * ((float)py + 0.5f) / (float)J.H;
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
  const float t0 = fmaxf(tn, 0.0f), t1 = tf;
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
  uint32_t cnt = 0;
  // a degenerate matrix gives a NaN direction and an unbounded segment: no hit
  const bool hit = active && isfinite(t0) && isfinite(t1) && t1 > t0 && (t1 - t0) * a.inv_step < 16.0e6f &&
                   isfinite(d.x + d.y + d.z);

  if (hit) {
    const float Bf = (float)a.B;
    int cx = cell_of(fmaf(t0, d.x, o.x), Bf, 0, a.nb0[0] - 1);
    int cy = cell_of(fmaf(t0, d.y, o.y), Bf, 0, a.nb0[1] - 1);
    int cz = cell_of(fmaf(t0, d.z, o.z), Bf, 0, a.nb0[2] - 1);
    int knext = 0;
    float tcur = t0;
    bool done = false;
    for (int guard = 0; guard < 4096 && !done; ++guard) {
      const uint32_t e = __ldg(J.leaf + ((size_t)cz * a.nb0[1] + cy) * a.nb0[0] + cx);
      const int L = e & 15;
      // the block of level L holding this cell: cells [nl, nh), level-0 box [lo, hi]
      const int nlx = (cx >> L) << L, nly = (cy >> L) << L, nlz = (cz >> L) << L;
      const int nhx = min(nlx + (1 << L), a.nb0[0]), nhy = min(nly + (1 << L), a.nb0[1]),
                nhz = min(nlz + (1 << L), a.nb0[2]);
      const float lox = (float)nlx * Bf, loy = (float)nly * Bf, loz = (float)nlz * Bf;
      const float span = (float)(a.B << L);
      const float hix = fminf(lox + span, a.dims0[0]), hiy = fminf(loy + span, a.dims0[1]),
                  hiz = fminf(loz + span, a.dims0[2]);
      const float ex = axis_exit(o.x, d.x, inv.x, lox, hix), ey = axis_exit(o.y, d.y, inv.y, loy, hiy),
                  ez = axis_exit(o.z, d.z, inv.z, loz, hiz);
      int ax = 0;
      float tx = ex;
      if (ey < tx) { tx = ey; ax = 1; }
      if (ez < tx) { tx = ez; ax = 2; }
      const float tend = fminf(tx, t1);
      const bool none = (e & kLeafNone) != 0;
      const bool own_empty = (e & 16u) != 0;
      if (!none && !(a.empty_skip && own_empty) && tend > tcur) {
        const uint32_t slot = (e & ~kLeafNone) >> 5;
        const T* brick0 = reinterpret_cast<const T*>(a.pool + (size_t)slot * a.nch * a.brick_bytes);
        const float s = __int_as_float((127 - L) << 23);  // 2^-L
        // brick-local coordinate = level-L position - block origin + 1 (apron) - 0.5 (voxel centre)
        const float3 nlo = make_float3(lox * s - 0.5f, loy * s - 0.5f, loz * s - 0.5f);
        if (!a.empty_skip) {
          done = sample_run<T>(a, brick0, L, o, d, t0, tend, knext, nlo, acc, cnt);
        } else {
          // walk the 8^3 sub-blocks of this block between tcur and tend
          const float S = (float)(kSub << L);
          const uint64_t* bits = a.subempty + (size_t)slot * a.sub_words;
          const int nsm = a.nsub - 1;
          int sx = min(max((int)floorf((fmaf(tcur, d.x, o.x) - lox) / S), 0), nsm);
          int sy = min(max((int)floorf((fmaf(tcur, d.y, o.y) - loy) / S), 0), nsm);
          int sz = min(max((int)floorf((fmaf(tcur, d.z, o.z) - loz) / S), 0), nsm);
          const int stx = d.x > 0.0f ? 1 : -1, sty = d.y > 0.0f ? 1 : -1, stz = d.z > 0.0f ? 1 : -1;
          float tmx = d.x != 0.0f ? (lox + (sx + (d.x > 0.0f)) * S - o.x) * inv.x : INFINITY;
          float tmy = d.y != 0.0f ? (loy + (sy + (d.y > 0.0f)) * S - o.y) * inv.y : INFINITY;
          float tmz = d.z != 0.0f ? (loz + (sz + (d.z > 0.0f)) * S - o.z) * inv.z : INFINITY;
          const float tdx = fabsf(S * inv.x), tdy = fabsf(S * inv.y), tdz = fabsf(S * inv.z);
          int kk = knext;
          for (int g2 = 0; g2 < 1024; ++g2) {
            int sa = 0;
            float ts = tmx;
            if (tmy < ts) { ts = tmy; sa = 1; }
            if (tmz < ts) { ts = tmz; sa = 2; }
            const float tsb = fminf(ts, tend);
            const int sid = (sz * a.nsub + sy) * a.nsub + sx;
            const bool sub_empty = (__ldg(bits + (sid >> 6)) >> (sid & 63)) & 1ull;
            if (!sub_empty) {
              done = sample_run<T>(a, brick0, L, o, d, t0, tsb, kk, nlo, acc, cnt);
              if (done) break;
            }
            kk = first_k_at(tsb, t0, a, kk);
            if (tsb >= tend) break;
            if (sa == 0) {
              sx += stx;
              if (sx < 0 || sx > nsm) break;
              tmx += tdx;
            } else if (sa == 1) {
              sy += sty;
              if (sy < 0 || sy > nsm) break;
              tmy += tdy;
            } else {
              sz += stz;
              if (sz < 0 || sz > nsm) break;
              tmz += tdz;
            }
          }
        }
      }
      if (done) break;
      knext = first_k_at(tend, t0, a, knext);
      if (tx >= t1) break;
      // step into the neighbour across the exit face; the other coordinates
      // stay inside this block's cell range
      if (ax == 0) {
        const int c = d.x > 0.0f ? nhx : nlx - 1;
        if (c < 0 || c >= a.nb0[0]) break;
        cx = c;
        cy = cell_of(fmaf(tx, d.y, o.y), Bf, nly, nhy - 1);
        cz = cell_of(fmaf(tx, d.z, o.z), Bf, nlz, nhz - 1);
      } else if (ax == 1) {
        const int c = d.y > 0.0f ? nhy : nly - 1;
        if (c < 0 || c >= a.nb0[1]) break;
        cy = c;
        cx = cell_of(fmaf(tx, d.x, o.x), Bf, nlx, nhx - 1);
        cz = cell_of(fmaf(tx, d.z, o.z), Bf, nlz, nhz - 1);
      } else {
        const int c = d.z > 0.0f ? nhz : nlz - 1;
        if (c < 0 || c >= a.nb0[2]) break;
        cz = c;
        cx = cell_of(fmaf(tx, d.x, o.x), Bf, nlx, nhx - 1);
        cy = cell_of(fmaf(tx, d.y, o.y), Bf, nly, nhy - 1);
      }
      tcur = tend;
    }
  }
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

template <int MAXI>
cudaError_t launch_impl(sg_volume* v, const sg_pose* poses, int n, const sg_render_params* prm, float* const* outs,
                        cudaStream_t s) {
  Args a;
  a.pool = v->d_pool;
  a.brick_bytes = v->brick_bytes;
  a.subempty = v->d_subempty;
  a.lut = v->d_lut;
  a.nch = v->nch;
  a.levels = v->levels;
  a.B = v->B;
  a.nsub = v->nsub;
  a.sub_words = v->sub_words;
  for (int k = 0; k < 3; ++k) {
    a.nb0[k] = v->geom[0].nb[k];
    a.dims0[k] = (float)v->geom[0].dims[k];
  }
  for (int c = 0; c < kMaxCh; ++c) {
    a.n[c] = c < v->nch ? v->tf[c].n : 2;
    a.lo[c] = c < v->nch ? v->tf[c].lo : 0.f;
    a.inv_w[c] = c < v->nch ? 1.0f / (v->tf[c].hi - v->tf[c].lo) : 1.f;
  }
  a.step = prm->step;
  a.inv_step = 1.0f / prm->step;
  a.term = prm->term_alpha > 0.0f ? prm->term_alpha : 0.99f;
  a.empty_skip = prm->empty_skip;
  a.total_samples = prm->sample_total;

  Jobs<MAXI> jobs;
  int ni = 0, tiles = 0;
  for (int i = 0; i < n; ++i)
    for (int e = 0; e < 2; ++e) {
      ImageJob& J = jobs.img[ni];
      if (!setup_image(v, &poses[i], e, &J)) return cudaErrorInvalidValue;
      J.out = reinterpret_cast<float4*>(outs[2 * i + e]);
      J.cnt = (n == 1 && prm->sample_count[e]) ? prm->sample_count[e] : nullptr;
      J.tiles_x = (J.W + kTileW - 1) / kTileW;
      J.tile_begin = tiles;
      tiles += J.tiles_x * ((J.H + kTileH - 1) / kTileH);
      ++ni;
    }
  jobs.n = ni;
  jobs.total_tiles = tiles;
  if (v->esize == 1)
    k_render<uint8_t, MAXI><<<tiles, kThreads, 0, s>>>(a, jobs);
  else
    k_render<uint16_t, MAXI><<<tiles, kThreads, 0, s>>>(a, jobs);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_render(sg_volume* v, const sg_pose* poses, int n, const sg_render_params* prm, float* const* outs,
                          cudaStream_t s) {
  if (n <= 1) return launch_impl<2>(v, poses, n, prm, outs, s);
  if (n <= 64) return launch_impl<128>(v, poses, n, prm, outs, s);
  return cudaErrorInvalidValue;
}

}  // namespace sg
