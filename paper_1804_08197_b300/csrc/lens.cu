// Unwarping of a lens-warped render ("DVR for HMD"): every pixel of the
// undistorted image takes the preimage of its NDC centre under the radial
// lens map and a bilinear tap of the warped image.
#include "internal.h"

namespace sg {
namespace {

struct UnwarpArgs {
  float k1, k2, scale, aspect, cx, cy;
  const float4* warped;
  int Ww, Hw;
  float4* out;
  int W, H;
};

// r f(r) = rho with f(r) = 1 + k1 r^2 + k2 r^4 (k1, k2 >= 0): increasing and
// convex in r, so Newton's method from r = rho (an upper bound) descends
// monotonically onto the root; 8 steps reach FP32 precision for the radii an
// image spans.
__device__ __forceinline__ float solve_radius(float rho, float k1, float k2) {
  float r = rho;
#pragma unroll
  for (int it = 0; it < 8; ++it) {
    const float r2 = r * r;
    const float g = r * (1.0f + r2 * (k1 + k2 * r2)) - rho;
    const float dg = 1.0f + r2 * (3.0f * k1 + 5.0f * k2 * r2);
    r -= g / dg;
  }
  return r;
}

__global__ void k_unwarp(UnwarpArgs a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y;
  if (i >= a.W) return;
  const float ux = 2.0f * ((float)i + 0.5f) / (float)a.W - 1.0f, uy = 1.0f - 2.0f * ((float)j + 0.5f) / (float)a.H;
  const float ex = (ux - a.cx) / a.scale, ey = (uy - a.cy) / a.scale;
  const float rho = sqrtf((ex * a.aspect) * (ex * a.aspect) + ey * ey);
  float wx = a.cx, wy = a.cy;
  if (rho > 0.0f) {
    const float r = solve_radius(rho, a.k1, a.k2);
    const float f = 1.0f + r * r * (a.k1 + a.k2 * r * r);
    wx = a.cx + ex / f;
    wy = a.cy + ey / f;
  }
  float4 o = make_float4(0.f, 0.f, 0.f, 0.f);
  if (wx >= -1.0f && wx <= 1.0f && wy >= -1.0f && wy <= 1.0f) {
    const float px = (wx + 1.0f) * 0.5f * (float)a.Ww - 0.5f, py = (1.0f - wy) * 0.5f * (float)a.Hw - 0.5f;
    const float fx = floorf(px), fy = floorf(py);
    const float ax = px - fx, ay = py - fy;
    const int x0 = (int)fx, y0 = (int)fy;
    const int xa = min(max(x0, 0), a.Ww - 1), xb = min(max(x0 + 1, 0), a.Ww - 1);
    const int ya = min(max(y0, 0), a.Hw - 1), yb = min(max(y0 + 1, 0), a.Hw - 1);
    const float4 p00 = __ldg(a.warped + (size_t)ya * a.Ww + xa), p10 = __ldg(a.warped + (size_t)ya * a.Ww + xb);
    const float4 p01 = __ldg(a.warped + (size_t)yb * a.Ww + xa), p11 = __ldg(a.warped + (size_t)yb * a.Ww + xb);
    const float w00 = (1.0f - ax) * (1.0f - ay), w10 = ax * (1.0f - ay), w01 = (1.0f - ax) * ay, w11 = ax * ay;
    o.x = w00 * p00.x + w10 * p10.x + w01 * p01.x + w11 * p11.x;
    o.y = w00 * p00.y + w10 * p10.y + w01 * p01.y + w11 * p11.y;
    o.z = w00 * p00.z + w10 * p10.z + w01 * p01.z + w11 * p11.z;
    o.w = w00 * p00.w + w10 * p10.w + w01 * p01.w + w11 * p11.w;
  }
  a.out[(size_t)j * a.W + i] = o;
}

}  // namespace

cudaError_t launch_unwarp(const sg_lens* lens, int e, const float* warped, int Ww, int Hw, float* out, int W, int H,
                          cudaStream_t s) {
  UnwarpArgs a;
  a.k1 = lens->k1;
  a.k2 = lens->k2;
  a.scale = lens->scale > 0.0f ? lens->scale : 1.0f / (1.0f + lens->k1 + lens->k2);
  a.aspect = lens->aspect > 0.0f ? lens->aspect : (float)Ww / (float)Hw;
  a.cx = lens->centre[e][0];
  a.cy = lens->centre[e][1];
  a.warped = reinterpret_cast<const float4*>(warped);
  a.Ww = Ww;
  a.Hw = Hw;
  a.out = reinterpret_cast<float4*>(out);
  a.W = W;
  a.H = H;
  k_unwarp<<<dim3((unsigned)((W + 127) / 128), (unsigned)H), 128, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace sg
