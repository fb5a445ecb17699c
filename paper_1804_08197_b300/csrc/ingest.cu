// Ingest kernels: multi-resolution pyramid, brick packing with aprons, value
// ranges ("Octree Representation": blocks of a multi-resolution pyramid;
// "Volumetric Data Storage": bricks uploaded as ready, aligned chunks).
#include "internal.h"

namespace sg {
namespace {

template <typename T>
__global__ void k_pyramid(const T* __restrict__ src, int64_t sx, int64_t sy, int64_t sz, T* __restrict__ dst,
                          int64_t dx, int64_t dy, int64_t dz) {
  // Level L+1 voxel = floor((sum of its 8 level-L children + 4) / 8); children
  // beyond the edge are replicated (clamped index).
  const int64_t total = dx * dy * dz;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    int64_t x = i % dx, y = (i / dx) % dy, z = i / (dx * dy);
    int64_t x0 = 2 * x, y0 = 2 * y, z0 = 2 * z;
    int64_t x1 = min(x0 + 1, sx - 1), y1 = min(y0 + 1, sy - 1), z1 = min(z0 + 1, sz - 1);
    uint32_t s = 0;
    s += src[(z0 * sy + y0) * sx + x0];
    s += src[(z0 * sy + y0) * sx + x1];
    s += src[(z0 * sy + y1) * sx + x0];
    s += src[(z0 * sy + y1) * sx + x1];
    s += src[(z1 * sy + y0) * sx + x0];
    s += src[(z1 * sy + y0) * sx + x1];
    s += src[(z1 * sy + y1) * sx + x0];
    s += src[(z1 * sy + y1) * sx + x1];
    dst[i] = (T)((s + 4u) >> 3);
  }
}

__device__ inline void block_minmax(uint32_t& mn, uint32_t& mx) {
  __shared__ uint32_t smn[32], smx[32];
  for (int o = 16; o > 0; o >>= 1) {
    mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, o));
    mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  }
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) { smn[w] = mn; smx[w] = mx; }
  __syncthreads();
  if (w == 0) {
    int nw = blockDim.x >> 5;
    mn = l < nw ? smn[l] : 0xffffffffu;
    mx = l < nw ? smx[l] : 0u;
    for (int o = 16; o > 0; o >>= 1) {
      mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, o));
      mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
  }
}

// One CTA per brick of level L: copy the (B+2)^3 voxels (global level index
// b*B - 1 + local, clamped into the level) into the brick's pool slot and
// record the min/max over them (the brick plus its apron).
template <typename T>
__global__ void k_pack(const T* __restrict__ lvl, int64_t nx, int64_t ny, int64_t nz, int B, int nbx, int nby,
                       const int32_t* __restrict__ slot_of_node, int64_t node_off, uint8_t* __restrict__ pool,
                       size_t brick_bytes, int nch, int c, uint32_t* __restrict__ range) {
  const int64_t b = blockIdx.x;
  const int bx = (int)(b % nbx), by = (int)((b / nbx) % nby), bz = (int)(b / ((int64_t)nbx * nby));
  const int32_t slot = slot_of_node[node_off + b];
  if (slot < 0) return;
  T* dst = reinterpret_cast<T*>(pool + ((size_t)slot * nch + c) * brick_bytes);
  const int R = B + 2;
  const int64_t R3 = (int64_t)R * R * R;
  uint32_t mn = 0xffffffffu, mx = 0u;
  for (int64_t i = threadIdx.x; i < R3; i += blockDim.x) {
    int lx = (int)(i % R), ly = (int)((i / R) % R), lz = (int)(i / ((int64_t)R * R));
    int64_t gx = min(max((int64_t)bx * B - 1 + lx, (int64_t)0), nx - 1);
    int64_t gy = min(max((int64_t)by * B - 1 + ly, (int64_t)0), ny - 1);
    int64_t gz = min(max((int64_t)bz * B - 1 + lz, (int64_t)0), nz - 1);
    T v = lvl[(gz * ny + gy) * nx + gx];
    dst[i] = v;
    mn = min(mn, (uint32_t)v);
    mx = max(mx, (uint32_t)v);
  }
  block_minmax(mn, mx);
  if (threadIdx.x == 0) {
    range[((node_off + b) * nch + c) * 2 + 0] = mn;
    range[((node_off + b) * nch + c) * 2 + 1] = mx;
  }
}

// Min/max of every sub-block's trilinear footprint: with sub-block edge S,
// sub-block s covers level-L positions [bB + Ss, bB + Ss + S] per axis, whose
// samples read brick-local voxels Ss .. Ss + S + 1. Grid: (brick, layer sz);
// a CTA covers one z-layer of nsub^2 sub-blocks of one brick, so a handful
// of bricks still fills the machine.
template <typename T>
__global__ void k_subranges(const uint8_t* __restrict__ pool, size_t brick_bytes, int nch, int c, int B, int nsub,
                            int S, const int32_t* __restrict__ slots, int32_t slot_base,
                            uint16_t* __restrict__ subrange) {
  const int32_t slot = slots ? slots[blockIdx.x] : slot_base + (int32_t)blockIdx.x;
  if (slot < 0) return;
  const T* src = reinterpret_cast<const T*>(pool + ((size_t)slot * nch + c) * brick_bytes);
  const int R = B + 2;
  const int n2 = nsub * nsub, ns3 = n2 * nsub;
  const int sz = blockIdx.y;
  for (int q = threadIdx.x; q < n2; q += blockDim.x) {
    const int sx = q % nsub, sy = q / nsub;
    uint32_t mn = 0xffffffffu, mx = 0u;
    for (int z = 0; z < S + 2; ++z)
      for (int y = 0; y < S + 2; ++y) {
        const T* row = src + ((size_t)(sz * S + z) * R + (sy * S + y)) * R + sx * S;
        for (int x = 0; x < S + 2; ++x) {
          const uint32_t v = __ldg(row + x);
          mn = min(mn, v);
          mx = max(mx, v);
        }
      }
    uint16_t* o = subrange + (((size_t)slot * ns3 + (size_t)sz * n2 + q) * nch + c) * 2;
    o[0] = (uint16_t)mn;
    o[1] = (uint16_t)mx;
  }
}

// Range of a whole brick with its apron from its sub-block ranges: the
// sub-block footprints cover the (B+2)^3 brick, so their min of mins and max
// of maxes is the brick's range (one pass over the small table instead of
// the brick).
__global__ void k_brick_range_from_sub(const uint16_t* __restrict__ subrange, int ns3, int nch, int c,
                                       const int32_t* __restrict__ slot_of_node, const int32_t* __restrict__ nodes,
                                       uint32_t* __restrict__ range) {
  const int32_t node = nodes[blockIdx.x];
  const int64_t slot = slot_of_node[node];
  uint32_t mn = 0xffffffffu, mx = 0u;
  for (int i = threadIdx.x; i < ns3; i += blockDim.x) {
    const uint16_t* r = subrange + ((slot * ns3 + i) * nch + c) * 2;
    mn = min(mn, (uint32_t)r[0]);
    mx = max(mx, (uint32_t)r[1]);
  }
  block_minmax(mn, mx);
  if (threadIdx.x == 0) {
    range[((int64_t)node * nch + c) * 2 + 0] = mn;
    range[((int64_t)node * nch + c) * 2 + 1] = mx;
  }
}

}  // namespace

cudaError_t launch_pyramid(const void* src, const int64_t* sd, void* dst, const int64_t* dd, int esize,
                           cudaStream_t s) {
  int64_t total = dd[0] * dd[1] * dd[2];
  int threads = 256;
  int64_t blocks = (total + threads - 1) / threads;
  if (blocks > 148 * 64) blocks = 148 * 64;
  if (blocks < 1) blocks = 1;
  if (esize == 1)
    k_pyramid<uint8_t><<<(unsigned)blocks, threads, 0, s>>>((const uint8_t*)src, sd[0], sd[1], sd[2], (uint8_t*)dst,
                                                             dd[0], dd[1], dd[2]);
  else
    k_pyramid<uint16_t><<<(unsigned)blocks, threads, 0, s>>>((const uint16_t*)src, sd[0], sd[1], sd[2],
                                                              (uint16_t*)dst, dd[0], dd[1], dd[2]);
  return cudaGetLastError();
}

cudaError_t launch_pack_level(sg_volume* v, int t, int c, int L, const void* data, cudaStream_t s) {
  const LevelGeom& g = v->geom[L];
  int64_t nblk = (int64_t)g.nb[0] * g.nb[1] * g.nb[2];
  const int32_t* slot_of_node = v->d_slot + (int64_t)t * v->nodes;
  uint32_t* range = v->d_range + (int64_t)t * v->nodes * v->nch * 2;
  if (v->esize == 1)
    k_pack<uint8_t><<<(unsigned)nblk, 512, 0, s>>>((const uint8_t*)data, g.dims[0], g.dims[1], g.dims[2], v->B,
                                                    g.nb[0], g.nb[1], slot_of_node, g.off, v->d_pool, v->brick_bytes,
                                                    v->nch, c, range);
  else
    k_pack<uint16_t><<<(unsigned)nblk, 512, 0, s>>>((const uint16_t*)data, g.dims[0], g.dims[1], g.dims[2], v->B,
                                                     g.nb[0], g.nb[1], slot_of_node, g.off, v->d_pool,
                                                     v->brick_bytes, v->nch, c, range);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // resident volumes: the slots of (t, L) are contiguous, t * nodes + node
  if (!v->pooled) {
    int32_t base = (int32_t)((int64_t)t * v->nodes + g.off);
    if (v->esize == 1)
      k_subranges<uint8_t><<<dim3((unsigned)nblk, v->nsub), 256, 0, s>>>(v->d_pool, v->brick_bytes, v->nch, c, v->B,
                                                                          v->nsub, v->sub, nullptr, base, v->d_subrange);
    else
      k_subranges<uint16_t><<<dim3((unsigned)nblk, v->nsub), 256, 0, s>>>(v->d_pool, v->brick_bytes, v->nch, c, v->B,
                                                                           v->nsub, v->sub, nullptr, base,
                                                                           v->d_subrange);
    e = cudaGetLastError();
  }
  return e;
}

cudaError_t launch_subranges(sg_volume* v, const int32_t* d_slots, int nslots, int c, cudaStream_t s) {
  if (nslots <= 0) return cudaSuccess;
  if (v->esize == 1)
    k_subranges<uint8_t><<<dim3(nslots, v->nsub), 256, 0, s>>>(v->d_pool, v->brick_bytes, v->nch, c, v->B, v->nsub,
                                                                v->sub, d_slots, 0, v->d_subrange);
  else
    k_subranges<uint16_t><<<dim3(nslots, v->nsub), 256, 0, s>>>(v->d_pool, v->brick_bytes, v->nch, c, v->B, v->nsub,
                                                                 v->sub, d_slots, 0, v->d_subrange);
  return cudaGetLastError();
}

cudaError_t launch_brick_ranges(sg_volume* v, int t, int c, int L, const int32_t* d_nodes, int n, cudaStream_t s) {
  (void)L;
  if (n <= 0) return cudaSuccess;
  // needs the bricks' sub-block ranges (launch_subranges first, same stream)
  const int32_t* slot_of_node = v->d_slot + (int64_t)t * v->nodes;
  uint32_t* range = v->d_range + (int64_t)t * v->nodes * v->nch * 2;
  const int ns3 = v->nsub * v->nsub * v->nsub;
  k_brick_range_from_sub<<<n, 256, 0, s>>>(v->d_subrange, ns3, v->nch, c, slot_of_node, d_nodes, range);
  return cudaGetLastError();
}

}  // namespace sg
