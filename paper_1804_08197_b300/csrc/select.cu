// LOD + residency selection ("Octree Representation", last paragraph): the
// octree is walked top-down from the roots; a block is accepted when its
// level's voxel subtends no more than tau pixels at the block's closest point
// to the nearer eye; invisible blocks are culled; when a needed child is not
// cached the children are requested and the block renders one level coarser.
//
// The decision is exact: the host turns the FP32 matrices into integers once
// (eyes at 1/64 voxel, side planes at 2^-16, K = floor((tau theta)^2 2^40)),
// and the kernel compares 128-bit products, so the result is bit-exact and
// independent of evaluation order. One CTA per pose walks the tree level by
// level (frontier in global scratch), then fills the per-cell leaf map.
#include <math.h>

#include <mutex>

#include "internal.h"

namespace sg {

// ---------------------------------------------------------------- host: FP64 quantisation

namespace {

void mul4(const double* a, const double* b, double* o) {  // column major o = a b
  double r[16];
  for (int c = 0; c < 4; ++c)
    for (int rr = 0; rr < 4; ++rr) {
      double s = 0.0;
      for (int k = 0; k < 4; ++k) s += a[k * 4 + rr] * b[c * 4 + k];
      r[c * 4 + rr] = s;
    }
  for (int i = 0; i < 16; ++i) o[i] = r[i];
}

// inverse by cofactor expansion (adjugate / determinant)
bool inv4(const double* m, double* out) {
  double inv[16];
  inv[0] = m[5] * m[10] * m[15] - m[5] * m[11] * m[14] - m[9] * m[6] * m[15] + m[9] * m[7] * m[14] +
           m[13] * m[6] * m[11] - m[13] * m[7] * m[10];
  inv[4] = -m[4] * m[10] * m[15] + m[4] * m[11] * m[14] + m[8] * m[6] * m[15] - m[8] * m[7] * m[14] -
           m[12] * m[6] * m[11] + m[12] * m[7] * m[10];
  inv[8] = m[4] * m[9] * m[15] - m[4] * m[11] * m[13] - m[8] * m[5] * m[15] + m[8] * m[7] * m[13] +
           m[12] * m[5] * m[11] - m[12] * m[7] * m[9];
  inv[12] = -m[4] * m[9] * m[14] + m[4] * m[10] * m[13] + m[8] * m[5] * m[14] - m[8] * m[6] * m[13] -
            m[12] * m[5] * m[10] + m[12] * m[6] * m[9];
  inv[1] = -m[1] * m[10] * m[15] + m[1] * m[11] * m[14] + m[9] * m[2] * m[15] - m[9] * m[3] * m[14] -
           m[13] * m[2] * m[11] + m[13] * m[3] * m[10];
  inv[5] = m[0] * m[10] * m[15] - m[0] * m[11] * m[14] - m[8] * m[2] * m[15] + m[8] * m[3] * m[14] +
           m[12] * m[2] * m[11] - m[12] * m[3] * m[10];
  inv[9] = -m[0] * m[9] * m[15] + m[0] * m[11] * m[13] + m[8] * m[1] * m[15] - m[8] * m[3] * m[13] -
           m[12] * m[1] * m[11] + m[12] * m[3] * m[9];
  inv[13] = m[0] * m[9] * m[14] - m[0] * m[10] * m[13] - m[8] * m[1] * m[14] + m[8] * m[2] * m[13] +
            m[12] * m[1] * m[10] - m[12] * m[2] * m[9];
  inv[2] = m[1] * m[6] * m[15] - m[1] * m[7] * m[14] - m[5] * m[2] * m[15] + m[5] * m[3] * m[14] +
           m[13] * m[2] * m[7] - m[13] * m[3] * m[6];
  inv[6] = -m[0] * m[6] * m[15] + m[0] * m[7] * m[14] + m[4] * m[2] * m[15] - m[4] * m[3] * m[14] -
           m[12] * m[2] * m[7] + m[12] * m[3] * m[6];
  inv[10] = m[0] * m[5] * m[15] - m[0] * m[7] * m[13] - m[4] * m[1] * m[15] + m[4] * m[3] * m[13] +
            m[12] * m[1] * m[7] - m[12] * m[3] * m[5];
  inv[14] = -m[0] * m[5] * m[14] + m[0] * m[6] * m[13] + m[4] * m[1] * m[14] - m[4] * m[2] * m[13] -
            m[12] * m[1] * m[6] + m[12] * m[2] * m[5];
  inv[3] = -m[1] * m[6] * m[11] + m[1] * m[7] * m[10] + m[5] * m[2] * m[11] - m[5] * m[3] * m[10] -
           m[9] * m[2] * m[7] + m[9] * m[3] * m[6];
  inv[7] = m[0] * m[6] * m[11] - m[0] * m[7] * m[10] - m[4] * m[2] * m[11] + m[4] * m[3] * m[10] +
           m[8] * m[2] * m[7] - m[8] * m[3] * m[6];
  inv[11] = -m[0] * m[5] * m[11] + m[0] * m[7] * m[9] + m[4] * m[1] * m[11] - m[4] * m[3] * m[9] -
            m[8] * m[1] * m[7] + m[8] * m[3] * m[5];
  inv[15] = m[0] * m[5] * m[10] - m[0] * m[6] * m[9] - m[4] * m[1] * m[10] + m[4] * m[2] * m[9] +
            m[8] * m[1] * m[6] - m[8] * m[2] * m[5];
  double det = m[0] * inv[0] + m[1] * inv[4] + m[2] * inv[8] + m[3] * inv[12];
  if (!(fabs(det) > 1e-300)) return false;
  for (int i = 0; i < 16; ++i) out[i] = inv[i] / det;
  return true;
}

int64_t clamp_round(double q, double lim) {
  if (q > lim) q = lim;
  if (q < -lim) q = -lim;
  return llround(q);
}

}  // namespace

// Shared with the render path (same translation-unit-free helpers are not
// exported; render.cu has its own FP64 setup).
void compute_select_inputs(const sg_volume* v, const sg_pose* p, SelectInputs* out) {
  double M[16];
  for (int i = 0; i < 16; ++i) M[i] = v->desc.model[i];
  for (int e = 0; e < 2; ++e) {
    double V[16], P[16], VM[16], VMi[16], C[16];
    for (int i = 0; i < 16; ++i) {
      V[i] = p->view[e][i];
      P[i] = p->proj[e][i];
    }
    mul4(V, M, VM);
    if (!inv4(VM, VMi)) {
      for (int a = 0; a < 3; ++a) out->eye[e][a] = 0;
    } else {
      // eye = (V M)^-1 (0,0,0,1): the fourth column, divided by w
      double w = VMi[15];
      for (int a = 0; a < 3; ++a) out->eye[e][a] = clamp_round(VMi[12 + a] / w * 64.0, 68719476736.0);
    }
    mul4(P, VM, C);
    // side planes of the view pyramid: w + x, w - x, w + y, w - y >= 0
    for (int q = 0; q < 4; ++q) {
      int row = q >> 1;
      double sgn = (q & 1) ? -1.0 : 1.0;
      double pl[4];
      for (int k = 0; k < 4; ++k) pl[k] = C[k * 4 + 3] + sgn * C[k * 4 + row];
      double n = sqrt(pl[0] * pl[0] + pl[1] * pl[1] + pl[2] * pl[2]);
      if (n < 1e-300) {
        out->plane[e][q][0] = out->plane[e][q][1] = out->plane[e][q][2] = 0;
        out->plane[e][q][3] = 1;
        continue;
      }
      for (int k = 0; k < 3; ++k) out->plane[e][q][k] = llround(pl[k] / n * 65536.0);
      double d = pl[3] / n;
      if (d > 1048576.0) d = 1048576.0;
      if (d < -1048576.0) d = -1048576.0;
      out->plane[e][q][3] = llround(d * 65536.0 * 64.0) + 65536LL * 64LL;
    }
  }
  double theta = 2.0 / ((double)p->proj[0][5] * (double)p->height);
  double tt = (double)p->pixel_error * theta;
  double kf = floor(tt * tt * 1099511627776.0);
  if (!(kf >= 0.0)) kf = 0.0;
  if (kf > 1099511627776.0) kf = 1099511627776.0;
  out->K = (uint64_t)kf;
}

// ---------------------------------------------------------------- device

namespace {

constexpr int kSelThreads = 1024;
constexpr int kMaxSelJobs = 48;

struct SelJob {
  SelectInputs in;
  int32_t t;
  uint32_t* leaf;
  int32_t* cell_node;
  uint8_t* state;
  int32_t* req;
  uint32_t* counters;
  int32_t* frontier;  // [2][max level nodes]
};

struct SelJobs {
  SelJob j[kMaxSelJobs];
};

struct SelGeom {
  int levels, B;
  int64_t dims0[3];
  int32_t nb[kMaxLevels][3];
  int64_t off[kMaxLevels];
  int64_t nodes, max_level_nodes;
  const int32_t* slot;     // [T][nodes]
  const uint8_t* flags;    // [T][nodes]
  uint64_t* stamp;         // [slots] LRU stamps (pooled volumes) or NULL
  uint64_t frame;
};

__device__ inline void node_box(const SelGeom& g, int L, int bx, int by, int bz, int64_t* lo, int64_t* hi) {
  const int64_t span = (int64_t)g.B << L;
  const int b[3] = {bx, by, bz};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    int64_t l = b[a] * span, h = l + span;
    if (h > g.dims0[a]) h = g.dims0[a];
    lo[a] = l * 64;
    hi[a] = h * 64;
  }
}

__device__ bool culled(const SelectInputs& in, const int64_t* lo, const int64_t* hi) {
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    bool outside = false;
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      const int64_t* P = in.plane[e][p];
      int64_t val = P[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) val += P[a] * (P[a] >= 0 ? hi[a] : lo[a]);
      outside |= (val < 0);
    }
    if (!outside) return false;
  }
  return true;
}

__device__ bool accept(const SelectInputs& in, int L, const int64_t* lo, const int64_t* hi) {
  if (L == 0) return true;
  unsigned __int128 best = 0;
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    unsigned __int128 d2 = 0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      int64_t q = in.eye[e][a];
      int64_t dd = q < lo[a] ? lo[a] - q : (q > hi[a] ? q - hi[a] : 0);
      d2 += (unsigned __int128)(uint64_t)dd * (uint64_t)dd;
    }
    if (e == 0 || d2 < best) best = d2;
  }
  unsigned __int128 lhs = (unsigned __int128)1 << (52 + 2 * L);
  return lhs <= (unsigned __int128)in.K * best;
}

__global__ void __launch_bounds__(kSelThreads) k_select(SelJobs jobs, SelGeom g) {
  const SelJob& J = jobs.j[blockIdx.x];
  const int32_t* slot = g.slot + (int64_t)J.t * g.nodes;
  const uint8_t* flags = g.flags + (int64_t)J.t * g.nodes;
  __shared__ int s_next, s_nreq, s_sel, s_cull, s_empty, s_fb, s_ne;
  for (int64_t i = threadIdx.x; i < g.nodes; i += blockDim.x) J.state[i] = kUnseen;
  if (threadIdx.x == 0) { s_next = 0; s_nreq = 0; s_sel = 0; s_cull = 0; s_empty = 0; s_fb = 0; s_ne = 0; }
  __syncthreads();

  const int top = g.levels - 1;
  int ncur = g.nb[top][0] * g.nb[top][1] * g.nb[top][2];
  int32_t* cur = J.frontier;
  int32_t* nxt = J.frontier + g.max_level_nodes;
  for (int L = top; L >= 0; --L) {
    const int nbx = g.nb[L][0], nby = g.nb[L][1];
    for (int i = threadIdx.x; i < ncur; i += blockDim.x) {
      const int b = (L == top) ? i : cur[i];
      const int bx = b % nbx, by = (b / nbx) % nby, bz = b / (nbx * nby);
      const int64_t id = g.off[L] + b;
      int64_t lo[3], hi[3];
      node_box(g, L, bx, by, bz, lo, hi);
      if (L == top) {
        if (culled(J.in, lo, hi)) { J.state[id] = kCulled; atomicAdd(&s_cull, 1); continue; }
        if (flags[id] & kSubtreeEmpty) { J.state[id] = kEmpty; atomicAdd(&s_empty, 1); continue; }
      }
      if (accept(J.in, L, lo, hi)) {
        J.state[id] = kSelected;
        atomicAdd(&s_sel, 1);
        if (!(flags[id] & kOwnEmpty)) atomicAdd(&s_ne, 1);
        continue;
      }
      // children of a refined block
      const int cnx = g.nb[L - 1][0], cny = g.nb[L - 1][1], cnz = g.nb[L - 1][2];
      int need = 0, miss = 0;
      for (int k = 0; k < 8; ++k) {
        int cx = 2 * bx + (k & 1), cy = 2 * by + ((k >> 1) & 1), cz = 2 * bz + ((k >> 2) & 1);
        if (cx >= cnx || cy >= cny || cz >= cnz) continue;
        int cb = (cz * cny + cy) * cnx + cx;
        int64_t cid = g.off[L - 1] + cb;
        int64_t clo[3], chi[3];
        node_box(g, L - 1, cx, cy, cz, clo, chi);
        if (culled(J.in, clo, chi)) { J.state[cid] = kCulled; atomicAdd(&s_cull, 1); continue; }
        if (flags[cid] & kSubtreeEmpty) { J.state[cid] = kEmpty; atomicAdd(&s_empty, 1); continue; }
        need |= 1 << k;
        if (slot[cid] < 0) miss |= 1 << k;
      }
      if (miss) {
        for (int k = 0; k < 8; ++k) {
          if (!(need & (1 << k))) continue;
          int cx = 2 * bx + (k & 1), cy = 2 * by + ((k >> 1) & 1), cz = 2 * bz + ((k >> 2) & 1);
          const int64_t cid = g.off[L - 1] + (cz * cny + cy) * cnx + cx;
          if (miss & (1 << k)) {
            int r = atomicAdd(&s_nreq, 1);
            J.req[r] = (int32_t)cid;
          } else if (g.stamp) {
            // the resident siblings of the missing children are in use too:
            // evicting them would keep this block from ever refining
            g.stamp[slot[cid]] = g.frame;
          }
        }
        J.state[id] = kFallback;
        atomicAdd(&s_sel, 1);
        atomicAdd(&s_fb, 1);
        if (!(flags[id] & kOwnEmpty)) atomicAdd(&s_ne, 1);
        continue;
      }
      J.state[id] = kRefined;
      for (int k = 0; k < 8; ++k)
        if (need & (1 << k)) {
          int cx = 2 * bx + (k & 1), cy = 2 * by + ((k >> 1) & 1), cz = 2 * bz + ((k >> 2) & 1);
          int pos = atomicAdd(&s_next, 1);
          nxt[pos] = (cz * cny + cy) * cnx + cx;
        }
    }
    __syncthreads();
    ncur = s_next;
    __syncthreads();
    if (threadIdx.x == 0) s_next = 0;
    int32_t* tmp = cur;
    cur = nxt;
    nxt = tmp;
    __syncthreads();
  }

  // leaf map: for every level-0 cell, walk down to the block that renders it
  const int ncx = g.nb[0][0], ncy = g.nb[0][1], ncz = g.nb[0][2];
  const int ncell = ncx * ncy * ncz;
  for (int c = threadIdx.x; c < ncell; c += blockDim.x) {
    const int x = c % ncx, y = (c / ncx) % ncy, z = c / (ncx * ncy);
    uint32_t e = kLeafNone | (uint32_t)top;
    int32_t node = -1;
    for (int L = top; L >= 0; --L) {
      int bx = x >> L, by = y >> L, bz = z >> L;
      int64_t id = g.off[L] + ((int64_t)bz * g.nb[L][1] + by) * g.nb[L][0] + bx;
      uint8_t s = J.state[id];
      if (s == kSelected || s == kFallback) {
        e = leaf_pack((uint32_t)slot[id], L, (flags[id] & kOwnEmpty) != 0);
        node = (int32_t)id;
        break;
      }
      if (s != kRefined) {
        e = kLeafNone | (uint32_t)L;
        break;
      }
    }
    J.leaf[c] = e;
    J.cell_node[c] = node;
  }
  // LRU: every block the traversal used this frame (rendered or refined)
  if (g.stamp)
    for (int64_t i = threadIdx.x; i < g.nodes; i += blockDim.x) {
      uint8_t s = J.state[i];
      if ((s == kSelected || s == kFallback || s == kRefined) && slot[i] >= 0) g.stamp[slot[i]] = g.frame;
    }
  if (threadIdx.x == 0) {
    J.counters[0] = (uint32_t)s_nreq;
    J.counters[1] = (uint32_t)s_sel;
    J.counters[2] = (uint32_t)s_cull;
    J.counters[3] = (uint32_t)s_empty;
    J.counters[4] = (uint32_t)s_fb;
    J.counters[5] = (uint32_t)s_ne;
  }
}

}  // namespace

cudaError_t launch_select(sg_volume* v, const sg_pose* poses, int n, cudaStream_t s) {
  SelGeom g;
  g.levels = v->levels;
  g.B = v->B;
  for (int a = 0; a < 3; ++a) g.dims0[a] = v->geom[0].dims[a];
  for (int L = 0; L < kMaxLevels; ++L) {
    for (int a = 0; a < 3; ++a) g.nb[L][a] = L < v->levels ? v->geom[L].nb[a] : 0;
    g.off[L] = L < v->levels ? v->geom[L].off : 0;
  }
  g.nodes = v->nodes;
  g.max_level_nodes = v->max_level_nodes;
  g.slot = v->d_slot;
  g.flags = v->d_nodeflags;
  g.stamp = v->pooled ? v->d_stamp : nullptr;
  g.frame = v->frame;
  for (int base = 0; base < n; base += kMaxSelJobs) {
    int m = n - base < kMaxSelJobs ? n - base : kMaxSelJobs;
    SelJobs jobs;
    for (int i = 0; i < m; ++i) {
      const sg_pose* p = &poses[base + i];
      SelSlot& sl = v->sel[p->slot];
      SelJob& J = jobs.j[i];
      compute_select_inputs(v, p, &J.in);
      J.t = p->t;
      J.leaf = sl.d_leaf;
      J.cell_node = sl.d_cell_node;
      J.state = sl.d_state;
      J.req = sl.d_req;
      J.counters = sl.d_counters;
      J.frontier = sl.d_frontier;
    }
    k_select<<<m, kSelThreads, 0, s>>>(jobs, g);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace sg

// ---------------------------------------------------------------- selection without allocation
//
// For callers that must not allocate device memory while they render (a
// thread under a hard frame budget, or one recording a CUDA graph, cannot
// call cudaMalloc: it may synchronise the device and cannot be captured).
// The breadth-first frontier that the selection kernel needs comes from this
// fixed array instead of the volume's per-slot buffers.

namespace {
constexpr int64_t kStaticFrontierNodes = 65536;  // blocks per level; 2 x 256 KiB
}  // namespace

static __device__ __align__(256) int32_t g_static_frontier[2 * kStaticFrontierNodes];

namespace {
std::mutex g_static_mu;
int32_t* g_static_ptr[256] = {};  // device address of g_static_frontier, per device ordinal
}  // namespace

extern "C" sg_status sg_select_lod_noalloc(sg_volume* v, const sg_pose* p, uint32_t* leaf, int32_t* cell_node,
                                           uint8_t* node_state, int32_t* req, uint32_t* counters, void* stream) {
  using namespace sg;
  if (!v || !p || !leaf || !cell_node || !node_state || !req || !counters) {
    set_error("sg_select_lod_noalloc: volume, pose and every output must be non-NULL");
    return SG_ERR_INVALID_ARG;
  }
  sg_status pst = check_pose_fields(v, p);
  if (pst != SG_OK) return pst;
  if (v->max_level_nodes > kStaticFrontierNodes) {
    set_error("sg_select_lod_noalloc: the volume has more than 65536 blocks on one level; its fixed scratch "
              "holds at most 65536 (use sg_select_lod)");
    return SG_ERR_INVALID_ARG;
  }
  for (int c = 0; c < v->nch; ++c)
    if (!v->tf[c].set || !v->has_data[(size_t)p->t * v->nch + c]) {
      set_error("sg_select_lod_noalloc: set a transfer function and upload data for every channel first");
      return SG_ERR_STATE;
    }
  if (v->pooled) {
    const LevelGeom& g = v->geom[v->levels - 1];
    const int64_t nt = (int64_t)g.nb[0] * g.nb[1] * g.nb[2];
    for (int64_t b = 0; b < nt; ++b)
      if (v->h_slot[(int64_t)p->t * v->nodes + g.off + b] < 0) {
        set_error("sg_select_lod_noalloc: the coarsest level must be resident");
        return SG_ERR_STATE;
      }
  }
  // set-up, once per device with that device current: the array's device
  // address (host code cannot use the symbol itself as a pointer)
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "sg_select_lod_noalloc: cudaGetDevice");
  if (dev < 0 || dev >= 256) {
    set_error("sg_select_lod_noalloc: device ordinal out of range");
    return SG_ERR_INVALID_ARG;
  }
  int32_t* frontier = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (!g_static_ptr[dev]) {
      void* ptr = nullptr;
      e = cudaGetSymbolAddress(&ptr, g_static_frontier);
      if (e != cudaSuccess) return cuda_fail(e, "sg_select_lod_noalloc: cudaGetSymbolAddress");
      g_static_ptr[dev] = static_cast<int32_t*>(ptr);
    }
    frontier = g_static_ptr[dev];
  }
  SelGeom g;
  g.levels = v->levels;
  g.B = v->B;
  for (int a = 0; a < 3; ++a) g.dims0[a] = v->geom[0].dims[a];
  for (int L = 0; L < kMaxLevels; ++L) {
    for (int a = 0; a < 3; ++a) g.nb[L][a] = L < v->levels ? v->geom[L].nb[a] : 0;
    g.off[L] = L < v->levels ? v->geom[L].off : 0;
  }
  g.nodes = v->nodes;
  g.max_level_nodes = kStaticFrontierNodes;  // the two halves of the fixed array
  g.slot = v->d_slot;
  g.flags = v->d_nodeflags;
  g.stamp = nullptr;  // a pure function of its inputs: LRU stamps are left alone
  g.frame = 0;
  SelJobs jobs;
  SelJob& J = jobs.j[0];
  compute_select_inputs(v, p, &J.in);
  J.t = p->t;
  J.leaf = leaf;
  J.cell_node = cell_node;
  J.state = node_state;
  J.req = req;
  J.counters = counters;
  J.frontier = frontier;
  const cudaStream_t s = (cudaStream_t)stream;
  // after the brick uploads queued so far (page table, flags)
  e = wait_uploads(v, s);
  if (e != cudaSuccess) return cuda_fail(e, "sg_select_lod_noalloc: upload order");
  k_select<<<1, kSelThreads, 0, s>>>(jobs, g);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "sg_select_lod_noalloc: launch");
  // an upload on another stream rewrites the page table and node flags this
  // launch reads: uploads wait on the selection event, so record it here too
  // (not during capture, where a recorded event cannot be waited on later)
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  e = cudaStreamIsCapturing(s, &cap);
  if (e != cudaSuccess) return cuda_fail(e, "sg_select_lod_noalloc: capture status");
  if (cap == cudaStreamCaptureStatusNone) {
    e = cudaEventRecord(v->ev_select, s);
    if (e != cudaSuccess) return cuda_fail(e, "sg_select_lod_noalloc: event");
  }
  return SG_OK;
}
