// C ABI of the B300 DVR library: argument checks, ownership, the brick pool
// and its LRU ("Volumetric Data Cashing": a GPU cache of chunks with
// timestamps, evicting the oldest when full), and the launches.
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <set>
#include <string>
#include <tuple>
#include <utility>
#include <vector>

#include "internal.h"

namespace sg {

static thread_local std::string g_err;

void set_error(const std::string& msg) { g_err = msg; }

sg_status cuda_fail(cudaError_t e, const char* what) {
  g_err = std::string(what) + ": " + cudaGetErrorString(e);
  return SG_ERR_CUDA;
}

sg_status check_pose_fields(const sg_volume* v, const sg_pose* p) {
  auto bad = [](const char* msg) {
    set_error(msg);
    return SG_ERR_INVALID_ARG;
  };
  if (!p) return bad("pose is NULL");
  if (!(p->t >= 0 && p->t < v->T)) return bad("pose.t out of range");
  if (!(p->width > 0 && p->height > 0 && p->width <= 32768 && p->height <= 32768)) return bad("pose image size");
  if (!(p->pixel_error > 0.0f)) return bad("pose.pixel_error must be > 0");
  if (p->proj[0][5] == 0.0f) return bad("projection has P11 == 0");
  return SG_OK;
}

}  // namespace sg

using namespace sg;

#define SG_CHECK_ARG(cond, msg)      \
  do {                               \
    if (!(cond)) {                   \
      set_error(msg);                \
      return SG_ERR_INVALID_ARG;     \
    }                                \
  } while (0)

#define SG_CUDA(call, what)                          \
  do {                                               \
    cudaError_t e_ = (call);                         \
    if (e_ != cudaSuccess) return cuda_fail(e_, what); \
  } while (0)

namespace {

// LRU order of occupied, unpinned slots: (stamp, tie, slot). The eviction
// victim is the first: the smallest stamp, ties going to the coarser block,
// then to the lower (time point, node) key.
using LruKey = std::tuple<uint64_t, int64_t, int64_t>;

struct VolumeExtra {
  std::set<LruKey> lru;
  std::vector<int64_t> free_slots;
  int32_t* d_scratch = nullptr;                // upload bookkeeping
  size_t scratch_n = 0;
  // page-locked staging of an upload's lists when the call does not wait
  // for its copies: a ring, each buffer reused once its event has passed
  struct Stage {
    int32_t* h = nullptr;
    size_t n = 0;  // int32 words
    cudaEvent_t ev = nullptr;
  } stage[4];
  int stage_next = 0;
  // the host's reads of selection stamps and requests: a stream of their
  // own, so that they wait for the last selection only and not for copies
  // queued on the caller's stream (made at first use, as is the page-locked
  // array of stamps)
  cudaStream_t side_s = nullptr;
  uint64_t* h_stamp = nullptr;
};

std::vector<std::pair<sg_volume*, VolumeExtra*>>& extras() {
  static std::vector<std::pair<sg_volume*, VolumeExtra*>> x;
  return x;
}

VolumeExtra* extra_of(sg_volume* v) {
  for (auto& p : extras())
    if (p.first == v) return p.second;
  return nullptr;
}

// tie rank of the block with page-table key `key`: coarser levels first,
// then ascending key
int64_t lru_tie(const sg_volume* v, int64_t key) {
  const int64_t node = key % v->nodes;
  int level = 0;
  while (level + 1 < v->levels && node >= v->geom[level + 1].off) ++level;
  return (int64_t)(v->levels - 1 - level) * ((int64_t)v->T * v->nodes) + key;
}

template <typename T>
cudaError_t dalloc(T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  return cudaMalloc(reinterpret_cast<void**>(p), count * sizeof(T));
}

void free_volume(sg_volume* v) {
  if (!v) return;
  if (v->ev_upload) cudaEventSynchronize(v->ev_upload);  // no copy may still read or write freed memory
  cudaFree(v->d_pool);
  cudaFree(v->d_slot);
  cudaFree(v->d_range);
  cudaFree(v->d_subrange);
  cudaFree(v->d_subempty);
  cudaFree(v->d_subdist);
  cudaFree(v->d_nodeflags);
  cudaFree(v->d_tf_raw);
  cudaFree(v->d_palette);
  cudaFree(v->d_lut);
  cudaFree(v->d_stage);
  cudaFree(v->d_pipe);
  for (int k = 0; k < sg_volume::kPipeDepth; ++k) {
    if (v->ev_rendered[k]) cudaEventDestroy(v->ev_rendered[k]);
    if (v->ev_copied[k]) cudaEventDestroy(v->ev_copied[k]);
  }
  if (v->copy_stream) cudaStreamDestroy(v->copy_stream);
  cudaFree(v->d_err);
  cudaFree(v->d_stamp);
  if (v->ev_select) cudaEventDestroy(v->ev_select);
  if (v->ev_upload) cudaEventDestroy(v->ev_upload);
  for (auto& s : v->sel) {
    cudaFree(s.d_leaf);
    cudaFree(s.d_cell_node);
    cudaFree(s.d_state);
    cudaFree(s.d_req);
    cudaFree(s.d_counters);
    cudaFree(s.d_frontier);
  }
  auto& xs = extras();
  for (size_t i = 0; i < xs.size(); ++i)
    if (xs[i].first == v) {
      cudaFree(xs[i].second->d_scratch);
      for (auto& g : xs[i].second->stage) {
        if (g.ev) cudaEventDestroy(g.ev);
        cudaFreeHost(g.h);
      }
      if (xs[i].second->side_s) cudaStreamDestroy(xs[i].second->side_s);
      cudaFreeHost(xs[i].second->h_stamp);
      delete xs[i].second;
      xs.erase(xs.begin() + i);
      break;
    }
  delete v;
}

bool tfs_ready(const sg_volume* v) {
  for (int c = 0; c < v->nch; ++c)
    if (!v->tf[c].set) return false;
  return true;
}

sg_status refresh_flags(sg_volume* v, cudaStream_t s, const int32_t* d_slots = nullptr, int nslots = 0) {
  if (!tfs_ready(v)) return SG_OK;
  // the flags read the ranges of bricks that queued uploads may still be writing
  SG_CUDA(wait_uploads(v, s), "transfer-function flags");
  SG_CUDA(launch_tf_flags(v, s, d_slots, nslots), "transfer-function flags");
  return SG_OK;
}

__global__ void k_page_update(int32_t* __restrict__ slot_of_key, const int64_t* __restrict__ upd, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) slot_of_key[upd[2 * i]] = (int32_t)upd[2 * i + 1];
}

// Places bricks nodes[0..n) of (t, c) in the cache in list order, copying
// brick i from host[i]; stops at the first brick that finds the cache full of
// bricks used by the current frame (*done = bricks placed, a prefix of the
// list). Page-table entries, value ranges and transparency flags of every
// placed brick are consistent once the stream reaches v->ev_upload; with
// wait the call returns only then, else as soon as everything is queued.
sg_status upload_list(sg_volume* v, int t, int c, int n, const int32_t* nodes, const void* const* host, int* done,
                      cudaStream_t s, bool wait = true) {
  VolumeExtra* x = extra_of(v);
  const int R = v->B + 2;
  const size_t raw = (size_t)R * R * R * v->esize;
  *done = 0;
  // after every earlier upload, on whatever stream (its scratch and page-table writes)
  SG_CUDA(cudaStreamWaitEvent(s, v->ev_upload, 0), "upload");
  if (v->pooled && v->stamps_read != v->frame) {
    // stamps of slots used by recent selections, read once the last
    // selection launch (on whatever stream) has written them
    cudaStream_t rs = side_stream(v);
    if (!rs) {
      set_error("stamps: no stream could be made");
      return SG_ERR_CUDA;
    }
    if (!x->h_stamp)
      SG_CUDA(cudaHostAlloc(reinterpret_cast<void**>(&x->h_stamp), v->pool_slots * sizeof(uint64_t),
                            cudaHostAllocDefault),
              "stamps");
    const uint64_t* st = x->h_stamp;
    SG_CUDA(cudaStreamWaitEvent(rs, v->ev_select, 0), "upload");
    SG_CUDA(cudaMemcpyAsync(x->h_stamp, v->d_stamp, v->pool_slots * sizeof(uint64_t), cudaMemcpyDeviceToHost, rs),
            "stamps");
    SG_CUDA(cudaStreamSynchronize(rs), "upload");
    // a slot's stamp only moves forward: the device array holds the stamps
    // selections wrote, so a slot placed since the last selection still
    // carries its previous occupant's (older) stamp there
    for (int64_t sl = 0; sl < v->pool_slots; ++sl)
      if (v->slot_owner[sl] >= 0 && !v->slot_pinned[sl] && st[sl] > v->slot_stamp[sl]) {
        const int64_t tie = lru_tie(v, v->slot_owner[sl]);
        x->lru.erase(LruKey{v->slot_stamp[sl], tie, sl});
        v->slot_stamp[sl] = st[sl];
        x->lru.insert(LruKey{st[sl], tie, sl});
      }
    // only a selection moves the device stamps: once per frame is enough
    v->stamps_read = v->frame;
  }
  std::vector<int32_t> lists(2 * (size_t)n);  // [nodes placed][their slots]
  std::vector<int64_t> touched;               // page-table keys whose entry changed
  int m = 0;
  for (; m < n; ++m) {
    const int32_t node = nodes[m];
    const int64_t key = (int64_t)t * v->nodes + node;
    int32_t slot = v->h_slot[key];
    if (slot < 0) {
      int64_t sl;
      if (!x->free_slots.empty()) {
        sl = x->free_slots.back();
        x->free_slots.pop_back();
      } else {
        // least recently used slot not used by the current frame
        auto it = x->lru.begin();
        if (it == x->lru.end() || std::get<0>(*it) >= v->frame) break;
        sl = std::get<2>(*it);
        x->lru.erase(it);
        const int64_t old = v->slot_owner[sl];
        v->h_slot[old] = -1;
        touched.push_back(old);
      }
      slot = (int32_t)sl;
      v->slot_owner[sl] = key;
      v->h_slot[key] = slot;
      touched.push_back(key);
      int level = 0;
      while (level + 1 < v->levels && node >= v->geom[level + 1].off) ++level;
      if (level == v->levels - 1) {
        v->slot_pinned[sl] = 1;
      } else {
        v->slot_stamp[sl] = v->frame;
        x->lru.insert(LruKey{v->frame, lru_tie(v, key), sl});
      }
    }
    lists[m] = node;
    lists[n + m] = slot;
    SG_CUDA(cudaMemcpyAsync(v->d_pool + ((size_t)slot * v->nch + c) * v->brick_bytes, host[m], raw,
                            cudaMemcpyHostToDevice, s),
            "brick upload");
  }
  *done = m;
  if (m == 0) return SG_OK;
  // final page-table value of every touched key (a key evicted and placed
  // again in the same list keeps its last value)
  std::sort(touched.begin(), touched.end());
  touched.erase(std::unique(touched.begin(), touched.end()), touched.end());
  const size_t nupd = touched.size();
  std::vector<int64_t> upd(2 * nupd);
  for (size_t i = 0; i < nupd; ++i) {
    upd[2 * i] = touched[i];
    upd[2 * i + 1] = v->h_slot[touched[i]];
  }
  // device copies of the lists for the range kernels and the page update
  const size_t need = 2 * (size_t)m + 4 * nupd;  // int32 words: lists + int64 pairs
  // sized at first use for a list of up to 65536 blocks (nupd <= 2 m, so
  // 10 words a block): growing later frees and allocates, and both wait for
  // the whole device, a render in flight included
  const size_t cap = std::max(need + 2, 10 * (size_t)std::min<int64_t>(v->nodes * v->T, 1 << 16) + 2);
  if (x->scratch_n < need) {
    cudaFree(x->d_scratch);
    x->d_scratch = nullptr;
    x->scratch_n = 0;
    cudaError_t e = dalloc(&x->d_scratch, cap);
    if (e != cudaSuccess) {
      set_error(std::string("upload scratch: ") + cudaGetErrorString(e));
      return SG_ERR_OOM;
    }
    x->scratch_n = cap - 2;
  }
  int32_t* d_nodes = x->d_scratch;
  int32_t* d_slots = x->d_scratch + m;
  int64_t* d_upd = reinterpret_cast<int64_t*>(x->d_scratch + ((2 * (size_t)m + 1) & ~(size_t)1));
  // the lists' host side: the vectors above when the call waits; else a
  // page-locked staging buffer that stays put until its copies are done
  const int32_t* h_nodes = lists.data();
  const int32_t* h_slots = lists.data() + n;
  const int64_t* h_upd = upd.data();
  VolumeExtra::Stage* g = nullptr;
  if (!wait) {
    g = &x->stage[x->stage_next];
    x->stage_next = (x->stage_next + 1) % 4;
    if (g->ev) SG_CUDA(cudaEventSynchronize(g->ev), "upload staging");
    else SG_CUDA(cudaEventCreateWithFlags(&g->ev, cudaEventDisableTiming), "upload staging");
    if (g->n < need + 2) {
      cudaFreeHost(g->h);
      g->h = nullptr;
      g->n = 0;
      SG_CUDA(cudaHostAlloc(reinterpret_cast<void**>(&g->h), cap * sizeof(int32_t), cudaHostAllocDefault),
              "upload staging");
      g->n = cap;
    }
    int32_t* gl = g->h;
    int64_t* gu = reinterpret_cast<int64_t*>(g->h + ((2 * (size_t)m + 1) & ~(size_t)1));
    memcpy(gl, lists.data(), m * sizeof(int32_t));
    memcpy(gl + m, lists.data() + n, m * sizeof(int32_t));
    if (nupd) memcpy(gu, upd.data(), upd.size() * sizeof(int64_t));
    h_nodes = gl;
    h_slots = gl + m;
    h_upd = gu;
  }
  SG_CUDA(cudaMemcpyAsync(d_nodes, h_nodes, m * sizeof(int32_t), cudaMemcpyHostToDevice, s), "upload");
  SG_CUDA(cudaMemcpyAsync(d_slots, h_slots, m * sizeof(int32_t), cudaMemcpyHostToDevice, s), "upload");
  if (nupd) {
    SG_CUDA(cudaMemcpyAsync(d_upd, h_upd, upd.size() * sizeof(int64_t), cudaMemcpyHostToDevice, s), "upload");
    k_page_update<<<(unsigned)((nupd + 255) / 256), 256, 0, s>>>(v->d_slot, d_upd, (int)nupd);
    SG_CUDA(cudaGetLastError(), "page table update");
  }
  SG_CUDA(launch_subranges(v, d_slots, m, c, s), "sub-block ranges");
  SG_CUDA(launch_brick_ranges(v, t, c, 0, d_nodes, m, s), "brick ranges");  // from the sub-block ranges
  v->has_data[(size_t)t * v->nch + c] = 1;
  // node flags everywhere, sub-block flags of the uploaded slots only
  sg_status st = refresh_flags(v, s, d_slots, m);
  SG_CUDA(cudaEventRecord(v->ev_upload, s), "upload");
  if (g) {
    SG_CUDA(cudaEventRecord(g->ev, s), "upload staging");
    return st;
  }
  // the host vectors above are consumed by the copies before they return
  SG_CUDA(cudaStreamSynchronize(s), "upload");
  return st;
}

sg_status ensure_selection(sg_volume* v, int slot) {
  SelSlot& s = v->sel[slot];
  if (s.d_leaf) return SG_OK;
  cudaError_t e;
  if ((e = dalloc(&s.d_leaf, v->ncell)) != cudaSuccess || (e = dalloc(&s.d_cell_node, v->ncell)) != cudaSuccess ||
      (e = dalloc(&s.d_state, v->nodes)) != cudaSuccess || (e = dalloc(&s.d_req, v->nodes)) != cudaSuccess ||
      (e = dalloc(&s.d_counters, 8)) != cudaSuccess ||
      (e = dalloc(&s.d_frontier, 2 * v->max_level_nodes)) != cudaSuccess) {
    set_error(std::string("selection buffers: ") + cudaGetErrorString(e));
    return SG_ERR_OOM;
  }
  return SG_OK;
}

sg_status check_pose(const sg_volume* v, const sg_pose* p) {
  SG_CHECK_ARG(p, "pose is NULL");
  SG_CHECK_ARG(p->slot >= 0 && p->slot < kMaxSlots, "pose.slot out of range [0, 255]");
  return check_pose_fields(v, p);
}

sg_status check_render_params(const sg_render_params* r) {
  SG_CHECK_ARG(r, "render params are NULL");
  SG_CHECK_ARG(r->step > 0.0f && r->step < 1e6f, "render step must be > 0");
  SG_CHECK_ARG(r->term_alpha <= 1.0f, "term_alpha must be <= 1");
  SG_CHECK_ARG(r->mode == SG_MODE_EMISSION_ABSORPTION || r->mode == SG_MODE_EMISSION || r->mode == SG_MODE_MIP,
               "unknown render mode");
  for (int e = 0; e < 2; ++e)
    SG_CHECK_ARG(((uintptr_t)r->depth[e] % 4) == 0, "depth buffers must be 4-byte aligned");
  if (r->lens)
    SG_CHECK_ARG(r->lens->k1 >= 0.0f && r->lens->k2 >= 0.0f && r->lens->scale >= 0.0f && r->lens->aspect >= 0.0f &&
                     r->lens->k1 < 100.0f && r->lens->k2 < 100.0f,
                 "lens: k1, k2 in [0, 100), scale and aspect >= 0");
  return SG_OK;
}

sg_status check_ready_for_render(sg_volume* v, const sg_pose* p) {
  const SelSlot& s = v->sel[p->slot];
  if (!s.valid || s.t != p->t) {
    set_error("sg_render: the pose's selection slot was not selected for this time point");
    return SG_ERR_STATE;
  }
  if (s.tf_version != v->tf_version) {
    set_error("sg_render: selection is stale (transfer function or data changed); call sg_select_lod again");
    return SG_ERR_STATE;
  }
  return SG_OK;
}

sg_status prepare_lut(sg_volume* v, float step, int mode, cudaStream_t s) {
  if (v->lut_step != step || v->lut_mode != mode) {
    SG_CUDA(launch_lut(v, step, mode, s), "opacity-corrected tables");
    v->lut_step = step;
    v->lut_mode = mode;
  }
  return SG_OK;
}

}  // namespace

namespace sg {

cudaStream_t side_stream(sg_volume* v) {
  VolumeExtra* x = extra_of(v);
  if (!x) return nullptr;
  if (!x->side_s && cudaStreamCreateWithFlags(&x->side_s, cudaStreamNonBlocking) != cudaSuccess) x->side_s = nullptr;
  return x->side_s;
}

cudaError_t wait_uploads(sg_volume* v, cudaStream_t s) {
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  cudaError_t e = cudaStreamIsCapturing(s, &cap);
  if (e != cudaSuccess || cap != cudaStreamCaptureStatusNone) return e;
  return cudaStreamWaitEvent(s, v->ev_upload, 0);
}

sg_status upload_list_nowait(sg_volume* v, int t, int c, int n, const int32_t* nodes, const void* const* host,
                             int32_t* done, cudaStream_t s) {
  int d = 0;
  const sg_status st = upload_list(v, t, c, n, nodes, host, &d, s, false);
  *done = d;
  return st;
}

}  // namespace sg

extern "C" {

const char* sg_last_error(void) { return g_err.c_str(); }

const char* sg_version(void) { return "sg-b300 0.1 (sm_103a)"; }

sg_status sg_volume_create(const sg_volume_desc* d, sg_volume** out) {
  return sg::guarded("sg_volume_create", [&]() -> sg_status {
    SG_CHECK_ARG(d && out, "desc and out must not be NULL");
    *out = nullptr;
    SG_CHECK_ARG(d->dims[0] >= 1 && d->dims[1] >= 1 && d->dims[2] >= 1, "dims must be >= 1");
    SG_CHECK_ARG(d->dtype == SG_U8 || d->dtype == SG_U16, "dtype must be SG_U8 or SG_U16");
    SG_CHECK_ARG(d->channels >= 1 && d->channels <= kMaxCh, "channels must be 1..4");
    SG_CHECK_ARG(d->timepoints >= 1 && d->timepoints <= 4096, "timepoints must be 1..4096");
    SG_CHECK_ARG(d->brick_size >= 8 && d->brick_size <= 256 && d->brick_size % 8 == 0,
                 "brick_size must be a multiple of 8 in [8, 256]");
    SG_CHECK_ARG(d->apron == 1, "apron must be 1");
    SG_CHECK_ARG(d->lod_levels >= 1 && d->lod_levels <= kMaxLevels, "lod_levels must be 1..16");
    // default: the finest cell that keeps at most kMaxSubPerEdge cells per brick edge
    const int sub = d->skip_block ? d->skip_block : (d->brick_size <= 64 ? 2 : (d->brick_size <= 128 ? 4 : 8));
    SG_CHECK_ARG((sub == 2 || sub == 4 || sub == 8 || sub == 16) && d->brick_size % sub == 0 &&
                     d->brick_size / sub <= kMaxSubPerEdge,
                 "skip_block must be 0 or 2/4/8/16 dividing brick_size, at most 32 cells per brick edge");

    sg_volume* v = new (std::nothrow) sg_volume();
    if (!v) {
      set_error("host allocation failed");
      return SG_ERR_OOM;
    }
    v->desc = *d;
    v->levels = d->lod_levels;
    v->B = d->brick_size;
    v->nch = d->channels;
    v->T = d->timepoints;
    v->esize = d->dtype == SG_U8 ? 1 : 2;
    int64_t off = 0;
    int64_t dims[3] = {d->dims[0], d->dims[1], d->dims[2]};
    for (int L = 0; L < v->levels; ++L) {
      LevelGeom& g = v->geom[L];
      for (int a = 0; a < 3; ++a) {
        g.dims[a] = dims[a];
        g.nb[a] = (int32_t)((dims[a] + v->B - 1) / v->B);
        dims[a] = (dims[a] + 1) / 2;
      }
      g.off = off;
      int64_t n = (int64_t)g.nb[0] * g.nb[1] * g.nb[2];
      off += n;
      v->max_level_nodes = std::max(v->max_level_nodes, n);
    }
    v->nodes = off;
    v->ncell = (int64_t)v->geom[0].nb[0] * v->geom[0].nb[1] * v->geom[0].nb[2];
    if (v->ncell > (1 << 24) || v->nodes * v->T > ((int64_t)1 << 30)) {
      delete v;
      set_error("volume has too many blocks (use a larger brick_size)");
      return SG_ERR_INVALID_ARG;
    }
    const int R = v->B + 2;
    v->brick_bytes = ((size_t)R * R * R * v->esize + 255) / 256 * 256;
    v->sub = sub;
    v->sub_shift = sub == 2 ? 1 : (sub == 4 ? 2 : (sub == 8 ? 3 : 4));
    v->nsub = v->B / sub;
    const int ns3 = v->nsub * v->nsub * v->nsub;
    v->sub_words = (ns3 + 63) / 64;
    const int top = v->levels - 1;
    const int64_t top_nodes = (int64_t)v->geom[top].nb[0] * v->geom[top].nb[1] * v->geom[top].nb[2];
    if (d->device_pool_bytes == 0) {
      v->pool_slots = v->nodes * v->T;
    } else {
      v->pooled = true;
      v->pool_slots = (int64_t)(d->device_pool_bytes / (v->brick_bytes * v->nch));
      if (v->pool_slots < top_nodes * v->T) {
        delete v;
        set_error("device_pool_bytes cannot hold the coarsest level of every time point");
        return SG_ERR_INVALID_ARG;
      }
      v->pool_slots = std::min(v->pool_slots, v->nodes * v->T);
    }
    if (v->pool_slots >= (1 << 26)) {
      delete v;
      set_error("brick pool has too many slots");
      return SG_ERR_INVALID_ARG;
    }

    cudaError_t e = cudaSuccess;
    const int64_t tn = v->nodes * v->T;
    if ((e = dalloc(&v->d_pool, (size_t)v->pool_slots * v->nch * v->brick_bytes)) != cudaSuccess ||
        (e = dalloc(&v->d_slot, tn)) != cudaSuccess || (e = dalloc(&v->d_range, tn * v->nch * 2)) != cudaSuccess ||
        (e = dalloc(&v->d_subrange, (size_t)v->pool_slots * ns3 * v->nch * 2)) != cudaSuccess ||
        (e = dalloc(&v->d_subempty, (size_t)v->pool_slots * v->sub_words)) != cudaSuccess ||
        (e = dalloc(&v->d_subdist, (size_t)v->pool_slots * 8 * ns3)) != cudaSuccess ||
        (e = dalloc(&v->d_nodeflags, tn)) != cudaSuccess ||
        (e = dalloc(&v->d_tf_raw, (size_t)v->nch * kMaxTF * 4)) != cudaSuccess ||
        (e = dalloc(&v->d_palette, (size_t)v->nch * kMaxTF)) != cudaSuccess ||
        (e = dalloc(&v->d_lut, (size_t)2 * v->nch * v->levels * kMaxTF)) != cudaSuccess ||
        (e = dalloc(&v->d_err, 4)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&v->ev_select, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&v->ev_upload, cudaEventDisableTiming)) != cudaSuccess) {
      free_volume(v);
      set_error(std::string("device allocation: ") + cudaGetErrorString(e));
      return SG_ERR_OOM;
    }
    // page table: resident volumes map (t, node) -> t * nodes + node
    v->h_slot.assign(tn, -1);
    if (!v->pooled)
      for (int64_t i = 0; i < tn; ++i) v->h_slot[i] = (int32_t)i;
    // value ranges start unknown (min > max), which is never transparent
    if ((e = cudaMemcpy(v->d_slot, v->h_slot.data(), tn * sizeof(int32_t), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemset(v->d_range, 0, tn * v->nch * 2 * sizeof(uint32_t))) != cudaSuccess ||
        (e = cudaMemset2D(v->d_range, 8, 0xff, 4, tn * v->nch)) != cudaSuccess ||
        (e = cudaMemset(v->d_subempty, 0, (size_t)v->pool_slots * v->sub_words * 8)) != cudaSuccess ||
        (e = cudaMemset(v->d_subdist, 0, (size_t)v->pool_slots * 8 * ns3)) != cudaSuccess ||
        (e = cudaMemset(v->d_nodeflags, 0, tn)) != cudaSuccess ||
        (e = cudaMemset(v->d_tf_raw, 0, (size_t)v->nch * kMaxTF * 16)) != cudaSuccess) {
      free_volume(v);
      return cuda_fail(e, "volume initialisation");
    }
    v->has_data.assign((size_t)v->T * v->nch, 0);
    VolumeExtra* x = new VolumeExtra();
    extras().push_back({v, x});
    if (v->pooled) {
      v->slot_owner.assign(v->pool_slots, -1);
      v->slot_stamp.assign(v->pool_slots, 0);
      v->slot_pinned.assign(v->pool_slots, 0);
      for (int64_t s = v->pool_slots - 1; s >= 0; --s) x->free_slots.push_back(s);
      if ((e = dalloc(&v->d_stamp, v->pool_slots)) != cudaSuccess ||
          (e = cudaMemset(v->d_stamp, 0, v->pool_slots * sizeof(uint64_t))) != cudaSuccess) {
        free_volume(v);
        set_error(std::string("stamp table: ") + cudaGetErrorString(e));
        return SG_ERR_OOM;
      }
    }
    *out = v;
    return SG_OK;
  });
}

sg_status sg_volume_destroy(sg_volume* v) {
  if (!v) return SG_OK;
  cudaDeviceSynchronize();
  free_volume(v);
  return SG_OK;
}

sg_status sg_upload_volume_device(sg_volume* v, int t, int c, const void* dev_level0, void* stream) {
  sg::NvtxRange nvtx_range("sg_upload_volume_device");
  SG_CHECK_ARG(v && dev_level0, "volume and dev_level0 must not be NULL");
  SG_CHECK_ARG(t >= 0 && t < v->T && c >= 0 && c < v->nch, "t or c out of range");
  if (v->pooled) {
    set_error("sg_upload_volume_device needs a fully resident volume (device_pool_bytes == 0)");
    return SG_ERR_STATE;
  }
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<void*> lv(v->levels, nullptr);
  lv[0] = const_cast<void*>(dev_level0);
  for (int L = 1; L < v->levels; ++L) {
    const LevelGeom& g = v->geom[L];
    size_t bytes = (size_t)g.dims[0] * g.dims[1] * g.dims[2] * v->esize;
    cudaError_t e = cudaMallocAsync(&lv[L], bytes, s);
    if (e != cudaSuccess) {
      for (int k = 1; k < L; ++k) cudaFreeAsync(lv[k], s);
      set_error(std::string("pyramid scratch: ") + cudaGetErrorString(e));
      return SG_ERR_OOM;
    }
    SG_CUDA(launch_pyramid(lv[L - 1], v->geom[L - 1].dims, lv[L], g.dims, v->esize, s), "pyramid");
  }
  for (int L = 0; L < v->levels; ++L) SG_CUDA(launch_pack_level(v, t, c, L, lv[L], s), "brick packing");
  for (int L = 1; L < v->levels; ++L) cudaFreeAsync(lv[L], s);
  v->has_data[(size_t)t * v->nch + c] = 1;
  ++v->tf_version;  // block ranges changed: earlier selections are stale
  return refresh_flags(v, s);
}

// ---------------------------------------------------------------- autotuner cache
//
// A text file of lines "<key>\t<persistent> <tile_w> <tile_h> <rays_per_thread>";
// a later line for a key replaces an earlier one.

sg_status sg_render_config_store(const char* path, const char* key, const sg_render_config* cfg) {
  return sg::guarded("sg_render_config_store", [&]() -> sg_status {
    SG_CHECK_ARG(path && key && cfg, "path, key and cfg must not be NULL");
    SG_CHECK_ARG(key[0] && !strpbrk(key, "\t\n") && strlen(key) < 1024, "key: 1..1023 characters, no tab or newline");
    SG_CHECK_ARG(render_config_supported(cfg), "unsupported render configuration");
    FILE* f = fopen(path, "a");
    if (!f) {
      set_error(std::string("sg_render_config_store: cannot open ") + path);
      return SG_ERR_IO;
    }
    const int n = fprintf(f, "%s\t%d %d %d %d\n", key, cfg->persistent, cfg->tile_w, cfg->tile_h, cfg->rays_per_thread);
    if (fclose(f) != 0 || n < 0) {
      set_error(std::string("sg_render_config_store: write failed: ") + path);
      return SG_ERR_IO;
    }
    return SG_OK;
  });
}

sg_status sg_render_config_lookup(const char* path, const char* key, sg_render_config* cfg, int* found) {
  return sg::guarded("sg_render_config_lookup", [&]() -> sg_status {
    SG_CHECK_ARG(path && key && cfg && found, "path, key, cfg and found must not be NULL");
    *found = 0;
    FILE* f = fopen(path, "r");
    if (!f) return SG_OK;  // no cache yet
    char line[1200];
    while (fgets(line, sizeof line, f)) {
      char* tab = strchr(line, '\t');
      if (!tab) continue;
      *tab = 0;
      if (strcmp(line, key) != 0) continue;
      sg_render_config c;
      memset(&c, 0, sizeof c);
      if (sscanf(tab + 1, "%d %d %d %d", &c.persistent, &c.tile_w, &c.tile_h, &c.rays_per_thread) == 4 &&
          render_config_supported(&c)) {
        *cfg = c;
        *found = 1;
      }
    }
    fclose(f);
    return SG_OK;
  });
}

sg_status sg_set_brick_ranges(sg_volume* v, int t, int c, int level, int n, const int32_t* xyz,
                              const uint32_t* minmax, void* stream) {
  return sg::guarded("sg_set_brick_ranges", [&]() -> sg_status {
    SG_CHECK_ARG(v && xyz && minmax && n >= 1, "volume/brick_xyz/minmax NULL or n < 1");
    SG_CHECK_ARG(t >= 0 && t < v->T && c >= 0 && c < v->nch && level >= 0 && level < v->levels,
                 "t, c or level out of range");
    const LevelGeom& g = v->geom[level];
    cudaStream_t s = (cudaStream_t)stream;
    // host-side scatter into a copy of the level's range table, one upload
    const int64_t nlev = (int64_t)g.nb[0] * g.nb[1] * g.nb[2];
    std::vector<uint32_t> tab((size_t)nlev * v->nch * 2);
    uint32_t* dst = v->d_range + ((int64_t)t * v->nodes + g.off) * v->nch * 2;
    SG_CUDA(cudaMemcpyAsync(tab.data(), dst, tab.size() * sizeof(uint32_t), cudaMemcpyDeviceToHost, s), "ranges");
    SG_CUDA(cudaStreamSynchronize(s), "ranges");
    for (int i = 0; i < n; ++i) {
      SG_CHECK_ARG(xyz[3 * i] >= 0 && xyz[3 * i] < g.nb[0] && xyz[3 * i + 1] >= 0 && xyz[3 * i + 1] < g.nb[1] &&
                       xyz[3 * i + 2] >= 0 && xyz[3 * i + 2] < g.nb[2],
                   "brick coordinates out of range");
      SG_CHECK_ARG(minmax[2 * i] <= minmax[2 * i + 1], "range with min > max");
      int64_t b = ((int64_t)xyz[3 * i + 2] * g.nb[1] + xyz[3 * i + 1]) * g.nb[0] + xyz[3 * i];
      tab[(b * v->nch + c) * 2] = minmax[2 * i];
      tab[(b * v->nch + c) * 2 + 1] = minmax[2 * i + 1];
    }
    SG_CUDA(cudaMemcpyAsync(dst, tab.data(), tab.size() * sizeof(uint32_t), cudaMemcpyHostToDevice, s), "ranges");
    SG_CUDA(cudaStreamSynchronize(s), "ranges");
    ++v->tf_version;
    return refresh_flags(v, s);
  });
}

sg_status sg_set_transfer_function(sg_volume* v, int c, const float* rgba, int n, float lo, float hi, float ref_step,
                                   void* stream) {
  sg::NvtxRange nvtx_range("sg_set_transfer_function");
  SG_CHECK_ARG(v && rgba, "volume and rgba must not be NULL");
  SG_CHECK_ARG(c >= 0 && c < v->nch, "channel out of range");
  SG_CHECK_ARG(n >= 2 && n <= kMaxTF, "table size must be 2..4096");
  SG_CHECK_ARG(hi > lo, "window needs hi > lo");
  SG_CHECK_ARG(ref_step > 0.0f, "ref_step must be > 0");
  for (int i = 0; i < 4 * n; ++i)
    SG_CHECK_ARG(rgba[i] >= 0.0f && rgba[i] <= 1.0f, "table entries must be in [0, 1]");
  cudaStream_t s = (cudaStream_t)stream;
  TFHost& t = v->tf[c];
  t.set = true;
  t.n = n;
  t.lo = lo;
  t.hi = hi;
  t.ref_step = ref_step;
  t.rgba.assign(rgba, rgba + 4 * n);
  {
    int e = 0;
    while (e < n && rgba[4 * e + 3] == 0.0f) ++e;
    bool positive_after = true;
    for (int k = e; k < n; ++k) positive_after &= rgba[4 * k + 3] > 0.0f;
    t.low_end_transparent = positive_after;
    t.zero_run = e;
  }
  SG_CUDA(cudaMemcpyAsync(v->d_tf_raw + (size_t)c * kMaxTF * 4, t.rgba.data(), sizeof(float) * 4 * n,
                          cudaMemcpyHostToDevice, s),
          "transfer-function upload");
  // the host vector stays alive in the volume until the next call for c; a
  // stream sync keeps it valid for an asynchronous copy from pageable memory
  SG_CUDA(cudaStreamSynchronize(s), "transfer-function upload");
  v->lut_step = -1.0f;
  v->lut_mode = -1;
  ++v->tf_version;
  return refresh_flags(v, s);
}

sg_status sg_set_channel_shading(sg_volume* v, int c, int input, const float* palette_rgb, int m, float near,
                                 float far, void* stream) {
  SG_CHECK_ARG(v && c >= 0 && c < v->nch, "volume NULL or channel out of range");
  SG_CHECK_ARG(input == SG_INPUT_VALUE || input == SG_INPUT_GRADIENT, "input must be SG_INPUT_VALUE or _GRADIENT");
  SG_CHECK_ARG(m == 0 || (palette_rgb && m >= 1 && m <= kMaxTF && far > near), "palette: 1..4096 entries, far > near");
  for (int i = 0; i < 3 * m; ++i)
    SG_CHECK_ARG(palette_rgb[i] >= 0.0f && palette_rgb[i] <= 1.0f, "palette entries must be in [0, 1]");
  cudaStream_t s = (cudaStream_t)stream;
  TFHost& t = v->tf[c];
  t.gradient = input == SG_INPUT_GRADIENT;
  t.pal_m = m;
  t.pal_near = near;
  t.pal_far = far;
  if (m > 0) {
    std::vector<float4> pal(m);
    for (int i = 0; i < m; ++i) pal[i] = make_float4(palette_rgb[3 * i], palette_rgb[3 * i + 1], palette_rgb[3 * i + 2], 0.f);
    SG_CUDA(cudaMemcpyAsync(v->d_palette + (size_t)c * kMaxTF, pal.data(), sizeof(float4) * m, cudaMemcpyHostToDevice,
                            s),
            "palette upload");
    SG_CUDA(cudaStreamSynchronize(s), "palette upload");
  }
  ++v->tf_version;  // transparency follows the table's input
  return refresh_flags(v, s);
}

sg_status sg_select_lod(sg_volume* v, const sg_pose* p, sg_select_stats* stats, void* stream) {
  sg::NvtxRange nvtx_range("sg_select_lod");
  SG_CHECK_ARG(v, "volume is NULL");
  sg_status st = check_pose(v, p);
  if (st != SG_OK) return st;
  st = sg_select_lod_batch(v, p, 1, stream);
  if (st != SG_OK || !stats) return st;
  uint32_t c[8];
  cudaStream_t s = (cudaStream_t)stream;
  SG_CUDA(cudaMemcpyAsync(c, v->sel[p->slot].d_counters, sizeof c, cudaMemcpyDeviceToHost, s), "select stats");
  SG_CUDA(cudaStreamSynchronize(s), "select stats");
  memset(stats, 0, sizeof *stats);
  stats->requested = c[0];
  stats->selected = c[1];
  stats->culled = c[2];
  stats->empty = c[3];
  stats->fallback = c[4];
  stats->nonempty = c[5];
  return SG_OK;
}

sg_status sg_select_lod_batch(sg_volume* v, const sg_pose* poses, int n, void* stream) {
  SG_CHECK_ARG(v && poses && n >= 1, "volume/poses NULL or n < 1");
  if (!tfs_ready(v)) {
    set_error("sg_select_lod: set a transfer function for every channel first");
    return SG_ERR_STATE;
  }
  for (int i = 0; i < n; ++i) {
    sg_status st = check_pose(v, &poses[i]);
    if (st != SG_OK) return st;
    for (int c = 0; c < v->nch; ++c)
      if (!v->has_data[(size_t)poses[i].t * v->nch + c]) {
        set_error("sg_select_lod: no data uploaded for this time point / channel");
        return SG_ERR_STATE;
      }
    if (v->pooled) {
      const LevelGeom& g = v->geom[v->levels - 1];
      int64_t nt = (int64_t)g.nb[0] * g.nb[1] * g.nb[2];
      for (int64_t b = 0; b < nt; ++b)
        if (v->h_slot[(int64_t)poses[i].t * v->nodes + g.off + b] < 0) {
          set_error("sg_select_lod: the coarsest level must be resident (upload it first)");
          return SG_ERR_STATE;
        }
    }
    for (int j = 0; j < i; ++j)
      SG_CHECK_ARG(poses[j].slot != poses[i].slot, "poses of one batch must use different selection slots");
    st = ensure_selection(v, poses[i].slot);
    if (st != SG_OK) return st;
  }
  cudaStream_t s = (cudaStream_t)stream;
  // the page table, ranges and flags of every brick upload queued so far
  SG_CUDA(wait_uploads(v, s), "selection");
  ++v->frame;
  SG_CUDA(launch_select(v, poses, n, s), "selection");
  // uploads and reads on other streams wait for the stamps and results this
  // launch writes. A launch captured into a CUDA graph is not recorded: an
  // event recorded during capture cannot be waited on outside it, so the
  // event keeps the last selection launched directly, and a caller replaying
  // the graph orders what follows through its own streams.
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  SG_CUDA(cudaStreamIsCapturing(s, &cap), "selection");
  if (cap == cudaStreamCaptureStatusNone) SG_CUDA(cudaEventRecord(v->ev_select, s), "selection");
  for (int i = 0; i < n; ++i) {
    SelSlot& sl = v->sel[poses[i].slot];
    sl.valid = true;
    sl.t = poses[i].t;
    sl.tf_version = v->tf_version;
  }
  return SG_OK;
}

sg_status sg_read_selection(sg_volume* v, int slot, int32_t* cell_node, int64_t ncell, uint8_t* node_state,
                            int64_t nnode, int32_t* req, int32_t req_cap, int32_t* nreq, void* stream) {
  return sg::guarded("sg_read_selection", [&]() -> sg_status {
    SG_CHECK_ARG(v && slot >= 0 && slot < kMaxSlots, "volume NULL or slot out of range");
    const SelSlot& sl = v->sel[slot];
    if (!sl.valid) {
      set_error("sg_read_selection: slot was never selected");
      return SG_ERR_STATE;
    }
    cudaStream_t s = (cudaStream_t)stream;
    SG_CHECK_ARG(!cell_node || ncell >= v->ncell, "cell_node buffer too small");
    SG_CHECK_ARG(!node_state || nnode >= v->nodes, "node_state buffer too small");
    uint32_t c[8];
    // the selection may have been launched on another stream
    SG_CUDA(cudaStreamWaitEvent(s, v->ev_select, 0), "read selection");
    SG_CUDA(cudaMemcpyAsync(c, sl.d_counters, sizeof c, cudaMemcpyDeviceToHost, s), "read selection");
    if (cell_node)
      SG_CUDA(cudaMemcpyAsync(cell_node, sl.d_cell_node, v->ncell * sizeof(int32_t), cudaMemcpyDeviceToHost, s),
              "read selection");
    if (node_state)
      SG_CUDA(cudaMemcpyAsync(node_state, sl.d_state, v->nodes, cudaMemcpyDeviceToHost, s), "read selection");
    SG_CUDA(cudaStreamSynchronize(s), "read selection");
    if (nreq) *nreq = (int32_t)c[0];
    if (req && req_cap > 0) {
      std::vector<int32_t> r(c[0]);
      if (c[0]) {
        SG_CUDA(cudaMemcpyAsync(r.data(), sl.d_req, c[0] * sizeof(int32_t), cudaMemcpyDeviceToHost, s),
                "read requests");
        SG_CUDA(cudaStreamSynchronize(s), "read requests");
      }
      std::sort(r.begin(), r.end());
      for (int32_t i = 0; i < req_cap && i < (int32_t)r.size(); ++i) req[i] = r[i];
    }
    return SG_OK;
  });
}

sg_status sg_read_ranges(sg_volume* v, int t, uint32_t* minmax, int64_t nnode) {
  SG_CHECK_ARG(v && minmax, "volume or output NULL");
  SG_CHECK_ARG(t >= 0 && t < v->T, "t out of range");
  SG_CHECK_ARG(nnode >= v->nodes, "output too small");
  SG_CUDA(cudaDeviceSynchronize(), "read ranges");
  SG_CUDA(cudaMemcpy(minmax, v->d_range + (int64_t)t * v->nodes * v->nch * 2, v->nodes * v->nch * 2 * sizeof(uint32_t),
                     cudaMemcpyDeviceToHost),
          "read ranges");
  return SG_OK;
}

sg_status sg_read_residency(sg_volume* v, int t, int32_t* slot_of_node, int64_t nnode) {
  SG_CHECK_ARG(v && slot_of_node, "volume or output NULL");
  SG_CHECK_ARG(t >= 0 && t < v->T, "t out of range");
  SG_CHECK_ARG(nnode >= v->nodes, "output too small");
  memcpy(slot_of_node, v->h_slot.data() + (size_t)t * v->nodes, v->nodes * sizeof(int32_t));
  return SG_OK;
}

sg_status sg_read_brick(sg_volume* v, int t, int c, int level, int bx, int by, int bz, void* host_out,
                        void* stream) {
  SG_CHECK_ARG(v && host_out, "volume or host_out NULL");
  SG_CHECK_ARG(t >= 0 && t < v->T && c >= 0 && c < v->nch && level >= 0 && level < v->levels,
               "t, c or level out of range");
  const LevelGeom& g = v->geom[level];
  SG_CHECK_ARG(bx >= 0 && bx < g.nb[0] && by >= 0 && by < g.nb[1] && bz >= 0 && bz < g.nb[2],
               "brick coordinates out of range");
  int64_t node = g.off + ((int64_t)bz * g.nb[1] + by) * g.nb[0] + bx;
  int32_t slot = v->h_slot[(int64_t)t * v->nodes + node];
  if (slot < 0) {
    set_error("sg_read_brick: brick not resident");
    return SG_ERR_NOT_RESIDENT;
  }
  const int R = v->B + 2;
  cudaStream_t s = (cudaStream_t)stream;
  SG_CUDA(wait_uploads(v, s), "brick download");
  SG_CUDA(cudaMemcpyAsync(host_out, v->d_pool + ((size_t)slot * v->nch + c) * v->brick_bytes,
                          (size_t)R * R * R * v->esize, cudaMemcpyDeviceToHost, s),
          "brick download");
  SG_CUDA(cudaStreamSynchronize(s), "brick download");
  return SG_OK;
}

sg_status sg_render(sg_volume* v, const sg_pose* p, const sg_render_params* prm, float* out_rgba[2], void* stream) {
  sg::NvtxRange nvtx_range("sg_render");
  SG_CHECK_ARG(v && out_rgba && out_rgba[0] && out_rgba[1], "volume or outputs NULL");
  SG_CHECK_ARG(((uintptr_t)out_rgba[0] % 16) == 0 && ((uintptr_t)out_rgba[1] % 16) == 0,
               "output buffers must be 16-byte aligned");
  sg_status st = check_pose(v, p);
  if (st != SG_OK) return st;
  if ((st = check_render_params(prm)) != SG_OK) return st;
  if ((st = check_ready_for_render(v, p)) != SG_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  if ((st = prepare_lut(v, prm->step, prm->mode, s)) != SG_OK) return st;
  SG_CUDA(launch_render(v, p, 1, prm, out_rgba, s), "render");
  return SG_OK;
}

sg_status sg_render_host(sg_volume* v, const sg_pose* p, const sg_render_params* prm, float* host_rgba[2],
                         void* stream) {
  sg::NvtxRange nvtx_range("sg_render_host");
  SG_CHECK_ARG(v && host_rgba && host_rgba[0] && host_rgba[1], "volume or outputs NULL");
  sg_status st = check_pose(v, p);
  if (st != SG_OK) return st;
  const size_t per = (size_t)p->width * p->height * 4 * sizeof(float);
  if (v->stage_bytes < 2 * per) {
    cudaFree(v->d_stage);
    v->d_stage = nullptr;
    v->stage_bytes = 0;
    cudaError_t e = cudaMalloc(&v->d_stage, 2 * per);
    if (e != cudaSuccess) {
      set_error(std::string("staging allocation: ") + cudaGetErrorString(e));
      return SG_ERR_OOM;
    }
    v->stage_bytes = 2 * per;
  }
  float* dev[2] = {v->d_stage, v->d_stage + per / sizeof(float)};
  st = sg_render(v, p, prm, dev, stream);
  if (st != SG_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  SG_CUDA(cudaMemcpyAsync(host_rgba[0], dev[0], per, cudaMemcpyDeviceToHost, s), "image download");
  SG_CUDA(cudaMemcpyAsync(host_rgba[1], dev[1], per, cudaMemcpyDeviceToHost, s), "image download");
  SG_CUDA(cudaStreamSynchronize(s), "image download");
  return SG_OK;
}

sg_status sg_render_host_wait(sg_volume* v, int all) {
  SG_CHECK_ARG(v, "volume NULL");
  // from pipe_next (the pair of the oldest frame) on, oldest first
  for (int i = 0; i < sg_volume::kPipeDepth; ++i) {
    const int k = (v->pipe_next + i) % sg_volume::kPipeDepth;
    if (!v->copy_pending[k]) continue;
    SG_CUDA(cudaEventSynchronize(v->ev_copied[k]), "image download");
    v->copy_pending[k] = false;
    if (!all) break;
  }
  return SG_OK;
}

sg_status sg_render_host_async(sg_volume* v, const sg_pose* p, const sg_render_params* prm, float* host_rgba[2],
                               void* stream) {
  SG_CHECK_ARG(v && host_rgba && host_rgba[0] && host_rgba[1], "volume or outputs NULL");
  sg_status st = check_pose(v, p);
  if (st != SG_OK) return st;
  const size_t per = (size_t)p->width * p->height * 4 * sizeof(float);
  cudaStream_t s = (cudaStream_t)stream;
  if (!v->copy_stream) {
    SG_CUDA(cudaStreamCreateWithFlags(&v->copy_stream, cudaStreamNonBlocking), "copy stream");
    for (int k = 0; k < sg_volume::kPipeDepth; ++k) {
      SG_CUDA(cudaEventCreateWithFlags(&v->ev_rendered[k], cudaEventDisableTiming), "pipeline events");
      SG_CUDA(cudaEventCreateWithFlags(&v->ev_copied[k], cudaEventDisableTiming), "pipeline events");
    }
  }
  if (v->pipe_bytes < 2 * per) {
    // larger images: the copies in flight still read the old staging
    if ((st = sg_render_host_wait(v, 1)) != SG_OK) return st;
    cudaFree(v->d_pipe);
    v->d_pipe = nullptr;
    v->pipe_bytes = 0;
    cudaError_t e = cudaMalloc(&v->d_pipe, 2 * sg_volume::kPipeDepth * per);
    if (e != cudaSuccess) {
      set_error(std::string("staging allocation: ") + cudaGetErrorString(e));
      return SG_ERR_OOM;
    }
    v->pipe_bytes = 2 * per;
  }
  const int k = v->pipe_next;
  float* dev[2] = {reinterpret_cast<float*>(v->d_pipe + k * v->pipe_bytes),
                   reinterpret_cast<float*>(v->d_pipe + k * v->pipe_bytes + per)};
  // the pair's previous frame (kPipeDepth calls back) must be copied out
  // before this render overwrites it: a wait on the GPU, not the host (the
  // copy stream's next event covers that frame's copy too)
  if (v->copy_pending[k]) SG_CUDA(cudaStreamWaitEvent(s, v->ev_copied[k], 0), "pipeline order");
  st = sg_render(v, p, prm, dev, stream);
  if (st != SG_OK) return st;
  SG_CUDA(cudaEventRecord(v->ev_rendered[k], s), "pipeline order");
  SG_CUDA(cudaStreamWaitEvent(v->copy_stream, v->ev_rendered[k], 0), "pipeline order");
  SG_CUDA(cudaMemcpyAsync(host_rgba[0], dev[0], per, cudaMemcpyDeviceToHost, v->copy_stream), "image download");
  SG_CUDA(cudaMemcpyAsync(host_rgba[1], dev[1], per, cudaMemcpyDeviceToHost, v->copy_stream), "image download");
  SG_CUDA(cudaEventRecord(v->ev_copied[k], v->copy_stream), "pipeline order");
  v->copy_pending[k] = true;
  v->pipe_next = (k + 1) % sg_volume::kPipeDepth;
  return SG_OK;
}

sg_status sg_render_batch(sg_volume* v, const sg_pose* poses, int n, const sg_render_params* prm, float** outs,
                          void* stream) {
  sg::NvtxRange nvtx_range("sg_render_batch");
  SG_CHECK_ARG(v && poses && outs && n >= 1 && n <= 64, "volume/poses/outs NULL or n not in 1..64");
  sg_status st = check_render_params(prm);
  if (st != SG_OK) return st;
  SG_CHECK_ARG(!prm->depth[0] && !prm->depth[1], "depth buffers apply to sg_render only");
  SG_CHECK_ARG(!prm->lens, "lens-warped rendering applies to sg_render only");
  for (int i = 0; i < n; ++i) {
    if ((st = check_pose(v, &poses[i])) != SG_OK) return st;
    if ((st = check_ready_for_render(v, &poses[i])) != SG_OK) return st;
    SG_CHECK_ARG(outs[2 * i] && outs[2 * i + 1], "batch output NULL");
    SG_CHECK_ARG(((uintptr_t)outs[2 * i] % 16) == 0 && ((uintptr_t)outs[2 * i + 1] % 16) == 0,
                 "output buffers must be 16-byte aligned");
  }
  cudaStream_t s = (cudaStream_t)stream;
  if ((st = prepare_lut(v, prm->step, prm->mode, s)) != SG_OK) return st;
  SG_CUDA(launch_render(v, poses, n, prm, outs, s), "batched render");
  return SG_OK;
}

sg_status sg_unwarp(const sg_lens* lens, const float* warped[2], int Ww, int Hw, float* out[2], int W, int H,
                    void* stream) {
  SG_CHECK_ARG(lens && warped && out && warped[0] && warped[1] && out[0] && out[1], "lens or buffers NULL");
  SG_CHECK_ARG(Ww > 0 && Hw > 0 && W > 0 && H > 0 && Ww <= 32768 && Hw <= 32768 && W <= 32768 && H <= 32768,
               "image sizes must be in 1..32768");
  SG_CHECK_ARG(lens->k1 >= 0.0f && lens->k2 >= 0.0f && lens->scale >= 0.0f && lens->aspect >= 0.0f &&
                   lens->k1 < 100.0f && lens->k2 < 100.0f,
               "lens: k1, k2 in [0, 100), scale and aspect >= 0");
  for (int e = 0; e < 2; ++e)
    SG_CHECK_ARG(((uintptr_t)warped[e] % 16) == 0 && ((uintptr_t)out[e] % 16) == 0, "buffers must be 16-byte aligned");
  cudaStream_t s = (cudaStream_t)stream;
  for (int e = 0; e < 2; ++e) SG_CUDA(launch_unwarp(lens, e, warped[e], Ww, Hw, out[e], W, H, s), "unwarp");
  return SG_OK;
}

sg_status sg_set_render_config(sg_volume* v, const sg_render_config* cfg) {
  SG_CHECK_ARG(v && cfg, "volume or config NULL");
  SG_CHECK_ARG(render_config_supported(cfg), "unsupported tile shape / rays per thread");
  v->render_cfg = *cfg;
  return SG_OK;
}

sg_status sg_get_render_config(sg_volume* v, sg_render_config* cfg) {
  SG_CHECK_ARG(v && cfg, "volume or config NULL");
  *cfg = v->render_cfg;
  return SG_OK;
}

sg_status sg_autotune_render(sg_volume* v, const sg_pose* poses, int n, const sg_render_params* prm, float** outs,
                             int reps, sg_render_config* best, float* best_ms, void* stream) {
  return sg::guarded("sg_autotune_render", [&]() -> sg_status {
    SG_CHECK_ARG(v && reps >= 1 && reps <= 1000, "volume NULL or reps not in 1..1000");
    cudaStream_t s = (cudaStream_t)stream;
    sg_render_config cand[32];
    int nc = render_config_candidates(cand, 32);
    cudaEvent_t e0, e1;
    SG_CUDA(cudaEventCreate(&e0), "autotune events");
    SG_CUDA(cudaEventCreate(&e1), "autotune events");
    const sg_render_config keep = v->render_cfg;
    float best_t = 1e30f;
    sg_render_config best_c = keep;
    sg_status st = SG_OK;
    for (int i = 0; i < nc && st == SG_OK; ++i) {
      v->render_cfg = cand[i];
      st = sg_render_batch(v, poses, n, prm, outs, stream);  // warm-up, also validates the arguments
      if (st != SG_OK) break;
      cudaEventRecord(e0, s);
      for (int r = 0; r < reps && st == SG_OK; ++r) st = sg_render_batch(v, poses, n, prm, outs, stream);
      cudaEventRecord(e1, s);
      cudaError_t ce = cudaEventSynchronize(e1);
      if (ce != cudaSuccess) {
        st = cuda_fail(ce, "autotune");
        break;
      }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      ms /= reps;
      if (ms < best_t) {
        best_t = ms;
        best_c = cand[i];
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    v->render_cfg = st == SG_OK ? best_c : keep;
    if (st != SG_OK) return st;
    if (best) *best = best_c;
    if (best_ms) *best_ms = best_t;
    return SG_OK;
  });
}

sg_status sg_upload_bricks(sg_volume* v, int t, int c, int level, int n, const int32_t* xyz, const void* host,
                           void* stream) {
  return sg::guarded("sg_upload_bricks", [&]() -> sg_status {
    SG_CHECK_ARG(v && xyz && host && n >= 1, "volume/brick_xyz/host NULL or n < 1");
    SG_CHECK_ARG(t >= 0 && t < v->T && c >= 0 && c < v->nch, "t or c out of range");
    SG_CHECK_ARG(level >= 0 && level < v->levels, "level out of range");
    const LevelGeom& g = v->geom[level];
    for (int i = 0; i < n; ++i)
      SG_CHECK_ARG(xyz[3 * i] >= 0 && xyz[3 * i] < g.nb[0] && xyz[3 * i + 1] >= 0 && xyz[3 * i + 1] < g.nb[1] &&
                       xyz[3 * i + 2] >= 0 && xyz[3 * i + 2] < g.nb[2],
                   "brick coordinates out of range");
    const size_t raw = (size_t)(v->B + 2) * (v->B + 2) * (v->B + 2) * v->esize;
    std::vector<int32_t> nodes(n);
    std::vector<const void*> ptrs(n);
    for (int i = 0; i < n; ++i) {
      nodes[i] = (int32_t)(g.off + ((int64_t)xyz[3 * i + 2] * g.nb[1] + xyz[3 * i + 1]) * g.nb[0] + xyz[3 * i]);
      ptrs[i] = static_cast<const uint8_t*>(host) + raw * i;
    }
    int done = 0;
    sg_status st = upload_list(v, t, c, n, nodes.data(), ptrs.data(), &done, (cudaStream_t)stream);
    if (st == SG_OK && done < n) {
      set_error("sg_upload_bricks: brick cache full of bricks used by the current frame");
      return SG_ERR_OOM;
    }
    return st;
  });
}

sg_status sg_upload_brick_list(sg_volume* v, int t, int c, int n, const int32_t* nodes, const void* const* host,
                               int32_t* n_done, void* stream) {
  return sg::guarded("sg_upload_brick_list", [&]() -> sg_status {
    sg::NvtxRange nvtx_range("sg_upload_brick_list");
    SG_CHECK_ARG(v && n_done && n >= 0 && (n == 0 || (nodes && host)), "volume/nodes/host/n_done NULL or n < 0");
    SG_CHECK_ARG(t >= 0 && t < v->T && c >= 0 && c < v->nch, "t or c out of range");
    *n_done = 0;
    for (int i = 0; i < n; ++i) {
      SG_CHECK_ARG(nodes[i] >= 0 && nodes[i] < v->nodes, "node id out of range");
      SG_CHECK_ARG(host[i], "host pointer NULL");
    }
    if (n == 0) return SG_OK;
    int done = 0;
    sg_status st = upload_list(v, t, c, n, nodes, host, &done, (cudaStream_t)stream);
    *n_done = done;
    return st;
  });
}

sg_status sg_upload_brick_list_async(sg_volume* v, int t, int c, int n, const int32_t* nodes,
                                     const void* const* host, int32_t* n_done, void* stream) {
  return sg::guarded("sg_upload_brick_list_async", [&]() -> sg_status {
    sg::NvtxRange nvtx_range("sg_upload_brick_list_async");
    SG_CHECK_ARG(v && n_done && n >= 0 && (n == 0 || (nodes && host)), "volume/nodes/host/n_done NULL or n < 0");
    SG_CHECK_ARG(t >= 0 && t < v->T && c >= 0 && c < v->nch, "t or c out of range");
    *n_done = 0;
    for (int i = 0; i < n; ++i) {
      SG_CHECK_ARG(nodes[i] >= 0 && nodes[i] < v->nodes, "node id out of range");
      SG_CHECK_ARG(host[i], "host pointer NULL");
    }
    if (n == 0) return SG_OK;
    int done = 0;
    sg_status st = upload_list(v, t, c, n, nodes, host, &done, (cudaStream_t)stream, false);
    *n_done = done;
    return st;
  });
}

}  // extern "C"
