// Internal declarations of the B300 DVR library (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <exception>
#include <string>
#include <utility>
#include <vector>

#include "../../include/sg.h"
#include <nvtx3/nvToolsExt.h>

namespace sg {

// A named NVTX range over the C-ABI call it is declared in, so a profiler
// that reads NVTX (ncu --nvtx) can pick a stage's kernels; without an
// attached tool a push or pop is a test of an unset function pointer.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

constexpr int kMaxLevels = 16;
constexpr int kMaxCh = 4;
constexpr int kMaxSlots = 256;   // selection slots per volume
constexpr int kMaxSubPerEdge = 32;  // empty-skipping cells per brick edge (distance map fits shared memory)
constexpr int kMaxTF = 4096;

// A leaf-map entry tells the ray caster what renders one level-0 block cell.
//   bit 31      : nothing renders here (culled or transparent); bits 0..3 give
//                 the level of the dropped block so a ray can jump all of it
//   bits 0..3   : level L of the rendering block
//   bit 4       : the block itself is transparent under the current tables
//   bits 5..30  : pool slot of the block's brick group
constexpr uint32_t kLeafNone = 0x80000000u;
__host__ __device__ inline uint32_t leaf_pack(uint32_t slot, int level, bool own_empty) {
  return (slot << 5) | (own_empty ? 16u : 0u) | (uint32_t)level;
}

// Node traversal states (match the C ABI's sg_read_selection documentation).
enum : uint8_t { kUnseen = 0, kCulled = 1, kEmpty = 2, kSelected = 3, kFallback = 4, kRefined = 5 };

// Node flags derived from the transfer functions.
enum : uint8_t { kOwnEmpty = 1, kSubtreeEmpty = 2 };

struct LevelGeom {
  int64_t dims[3];  // voxels of this level
  int32_t nb[3];    // blocks per axis
  int64_t off;      // first node id of this level
};

// Quantised inputs of the integer selection test for one pose.
struct SelectInputs {
  int64_t eye[2][3];      // 1/64 level-0 voxel
  int64_t plane[2][4][4]; // A, B, C (x 2^16), D (x 2^16 x 64, one voxel outward)
  uint64_t K;             // floor((tau theta)^2 2^40)
};

struct SelSlot {
  bool valid = false;
  int t = -1;
  uint64_t tf_version = 0;
  uint32_t* d_leaf = nullptr;      // [ncell]
  int32_t* d_cell_node = nullptr;  // [ncell]
  uint8_t* d_state = nullptr;      // [nodes]
  int32_t* d_req = nullptr;        // [nodes]
  uint32_t* d_counters = nullptr;  // [8]: nreq, selected, culled, empty, fallback
  int32_t* d_frontier = nullptr;   // [2][max level count]
};

struct TFHost {
  bool set = false;
  int n = 0;
  float lo = 0, hi = 1, ref_step = 0.5f;
  std::vector<float> rgba;
  // alpha is 0 exactly on a run of entries starting at entry 0 and positive
  // after it (so every transparent value lies below every visible one)
  bool low_end_transparent = false;
  int zero_run = 0;                 // entries 0 .. zero_run - 1 have alpha exactly 0
  int gradient = 0;                 // the table reads the gradient magnitude
  int pal_m = 0;                    // depth palette entries (0: the table's colour)
  float pal_near = 0.0f, pal_far = 1.0f;
};

}  // namespace sg

struct sg_volume {
  sg_volume_desc desc;
  int levels = 0, B = 0, nch = 0, T = 0, esize = 0;
  sg::LevelGeom geom[sg::kMaxLevels];
  int64_t nodes = 0;        // per time point
  int64_t ncell = 0;        // level-0 block cells
  int64_t max_level_nodes = 0;
  int sub = 0, sub_shift = 0;  // empty-skipping cell edge (level-L voxels) and its log2
  int nsub = 0;             // sub-blocks per axis in a brick
  int sub_words = 0;        // 64-bit words of sub-block empty bits per slot

  // brick pool: slot s, channel c at d_pool + (s * nch + c) * brick_bytes
  uint8_t* d_pool = nullptr;
  int64_t pool_slots = 0;
  size_t brick_bytes = 0;   // (B+2)^3 * esize, padded to 256
  bool pooled = false;      // LRU cache instead of everything resident

  int32_t* d_slot = nullptr;       // [T][nodes] slot or -1
  std::vector<int32_t> h_slot;     // host mirror
  uint32_t* d_range = nullptr;     // [T][nodes][nch][2]
  uint16_t* d_subrange = nullptr;  // [slots][nsub^3][nch][2]
  uint64_t* d_subempty = nullptr;  // [slots][sub_words]
  uint8_t* d_subdist = nullptr;    // [slots][8 octants][nsub^3] sub-blocks ahead that are all transparent
  uint8_t* d_nodeflags = nullptr;  // [T][nodes]
  std::vector<uint8_t> has_data;   // [T][nch]

  // transfer functions
  sg::TFHost tf[sg::kMaxCh];
  float* d_tf_raw = nullptr;       // [nch][kMaxTF][4]
  float4* d_palette = nullptr;     // [nch][kMaxTF] depth palette RGB (w unused)
  float4* d_lut = nullptr;         // [nch][levels][kMaxTF][2] opacity-corrected (entry, delta to next)
  float lut_step = -1.0f;
  int lut_mode = -1;
  uint64_t tf_version = 0;

  // LRU state (pooled volumes)
  std::vector<int64_t> slot_owner;    // slot -> t*nodes+node or -1
  std::vector<uint64_t> slot_stamp;   // last frame the slot was used
  std::vector<uint8_t> slot_pinned;   // coarsest level: never evicted
  uint64_t frame = 0;
  uint64_t* d_stamp = nullptr;        // [slots] frame of last use, written by the selection kernel
  cudaEvent_t ev_select = nullptr;    // recorded after each stamping selection launch
  cudaEvent_t ev_upload = nullptr;    // recorded after each brick upload's copies and kernels
  uint64_t stamps_read = ~0ull;       // the frame whose device stamps the host LRU last took in

  sg::SelSlot sel[sg::kMaxSlots];

  sg_render_config render_cfg = {};  // tile shape / persistence; zero = default
  float* d_stage = nullptr;  // sg_render_host staging
  size_t stage_bytes = 0;
  // sg_render_host_async: kPipeDepth staging pairs (frames in flight), a copy
  // stream, per-pair events; the calls take the pairs in turn
  static constexpr int kPipeDepth = 3;
  uint8_t* d_pipe = nullptr;
  size_t pipe_bytes = 0;  // one pair (both eyes)
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t ev_rendered[kPipeDepth] = {}, ev_copied[kPipeDepth] = {};
  bool copy_pending[kPipeDepth] = {};
  int pipe_next = 0;  // the pair of the next call: the oldest frame's
  uint32_t* d_err = nullptr; // device control block: [0] tile queue head of the persistent render
};

namespace sg {

void set_error(const std::string& msg);

// Runs an entry point's body; a C++ exception from host bookkeeping (a
// container that could not grow, a thread that could not start) becomes
// SG_ERR_OOM with a message, so that none crosses the C ABI.
template <typename F>
sg_status guarded(const char* name, F&& body) {
  try {
    return body();
  } catch (const std::exception& e) {
    set_error(std::string(name) + ": host resources exhausted (" + e.what() + ")");
  } catch (...) {
    set_error(std::string(name) + ": host resources exhausted");
  }
  return SG_ERR_OOM;
}
sg_status cuda_fail(cudaError_t e, const char* what);
// the checks of a pose that do not involve its selection slot (time point,
// image size, pixel error, projection)
sg_status check_pose_fields(const sg_volume* v, const sg_pose* p);

// ingest.cu
cudaError_t launch_pyramid(const void* src, const int64_t* sdims, void* dst, const int64_t* ddims, int esize,
                           cudaStream_t s);
cudaError_t launch_pack_level(sg_volume* v, int t, int c, int L, const void* level_data, cudaStream_t s);
cudaError_t launch_subranges(sg_volume* v, const int32_t* d_slots, int nslots, int c, cudaStream_t s);
cudaError_t launch_brick_ranges(sg_volume* v, int t, int c, int L, const int32_t* d_nodes, int n,
                                cudaStream_t s);

// tf.cu
// node flags for every node; sub-block bits / distances for every slot, or
// only the nslots slots listed in device array d_slots
cudaError_t launch_tf_flags(sg_volume* v, cudaStream_t s, const int32_t* d_slots = nullptr, int nslots = 0);
cudaError_t launch_lut(sg_volume* v, float step, int mode, cudaStream_t s);
cudaError_t launch_unwarp(const sg_lens* lens, int e, const float* warped, int Ww, int Hw, float* out, int W, int H,
                          cudaStream_t s);

// select.cu
void compute_select_inputs(const sg_volume* v, const sg_pose* p, SelectInputs* out);
cudaError_t launch_select(sg_volume* v, const sg_pose* poses, int n, cudaStream_t s);

// render.cu
cudaError_t launch_render(sg_volume* v, const sg_pose* poses, int n, const sg_render_params* prm,
                          float* const* outs, cudaStream_t s);
bool render_config_supported(const sg_render_config* c);
int render_config_candidates(sg_render_config* out, int cap);

}  // namespace sg

// Container and host cache (host code shared by container.cpp and stream.cpp)
namespace sg {
size_t lz4_bound(size_t n);
size_t lz4_compress(const uint8_t* src, size_t n, uint8_t* dst);
bool lz4_decompress(const uint8_t* src, size_t csize, uint8_t* dst, size_t n);
sg_status container_read_chunk(sg_container* k, uint64_t off, void* out, uint32_t* minmax, uint32_t* comp_bytes);
const sg_volume_desc& container_desc(const sg_container* k);
uint64_t container_chunk_offset(const sg_container* k, int t, int c, int64_t node, bool* found);
size_t container_brick_bytes(const sg_container* k);
int64_t container_nodes(const sg_container* k);
sg_status host_cache_lookup(sg_host_cache* hc, int t, int c, int64_t node, int64_t* entry, int* hit,
                            std::vector<std::pair<int64_t, int64_t>>* todo);
void host_cache_drop(sg_host_cache* hc, int64_t e);
// sg_upload_brick_list without the final wait: returns once the copies and
// kernels are queued on s (the host bricks must stay untouched until
// v->ev_upload has passed; later selections wait for it on the device)
sg_status upload_list_nowait(sg_volume* v, int t, int c, int n, const int32_t* nodes, const void* const* host,
                             int32_t* done, cudaStream_t s);
// the stream waits (on the device) for every brick upload queued so far
// (not while it is being captured into a graph)
cudaError_t wait_uploads(sg_volume* v, cudaStream_t s);
void host_cache_collect(sg_host_cache* hc, bool wait, int32_t* reads, uint64_t* bytes, int32_t* failed);
void host_cache_drain(sg_host_cache* hc);
void host_cache_quiesce(sg_host_cache* hc);
// clears the pending state of the copies once they are done, without waiting
void host_cache_poll(sg_host_cache* hc);
// a non-blocking stream of the volume for the host's reads of selection
// results and stamps (made at first use; nullptr if none could be made)
cudaStream_t side_stream(sg_volume* v);
}  // namespace sg
