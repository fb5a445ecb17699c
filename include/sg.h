/* sg.h: C ABI of the B300 direct-volume-rendering library.
 *
 * The library renders bricked, multi-resolution 8/16-bit volumes by per-pixel
 * ray casting under the emission-absorption optical model, as a stereo pair
 * per head pose. It follows the "Volume Rendering" section of syGlass
 * (arXiv:1804.08197):
 *   - "DVR Techniques": one ray per pixel, sampled at a fixed step, trilinear
 *     interpolation, transfer function, emission-absorption compositing with
 *     early ray termination;
 *   - "Octree Representation": blocks in a multi-resolution pyramid, chosen
 *     top-down by comparing the block's angular voxel size with the pixel
 *     angle, front to back, with frustum culling and a one-level-coarser
 *     fallback while children are not cached;
 *   - "Volumetric Data Cashing": a GPU brick cache with least-recently-used
 *     eviction by timestamp.
 *
 * Conventions shared by every call
 *  - Every call returns sg_status; no exception crosses the ABI. On failure,
 *    sg_last_error() returns a thread-local message naming the cause.
 *  - "stream" is a cudaStream_t (NULL = the legacy default stream). Calls that
 *    take a stream enqueue their GPU work on it and return without waiting,
 *    unless stated otherwise.
 *  - Matrices are 4x4 float, column major, OpenGL conventions (clip z in
 *    [-1, 1]). Voxel space is [0, N]^3 in level-0 voxels, voxel i has its
 *    centre at i + 0.5; the model matrix maps voxel space to world space.
 *  - Images are row-major RGBA float32, row 0 = top, colour premultiplied by
 *    alpha (associated colour), background (0, 0, 0, 0).
 *  - Host arrays are owned by the caller and only read during the call
 *    (asynchronous uploads read them until the stream reaches the copy:
 *    keep them alive and unchanged until then; pinned memory makes the copy
 *    asynchronous). Device output buffers are owned by the caller. All other
 *    device memory (brick pool, page tables, transfer functions, selections)
 *    is owned by the volume and released by sg_volume_destroy.
 */
#ifndef SG_H
#define SG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SG_OK = 0,
  SG_ERR_INVALID_ARG = 1, /* a pointer, size, index or enum is out of range */
  SG_ERR_OOM = 2,         /* a device or pinned-host allocation failed; no state was changed */
  SG_ERR_CUDA = 3,        /* a CUDA runtime call failed (message has the CUDA error string) */
  SG_ERR_NOT_RESIDENT = 4,/* a brick the call needs is not in the device cache */
  SG_ERR_TIMEOUT = 5,     /* a bounded device-side wait gave up */
  SG_ERR_STATE = 6,       /* calls out of order (e.g. render before select, TF missing) */
  SG_ERR_IO = 7           /* a container file could not be read or written, or holds a corrupt chunk */
} sg_status;

typedef enum { SG_U8 = 1, SG_U16 = 2 } sg_dtype;

typedef struct sg_volume sg_volume; /* opaque, owned by the library */

/* Volume description ("Octree Representation": blocks of a multi-resolution
 * pyramid). Level 0 has dims; level L+1 has ceil(N_L / 2) voxels per axis and
 * is the 2x box filter of level L: floor((sum of the 8 children + 4) / 8),
 * children beyond the edge replicated. A block (brick) of level L covers
 * level-L voxels [b B, (b+1) B) per axis and is stored with a one-voxel apron
 * on every side ((B+2)^3 voxels, x fastest), apron voxels taken from the
 * neighbours or replicated at the volume edge. Node ids number the blocks
 * level by level from 0, x fastest within a level. */
typedef struct {
  int32_t dims[3];            /* level-0 voxels x, y, z (>= 1) */
  int32_t dtype;              /* SG_U8 or SG_U16 */
  int32_t channels;           /* 1..4, blended additively */
  int32_t timepoints;         /* >= 1 (3D movies) */
  int32_t brick_size;         /* B: multiple of 8, 8..256 */
  int32_t apron;              /* must be 1 */
  int32_t lod_levels;         /* 1..16 */
  int32_t skip_block;         /* edge in voxels of the empty-space skipping cells within a brick:
                                 2, 4, 8 or 16, dividing brick_size, at most 32 per brick edge;
                                 0 = the finest of 2, 4, 8 with at most 32 cells per edge */
  uint64_t device_pool_bytes; /* 0: every brick of every level resident; else the
                                 brick cache budget (bricks stream in by LRU) */
  float model[16];            /* voxel space -> world, column major; uniform scale */
} sg_volume_desc;

/* Creates a volume and allocates its page tables. With device_pool_bytes == 0
 * the brick pool holds every brick; otherwise it holds as many brick groups
 * (all channels of one brick) as fit the budget, and the coarsest level of
 * every time point must fit. Errors: INVALID_ARG (bad desc), OOM. */
sg_status sg_volume_create(const sg_volume_desc* desc, sg_volume** out);

/* Waits for the volume's work and frees everything it owns. NULL is a no-op. */
sg_status sg_volume_destroy(sg_volume* vol);

/* Ingest from a device array: dev_level0 holds the whole level-0 volume of
 * time point t, channel c (dims[0]*dims[1]*dims[2] voxels of dtype, x
 * fastest, caller-owned device memory). The library builds levels
 * 1..lod_levels-1 with the box filter, packs every brick with its apron into
 * the pool and records each brick's value range (min/max over the brick and
 * its apron) and the ranges of its skip_block^3-voxel sub-blocks. Only valid when
 * every brick is resident (device_pool_bytes == 0). Temporary device memory:
 * about 1/7 of the level-0 bytes, released before return. Errors:
 * INVALID_ARG, STATE (pooled volume), OOM, CUDA. */
sg_status sg_upload_volume_device(sg_volume* vol, int t, int c, const void* dev_level0, void* stream);

/* Ingest of ready bricks from host memory (the container's "already memory
 * aligned" chunks, "Volumetric Data Storage"): n bricks of one (t, c, level),
 * brick i at block coordinates brick_xyz[3i..3i+2], each (B+2)^3 voxels with
 * its apron, x fastest, stored back to back in host. Bricks not yet cached
 * get a pool slot (evicting the least recently used unpinned brick groups
 * when the pool is full). The brick's value ranges are recomputed on the GPU.
 * Errors: INVALID_ARG, OOM (pool full of bricks in use this frame: the
 * bricks before the one that found no slot are cached and consistent),
 * CUDA. */
sg_status sg_upload_bricks(sg_volume* vol, int t, int c, int level, int n, const int32_t* brick_xyz,
                           const void* host, void* stream);

/* Streaming ingest by node id: n bricks of (t, c), brick i the node nodes[i]
 * (the ids sg_read_selection lists as requests; levels may be mixed), copied
 * from host[i]: (B+2)^3 voxels of dtype with the apron, x fastest (pinned
 * host memory makes the copies asynchronous; all are complete on return).
 * Bricks are placed in list order, so a coarse-first list keeps the coarse
 * ones when the cache runs short: placement stops, without an error, at the
 * first brick that finds the cache full of bricks used by the current frame,
 * and *n_done receives how many bricks (a prefix of the list) are cached.
 * The page table, value ranges and transparency flags of every placed brick
 * are updated before return. Streams: the call first waits (on its stream)
 * for the last selection launch, whose slot stamps decide what may be
 * evicted; it never evicts a brick that selection used, so it may run on a
 * copy stream while that selection's render runs on another.
 * Errors: INVALID_ARG (node id out of range, NULL pointer), OOM (bookkeeping
 * memory), CUDA. */
sg_status sg_upload_brick_list(sg_volume* vol, int t, int c, int n, const int32_t* nodes, const void* const* host,
                               int32_t* n_done, void* stream);

/* sg_upload_brick_list without the wait: placement (page table, LRU state,
 * *n_done) is decided on return, the copies and the placed bricks' ranges
 * and flags are queued on stream. The caller keeps host[0..*n_done) unchanged
 * (page-locked, for the copies to run asynchronously) until the stream has
 * passed the upload. Later selections, transfer-function changes and brick
 * reads, on any stream, wait for it on the device (not while their stream
 * is captured into a graph). Errors: as sg_upload_brick_list. */
sg_status sg_upload_brick_list_async(sg_volume* vol, int t, int c, int n, const int32_t* nodes,
                                     const void* const* host, int32_t* n_done, void* stream);

/* ---- Brick container and host cache ("Volumetric Data Storage",
 * "Volumetric Data Cashing") ----------------------------------------------
 * A container is one file of LZ4-compressed chunks, one per brick with its
 * apron ((B+2)^3 voxels of the layout's dtype, x fastest) of any (t, c,
 * level). Chunks are appended (a chunk has a header and a checksum, so a
 * conversion that stopped part way resumes after its last complete chunk);
 * sg_container_finish writes the index table of chunk offsets and a footer.
 * The host cache keeps decompressed bricks in (optionally page-locked) host
 * memory, least recently used out first, in front of a volume's GPU cache.
 * Container and cache calls are host-only: no GPU is needed except for a
 * page-locked cache and sg_stream_requests. */
typedef struct sg_container sg_container;   /* opaque */
typedef struct sg_host_cache sg_host_cache; /* opaque */

typedef struct {
  sg_volume_desc desc;        /* the layout (device_pool_bytes and model as written) */
  int64_t chunks;             /* chunks present */
  int64_t nodes;              /* blocks per (t, c) */
  uint64_t raw_bytes;         /* total decompressed bytes of the chunks */
  uint64_t compressed_bytes;  /* total chunk payload bytes */
  int32_t complete;           /* 1: finished (indexed, read only); 0: appendable */
  int32_t reserved;
} sg_container_info;

/* Creates (truncates) path as an empty container for the layout desc.
 * Errors: INVALID_ARG, OOM, IO. */
sg_status sg_container_create(const char* path, const sg_volume_desc* desc, sg_container** out);

/* Opens a container. A finished one is read through its index (read only);
 * an unfinished one is scanned chunk by chunk, a torn last chunk is cut off,
 * and appending resumes after the last complete chunk. Errors: INVALID_ARG,
 * OOM, IO (missing file, bad header). */
sg_status sg_container_open(const char* path, sg_container** out);

/* Compresses and appends the brick (t, c, level, bx, by, bz) with its value
 * range [vmin, vmax] (over the brick and its apron, as the index of
 * sg_set_brick_ranges). A brick appended twice keeps its last chunk. Safe
 * to call from several threads at once (compression runs in parallel, the
 * writes are serialised). Errors: INVALID_ARG, STATE (finished container),
 * IO. */
sg_status sg_container_append(sg_container* k, int t, int c, int level, int bx, int by, int bz, const void* brick,
                              uint32_t vmin, uint32_t vmax);

/* Writes the index table and the footer; the container becomes read only.
 * Errors: INVALID_ARG, IO. */
sg_status sg_container_finish(sg_container* k);

sg_status sg_container_get_info(sg_container* k, sg_container_info* info);

/* Reads and decompresses the brick of (t, c, node id) into out ((B+2)^3
 * voxels); minmax (optional) receives its stored range. Errors: INVALID_ARG,
 * NOT_RESIDENT (no chunk for it), IO (corrupt chunk). */
sg_status sg_container_read(sg_container* k, int t, int c, int64_t node, void* out, uint32_t* minmax);

sg_status sg_container_close(sg_container* k);

/* A host cache of floor(bytes / brick bytes) decompressed bricks of
 * container k (which must outlive it); pinned != 0 page-locks it for full
 * upload bandwidth; threads decompress misses in parallel (and, once
 * sg_stream_requests_async or sg_host_cache_prefetch is first called, as
 * many background loader threads run until sg_host_cache_destroy). Errors:
 * INVALID_ARG, OOM. */
sg_status sg_host_cache_create(sg_container* k, uint64_t bytes, int pinned, int threads, sg_host_cache** out);
sg_status sg_host_cache_destroy(sg_host_cache* hc);

/* The cached brick of (t, c, node), read and decompressed on a miss (*hit
 * = 0) into an entry that stays valid until the next cache call. Errors:
 * INVALID_ARG, NOT_RESIDENT, OOM, IO. */
sg_status sg_host_cache_fetch(sg_host_cache* hc, int t, int c, int64_t node, const void** brick, int* hit);

/* Forgets the chunks sg_stream_requests found unreadable, so the next calls
 * try them again (after a transient read error, say). Errors: INVALID_ARG. */
sg_status sg_host_cache_clear_failures(sg_host_cache* hc);

typedef struct {
  int32_t requested;     /* requests of the selection */
  int32_t served;        /* bricks placed in the GPU cache by this call */
  int32_t host_hits;     /* brick-channels found in the host cache */
  int32_t disk_reads;    /* brick-channels read and decompressed from the container */
  int32_t missing;       /* requests without a chunk in the container (skipped) */
  int32_t failed;        /* requests skipped: a chunk failed to read or decompress (now or earlier) */
  uint64_t disk_bytes;   /* compressed bytes read */
  uint64_t upload_bytes; /* bytes copied to the GPU cache */
  int32_t queued;        /* sg_stream_requests_async: brick-channels handed to the loaders by this call */
  int32_t in_flight;     /* sg_stream_requests_async: brick-channels being loaded after this call */
} sg_stream_stats;

/* Serves the requests of selection slot `slot` of vol from container-backed
 * host cache hc: coarse levels first (then node id), at most max_bytes of
 * bricks (all channels); each from the host cache or read + decompressed
 * (hc's threads), then placed in the GPU cache (sg_upload_brick_list per
 * channel, on stream; complete on return). Stops early, without error, when
 * either cache holds only bricks of the current frame. A brick whose chunk
 * fails to read or decompress (any channel) is left out: it stays
 * non-resident, so the next selections render its parent in its place
 * ("Octree Representation"), and hc remembers the chunk, so later calls
 * skip it without spending budget (sg_host_cache_clear_failures forgets).
 * The other bricks are served; the call then returns SG_ERR_IO with *stats
 * filled (stats->failed counts the skipped requests). Errors: INVALID_ARG
 * (layouts differ), STATE, IO (see above), OOM, CUDA. */
sg_status sg_stream_requests(sg_volume* vol, int slot, sg_host_cache* hc, uint64_t max_bytes, sg_stream_stats* stats,
                             void* stream);

/* The same requests served without waiting for the disk ("Volumetric Data
 * Cashing" with "Octree Representation"'s coarser stand-ins): the bricks
 * whose every channel the host cache holds are placed in the GPU cache (at
 * most max_bytes, coarse levels first): the page table is updated on return,
 * the copies and the bricks' ranges and flags are queued on stream and not
 * waited for; every later selection, transfer-function change or brick read
 * waits for them on the device, and the host cache reuses none of those
 * entries before they are done (the call waits for earlier calls' copies
 * only when it must reuse an entry they may still read; it reads the
 * selection's requests on a stream of the volume's own). The others are
 * handed to hc's background loader threads (at most max_bytes of new loads
 * per call) and placed by a later call once loaded. Until then the next
 * selections render their resident ancestors, so a frame never waits on a
 * read. stats->disk_reads / disk_bytes count the loads finished since the
 * previous call, stats->queued the loads this call started, stats->in_flight
 * those still running. A chunk that fails to load is remembered and skipped
 * as in sg_stream_requests (the call that learns of it returns SG_ERR_IO
 * with *stats filled). A host cache may serve both calls; sg_stream_requests
 * and sg_host_cache_fetch first wait for every load in flight. Errors: as
 * sg_stream_requests. */
sg_status sg_stream_requests_async(sg_volume* vol, int slot, sg_host_cache* hc, uint64_t max_bytes,
                                   sg_stream_stats* stats, void* stream);

/* Queues background loads of the bricks (t, c, nodes[0..n)) that hc does not
 * hold (bricks without a chunk, or whose chunk failed before, are skipped);
 * *queued (optional) receives how many were queued. Host only. Errors:
 * INVALID_ARG, OOM (every entry is in use this call or being loaded: the
 * bricks before are queued). */
sg_status sg_host_cache_prefetch(sg_host_cache* hc, int t, int c, const int64_t* nodes, int32_t n, int32_t* queued);

/* Waits for every background load of hc and takes the results in: loaded
 * bricks become hits, failed chunks are remembered (*failed, optional,
 * receives how many failed). Host only. Errors: INVALID_ARG. */
sg_status sg_host_cache_wait(sg_host_cache* hc, int32_t* failed);

/* Value ranges of bricks known without their data, as a container's index
 * table would hold them ("Volumetric Data Storage": chunks with an index):
 * minmax[2i], minmax[2i+1] are the min and max over brick i (at block
 * coordinates brick_xyz[3i..3i+2] of (t, c, level)) and its one-voxel apron.
 * With them, selection drops transparent subtrees before their bricks are
 * ever cached instead of requesting them (an unknown range is never
 * transparent). Marks earlier selections stale. Errors: INVALID_ARG, OOM,
 * CUDA. */
sg_status sg_set_brick_ranges(sg_volume* vol, int t, int c, int level, int n, const int32_t* brick_xyz,
                              const uint32_t* minmax, void* stream);

/* Transfer function of channel c ("DVR Techniques": tau for colour, T for
 * opacity; "Visualization Enhancements": one per channel). rgba holds n >= 2
 * entries of straight colour and opacity in [0, 1]; the opacities are those of
 * one sample every ref_step level-0 voxels. A voxel value v maps to
 * x = clamp((v - lo) / (hi - lo), 0, 1), table position q = x (n - 1), with
 * linear interpolation between entries floor(q) and floor(q) + 1. A sample
 * spaced s apart uses opacity 1 - (1 - alpha)^(s / ref_step). Also derives
 * which blocks and sub-blocks are transparent under the table and marks
 * earlier selections stale. Errors: INVALID_ARG (n < 2 or > 4096, hi <= lo,
 * ref_step <= 0), OOM, CUDA. */
sg_status sg_set_transfer_function(sg_volume* vol, int c, const float* rgba, int n, float lo, float hi,
                                   float ref_step, void* stream);

/* What a channel's table reads and where its colour comes from
 * ("Visualization Enhancements"). input SG_INPUT_VALUE: the voxel value (the
 * default); SG_INPUT_GRADIENT: the gradient magnitude |grad f| in value units
 * per level-0 voxel, from central differences of the trilinear field at
 * +-1/2 voxel of the sample's level along each axis (the window of
 * sg_set_transfer_function then applies to gradient magnitudes; a block's
 * gradient lies in [0, sqrt(3) (max - min)], which decides its
 * transparency). m > 0: the colour comes from palette_rgb (m RGB entries in
 * [0, 1]) at the sample's world distance d from the eye, x = clamp((d - near)
 * / (far - near), 0, 1), linear between entries floor(x (m-1)) and the next
 * (MIP: the distance of the first sample that reaches the maximum); the
 * table keeps deciding opacity. m = 0: the table's colour. Marks earlier
 * selections stale. Errors: INVALID_ARG, CUDA. */
enum { SG_INPUT_VALUE = 0, SG_INPUT_GRADIENT = 1 };
sg_status sg_set_channel_shading(sg_volume* vol, int c, int input, const float* palette_rgb, int m, float near,
                                 float far, void* stream);

/* One head pose: the two eyes' view and projection matrices, the per-eye image
 * size, the LOD tolerance in pixels (tau, 1.0 = a voxel may cover one pixel),
 * the time point, and the selection slot that sg_select_lod fills and
 * sg_render reads (0 .. 255; independent poses in flight use different slots). */
typedef struct {
  float view[2][16];
  float proj[2][16];
  int32_t width, height;
  float pixel_error;
  int32_t t;
  int32_t slot;
  int32_t reserved;
} sg_pose;

typedef struct {
  uint32_t selected;  /* blocks rendered (including fallbacks) */
  uint32_t culled;    /* blocks outside both view pyramids */
  uint32_t empty;     /* blocks dropped because they and all descendants are transparent */
  uint32_t requested; /* non-resident children requested */
  uint32_t fallback;  /* blocks rendered one level coarser than wanted */
  uint32_t nonempty;  /* selected blocks that are not transparent themselves (their bricks get sampled) */
  uint32_t reserved[2];
} sg_select_stats;

/* LOD and residency selection for one pose ("Octree Representation", last
 * paragraph). Top-down from the roots (every block of the coarsest level):
 * a block outside one side plane of the view pyramid of both eyes (planes
 * pushed one voxel outward) is culled; a block that is transparent together
 * with all its descendants is dropped; a block of level L is accepted when
 * L == 0 or 2^L <= tau theta d, with theta = 2 / (P11 height) the pixel angle
 * at the image centre and d the distance from the block to the nearer eye
 * (0 inside). The test runs in exact integers: eyes rounded to 1/64 voxel,
 * K = floor((tau theta)^2 2^40), accept iff 4^L 64^2 2^40 <= K d^2 (128-bit).
 * Otherwise, if a needed (not culled, not dropped) child is not resident,
 * those children are requested and the block itself is rendered; else the
 * needed children are visited. The result (which block renders each level-0
 * block cell, requests, counters) is kept in pose->slot. The launch waits
 * on the device for every brick upload queued before it, on any stream (an
 * upload of sg_stream_requests_async may still be running); not while the
 * stream is captured into a graph. If stats is not NULL the call waits for
 * the stream and fills it. Errors: INVALID_ARG, STATE (no transfer function
 * or no data for t), CUDA. */
sg_status sg_select_lod(sg_volume* vol, const sg_pose* pose, sg_select_stats* stats, void* stream);

/* Selection for n poses in one launch (batched frames); no stats.
 * Selections may be captured into a CUDA graph (stats = NULL). A captured
 * selection is not tracked for other streams: after replaying the graph,
 * order reads (sg_read_selection) and uploads after the replay through the
 * caller's streams, e.g. by synchronising. */
sg_status sg_select_lod_batch(sg_volume* vol, const sg_pose* poses, int n, void* stream);

/* Allocation-free selection. The paper has no counterpart: this entry point
 * exists for callers that cannot allocate device memory while they render,
 * such as a thread under a hard frame budget or one recording a CUDA graph
 * (cudaMalloc may synchronise the device and cannot be captured). It
 * computes what sg_select_lod computes for the pose, but writes into the
 * caller's device buffers and takes its breadth-first scratch from a fixed
 * array inside the library: 2 x 65536 int32 (512 KiB) that every GPU which
 * loads the library keeps until the process exits. Volumes with more than
 * 65536 blocks on one level are rejected (SG_ERR_INVALID_ARG); sg_select_lod
 * has no such limit. Outputs (device, caller-owned): leaf[ncell] render
 * entries, cell_node[ncell] node id or -1, node_state[nodes] as in
 * sg_read_selection, req[nodes] requested node ids in no particular order,
 * counters[8] = requested, selected, culled, empty, fallback, nonempty.
 * The first call on a device looks up the fixed array's device address (no
 * allocation); make that first call before any stream capture. The address
 * is kept for the life of the process: after cudaDeviceReset on a device
 * this entry point must not be called on it again. Brick uploads issued
 * later on other streams wait for the call when it was not captured (as
 * they do for sg_select_lod); after a captured call, and for
 * transfer-function changes in every case, order them after the call
 * yourself (one stream, or events). Every call
 * shares the array and it keeps the last call's contents (each call writes
 * before it reads, nothing needs clearing): calls whose work overlaps on the
 * GPU race, so order them (one stream, or events). pose.slot is ignored and
 * LRU timestamps are not updated. The call allocates nothing and does not
 * wait for the stream. Errors: INVALID_ARG, STATE (no transfer function or
 * data), CUDA. */
sg_status sg_select_lod_noalloc(sg_volume* vol, const sg_pose* pose, uint32_t* leaf, int32_t* cell_node,
                                uint8_t* node_state, int32_t* req, uint32_t* counters, void* stream);

/* Copies a selection to host memory (waits for the stream): per level-0 block
 * cell the rendering node id or -1 (ncell = product of ceil(dims/B)); per node
 * the traversal state (0 unseen, 1 culled, 2 dropped-empty, 3 selected,
 * 4 selected as fallback, 5 refined); the requested node ids in ascending
 * order (at most req_cap, *nreq gets the full count). Any output may be NULL.
 * Errors: INVALID_ARG, STATE (slot never selected), CUDA. */
sg_status sg_read_selection(sg_volume* vol, int slot, int32_t* cell_node, int64_t ncell, uint8_t* node_state,
                            int64_t nnode, int32_t* req, int32_t req_cap, int32_t* nreq, void* stream);

/* Copies the page table of time point t to host: per node the pool slot of
 * its brick group, or -1 when it is not cached ("Volumetric Data Cashing").
 * slot_of_node holds nnode >= nodes entries. Errors: INVALID_ARG. */
sg_status sg_read_residency(sg_volume* vol, int t, int32_t* slot_of_node, int64_t nnode);

/* Copies the value ranges of every brick of time point t to host:
 * minmax[(node * channels + c) * 2 + {0, 1}] = min, max over the brick and
 * its apron (min > max: never seen), nnode >= nodes. With
 * sg_set_brick_ranges this moves a volume's index between volumes
 * (synchronous). Errors: INVALID_ARG, CUDA. */
sg_status sg_read_ranges(sg_volume* vol, int t, uint32_t* minmax, int64_t nnode);

/* Copies the stored brick of (t, c, level, bx, by, bz) to host: (B+2)^3
 * voxels of dtype, x fastest, apron included (waits for the stream). For
 * inspection and tests of the ingest path. Errors: INVALID_ARG,
 * NOT_RESIDENT (brick not in the cache), CUDA. */
sg_status sg_read_brick(sg_volume* vol, int t, int c, int level, int bx, int by, int bz, void* host_out,
                        void* stream);

/* Radial lens model of an HMD eye ("DVR for HMD"): the image is rendered in
 * the lens's warped space, one ray per warped pixel, and unwarped afterwards
 * (sg_unwarp), so no rays are spent on detail the lens would discard. A
 * warped NDC point w (pixel (i,j) of a Ww x Hw image: (2(i+0.5)/Ww - 1,
 * 1 - 2(j+0.5)/Hw)) at offset d = w - c from the lens centre c looks through
 * the undistorted NDC point u = c + d (1 + k1 r^2 + k2 r^4) scale, with
 * r^2 = (d_x aspect)^2 + d_y^2. k1, k2 >= 0; scale > 0 (0: 1 / (1 + k1 +
 * k2), which maps the warped edge midpoints of a centred lens to the
 * undistorted ones); aspect > 0 (0: the image's width / height). A warped
 * image of scale * W x scale * H pixels has the undistorted W x H image's
 * pixel density at the lens centre. */
typedef struct {
  float k1, k2, scale, aspect;
  float centre[2][2]; /* lens centre per eye, NDC (x, y) */
} sg_lens;

/* Optical models ("DVR Techniques"):
 * - EMISSION_ABSORPTION: front-to-back compositing, C += (1 - A) colour_s,
 *   A += (1 - A) alpha_s, early termination at term_alpha (below).
 * - EMISSION: the emission-only integral, no absorption and no early
 *   termination: C += sum_c alpha_c colour_c (step 2^L / ref_step), with the
 *   table's alpha for one reference step; the output alpha is 0 (composite
 *   additively over the scene behind).
 * - MIP: maximum intensity projection: per channel the largest trilinear
 *   value along the ray, classified with the table as given, channels
 *   blended as above, output premultiplied. Empty-space skipping stays exact
 *   only when every channel's transparent entries are the lowest ones (a
 *   table whose alpha is 0 up to some entry and positive after it); other
 *   tables render MIP without skipping. Blocks that selection dropped as
 *   transparent are not sampled in any mode. */
enum { SG_MODE_EMISSION_ABSORPTION = 0, SG_MODE_EMISSION = 1, SG_MODE_MIP = 2 };

typedef struct {
  float step;             /* level-0 sample spacing in voxels (> 0); level L samples every 2^L-th point */
  float term_alpha;       /* early ray termination threshold, e.g. 0.99 (<= 0: 0.99); EMISSION_ABSORPTION only */
  int32_t mode;           /* SG_MODE_* */
  int32_t empty_skip;     /* 1: skip transparent blocks and sub-blocks (output unchanged) */
  uint32_t* sample_count[2]; /* optional device buffers (W*H per eye): samples composited per pixel */
  unsigned long long* sample_total; /* optional device counter: incremented by the samples composited */
  const float* depth[2];  /* optional device buffers (W*H per eye, row 0 = top, 4-byte aligned): the
                             distance in world units from the eye along each pixel's ray to an opaque
                             surface (a scene's depth buffer turned into distances, "Volumetric and
                             Mesh Data Compositing"); the ray ends there, taking no sample at or beyond it, and
                             the caller composites the premultiplied image over the scene; +inf = no
                             surface. sg_render / sg_render_host only. */
  const sg_lens* lens;    /* optional: rays through the lens-warped image (the pose's width/height are the
                             warped image's); sg_render / sg_render_host only */
  uint8_t* touched;       /* optional device buffer, one byte per cache slot: set to 1 for every brick a ray
                             took a sample from (the slot of node n at time point t is t * nodes + n for a
                             volume without a device_pool_bytes budget). A diagnostic of the bricks the frame
                             reads: sg_render and sg_render_host, emission-absorption without gradient or palette tables, the
                             default launch shape. */
} sg_render_params;

/* Ray casts both eyes of a selected pose ("DVR Techniques"). For pixel (i,j)
 * the ray leaves the eye towards the unprojection of NDC
 * (2(i+0.5)/W - 1, 1 - 2(j+0.5)/H); t is in level-0 voxels; the ray is
 * clipped to [0,N]^3: t0 = max(t_near, 0), t1 = t_far. Samples lie on the
 * lattice t0 + k step (k >= 0), every 2^L-th point inside a block of level L.
 * Each sample: trilinear value from the block's brick (exact trilinear
 * weights in FP32), table lookup per channel, channels blended additively
 * (alpha_s = min(1, sum alpha_c), colour scaled by alpha_s / max(alpha_s,
 * sum alpha_c)), then C += (1 - A) colour_s, A += (1 - A) alpha_s; the ray
 * stops after the sample that makes A >= term_alpha. out_rgba[e]: caller-owned
 * device buffers of W*H*4 floats, 16-byte aligned. Errors: INVALID_ARG,
 * STATE (slot not selected for this pose's t, or selection stale), CUDA. */
sg_status sg_render(sg_volume* vol, const sg_pose* pose, const sg_render_params* params, float* out_rgba[2],
                    void* stream);

/* As sg_render, but the images land in caller-owned HOST buffers (W*H*4
 * floats per eye; pinned memory gives full copy bandwidth). Renders into
 * library-owned device staging, copies back and waits for the stream. */
sg_status sg_render_host(sg_volume* vol, const sg_pose* pose, const sg_render_params* params,
                         float* host_rgba[2], void* stream);

/* Pipelined sg_render_host for a stream of frames: renders on `stream` into
 * one of three library-owned device staging pairs (taken in turn), then
 * copies both images to the caller's HOST buffers on a library-owned copy
 * stream, and returns without waiting. So the copy of one frame overlaps
 * the renders of the next two: a caller that waits for frame i - 2 after
 * queueing frame i keeps the GPU rendering while frame i - 1 is copied,
 * even when a render is shorter than a copy. A render waits on the GPU (not
 * the host) until the pair it reuses, three calls back, has been copied
 * out. The images of a call are complete once sg_render_host_wait has
 * covered it: all = 0 waits for the oldest of the (at most three) frames in
 * flight, all != 0 for all of them. Host buffers must stay valid and unread
 * until then; pinned memory is needed for the copies to run asynchronously.
 * Errors: as sg_render_host. */
sg_status sg_render_host_async(sg_volume* vol, const sg_pose* pose, const sg_render_params* params,
                               float* host_rgba[2], void* stream);
sg_status sg_render_host_wait(sg_volume* vol, int all);

/* Renders n selected poses (2n images of possibly different sizes) in one
 * persistent launch over a queue of ray tiles ("3D Movies": time points;
 * several viewers). outs[2i + e] is pose i's eye e (device, W*H*4 floats). */
sg_status sg_render_batch(sg_volume* vol, const sg_pose* poses, int n, const sg_render_params* params,
                          float** outs, void* stream);

/* Unwarps both eyes of a warped render ("DVR for HMD"): output pixel (i,j)
 * of the W x H undistorted image takes the preimage w of its NDC centre under
 * the lens map (solved by Newton iterations on the radial polynomial) and a
 * bilinear tap of the warped image's pixel centres, edge pixels replicated;
 * preimages outside the warped image give (0,0,0,0). warped[e] / out[e]:
 * device RGBA float buffers (Ww*Hw*4, W*H*4 floats, 16-byte aligned). Errors:
 * INVALID_ARG, CUDA. */
sg_status sg_unwarp(const sg_lens* lens, const float* warped[2], int Ww, int Hw, float* out[2], int W, int H,
                    void* stream);

/* How sg_render / sg_render_batch map rays onto the GPU. tile_w x tile_h
 * pixel tiles (warps cover 8 x 4 pixels), rays_per_thread rays per thread;
 * persistent != 0: a grid sized to the GPU pulls tiles from a queue shared by
 * all images of the launch (balances uneven image sizes), else one CTA per
 * tile. Supported shapes (w, h, rays): (16,8,1) (8,16,1) (32,4,1) (8,8,1)
 * (16,16,2) (32,8,2); all zero = the default one-CTA-per-16x8-tile kernel.
 * Launches of one volume must not overlap on the GPU when persistent. */
typedef struct {
  int32_t persistent;
  int32_t tile_w, tile_h;
  int32_t rays_per_thread;
  int32_t reserved[4];
} sg_render_config;

/* Sets / reads the volume's render configuration. Errors: INVALID_ARG. */
sg_status sg_set_render_config(sg_volume* vol, const sg_render_config* cfg);
sg_status sg_get_render_config(sg_volume* vol, sg_render_config* cfg);

/* The autotuner's picks, kept across runs in a text file of lines
 * "<key> TAB <persistent> <tile_w> <tile_h> <rays_per_thread>" (the key names
 * the GPU and workload; a later line for a key replaces an earlier one).
 * store appends one; lookup sets *found and, when found, *cfg (a missing
 * file is an empty cache). Errors: INVALID_ARG (NULL, key with a tab or
 * newline, unsupported configuration), IO. */
sg_status sg_render_config_store(const char* path, const char* key, const sg_render_config* cfg);
sg_status sg_render_config_lookup(const char* path, const char* key, sg_render_config* cfg, int* found);

/* Autotuner: renders the n selected poses with every supported configuration
 * (one warm-up launch, then reps timed launches each, CUDA events on the
 * stream), keeps the fastest as the volume's configuration and returns it
 * with its mean launch time. Outputs are overwritten. Waits for the stream.
 * Errors: as sg_render_batch, CUDA. */
sg_status sg_autotune_render(sg_volume* vol, const sg_pose* poses, int n, const sg_render_params* params,
                             float** outs, int reps, sg_render_config* best, float* best_ms, void* stream);

/* ---------------------------------------------------------------------------
 * Learned reconstruction (not in the paper): a residual U-Net that turns a
 * half-resolution render (h x w, rendered at twice the step) into the
 * full-resolution image (2h x 2w): out = bilinear_2x(in) +
 * pixel_shuffle_2x(head(unet(in))). Three levels of 3x3 convolutions with
 * 32 / 64 / 128 channels, ReLU, 2x2 average pooling, nearest upsampling and
 * skip concatenation; BF16 weights and activations, FP32 accumulation on the
 * tensor cores. Parameters (FP32 master copy), in order, per layer
 * c1a c1b c2a c2b c3a c3b d2a d2b d1a d1b head: W[Cout][9][Cin] (tap =
 * 3 (dy+1) + (dx+1)) then b[Cout], with (Cin, Cout) = (16,32) (32,32) (32,64)
 * (64,64) (64,128) (128,128) (192,64) (64,64) (96,32) (32,32) (32,16); input
 * channels 4..15 of c1a are zero padding. The head starts at zero, so an
 * untrained network is exactly the bilinear upsampling. */
typedef struct sg_unet sg_unet;

/* Allocates weights, optimizer state and activations for batches of up to
 * max_batch (<= 64) images of up to max_h x max_w half-resolution pixels
 * (multiples of 4); He-normal weights from seed. Errors: INVALID_ARG, OOM. */
sg_status sg_unet_create(int max_batch, int max_h, int max_w, uint64_t seed, sg_unet** out);
sg_status sg_unet_destroy(sg_unet* net);
sg_status sg_unet_param_count(sg_unet* net, int64_t* n);
/* Copies the FP32 parameters (which = 0) or their last gradients (which = 1)
 * to host (synchronous). */
sg_status sg_unet_get_params(sg_unet* net, float* host, int64_t n, int which);
/* Replaces the parameters from host (synchronous). */
sg_status sg_unet_set_params(sg_unet* net, const float* host, int64_t n);

/* Inference on n images: in[i] and out[i] are device pointers (host array of
 * n pointers) to RGBA FP32 rows, in_pitch / out_pitch floats apart (so crops
 * of larger images work in place); in is h x w, out is 2h x 2w. Keeps the
 * activations for sg_unet_backward. Errors: INVALID_ARG, CUDA. */
sg_status sg_unet_forward(sg_unet* net, const float* const* in, int64_t in_pitch, int n, int h, int w,
                          float* const* out, int64_t out_pitch, void* stream);

/* Gradients of the MSE between the last forward's outputs (out, as passed to
 * it) and target (n images, 2h x 2w RGBA rows target_pitch floats apart),
 * averaged over every output value; loss (device float, may be NULL) gets the
 * MSE. Overwrites the previous gradients. Errors: INVALID_ARG, CUDA. */
sg_status sg_unet_backward(sg_unet* net, const float* const* target, int64_t target_pitch, const float* const* out,
                           int64_t out_pitch, float* loss, void* stream);

/* Selects the tensor-core path of the convolutions (all: BF16 products, FP32
 * sums): 2 = tcgen05 with TMEM accumulators, each CTA computing four output
 * rows from input row segments loaded once per 32 channels (halo reuse); 3 = the same with the input row segments staged by TMA tensor
 * copies (identical results); 4 (default) = persistent warp-specialised halo reuse:
 * one CTA per SM walking tiles, a TMA producer, one MMA-issuing thread and
 * eight epilogue warps, a ring of 32-channel stages (16 for 16-channel
 * inputs) copied as swizzled 64-byte pixel rows, and two TMEM accumulators,
 * so loads, MMAs and stores of successive tiles overlap;
 * 1 = tcgen05 implicit GEMM gathering every tap; 0 = mma.sync. */
sg_status sg_unet_set_tensor_path(sg_unet* net, int tcgen05);

/* Reports (and clears) a timed-out bounded wait in a tcgen05 convolution since
 * the last check: SG_ERR_TIMEOUT means the affected outputs are invalid.
 * Synchronous. */
sg_status sg_unet_check(sg_unet* net);

/* Failure-detection self-test of the bounded waits (the paper has no
 * counterpart). Launches one small kernel on stream that waits, with the
 * tensor-core kernels' own bounded poll limited to `polls` polls (1 to
 * 2^24), on a shared-memory barrier that nothing ever arrives at; no copy,
 * MMA or tensor-memory allocation is in flight. The wait gives up and the
 * kernel raises the network's error word exactly as a stalled convolution
 * would, so the next sg_unet_check returns SG_ERR_TIMEOUT (and clears it).
 * Errors: INVALID_ARG, CUDA. */
sg_status sg_unet_wait_selftest(sg_unet* net, uint32_t polls, void* stream);

/* One Adam step on the FP32 master parameters with the last gradients
 * (bias-corrected moments), then refreshes the BF16 copies. */
sg_status sg_unet_adam_step(sg_unet* net, float lr, float beta1, float beta2, float eps, void* stream);

/* PSNR of a against b over count floats in [0, 1]: 10 log10(1 / MSE), into
 * the device float out_db (1000 when identical). */
sg_status sg_psnr(const float* a, const float* b, int64_t count, float* out_db, void* stream);

/* Saves the network's training state to a file: the FP32 parameters, both
 * Adam moments and the step count (a checkpoint to resume training from, or
 * to serve a trained network without retraining). Synchronous. Errors:
 * INVALID_ARG, IO, CUDA. */
sg_status sg_unet_save(sg_unet* net, const char* path);
/* Restores a checkpoint written by sg_unet_save for this network (same
 * parameter count) and refreshes the BF16 weights. Synchronous. Errors:
 * INVALID_ARG, IO (missing, truncated or another network's file), CUDA. */
sg_status sg_unet_load(sg_unet* net, const char* path);

/* One learned frame (the method's reconstruction path, not in the paper). */
typedef struct {
  float step;               /* full-rate sample spacing, level-0 voxels; the reduced render uses 2 step */
  float term_alpha;         /* early termination (0 = 0.99) */
  float pixel_error_half;   /* tau of the reduced render (0 = pose->pixel_error / 2: the full image's detail) */
  float threshold_db;       /* judging: fall back to the full-rate render below this stereo PSNR */
  int32_t judge;            /* 1: also render the full-rate frame, compute the PSNR, fall back */
  int32_t half_slot;        /* selection slot of the reduced pose (0..255, not pose->slot) */
  int32_t reserved[2];
  sg_render_config half_config, full_config; /* launch shapes (all zero: the volume's own) */
} sg_learned_params;

/* A learned stereo frame, all on the device, asynchronous on stream (no
 * host synchronisation): selects and renders the pose at half resolution
 * (width/2 x height/2 per eye, multiples of 4) and twice the step, then
 * reconstructs both eyes with the network into out_rgba[2] (caller-owned
 * device FP32, width x height x 4 each). With prm->judge it also selects
 * and renders the plain full-rate frame (the yardstick), writes psnr_db[0..2]
 * (device: eye 0, eye 1, and the stereo PSNR 10 log10(1 / mean of the two
 * eyes' MSE)) and *fell_back (device int32); a frame below
 * prm->threshold_db gets the full-rate render in out_rgba instead. The
 * reduced and full-rate images live in buffers of the network, grown on
 * first use. The pose's own selection slot takes the full-rate selection.
 * Errors: INVALID_ARG, STATE, OOM, CUDA. */
sg_status sg_render_learned(sg_volume* vol, sg_unet* net, const sg_pose* pose, const sg_learned_params* prm,
                            float* out_rgba[2], float* psnr_db, int32_t* fell_back, void* stream);

/* Thread-local message of the last failure on this thread ("" if none). */
const char* sg_last_error(void);

/* Library version string. */
const char* sg_version(void);

#ifdef __cplusplus
}
#endif
#endif /* SG_H */
