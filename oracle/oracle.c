/* FP64 CPU oracle for the syGlass direct-volume-rendering hot path.
 *
 * TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the bench's
 * CPU-baseline leg may load this library. It shares no code with the CUDA
 * path (no headers, helpers or tables), and nothing in it is blocked, fused
 * or reordered beyond what the definitions below state.
 *
 * What it computes, following the paper's "Volume Rendering" section:
 *  - the multi-resolution block pyramid ("Octree Representation"): level L+1
 *    is the 2x box filter of level L, floor((sum of 8 + 4) / 8), with the
 *    edge replicated for odd sizes;
 *  - per-block value ranges (block plus its one-voxel apron) and the
 *    transfer-function emptiness test derived from them;
 *  - the octree traversal that picks blocks whose resolution matches the
 *    pixel resolution ("Octree Representation", last paragraph): top-down
 *    from the roots, frustum culling, accept a block when one of its voxels
 *    subtends at most tau pixels at the block's closest point to the nearer
 *    eye, render one level coarser and request the children when any needed
 *    child is not resident;
 *  - per-pixel ray casting under the emission-absorption model ("DVR
 *    Techniques", second integral), discretised front to back with
 *    associated colours, early termination, trilinear sampling of the global
 *    level-L voxel arrays (never bricks or aprons) and a 1D transfer function.
 *
 * Readings of points the paper leaves open (opacity correction, the sample
 * lattice, voxel centres, the integer form of the LOD test, the culling
 * planes, the channel blend) are stated at each function.
 *
 * Parity pins: every function here is checked by the CPU tests against
 * closed forms (Beer-Lambert, linear fields, hand-computed 4^3 cases),
 * brute force (pyramid, selection) and invariants (coverage, monotonicity,
 * stereo mirror, opacity-correction step invariance).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <omp.h>

#define OR_MAX_LEVELS 16
#define OR_MAX_CH 4

typedef struct {
  int32_t dtype;  /* 1 = uint8, 2 = uint16 */
  int32_t levels; /* pyramid levels, 0 = finest */
  int32_t brick;  /* block edge B in voxels of the block's own level */
  int32_t nch;    /* channels, blended additively */
  int64_t dims[OR_MAX_LEVELS][3];
  const void* data[OR_MAX_LEVELS][OR_MAX_CH]; /* global level-L arrays, x fastest */
  double model[16]; /* voxel space [0,N]^3 -> world, column major */
} or_volume;

typedef struct {
  int32_t n;        /* table entries */
  float lo, hi;     /* intensity window mapped onto [0, n-1] */
  float ref_step;   /* step, in level-0 voxels, at which the table's alphas hold */
  const float* rgba; /* 4n, straight (not premultiplied) colour + opacity */
  /* "Visualization Enhancements": the table reads the voxel value (input 0)
   * or the gradient magnitude (input 1); with m > 0 the colour comes from a
   * palette of m RGB entries indexed by the sample's world distance from the
   * eye over [pnear, pfar] instead of the table's colour */
  int32_t input;
  int32_t m;
  float pnear, pfar;
  const float* palette; /* 3m */
} or_tf;

enum { OR_INPUT_VALUE = 0, OR_INPUT_GRADIENT = 1 };

/* ------------------------------------------------------------------------ */
/* small linear algebra (column-major 4x4, FP64)                             */

static void mat_mul(const double* a, const double* b, double* o) {
  double t[16];
  for (int c = 0; c < 4; ++c)
    for (int r = 0; r < 4; ++r) {
      double s = 0.0;
      for (int k = 0; k < 4; ++k) s += a[k * 4 + r] * b[c * 4 + k];
      t[c * 4 + r] = s;
    }
  memcpy(o, t, sizeof t);
}

/* Gauss-Jordan with partial pivoting; returns 0 if singular */
static int mat_inv(const double* m, double* inv) {
  double a[4][8];
  for (int r = 0; r < 4; ++r)
    for (int c = 0; c < 4; ++c) {
      a[r][c] = m[c * 4 + r];
      a[r][c + 4] = (r == c) ? 1.0 : 0.0;
    }
  for (int c = 0; c < 4; ++c) {
    int p = c;
    for (int r = c + 1; r < 4; ++r)
      if (fabs(a[r][c]) > fabs(a[p][c])) p = r;
    if (fabs(a[p][c]) < 1e-300) return 0;
    if (p != c)
      for (int k = 0; k < 8; ++k) { double t = a[p][k]; a[p][k] = a[c][k]; a[c][k] = t; }
    double d = a[c][c];
    for (int k = 0; k < 8; ++k) a[c][k] /= d;
    for (int r = 0; r < 4; ++r)
      if (r != c) {
        double f = a[r][c];
        if (f != 0.0)
          for (int k = 0; k < 8; ++k) a[r][k] -= f * a[c][k];
      }
  }
  for (int r = 0; r < 4; ++r)
    for (int c = 0; c < 4; ++c) inv[c * 4 + r] = a[r][c + 4];
  return 1;
}

static void mat_apply(const double* m, const double* v, double* o) {
  for (int r = 0; r < 4; ++r)
    o[r] = m[r] * v[0] + m[4 + r] * v[1] + m[8 + r] * v[2] + m[12 + r] * v[3];
}

/* ------------------------------------------------------------------------ */
/* pyramid                                                                   */

static inline uint32_t vox_get(const void* p, int dtype, int64_t idx) {
  return dtype == 1 ? ((const uint8_t*)p)[idx] : ((const uint16_t*)p)[idx];
}

/* One 2x box-filter step: dst[j] = floor((sum over the 2x2x2 children of src,
 * child indices clamped into src, + 4) / 8). dst dims are ceil(src/2). */
void or_pyramid_level(const void* src, int dtype, const int64_t* sdims, void* dst) {
  int64_t nx = sdims[0], ny = sdims[1], nz = sdims[2];
  int64_t mx = (nx + 1) / 2, my = (ny + 1) / 2, mz = (nz + 1) / 2;
#pragma omp parallel for schedule(static)
  for (int64_t z = 0; z < mz; ++z)
    for (int64_t y = 0; y < my; ++y)
      for (int64_t x = 0; x < mx; ++x) {
        uint64_t s = 0;
        for (int dz = 0; dz < 2; ++dz)
          for (int dy = 0; dy < 2; ++dy)
            for (int dx = 0; dx < 2; ++dx) {
              int64_t X = 2 * x + dx, Y = 2 * y + dy, Z = 2 * z + dz;
              if (X > nx - 1) X = nx - 1;
              if (Y > ny - 1) Y = ny - 1;
              if (Z > nz - 1) Z = nz - 1;
              s += vox_get(src, dtype, (Z * ny + Y) * nx + X);
            }
        uint32_t v = (uint32_t)((s + 4) / 8);
        int64_t o = (z * my + y) * mx + x;
        if (dtype == 1) ((uint8_t*)dst)[o] = (uint8_t)v;
        else ((uint16_t*)dst)[o] = (uint16_t)v;
      }
}

/* ------------------------------------------------------------------------ */
/* blocks (octree nodes)                                                     */

static void level_blocks(const or_volume* v, int L, int64_t nb[3]) {
  for (int a = 0; a < 3; ++a) nb[a] = (v->dims[L][a] + v->brick - 1) / v->brick;
}

/* Node ids: levels in order 0..levels-1, within a level x fastest. */
int64_t or_node_count(const or_volume* v, int64_t* level_offsets /* levels+1, may be NULL */) {
  int64_t off = 0;
  for (int L = 0; L < v->levels; ++L) {
    if (level_offsets) level_offsets[L] = off;
    int64_t nb[3];
    level_blocks(v, L, nb);
    off += nb[0] * nb[1] * nb[2];
  }
  if (level_offsets) level_offsets[v->levels] = off;
  return off;
}

/* Value range of every block of every level and channel: min and max over
 * the block's voxels plus a one-voxel apron on every side, with indices
 * clamped into the level (the voxels a trilinear sample anywhere inside the
 * block can touch). out: [node][channel][2]. */
void or_block_ranges(const or_volume* v, uint32_t* out) {
  int64_t off[OR_MAX_LEVELS + 1];
  or_node_count(v, off);
  const int64_t B = v->brick;
  for (int L = 0; L < v->levels; ++L) {
    int64_t nb[3];
    level_blocks(v, L, nb);
    const int64_t* D = v->dims[L];
    int64_t nblk = nb[0] * nb[1] * nb[2];
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t b = 0; b < nblk; ++b) {
      int64_t bx = b % nb[0], by = (b / nb[0]) % nb[1], bz = b / (nb[0] * nb[1]);
      int64_t lo[3] = {bx * B - 1, by * B - 1, bz * B - 1};
      int64_t hi[3] = {bx * B + B, by * B + B, bz * B + B}; /* inclusive */
      for (int a = 0; a < 3; ++a) {
        if (lo[a] < 0) lo[a] = 0;
        if (hi[a] > D[a] - 1) hi[a] = D[a] - 1;
      }
      for (int c = 0; c < v->nch; ++c) {
        uint32_t mn = 0xffffffffu, mx = 0;
        for (int64_t z = lo[2]; z <= hi[2]; ++z)
          for (int64_t y = lo[1]; y <= hi[1]; ++y)
            for (int64_t x = lo[0]; x <= hi[0]; ++x) {
              uint32_t q = vox_get(v->data[L][c], v->dtype, (z * D[1] + y) * D[0] + x);
              if (q < mn) mn = q;
              if (q > mx) mx = q;
            }
        out[((off[L] + b) * v->nch + c) * 2 + 0] = mn;
        out[((off[L] + b) * v->nch + c) * 2 + 1] = mx;
      }
    }
  }
}

/* Transfer-function emptiness of a value range [vmin, vmax] for one channel.
 * Decided in FP32, in this exact sequence, because it turns floating point
 * into a table index: x = (v - lo) / (hi - lo) clamped to [0,1], q = x (n-1);
 * the range is empty iff every entry from floor(q(vmin)) - 1 to
 * floor(q(vmax)) + 2 (clamped to the table) has alpha exactly 0. The one-entry
 * margins make the test conservative against a one-ulp difference in q. */
static int tf_range_empty(const or_tf* tf, uint32_t vmin, uint32_t vmax) {
  /* an unknown range (vmin > vmax: a block whose data was never seen) is
   * never transparent */
  if (vmin > vmax) return 0;
  /* the table's input over the block: the value range, or for gradient
   * input [0, sqrt(3) (vmax - vmin)]: each central difference of the
   * trilinear field spans at most vmax - vmin (its taps lie in the block and
   * its apron), and a level-L gradient is divided by 2^L >= 1 */
  volatile float in0 = (float)vmin, in1 = (float)vmax;
  if (tf->input == OR_INPUT_GRADIENT) {
    in0 = 0.0f;
    in1 = 1.7320508f * (float)(vmax - vmin);
  }
  volatile float width = tf->hi - tf->lo;
  volatile float x0 = (in0 - tf->lo) / width;
  volatile float x1 = (in1 - tf->lo) / width;
  float a = x0 < 0.0f ? 0.0f : (x0 > 1.0f ? 1.0f : x0);
  float b = x1 < 0.0f ? 0.0f : (x1 > 1.0f ? 1.0f : x1);
  volatile float q0 = a * (float)(tf->n - 1);
  volatile float q1 = b * (float)(tf->n - 1);
  int ilo = (int)floorf(q0) - 1, ihi = (int)floorf(q1) + 2;
  if (ilo < 0) ilo = 0;
  if (ihi > tf->n - 1) ihi = tf->n - 1;
  for (int i = ilo; i <= ihi; ++i)
    if (tf->rgba[4 * i + 3] != 0.0f) return 0;
  return 1;
}

/* ------------------------------------------------------------------------ */
/* LOD + residency selection                                                 */

typedef struct {
  const or_volume* v;
  const or_tf* tf;
  const uint32_t* ranges; /* [node][ch][2] */
  const uint8_t* resident;
  int64_t off[OR_MAX_LEVELS + 1];
  int64_t nb[OR_MAX_LEVELS][3];
  int64_t eye[2][3];       /* 1/64 level-0 voxel */
  int64_t plane[2][4][4];  /* A,B,C (x 2^16) and D (x 2^16 x 64), pushed out 1 voxel */
  uint64_t K;              /* floor(tau^2 theta^2 2^40) */
  uint8_t* own_empty;
  uint8_t* sub_empty;
  uint8_t* state;
  int32_t* leaf;
  int32_t* req;
  int req_cap, nreq;
  uint8_t* used;
} sel_t;

enum { ST_UNSEEN = 0, ST_CULLED = 1, ST_EMPTY = 2, ST_SELECTED = 3, ST_FALLBACK = 4, ST_REFINED = 5 };

static void node_box(const sel_t* s, int L, const int64_t* b, int64_t* lo, int64_t* hi) {
  int64_t span = (int64_t)s->v->brick << L;
  for (int a = 0; a < 3; ++a) {
    int64_t l = b[a] * span, h = (b[a] + 1) * span;
    if (h > s->v->dims[0][a]) h = s->v->dims[0][a];
    lo[a] = l * 64;
    hi[a] = h * 64;
  }
}

/* Culled iff the block lies entirely outside one of the four side planes of
 * the view pyramid of each eye (the near and far planes are not used: rays
 * start at the eye and run to the volume's exit). */
static int node_culled(const sel_t* s, int L, const int64_t* b) {
  int64_t lo[3], hi[3];
  node_box(s, L, b, lo, hi);
  for (int e = 0; e < 2; ++e) {
    int outside = 0;
    for (int p = 0; p < 4 && !outside; ++p) {
      const int64_t* P = s->plane[e][p];
      int64_t val = P[3];
      for (int a = 0; a < 3; ++a) val += P[a] * (P[a] >= 0 ? hi[a] : lo[a]);
      if (val < 0) outside = 1;
    }
    if (!outside) return 0;
  }
  return 1;
}

/* Accept level L iff L == 0 or a level-L voxel (2^L level-0 voxels wide)
 * subtends at most tau pixels at distance d, d the distance from the block's
 * box to the nearer eye: 2^L <= tau theta d. In integers, with d in 1/64
 * voxel: 4^L 64^2 2^40 <= K d^2, evaluated exactly in 128 bits. */
static int node_accept(const sel_t* s, int L, const int64_t* b) {
  if (L == 0) return 1;
  int64_t lo[3], hi[3];
  node_box(s, L, b, lo, hi);
  unsigned __int128 best = 0;
  for (int e = 0; e < 2; ++e) {
    unsigned __int128 d2 = 0;
    for (int a = 0; a < 3; ++a) {
      int64_t q = s->eye[e][a], dd = 0;
      if (q < lo[a]) dd = lo[a] - q;
      else if (q > hi[a]) dd = q - hi[a];
      d2 += (unsigned __int128)((uint64_t)dd) * (uint64_t)dd;
    }
    if (e == 0 || d2 < best) best = d2;
  }
  unsigned __int128 lhs = (unsigned __int128)1 << (52 + 2 * L);
  return lhs <= (unsigned __int128)s->K * best;
}

static int64_t node_id(const sel_t* s, int L, const int64_t* b) {
  return s->off[L] + (b[2] * s->nb[L][1] + b[1]) * s->nb[L][0] + b[0];
}

static void fill_leaf(sel_t* s, int L, const int64_t* b, int32_t id) {
  int64_t n = (int64_t)1 << L;
  for (int64_t z = b[2] * n; z < (b[2] + 1) * n && z < s->nb[0][2]; ++z)
    for (int64_t y = b[1] * n; y < (b[1] + 1) * n && y < s->nb[0][1]; ++y)
      for (int64_t x = b[0] * n; x < (b[0] + 1) * n && x < s->nb[0][0]; ++x)
        s->leaf[(z * s->nb[0][1] + y) * s->nb[0][0] + x] = id;
}

static void visit(sel_t* s, int L, const int64_t* b) {
  int64_t id = node_id(s, L, b);
  if (node_culled(s, L, b)) { s->state[id] = ST_CULLED; return; }
  if (s->sub_empty[id]) { s->state[id] = ST_EMPTY; return; }
  if (node_accept(s, L, b)) { s->state[id] = ST_SELECTED; fill_leaf(s, L, b, (int32_t)id); return; }
  int64_t need[8][3];
  int nneed = 0, nmiss = 0;
  for (int c = 0; c < 8; ++c) {
    int64_t cb[3] = {2 * b[0] + (c & 1), 2 * b[1] + ((c >> 1) & 1), 2 * b[2] + ((c >> 2) & 1)};
    if (cb[0] >= s->nb[L - 1][0] || cb[1] >= s->nb[L - 1][1] || cb[2] >= s->nb[L - 1][2]) continue;
    int64_t cid = node_id(s, L - 1, cb);
    if (node_culled(s, L - 1, cb)) { s->state[cid] = ST_CULLED; continue; }
    if (s->sub_empty[cid]) { s->state[cid] = ST_EMPTY; continue; }
    memcpy(need[nneed++], cb, sizeof cb);
    if (s->resident && !s->resident[cid]) ++nmiss;
  }
  if (nmiss > 0) {
    for (int i = 0; i < nneed; ++i) {
      int64_t cid = node_id(s, L - 1, need[i]);
      if (!s->resident[cid] && s->nreq < s->req_cap) s->req[s->nreq++] = (int32_t)cid;
      if (s->resident[cid] && s->used) s->used[cid] = 1;
    }
    s->state[id] = ST_FALLBACK;
    fill_leaf(s, L, b, (int32_t)id);
    return;
  }
  s->state[id] = ST_REFINED;
  for (int i = 0; i < nneed; ++i) visit(s, L - 1, need[i]);
}

static int cmp_i32(const void* a, const void* b) {
  int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
  return (x > y) - (x < y);
}

/* Quantised selection inputs for one eye, from FP64 copies of the FP32
 * matrices: the eye in voxel space rounded to 1/64 voxel, and the four side
 * planes of clip = P V M, normalised to unit normals in voxel space,
 * A,B,C = round(n 2^16), D = round(d 2^16 64) + 2^16 64 (one voxel outward). */
static void eye_inputs(const double* model, const double* view, const double* proj, int64_t* eye,
                       int64_t planes[4][4]) {
  double vm[16], vminv[16], clip[16];
  mat_mul(view, model, vm);
  mat_inv(vm, vminv);
  double o[4] = {0, 0, 0, 1}, e[4];
  mat_apply(vminv, o, e);
  for (int a = 0; a < 3; ++a) {
    double q = e[a] / e[3] * 64.0;
    if (q > 68719476736.0) q = 68719476736.0;
    if (q < -68719476736.0) q = -68719476736.0;
    eye[a] = llround(q);
  }
  mat_mul(proj, vm, clip);
  for (int p = 0; p < 4; ++p) {
    int row = p >> 1;
    double sg = (p & 1) ? -1.0 : 1.0;
    double pl[4];
    for (int k = 0; k < 4; ++k) pl[k] = clip[k * 4 + 3] + sg * clip[k * 4 + row];
    double n = sqrt(pl[0] * pl[0] + pl[1] * pl[1] + pl[2] * pl[2]);
    if (n < 1e-300) { planes[p][0] = planes[p][1] = planes[p][2] = 0; planes[p][3] = 1; continue; }
    for (int k = 0; k < 3; ++k) planes[p][k] = llround(pl[k] / n * 65536.0);
    double d = pl[3] / n;
    if (d > 1048576.0) d = 1048576.0;
    if (d < -1048576.0) d = -1048576.0;
    planes[p][3] = llround(d * 65536.0 * 64.0) + 65536LL * 64LL;
  }
}

/* view/proj: [2][16] column major (FP64 copies of FP32 inputs).
 * leaf: one int32 per level-0 block cell, -1 where nothing is rendered.
 * state: one byte per node (see ST_*). req: requested node ids, ascending.
 * used (optional, one byte per node): the blocks this traversal used, whose
 * cache time stamps it renews ("Volumetric Data Cashing"): every block
 * rendered, rendered in place of its children, or refined, and the resident
 * children a fallback block needs (evicting those to make room for the
 * missing ones would keep the block from ever refining).
 * Returns the number of selected nodes. */
int or_select(const or_volume* v, const or_tf* tfs, const uint32_t* ranges, const double* view,
              const double* proj, int height, double tau, const uint8_t* resident, int32_t* leaf,
              uint8_t* state, int32_t* req, int req_cap, int* nreq, uint8_t* used) {
  sel_t s;
  memset(&s, 0, sizeof s);
  s.v = v; s.tf = tfs; s.ranges = ranges; s.resident = resident;
  int64_t nn = or_node_count(v, s.off);
  for (int L = 0; L < v->levels; ++L) level_blocks(v, L, s.nb[L]);
  for (int e = 0; e < 2; ++e) eye_inputs(v->model, view + 16 * e, proj + 16 * e, s.eye[e], s.plane[e]);
  /* pixel angle at the image centre: theta = 2 tan(fovy/2) / H = 2 / (P11 H) */
  double theta = 2.0 / (proj[5] * (double)height);
  double tt = tau * theta;
  double kf = floor(tt * tt * 1099511627776.0);
  if (!(kf >= 0.0)) kf = 0.0;
  if (kf > 1099511627776.0) kf = 1099511627776.0;
  s.K = (uint64_t)kf;

  s.own_empty = (uint8_t*)calloc(nn, 1);
  s.sub_empty = (uint8_t*)calloc(nn, 1);
  s.state = state;
  memset(state, 0, nn);
  for (int64_t id = 0; id < nn; ++id) {
    int e = 1;
    for (int c = 0; c < v->nch && e; ++c)
      e = tf_range_empty(&tfs[c], ranges[(id * v->nch + c) * 2], ranges[(id * v->nch + c) * 2 + 1]);
    s.own_empty[id] = (uint8_t)e;
  }
  /* subtree emptiness: the block and all its descendants are empty */
  for (int L = 0; L < v->levels; ++L)
    for (int64_t bz = 0; bz < s.nb[L][2]; ++bz)
      for (int64_t by = 0; by < s.nb[L][1]; ++by)
        for (int64_t bx = 0; bx < s.nb[L][0]; ++bx) {
          int64_t b[3] = {bx, by, bz};
          int64_t id = node_id(&s, L, b);
          int e = s.own_empty[id];
          if (L > 0)
            for (int c = 0; c < 8 && e; ++c) {
              int64_t cb[3] = {2 * bx + (c & 1), 2 * by + ((c >> 1) & 1), 2 * bz + ((c >> 2) & 1)};
              if (cb[0] >= s.nb[L - 1][0] || cb[1] >= s.nb[L - 1][1] || cb[2] >= s.nb[L - 1][2]) continue;
              e = s.sub_empty[node_id(&s, L - 1, cb)];
            }
          s.sub_empty[id] = (uint8_t)e;
        }
  int64_t ncell = s.nb[0][0] * s.nb[0][1] * s.nb[0][2];
  for (int64_t i = 0; i < ncell; ++i) leaf[i] = -1;
  s.leaf = leaf; s.req = req; s.req_cap = req_cap; s.nreq = 0;
  s.used = used;
  if (used) memset(used, 0, nn);
  int top = v->levels - 1;
  for (int64_t bz = 0; bz < s.nb[top][2]; ++bz)
    for (int64_t by = 0; by < s.nb[top][1]; ++by)
      for (int64_t bx = 0; bx < s.nb[top][0]; ++bx) {
        int64_t b[3] = {bx, by, bz};
        visit(&s, top, b);
      }
  qsort(req, s.nreq, sizeof(int32_t), cmp_i32);
  *nreq = s.nreq;
  int nsel = 0;
  for (int64_t id = 0; id < nn; ++id) {
    nsel += (state[id] == ST_SELECTED || state[id] == ST_FALLBACK);
    if (used && (state[id] == ST_SELECTED || state[id] == ST_FALLBACK || state[id] == ST_REFINED)) used[id] = 1;
  }
  free(s.own_empty);
  free(s.sub_empty);
  return nsel;
}

/* ------------------------------------------------------------------------ */
/* brick cache ("Volumetric Data Cashing")                                   */

/* The GPU cache holds at most `slots` blocks. Each resident block carries
 * the time stamp of the last frame whose traversal used it (see or_select's
 * `used`). Blocks of the coarsest level are pinned: they are never evicted.
 * Requests are placed in the order given. A request already resident is
 * left as it is. Otherwise it takes a free slot if there is one, else the
 * slot of the resident block with the smallest stamp that is older than the
 * current frame, ties going to the coarser block and then to the lower node
 * id; the placed block is stamped with the current frame. Placement stops
 * at the first request that finds no such block (every unpinned block in
 * use this frame). Returns the number of requests processed, a prefix of
 * the list; evicted[0..*nevicted) lists the blocks evicted, in order. */
int or_cache_place(const or_volume* v, int64_t slots, uint64_t frame, uint8_t* resident, uint64_t* stamp,
                   const int32_t* req, int nreq, int32_t* evicted, int* nevicted) {
  int64_t off[OR_MAX_LEVELS + 1];
  int64_t nn = or_node_count(v, off);
  int64_t nres = 0;
  for (int64_t i = 0; i < nn; ++i) nres += resident[i] != 0;
  *nevicted = 0;
  int m = 0;
  for (; m < nreq; ++m) {
    int64_t id = req[m];
    if (resident[id]) continue;
    if (nres >= slots) {
      int64_t victim = -1;
      int vlevel = 0;
      for (int64_t j = 0; j < nn; ++j) {
        if (!resident[j] || j >= off[v->levels - 1] || stamp[j] >= frame) continue;
        int L = 0;
        while (L + 1 < v->levels && j >= off[L + 1]) ++L;
        /* smallest stamp, then the larger level, then the lower id (j
         * ascends, so a later j only wins on a strictly better key) */
        if (victim < 0 || stamp[j] < stamp[victim] || (stamp[j] == stamp[victim] && L > vlevel)) {
          victim = j;
          vlevel = L;
        }
      }
      if (victim < 0) break;
      resident[victim] = 0;
      evicted[(*nevicted)++] = (int32_t)victim;
      --nres;
    }
    resident[id] = 1;
    stamp[id] = frame;
    ++nres;
  }
  return m;
}

/* The integers the selection decides with, exposed for pins. */
void or_select_inputs(const or_volume* v, const double* view, const double* proj, int height, double tau,
                      int64_t* eyes /*2x3*/, int64_t* planes /*2x4x4*/, uint64_t* K) {
  for (int e = 0; e < 2; ++e)
    eye_inputs(v->model, view + 16 * e, proj + 16 * e, eyes + 3 * e, (int64_t(*)[4])(planes + 16 * e));
  double theta = 2.0 / (proj[5] * (double)height);
  double tt = tau * theta;
  double kf = floor(tt * tt * 1099511627776.0);
  if (!(kf >= 0.0)) kf = 0.0;
  if (kf > 1099511627776.0) kf = 1099511627776.0;
  *K = (uint64_t)kf;
}

/* ------------------------------------------------------------------------ */
/* sampling and classification                                               */

static inline double fetch(const or_volume* v, int L, int c, int64_t x, int64_t y, int64_t z) {
  const int64_t* D = v->dims[L];
  if (x < 0) x = 0; if (x > D[0] - 1) x = D[0] - 1;
  if (y < 0) y = 0; if (y > D[1] - 1) y = D[1] - 1;
  if (z < 0) z = 0; if (z > D[2] - 1) z = D[2] - 1;
  return (double)vox_get(v->data[L][c], v->dtype, (z * D[1] + y) * D[0] + x);
}

/* Trilinear value of level L, channel c at p (level-0 voxel units). Voxel j
 * of level L has its centre at (j + 0.5) 2^L; indices are clamped to the
 * level (clamp-to-edge). The blend is the exact trilinear weighting. */
double or_sample(const or_volume* v, int L, int c, const double* p) {
  double s = 1.0 / (double)((int64_t)1 << L);
  double u[3], f[3];
  int64_t i[3];
  for (int a = 0; a < 3; ++a) {
    u[a] = p[a] * s - 0.5;
    i[a] = (int64_t)floor(u[a]);
    f[a] = u[a] - (double)i[a];
  }
  double acc = 0.0;
  for (int dz = 0; dz < 2; ++dz)
    for (int dy = 0; dy < 2; ++dy)
      for (int dx = 0; dx < 2; ++dx) {
        double w = (dx ? f[0] : 1.0 - f[0]) * (dy ? f[1] : 1.0 - f[1]) * (dz ? f[2] : 1.0 - f[2]);
        acc += w * fetch(v, L, c, i[0] + dx, i[1] + dy, i[2] + dz);
      }
  return acc;
}

/* Opacity-corrected table for a sample spacing of `spacing` level-0 voxels:
 * alpha' = 1 - (1 - alpha)^(spacing / ref_step), colour unchanged. */
void or_tf_table(const or_tf* tf, double spacing, double* out /*4n*/) {
  double e = spacing / (double)tf->ref_step;
  for (int i = 0; i < tf->n; ++i) {
    for (int k = 0; k < 3; ++k) out[4 * i + k] = tf->rgba[4 * i + k];
    out[4 * i + 3] = 1.0 - pow(1.0 - (double)tf->rgba[4 * i + 3], e);
  }
}

/* Classification: x = clamp((v - lo)/(hi - lo), 0, 1), q = x (n-1), linear
 * interpolation between entries floor(q) and floor(q)+1 (clamped). */
void or_classify(const or_tf* tf, const double* table, double value, double* rgba) {
  double x = (value - (double)tf->lo) / ((double)tf->hi - (double)tf->lo);
  if (x < 0.0) x = 0.0;
  if (x > 1.0) x = 1.0;
  double q = x * (double)(tf->n - 1);
  int i = (int)floor(q);
  if (i > tf->n - 1) i = tf->n - 1;
  int i1 = i + 1 > tf->n - 1 ? tf->n - 1 : i + 1;
  double f = q - (double)i;
  for (int k = 0; k < 4; ++k) rgba[k] = table[4 * i + k] * (1.0 - f) + table[4 * i1 + k] * f;
}

/* Gradient magnitude of channel c's level-L field at level-0 position p, per
 * level-0 voxel: central differences of the trilinear field at +-1/2 level-L
 * voxel along each axis (the taps stay within a brick's one-voxel apron),
 * divided by 2^L. */
static double grad_mag(const or_volume* v, int L, int c, const double* p) {
  double h = 0.5 * (double)((int64_t)1 << L), g2 = 0.0;
  for (int ax = 0; ax < 3; ++ax) {
    double a[3] = {p[0], p[1], p[2]}, b[3] = {p[0], p[1], p[2]};
    a[ax] += h;
    b[ax] -= h;
    double d = or_sample(v, L, c, a) - or_sample(v, L, c, b);
    g2 += d * d;
  }
  return sqrt(g2) / (double)((int64_t)1 << L);
}

/* Palette colour at world distance d from the eye: x = clamp((d - near) /
 * (far - near), 0, 1), q = x (m - 1), linear between entries floor(q) and
 * floor(q) + 1. */
static void palette_rgb(const or_tf* tf, double d, double* rgb) {
  double x = (d - (double)tf->pnear) / ((double)tf->pfar - (double)tf->pnear);
  if (x < 0.0) x = 0.0;
  if (x > 1.0) x = 1.0;
  double q = x * (double)(tf->m - 1);
  int i = (int)floor(q);
  if (i > tf->m - 2) i = tf->m - 2;
  if (i < 0) i = 0;
  int i1 = i + 1 > tf->m - 1 ? tf->m - 1 : i + 1;
  double f = q - (double)i;
  for (int k = 0; k < 3; ++k) rgb[k] = tf->palette[3 * i + k] * (1.0 - f) + tf->palette[3 * i1 + k] * f;
}

/* ------------------------------------------------------------------------ */
/* ray casting                                                               */

/* Pixel flags. FL_FACE: a lattice point lies within eps of a face between
 * cells whose sampling differs (two levels, or a dropped cell next to a
 * rendered one); FL_TEDGE: a lattice point lies within eps of where the ray
 * ends (the volume's exit face or a depth-buffer surface). Both are resolved
 * by enumerating the legitimate assignments (or_render_variants). FL_TERM:
 * the termination threshold test is within term_tol. FL_ENTRY: the eye lies
 * within eps of a volume face, so the lattice anchor itself is uncertain;
 * FL_MANY: more assignments than the enumeration's cap. These two are not
 * resolved. */
enum { FL_FACE = 1, FL_TEDGE = 2, FL_TERM = 4, FL_ENTRY = 8, FL_MANY = 16 };

/* Optical models ("DVR Techniques"): emission-absorption (front-to-back
 * compositing with early termination), emission-only (the integral of the
 * emitted intensity along the ray, no absorption, alpha output 0), and
 * maximum intensity projection (the classified maximum along the ray). */
enum { OR_MODE_EA = 0, OR_MODE_EMISSION = 1, OR_MODE_MIP = 2 };

/* Radial lens model ("DVR for HMD"): the image is rendered in the lens's
 * warped space with one ray per warped pixel. A warped NDC point w at offset
 * d = w - c from the lens centre c looks through the undistorted NDC point
 * u = c + d f(r) s, with f(r) = 1 + k1 r^2 + k2 r^4, r^2 = (d_x aspect)^2 +
 * d_y^2 (aspect = width / height, so r is isotropic on the display) and s
 * the scale. */
typedef struct {
  double k1, k2, scale, aspect, cx, cy;
} or_lens;

static void lens_warp_to_undistorted(const or_lens* L, double wx, double wy, double* ux, double* uy) {
  double dx = wx - L->cx, dy = wy - L->cy;
  double r2 = dx * L->aspect * dx * L->aspect + dy * dy;
  double f = (1.0 + L->k1 * r2 + L->k2 * r2 * r2) * L->scale;
  *ux = L->cx + dx * f;
  *uy = L->cy + dy * f;
}

/* Inverse of the map above (k1, k2 >= 0, so r f(r) is increasing): given
 * the undistorted u, the warped w. rho = |(u - c) / s| (aspect-weighted)
 * equals r f(r); r is found by bisection on [0, rho] to full precision. */
void or_lens_unwarp_point(const or_lens* L, double ux, double uy, double* wx, double* wy) {
  double ex = (ux - L->cx) / L->scale, ey = (uy - L->cy) / L->scale;
  double rho = sqrt(ex * L->aspect * ex * L->aspect + ey * ey);
  if (rho == 0.0) { *wx = L->cx; *wy = L->cy; return; }
  double lo = 0.0, hi = rho;
  for (int it = 0; it < 200; ++it) {
    double mid = 0.5 * (lo + hi);
    double g = mid * (1.0 + L->k1 * mid * mid + L->k2 * mid * mid * mid * mid);
    if (g < rho) lo = mid; else hi = mid;
  }
  double r = 0.5 * (lo + hi);
  double f = 1.0 + L->k1 * r * r + L->k2 * r * r * r * r;
  *wx = L->cx + ex / f;
  *wy = L->cy + ey / f;
}

/* Resample a warped RGBA image (Ww x Hw, row 0 = top) to the undistorted
 * image (W x H): output pixel centre u -> warped point w -> bilinear tap of
 * the warped pixel centres (edge pixels replicated); points outside the
 * warped image [-1, 1]^2 give (0,0,0,0). */
void or_unwarp(const or_lens* L, const float* warped, int Ww, int Hw, double* out, int W, int H) {
#pragma omp parallel for schedule(static)
  for (int j = 0; j < H; ++j)
    for (int i = 0; i < W; ++i) {
      double ux = 2.0 * (i + 0.5) / W - 1.0, uy = 1.0 - 2.0 * (j + 0.5) / H, wx, wy;
      or_lens_unwarp_point(L, ux, uy, &wx, &wy);
      double* o = out + 4 * ((int64_t)j * W + i);
      if (!(wx >= -1.0 && wx <= 1.0 && wy >= -1.0 && wy <= 1.0)) {
        o[0] = o[1] = o[2] = o[3] = 0.0;
        continue;
      }
      double px = (wx + 1.0) * 0.5 * Ww - 0.5, py = (1.0 - wy) * 0.5 * Hw - 0.5;
      double fx = floor(px), fy = floor(py);
      double ax = px - fx, ay = py - fy;
      int x0 = (int)fx, y0 = (int)fy;
      for (int k = 0; k < 4; ++k) {
        double v = 0.0;
        for (int b = 0; b < 2; ++b)
          for (int a = 0; a < 2; ++a) {
            int xx = x0 + a, yy = y0 + b;
            xx = xx < 0 ? 0 : (xx > Ww - 1 ? Ww - 1 : xx);
            yy = yy < 0 ? 0 : (yy > Hw - 1 ? Hw - 1 : yy);
            double w = (a ? ax : 1.0 - ax) * (b ? ay : 1.0 - ay);
            v += w * (double)warped[4 * ((int64_t)yy * Ww + xx) + k];
          }
        o[k] = v;
      }
    }
}

typedef struct {
  const or_volume* v;
  const or_tf* tf;
  const int32_t* leaf;
  int64_t nb0[3];
  int64_t off[OR_MAX_LEVELS + 1];
  double* table[OR_MAX_LEVELS][OR_MAX_CH];
  double* raw[OR_MAX_CH]; /* the tables as given (opacity for one reference step) */
  double inv[16]; /* (P V M)^-1 */
  double eye[3];
  int W, H;
  double step, term, term_tol, eps;
  int mode;
  const double* tmax; /* per image pixel: the ray ends there (level-0 voxels from the eye); NULL = none */
  const or_lens* lens; /* rays through the warped image; NULL = none */
  double voxel;        /* world units per level-0 voxel (the model's uniform scale) */
} ray_t;

/* the table's input for channel c at level-0 position p, sampled at level L */
static double tf_input(const ray_t* r, int L, int c, const double* p) {
  return r->tf[c].input == OR_INPUT_GRADIENT ? grad_mag(r->v, L, c, p) : or_sample(r->v, L, c, p);
}

static int node_level(const ray_t* r, int32_t id) {
  if (id < 0) return -1;
  int L = 0;
  while (L + 1 < r->v->levels && id >= r->off[L + 1]) ++L;
  return L;
}

static int32_t cell_at(const ray_t* r, const int64_t* c) {
  return r->leaf[(c[2] * r->nb0[1] + c[1]) * r->nb0[0] + c[0]];
}

static void cell_of(const ray_t* r, const double* p, double shift, const int* dirs, int64_t* c) {
  for (int a = 0; a < 3; ++a) {
    int64_t q = (int64_t)floor((p[a] + shift * dirs[a]) / (double)r->v->brick);
    if (q < 0) q = 0;
    if (q > r->nb0[a] - 1) q = r->nb0[a] - 1;
    c[a] = q;
  }
}

/* ---- one ray: the lattice walk ------------------------------------------
 *
 * The ray takes the lattice points t0 + k step (k >= 0) in order; the point
 * belongs to the level-0 cell containing it, and the selected block rendering
 * that cell (level L) takes it iff k is a multiple of 2^L, sampling level L
 * there. The ray ends at the first point at or beyond t1 (volume exit or
 * depth-buffer surface), or after the sample that makes A >= term.
 *
 * Where exact arithmetic puts a point within eps of a face between cells
 * that would treat it differently, or within eps of the ray's end, a
 * floating-point implementation may legitimately assign it either way. Each
 * such point is a branch point with its candidate behaviours (sample at
 * level L, skip, or end the ray). The exact walk takes the exact assignment
 * everywhere; the enumeration walks every combination, with one constraint
 * that follows from the geometry: along a run of consecutive points near
 * one face (a ray grazing it) the ray crosses that face once, so once a
 * point of the run is given the far side, the later ones are too. */

enum { BEH_SKIP = -1, BEH_END = -2 };

typedef struct {
  double o[3], d[3];
  double t0, t1box, tsurf;
  uint8_t entry_flag;
} geom_t;

typedef struct {
  int64_t k;
  double C[3], A, Ce[3], Ae;
  uint32_t cnt, cnte;
  int early_done;
  double vmax[OR_MAX_CH], tat[OR_MAX_CH];
  int any;
  int run_ax;      /* face run in progress: axis, -1 for none */
  double run_face; /* its plane, level-0 voxels */
  int run_far;     /* the walk has given a point of the run the far side */
} walk_t;

typedef struct {
  int cap, n, overflow;
  double* early; /* [cap][4] */
  double* late;  /* [cap][4] */
  uint32_t* ce;  /* [cap] */
  uint32_t* cl;  /* [cap] */
  uint8_t flags;
} leaves_t;

#define OR_MAX_CAND 10

typedef struct {
  int n;
  int beh[OR_MAX_CAND];
  int far[OR_MAX_CAND]; /* 1: this candidate is the far side of the current run's face */
  int exact;            /* index of the exact assignment */
  uint8_t kind;         /* FL_FACE and/or FL_TEDGE when n > 1 */
} cand_t;

static int geom_setup(const ray_t* r, int64_t pix, geom_t* g) {
  int i = (int)(pix % r->W), j = (int)(pix / r->W);
  double x = 2.0 * (i + 0.5) / r->W - 1.0, y = 1.0 - 2.0 * (j + 0.5) / r->H;
  if (r->lens) lens_warp_to_undistorted(r->lens, x, y, &x, &y);
  double pn[4] = {x, y, -1.0, 1.0}, pf[4] = {x, y, 1.0, 1.0}, a[4], b[4];
  mat_apply(r->inv, pn, a);
  mat_apply(r->inv, pf, b);
  double dn = 0.0;
  for (int k = 0; k < 3; ++k) { g->d[k] = b[k] / b[3] - a[k] / a[3]; dn += g->d[k] * g->d[k]; }
  dn = sqrt(dn);
  for (int k = 0; k < 3; ++k) { g->d[k] /= dn; g->o[k] = r->eye[k]; }
  double tn = -INFINITY, tf = INFINITY;
  for (int k = 0; k < 3; ++k) {
    double N = (double)r->v->dims[0][k];
    if (g->d[k] == 0.0) {
      if (g->o[k] < 0.0 || g->o[k] > N) { tf = -INFINITY; break; }
      continue;
    }
    double t1 = (0.0 - g->o[k]) / g->d[k], t2 = (N - g->o[k]) / g->d[k];
    if (t1 > t2) { double t = t1; t1 = t2; t2 = t; }
    if (t1 > tn) tn = t1;
    if (t2 < tf) tf = t2;
  }
  g->t0 = tn > 0.0 ? tn : 0.0;
  g->t1box = tf;
  /* depth-buffer termination: an opaque surface at tmax ends the ray
   * ("Volumetric and Mesh Data Compositing") */
  g->tsurf = r->tmax ? r->tmax[pix] : INFINITY;
  g->entry_flag = (tf > g->t0 && fabs(tn) < r->eps) ? FL_ENTRY : 0;
  double t1 = tf < g->tsurf ? tf : g->tsurf;
  return t1 > g->t0;
}

/* behaviour of the cell holding node id at lattice point k */
static int cell_behaviour(const ray_t* r, int32_t id, int64_t k) {
  int L = node_level(r, id);
  if (L < 0) return BEH_SKIP;
  return (k & (((int64_t)1 << L) - 1)) == 0 ? L : BEH_SKIP;
}

static void cand_add(cand_t* c, int beh, int far) {
  for (int i = 0; i < c->n; ++i)
    if (c->beh[i] == beh) {
      if (!far) c->far[i] = 0; /* reachable without crossing */
      return;
    }
  if (c->n < OR_MAX_CAND) {
    c->beh[c->n] = beh;
    c->far[c->n] = far;
    ++c->n;
  }
}

/* Candidate behaviours of lattice point k at distance t, position p. Updates
 * the walk's face run. */
static void candidates(const ray_t* r, const geom_t* g, walk_t* s, double t, const double* p, cand_t* c) {
  const double B = (double)r->v->brick;
  c->n = 0;
  c->exact = 0;
  c->kind = 0;
  /* where the ray ends: out_dist = how far p lies outside the volume box,
   * exit_dist = its distance to the nearest face the ray leaves through */
  double out_dist = 0.0, exit_dist = INFINITY;
  for (int a = 0; a < 3; ++a) {
    const double N = (double)r->v->dims[0][a];
    const double o = p[a] - N > -p[a] ? p[a] - N : -p[a];
    if (o > out_dist) out_dist = o;
    if (g->d[a] != 0.0) {
      const double e = fabs(p[a] - (g->d[a] > 0.0 ? N : 0.0));
      if (e < exit_dist) exit_dist = e;
    }
  }
  const int inside = t < g->t1box && t < g->tsurf;
  const int beyond = (t >= g->t1box && out_dist >= r->eps) || t >= g->tsurf + r->eps;
  if (beyond) {
    c->n = 1;
    c->beh[0] = BEH_END;
    c->far[0] = 0;
    s->run_ax = -1;
    return;
  }
  /* not beyond but not inside: within eps past the end */
  const int end_amb = (t < g->t1box ? exit_dist < r->eps : out_dist < r->eps) || fabs(t - g->tsurf) < r->eps;
  /* the cells around p: faces within eps on each axis (interior faces only) */
  int zero[3] = {0, 0, 0};
  int64_t ce[3];
  cell_of(r, p, 0.0, zero, ce);
  const int exact_beh = cell_behaviour(r, cell_at(r, ce), s->k);
  int near_ax[3], nnear = 0, lone = -1;
  double face[3];
  for (int a = 0; a < 3; ++a) {
    double f = floor(p[a] / B + 0.5) * B;
    int64_t fi = (int64_t)floor(p[a] / B + 0.5);
    near_ax[a] = fabs(p[a] - f) < r->eps && fi >= 1 && fi <= r->nb0[a] - 1;
    face[a] = f;
    if (near_ax[a]) { ++nnear; lone = a; }
  }
  if (nnear == 1) {
    const int a = lone;
    if (s->run_ax != a || s->run_face != face[a]) {
      s->run_ax = a;
      s->run_face = face[a];
      s->run_far = 0;
    }
    int64_t lo[3] = {ce[0], ce[1], ce[2]}, hi[3] = {ce[0], ce[1], ce[2]};
    lo[a] = (int64_t)(face[a] / B) - 1;
    hi[a] = (int64_t)(face[a] / B);
    const int blo = cell_behaviour(r, cell_at(r, lo), s->k), bhi = cell_behaviour(r, cell_at(r, hi), s->k);
    /* near side: the one the ray comes from (for a ray in the face's plane,
     * the exact one) */
    int lo_near = g->d[a] > 0.0 ? 1 : (g->d[a] < 0.0 ? 0 : ce[a] == lo[a]);
    const int bnear = lo_near ? blo : bhi, bfar = lo_near ? bhi : blo;
    if (!s->run_far) cand_add(c, bnear, 0);
    cand_add(c, bfar, 1);
    if (c->n > 1) c->kind |= FL_FACE;
  } else if (nnear > 1) {
    s->run_ax = -1;
    for (int m = 0; m < 8; ++m) {
      int64_t cc[3];
      int skip = 0;
      for (int a = 0; a < 3; ++a) {
        int side = (m >> a) & 1;
        if (!near_ax[a]) {
          if (side) skip = 1;
          cc[a] = ce[a];
        } else {
          cc[a] = (int64_t)(face[a] / B) - 1 + side;
        }
      }
      if (skip) continue;
      cand_add(c, cell_behaviour(r, cell_at(r, cc), s->k), 0);
    }
    if (c->n > 1) c->kind |= FL_FACE;
  } else {
    s->run_ax = -1;
    cand_add(c, exact_beh, 0);
  }
  if (end_amb) {
    cand_add(c, BEH_END, 0);
    if (c->n > 1) c->kind |= FL_TEDGE;
  }
  /* index of the exact assignment */
  const int want = inside ? exact_beh : BEH_END;
  for (int i = 0; i < c->n; ++i)
    if (c->beh[i] == want) c->exact = i;
}

/* Takes the sample of lattice point s->k at level L. Returns 1 when the ray
 * stops (A >= term + term_tol). */
static int take_sample(const ray_t* r, walk_t* s, int L, double t, const double* p) {
  const int nch = r->v->nch;
  if (r->mode == OR_MODE_MIP) {
    /* the maximum table input per channel (the first sample that reaches it
     * keeps its distance), classified when the ray ends */
    for (int c = 0; c < nch; ++c) {
      double val = tf_input(r, L, c, p);
      if (val > s->vmax[c]) { s->vmax[c] = val; s->tat[c] = t; }
    }
    s->any = 1;
    ++s->cnt;
    return 0;
  }
  if (r->mode == OR_MODE_EMISSION) {
    /* emitted intensity per level-0 voxel of path: the table's colour times
     * its opacity for one reference step, over that step; a level-L sample
     * stands for step * 2^L of path */
    for (int c = 0; c < nch; ++c) {
      double val = tf_input(r, L, c, p), rgba[4];
      or_classify(&r->tf[c], r->raw[c], val, rgba);
      if (r->tf[c].m > 0) palette_rgb(&r->tf[c], t * r->voxel, rgba);
      double w = rgba[3] * (r->step * (double)((int64_t)1 << L)) / (double)r->tf[c].ref_step;
      for (int q = 0; q < 3; ++q) s->C[q] += w * rgba[q];
    }
    ++s->cnt;
    return 0;
  }
  /* classify every channel, blend additively (alpha capped at 1) */
  double sa = 0.0, sc[3] = {0, 0, 0};
  for (int c = 0; c < nch; ++c) {
    double val = tf_input(r, L, c, p), rgba[4];
    or_classify(&r->tf[c], r->table[L][c], val, rgba);
    if (r->tf[c].m > 0) palette_rgb(&r->tf[c], t * r->voxel, rgba);
    sa += rgba[3];
    for (int q = 0; q < 3; ++q) sc[q] += rgba[3] * rgba[q];
  }
  double as = sa < 1.0 ? sa : 1.0;
  double scale = sa > 0.0 ? as / (sa > as ? sa : as) : 0.0;
  for (int q = 0; q < 3; ++q) s->C[q] += (1.0 - s->A) * sc[q] * scale;
  s->A += (1.0 - s->A) * as;
  ++s->cnt;
  if (!s->early_done && s->A >= r->term - r->term_tol) {
    s->early_done = 1;
    memcpy(s->Ce, s->C, sizeof s->C);
    s->Ae = s->A;
    s->cnte = s->cnt;
  }
  return s->A >= r->term + r->term_tol;
}

/* The ray has ended: finish MIP, record early/late results. */
static void leaf(const ray_t* r, walk_t* s, leaves_t* out) {
  if (r->mode == OR_MODE_MIP && s->any) {
    /* classify each channel's maximum with its table for one reference
     * step, blend the channels additively (alpha capped at 1), premultiply */
    double sa = 0.0, sc[3] = {0, 0, 0};
    for (int c = 0; c < r->v->nch; ++c) {
      double rgba[4];
      or_classify(&r->tf[c], r->raw[c], s->vmax[c], rgba);
      if (r->tf[c].m > 0) palette_rgb(&r->tf[c], s->tat[c] * r->voxel, rgba);
      sa += rgba[3];
      for (int q = 0; q < 3; ++q) sc[q] += rgba[3] * rgba[q];
    }
    double as = sa < 1.0 ? sa : 1.0;
    double scale = sa > 0.0 ? as / (sa > as ? sa : as) : 0.0;
    for (int q = 0; q < 3; ++q) s->C[q] = sc[q] * scale;
    s->A = as;
  }
  if (!s->early_done) {
    memcpy(s->Ce, s->C, sizeof s->C);
    s->Ae = s->A;
    s->cnte = s->cnt;
  }
  if (s->cnte != s->cnt) out->flags |= FL_TERM;
  if (out->n >= out->cap) {
    out->overflow = 1;
    return;
  }
  double* e = out->early + 4 * out->n;
  double* l = out->late + 4 * out->n;
  for (int q = 0; q < 3; ++q) { e[q] = s->Ce[q]; l[q] = s->C[q]; }
  e[3] = s->Ae;
  l[3] = s->A;
  out->ce[out->n] = s->cnte;
  out->cl[out->n] = s->cnt;
  ++out->n;
}

/* Applies behaviour b at the walk's point. Returns 1 when the ray has ended. */
static int apply(const ray_t* r, walk_t* s, int b, double t, const double* p) {
  if (b == BEH_END) return 1;
  if (b == BEH_SKIP) return 0;
  return take_sample(r, s, b, t, p);
}

/* Walks the ray from s.k on. explore = 0: the exact assignment at every
 * point (one leaf); explore = 1: every candidate at every branch point,
 * depth-first (depth = branch points taken so far on this path). */
#define OR_MAX_BRANCH_DEPTH 400

static void walk(const ray_t* r, const geom_t* g, walk_t s, int explore, int depth, leaves_t* out) {
  if (depth > OR_MAX_BRANCH_DEPTH) {
    out->overflow = 1;
    return;
  }
  for (;; ++s.k) {
    if (out->overflow) return;
    const double t = g->t0 + (double)s.k * r->step;
    const double p[3] = {g->o[0] + t * g->d[0], g->o[1] + t * g->d[1], g->o[2] + t * g->d[2]};
    cand_t c;
    candidates(r, g, &s, t, p, &c);
    if (c.n > 1) out->flags |= c.kind;
    if (!explore || c.n == 1) {
      const int i = explore ? 0 : c.exact;
      if (c.far[i]) s.run_far = 1;
      if (apply(r, &s, c.beh[i], t, p)) {
        leaf(r, &s, out);
        return;
      }
      continue;
    }
    for (int i = 0; i < c.n && !out->overflow; ++i) {
      walk_t s2 = s;
      if (c.far[i]) s2.run_far = 1;
      if (apply(r, &s2, c.beh[i], t, p)) {
        leaf(r, &s2, out);
        continue;
      }
      s2.k += 1;
      walk(r, g, s2, 1, depth + 1, out);
    }
    return;
  }
}

static void walk_init(walk_t* s) {
  memset(s, 0, sizeof *s);
  for (int c = 0; c < OR_MAX_CH; ++c) s->vmax[c] = -INFINITY;
  s->run_ax = -1;
}

/* One ray, FP64, exact assignment. Two compositing results bracket the
 * termination decision: "early" stops after the first sample with
 * A >= term - term_tol, "late" after the first with A >= term + term_tol
 * (they differ only when a sample lands within term_tol of the threshold). */
static void cast(const ray_t* r, int64_t pix, double* early, double* late, uint32_t* ne, uint32_t* nl,
                 uint8_t* flag) {
  geom_t g;
  leaves_t out;
  memset(&out, 0, sizeof out);
  out.cap = 1;
  out.early = early;
  out.late = late;
  out.ce = ne;
  out.cl = nl;
  walk_t s;
  walk_init(&s);
  if (!geom_setup(r, pix, &g)) {
    for (int q = 0; q < 4; ++q) early[q] = late[q] = 0.0;
    *ne = *nl = 0;
    *flag = 0;
    return;
  }
  walk(r, &g, s, 0, 0, &out);
  *flag = out.flags | g.entry_flag;
}

static int ray_init(ray_t* r, const or_volume* v, const or_tf* tfs, const int32_t* leaf, const double* view,
                    const double* proj, int W, int H, double step, double term, double term_tol, double eps, int mode,
                    const double* tmax, const or_lens* lens) {
  memset(r, 0, sizeof *r);
  r->v = v; r->tf = tfs; r->leaf = leaf; r->W = W; r->H = H;
  r->step = step; r->term = term; r->term_tol = term_tol; r->eps = eps;
  r->mode = mode; r->tmax = tmax; r->lens = lens;
  r->voxel = sqrt(v->model[0] * v->model[0] + v->model[1] * v->model[1] + v->model[2] * v->model[2]);
  or_node_count(v, r->off);
  level_blocks(v, 0, r->nb0);
  double vm[16], pvm[16], vminv[16];
  mat_mul(view, v->model, vm);
  mat_mul(proj, vm, pvm);
  if (!mat_inv(pvm, r->inv) || !mat_inv(vm, vminv)) return 0;
  double o[4] = {0, 0, 0, 1}, e[4];
  mat_apply(vminv, o, e);
  for (int k = 0; k < 3; ++k) r->eye[k] = e[k] / e[3];
  for (int c = 0; c < v->nch; ++c) {
    r->raw[c] = (double*)malloc(sizeof(double) * 4 * tfs[c].n);
    for (int i = 0; i < 4 * tfs[c].n; ++i) r->raw[c][i] = (double)tfs[c].rgba[i];
  }
  for (int L = 0; L < v->levels; ++L)
    for (int c = 0; c < v->nch; ++c) {
      r->table[L][c] = (double*)malloc(sizeof(double) * 4 * tfs[c].n);
      or_tf_table(&tfs[c], step * (double)((int64_t)1 << L), r->table[L][c]);
    }
  return 1;
}

static void ray_free(ray_t* r) {
  for (int L = 0; L < r->v->levels; ++L)
    for (int c = 0; c < r->v->nch; ++c) free(r->table[L][c]);
  for (int c = 0; c < r->v->nch; ++c) free(r->raw[c]);
}

/* Render the pixels pix[0..npix) (row-major ids j*W+i, row 0 = top; NULL
 * means every pixel) of one eye with the exact assignment. leaf comes from
 * or_select. step is the level-0 sample spacing; level L samples every
 * 2^L-th lattice point t0 + k step, k >= 0, anchored at the volume entry t0.
 * Returns 0 on a singular matrix. nthreads <= 0 uses every core. */
int or_render(const or_volume* v, const or_tf* tfs, const int32_t* leaf, const double* view,
              const double* proj, int W, int H, double step, double term, double term_tol, double eps,
              const int64_t* pix, int64_t npix, double* rgba_early, double* rgba_late, uint32_t* cnt_early,
              uint32_t* cnt_late, uint8_t* flags, int nthreads, int mode, const double* tmax,
              const or_lens* lens) {
  ray_t r;
  if (!ray_init(&r, v, tfs, leaf, view, proj, W, H, step, term, term_tol, eps, mode, tmax, lens)) return 0;
  int64_t n = pix ? npix : (int64_t)W * H;
  const int nt = nthreads > 0 ? nthreads : omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 64) num_threads(nt)
  for (int64_t q = 0; q < n; ++q) {
    int64_t id = pix ? pix[q] : q;
    cast(&r, id, rgba_early + 4 * q, rgba_late + 4 * q, cnt_early + q, cnt_late + q, flags + q);
  }
  ray_free(&r);
  return 1;
}

/* Every legitimate result of the pixels pix[0..npix): one per combination of
 * candidate assignments at the ray's branch points (see the lattice walk
 * above), at most cap per pixel, each with its early/late bracket. nvar[q]
 * is the number written, 0 when the combinations exceed cap. Output layout:
 * [npix][cap][4] RGBA and [npix][cap] counts. */
int or_render_variants(const or_volume* v, const or_tf* tfs, const int32_t* leaf, const double* view,
                       const double* proj, int W, int H, double step, double term, double term_tol, double eps,
                       const int64_t* pix, int64_t npix, int cap, double* rgba_early, double* rgba_late,
                       uint32_t* cnt_early, uint32_t* cnt_late, int32_t* nvar, int nthreads, int mode,
                       const double* tmax, const or_lens* lens) {
  ray_t r;
  if (!ray_init(&r, v, tfs, leaf, view, proj, W, H, step, term, term_tol, eps, mode, tmax, lens)) return 0;
  const int nt = nthreads > 0 ? nthreads : omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nt)
  for (int64_t q = 0; q < npix; ++q) {
    geom_t g;
    leaves_t out;
    memset(&out, 0, sizeof out);
    out.cap = cap;
    out.early = rgba_early + (size_t)4 * cap * q;
    out.late = rgba_late + (size_t)4 * cap * q;
    out.ce = cnt_early + (size_t)cap * q;
    out.cl = cnt_late + (size_t)cap * q;
    walk_t s;
    walk_init(&s);
    if (!geom_setup(&r, pix[q], &g)) {
      for (int k = 0; k < 4; ++k) out.early[k] = out.late[k] = 0.0;
      out.ce[0] = out.cl[0] = 0;
      nvar[q] = 1;
      continue;
    }
    walk(&r, &g, s, 1, 0, &out);
    nvar[q] = out.overflow ? 0 : out.n;
  }
  ray_free(&r);
  return 1;
}

int or_max_threads(void) { return omp_get_max_threads(); }
