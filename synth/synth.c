/* Seeded synthetic inputs shaped like the paper's microscopy workloads.
 *
 * This module only produces inputs (volumes); it holds none of the rendering
 * method's arithmetic. Both the CUDA path's tests/bench and the CPU oracle
 * consume its output, and neither shares any other code.
 *
 * Randomness is counter based (splitmix64 finaliser over (seed, counter)), so
 * every voxel is a pure function of its coordinates and the seed and any
 * sub-region can be regenerated on its own (used for out-of-core bricks).
 *
 * Coordinates: voxel (i,j,k) has its centre at (i+0.5, j+0.5, k+0.5); arrays
 * are x fastest, then y, then z.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <omp.h>

static inline uint64_t mix64(uint64_t z) {
  z += 0x9e3779b97f4a7c15ULL;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}
/* uniform double in [0,1) for (seed, stream, counter) */
static inline double u01(uint64_t seed, uint64_t stream, uint64_t ctr) {
  uint64_t h = mix64(mix64(seed ^ (stream * 0xd1b54a32d192ed03ULL)) ^ ctr);
  return (double)(h >> 11) * (1.0 / 9007199254740992.0);
}
static inline double urange(uint64_t seed, uint64_t stream, uint64_t ctr, double a, double b) {
  return a + (b - a) * u01(seed, stream, ctr);
}

/* --- configuration "plain ray cast": sum of isotropic Gaussians + uniform noise, u8 --- */
void sy_gaussians_u8(uint8_t* out, int nx, int ny, int nz, uint64_t seed, int count,
                     double noise_max) {
  double c[64][3], s[64], a[64];
  if (count > 64) count = 64;
  for (int g = 0; g < count; ++g) {
    c[g][0] = urange(seed, 1, 8 * g + 0, 0.2, 0.8) * nx;
    c[g][1] = urange(seed, 1, 8 * g + 1, 0.2, 0.8) * ny;
    c[g][2] = urange(seed, 1, 8 * g + 2, 0.2, 0.8) * nz;
    s[g] = urange(seed, 1, 8 * g + 3, 6.0, 20.0);
    a[g] = urange(seed, 1, 8 * g + 4, 80.0, 255.0);
  }
#pragma omp parallel for schedule(static)
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        double v = 0.0;
        for (int g = 0; g < count; ++g) {
          double dx = x + 0.5 - c[g][0], dy = y + 0.5 - c[g][1], dz = z + 0.5 - c[g][2];
          v += a[g] * exp(-(dx * dx + dy * dy + dz * dz) / (2.0 * s[g] * s[g]));
        }
        uint64_t idx = ((uint64_t)z * ny + y) * nx + x;
        v += noise_max * u01(seed, 2, idx);
        double r = floor(v + 0.5);
        out[idx] = (uint8_t)(r > 255.0 ? 255.0 : r);
      }
}

/* --- configuration "bricked multi-LOD stereo": Catmull-Rom tubes over a Poisson background, u16 --- */
typedef struct { float x, y, z, r, I; } stamp_t;

static void catmull(const double* p0, const double* p1, const double* p2, const double* p3,
                    double t, double* o) {
  double t2 = t * t, t3 = t2 * t;
  for (int k = 0; k < 3; ++k)
    o[k] = 0.5 * (2.0 * p1[k] + (-p0[k] + p2[k]) * t + (2 * p0[k] - 5 * p1[k] + 4 * p2[k] - p3[k]) * t2 +
                  (-p0[k] + 3 * p1[k] - 3 * p2[k] + p3[k]) * t3);
}

static int cmp_stamp_z(const void* a, const void* b) {
  float za = ((const stamp_t*)a)->z, zb = ((const stamp_t*)b)->z;
  return (za > zb) - (za < zb);
}

/* Poisson(lambda) by inverse CDF of a counter-based uniform. */
static int build_poisson_cdf(double lambda, double** cdf_out) {
  int kmax = (int)(lambda + 20.0 * sqrt(lambda) + 40.0);
  double* cdf = (double*)malloc(sizeof(double) * (kmax + 1));
  double logp = -lambda, acc = 0.0;
  for (int k = 0; k <= kmax; ++k) {
    if (k > 0) logp += log(lambda) - log((double)k);
    acc += exp(logp);
    cdf[k] = acc;
  }
  cdf[kmax] = 2.0; /* absorb the tail */
  *cdf_out = cdf;
  return kmax;
}
static inline int poisson_draw(const double* cdf, int kmax, double u) {
  int lo = 0, hi = kmax;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (cdf[mid] > u) hi = mid; else lo = mid + 1;
  }
  return lo;
}

int sy_filaments_u16(uint16_t* out, int nx, int ny, int nz, uint64_t seed, int ntubes,
                     double lambda, double rmin, double rmax, double imin, double imax) {
  /* 1. stamps along every tube, spaced <= 0.5 voxel */
  size_t cap = 1 << 16, n = 0;
  stamp_t* st = (stamp_t*)malloc(cap * sizeof(stamp_t));
  double dims[3] = {nx, ny, nz};
  for (int tb = 0; tb < ntubes; ++tb) {
    uint64_t base = (uint64_t)tb * 64;
    int m = 4 + (int)(u01(seed, 3, base) * 3.0); /* 4..6 control points */
    double P[6][3];
    for (int i = 0; i < m; ++i)
      for (int k = 0; k < 3; ++k) P[i][k] = urange(seed, 3, base + 1 + 3 * i + k, 0.05, 0.95) * dims[k];
    double r = urange(seed, 3, base + 40, rmin, rmax);
    double I = urange(seed, 3, base + 41, imin, imax);
    for (int sgm = 0; sgm + 3 < m; ++sgm) {
      double len = 0.0, prev[3], cur[3];
      catmull(P[sgm], P[sgm + 1], P[sgm + 2], P[sgm + 3], 0.0, prev);
      for (int j = 1; j <= 64; ++j) {
        catmull(P[sgm], P[sgm + 1], P[sgm + 2], P[sgm + 3], j / 64.0, cur);
        len += sqrt((cur[0] - prev[0]) * (cur[0] - prev[0]) + (cur[1] - prev[1]) * (cur[1] - prev[1]) +
                    (cur[2] - prev[2]) * (cur[2] - prev[2]));
        memcpy(prev, cur, sizeof cur);
      }
      int steps = (int)ceil(len / 0.35) + 1;
      for (int j = 0; j <= steps; ++j) {
        catmull(P[sgm], P[sgm + 1], P[sgm + 2], P[sgm + 3], (double)j / steps, cur);
        if (n == cap) { cap *= 2; st = (stamp_t*)realloc(st, cap * sizeof(stamp_t)); }
        st[n].x = (float)cur[0]; st[n].y = (float)cur[1]; st[n].z = (float)cur[2];
        st[n].r = (float)r; st[n].I = (float)I;
        ++n;
      }
    }
  }
  qsort(st, n, sizeof(stamp_t), cmp_stamp_z);

  /* 2. Poisson background */
  double* cdf;
  int kmax = build_poisson_cdf(lambda, &cdf);
  const uint64_t plane = (uint64_t)nx * ny;
#pragma omp parallel for schedule(dynamic, 1)
  for (int z = 0; z < nz; ++z) {
    uint16_t* o = out + plane * z;
    for (uint64_t i = 0; i < plane; ++i) {
      int k = poisson_draw(cdf, kmax, u01(seed, 4, plane * z + i));
      o[i] = (uint16_t)(k > 65535 ? 65535 : k);
    }
  }
  free(cdf);

  /* 3. max-combine the tubes: value = I * clamp(r + 1 - dist, 0, 1), z-slabs in parallel */
  const int slab = 8;
  int nslab = (nz + slab - 1) / slab;
#pragma omp parallel for schedule(dynamic, 1)
  for (int s = 0; s < nslab; ++s) {
    int z0 = s * slab, z1 = z0 + slab < nz ? z0 + slab : nz;
    /* stamps sorted by z: find the first whose extent may reach z0 (r <= 7) */
    size_t lo = 0, hi = n;
    while (lo < hi) { size_t mid = (lo + hi) / 2; if (st[mid].z < z0 - 8.0f) lo = mid + 1; else hi = mid; }
    for (size_t q = lo; q < n && st[q].z <= z1 + 8.0f; ++q) {
      const stamp_t* p = &st[q];
      double R = p->r + 1.0;
      int xa = (int)floor(p->x - R - 0.5), xb = (int)ceil(p->x + R - 0.5);
      int ya = (int)floor(p->y - R - 0.5), yb = (int)ceil(p->y + R - 0.5);
      int za = (int)floor(p->z - R - 0.5), zb = (int)ceil(p->z + R - 0.5);
      if (xa < 0) xa = 0; if (ya < 0) ya = 0; if (za < z0) za = z0;
      if (xb > nx - 1) xb = nx - 1; if (yb > ny - 1) yb = ny - 1; if (zb > z1 - 1) zb = z1 - 1;
      for (int z = za; z <= zb; ++z)
        for (int y = ya; y <= yb; ++y)
          for (int x = xa; x <= xb; ++x) {
            double dx = x + 0.5 - p->x, dy = y + 0.5 - p->y, dz = z + 0.5 - p->z;
            double d = sqrt(dx * dx + dy * dy + dz * dz);
            double w = R - d;
            if (w <= 0.0) continue;
            if (w > 1.0) w = 1.0;
            double v = floor(p->I * w + 0.5);
            uint16_t* o = &out[plane * z + (uint64_t)y * nx + x];
            if (v > *o) *o = (uint16_t)(v > 65535.0 ? 65535.0 : v);
          }
    }
  }
  free(st);
  return (int)n;
}

/* --- configuration "batched 4D multichannel": drifting, growing Gaussian blobs, u16 --- */
void sy_blobs_u16(uint16_t* out, int nx, int ny, int nz, uint64_t seed, int channel, int t,
                  int nblobs, double noise_max) {
  double c[256][3], s[256], a[256];
  if (nblobs > 256) nblobs = 256;
  double dims[3] = {nx, ny, nz};
  uint64_t sd = seed * 1315423911ULL + (uint64_t)channel * 7919ULL;
  for (int b = 0; b < nblobs; ++b) {
    uint64_t base = (uint64_t)b * 16;
    double v[3], vn = 0.0;
    for (int k = 0; k < 3; ++k) { v[k] = urange(sd, 5, base + 3 + k, -1.0, 1.0); vn += v[k] * v[k]; }
    vn = sqrt(vn) + 1e-12;
    double speed = urange(sd, 5, base + 6, 1.0, 3.0);
    double growth = urange(sd, 5, base + 7, 0.01, 0.02);
    for (int k = 0; k < 3; ++k)
      c[b][k] = urange(sd, 5, base + k, 0.15, 0.85) * dims[k] + v[k] / vn * speed * t;
    s[b] = urange(sd, 5, base + 8, 4.0, 12.0) * pow(1.0 + growth, t);
    a[b] = urange(sd, 5, base + 9, 5000.0, 40000.0);
  }
  const uint64_t plane = (uint64_t)nx * ny;
  /* per z-slice: noise, then every blob whose 3.5 sigma ball reaches the slice */
#pragma omp parallel
  {
    double* acc = (double*)malloc(sizeof(double) * plane);
#pragma omp for schedule(dynamic, 4)
    for (int z = 0; z < nz; ++z) {
      for (uint64_t i = 0; i < plane; ++i) acc[i] = noise_max * u01(sd, 6 + (uint64_t)t * 131, plane * z + i);
      for (int b = 0; b < nblobs; ++b) {
        double lim = 3.5 * s[b], dz = z + 0.5 - c[b][2];
        if (fabs(dz) >= lim) continue;
        int x0 = (int)floor(c[b][0] - lim), x1 = (int)ceil(c[b][0] + lim);
        int y0 = (int)floor(c[b][1] - lim), y1 = (int)ceil(c[b][1] + lim);
        if (x0 < 0) x0 = 0; if (y0 < 0) y0 = 0;
        if (x1 > nx - 1) x1 = nx - 1; if (y1 > ny - 1) y1 = ny - 1;
        for (int y = y0; y <= y1; ++y)
          for (int x = x0; x <= x1; ++x) {
            double dx = x + 0.5 - c[b][0], dy = y + 0.5 - c[b][1];
            double r2 = dx * dx + dy * dy + dz * dz;
            if (r2 < lim * lim) acc[(uint64_t)y * nx + x] += a[b] * exp(-r2 / (2.0 * s[b] * s[b]));
          }
      }
      for (uint64_t i = 0; i < plane; ++i) {
        double r = floor(acc[i] + 0.5);
        out[plane * z + i] = (uint16_t)(r > 65535.0 ? 65535.0 : r);
      }
    }
    free(acc);
  }
}

/* --- configuration "large volume": jittered cell bodies with membrane shells, u8 ---
 * Procedural per voxel, so any box (coordinates clamped into the volume, which
 * replicates the edge as the bricks' aprons require) can be produced alone. */
static inline double gauss01(uint64_t seed, uint64_t idx) {
  double u1 = u01(seed, 8, idx), u2 = u01(seed, 9, idx);
  if (u1 < 1e-300) u1 = 1e-300;
  return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}
typedef struct { int present; double c[3], r, inner; } cell_t;
static void cell_params(uint64_t seed, int cs, long gx, long gy, long gz, long ng, cell_t* o) {
  uint64_t id = ((uint64_t)gz * ng + gy) * ng + gx;
  uint64_t b = id * 8;
  o->present = u01(seed, 7, b) < 0.6;
  double jit = cs * 0.25;
  o->c[0] = (gx + 0.5) * cs + urange(seed, 7, b + 1, -jit, jit);
  o->c[1] = (gy + 0.5) * cs + urange(seed, 7, b + 2, -jit, jit);
  o->c[2] = (gz + 0.5) * cs + urange(seed, 7, b + 3, -jit, jit);
  o->r = urange(seed, 7, b + 4, cs / 8.0, cs * 0.625);
  o->inner = urange(seed, 7, b + 5, 120.0, 160.0);
}
void sy_cells_u8_box(uint8_t* out, long N, uint64_t seed, long x0, long y0, long z0, int sx, int sy,
                     int sz, int cell) {
  long ng = (N + cell - 1) / cell;
#pragma omp parallel for schedule(static)
  for (int k = 0; k < sz; ++k) {
    long z = z0 + k; z = z < 0 ? 0 : (z > N - 1 ? N - 1 : z);
    for (int j = 0; j < sy; ++j) {
      long y = y0 + j; y = y < 0 ? 0 : (y > N - 1 ? N - 1 : y);
      long gy = y / cell, gz = z / cell;
      cell_t cc[3][3][3];
      long gx_cached = -1000;
      for (int i = 0; i < sx; ++i) {
        long x = x0 + i; x = x < 0 ? 0 : (x > N - 1 ? N - 1 : x);
        long gx = x / cell;
        if (gx != gx_cached) {
          for (int a = -1; a <= 1; ++a)
            for (int bb = -1; bb <= 1; ++bb)
              for (int c = -1; c <= 1; ++c) {
                long X = gx + c, Y = gy + bb, Z = gz + a;
                cell_t* o = &cc[a + 1][bb + 1][c + 1];
                if (X < 0 || Y < 0 || Z < 0 || X >= ng || Y >= ng || Z >= ng) { o->present = 0; continue; }
                cell_params(seed, cell, X, Y, Z, ng, o);
              }
          gx_cached = gx;
        }
        double v = 20.0;
        for (int q = 0; q < 27; ++q) {
          const cell_t* o = &((cell_t*)cc)[q];
          if (!o->present) continue;
          double dx = x + 0.5 - o->c[0], dy = y + 0.5 - o->c[1], dz = z + 0.5 - o->c[2];
          double d = sqrt(dx * dx + dy * dy + dz * dz);
          double w = d < o->r ? o->inner : (d < o->r + 2.0 ? 230.0 : 0.0);
          if (w > v) v = w;
        }
        uint64_t idx = ((uint64_t)z * N + y) * N + x;
        v += 8.0 * gauss01(seed, idx);
        double r = floor(v + 0.5);
        out[((size_t)k * sy + j) * sx + i] = (uint8_t)(r < 0 ? 0 : (r > 255 ? 255 : r));
      }
    }
  }
}

/* Parameters of every cell of the cell-body volume of edge N as float32, 8 per
 * cell (present, centre x/y/z, radius, interior value, 0, 0), cells x fastest
 * over a grid of ceil(N / cell)^3: the table the GPU generator reads. */
void sy_cell_table(float* out, long N, uint64_t seed, int cell) {
  long ng = (N + cell - 1) / cell;
#pragma omp parallel for schedule(static)
  for (long gz = 0; gz < ng; ++gz)
    for (long gy = 0; gy < ng; ++gy)
      for (long gx = 0; gx < ng; ++gx) {
        cell_t o;
        cell_params(seed, cell, gx, gy, gz, ng, &o);
        float* p = out + (((size_t)gz * ng + gy) * ng + gx) * 8;
        p[0] = (float)o.present;
        p[1] = (float)o.c[0];
        p[2] = (float)o.c[1];
        p[3] = (float)o.c[2];
        p[4] = (float)o.r;
        p[5] = (float)o.inner;
        p[6] = 0.0f;
        p[7] = 0.0f;
      }
}
