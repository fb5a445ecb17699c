// Brick container ("Volumetric Data Storage"): one file of LZ4-compressed
// chunks, one chunk per brick (with its apron) of every level, appended in
// any order. Every chunk has a header, so a conversion that stopped part
// way resumes after the last complete chunk; a finished file ends with an
// index table of chunk offsets and a footer. Layout (little endian):
//
//   file header  : "SGC1" u32 version, sg_volume_desc
//   chunk        : "CHNK" i32 t, c, level, bx, by, bz; u32 raw_bytes,
//                  comp_bytes, vmin, vmax; u32 checksum of the payload;
//                  payload (comp_bytes)
//   index        : per chunk i64 key (t, c, node), u64 offset of its header
//   footer       : "SGIX" u32 version, u64 index offset, u64 chunks
#include <stdio.h>
#include <string.h>
#include <unistd.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "internal.h"


using namespace sg;

namespace {

constexpr uint32_t kFileMagic = 0x31434753u;   // "SGC1"
constexpr uint32_t kChunkMagic = 0x4b4e4843u;  // "CHNK"
constexpr uint32_t kIndexMagic = 0x58494753u;  // "SGIX"
constexpr uint32_t kVersion = 1;

struct FileHeader {
  uint32_t magic, version;
  sg_volume_desc desc;
};

struct ChunkHeader {
  uint32_t magic;
  int32_t t, c, level, bx, by, bz;
  uint32_t raw_bytes, comp_bytes, vmin, vmax, checksum;
};

struct Footer {
  uint32_t magic, version;
  uint64_t index_offset, chunks;
};

// FNV-1a over the payload: detects a torn or overwritten chunk on resume
uint32_t checksum(const uint8_t* p, size_t n) {
  uint32_t h = 2166136261u;
  for (size_t i = 0; i < n; ++i) h = (h ^ p[i]) * 16777619u;
  return h;
}

struct Geometry {
  int levels = 0, B = 0, esize = 1, nch = 1, T = 1;
  int64_t nb[kMaxLevels][3] = {};
  int64_t off[kMaxLevels + 1] = {};
  int64_t nodes = 0;
  size_t raw_bytes = 0;  // one brick with its apron
};

Geometry geometry_of(const sg_volume_desc& d) {
  Geometry g;
  g.levels = d.lod_levels;
  g.B = d.brick_size;
  g.esize = d.dtype == SG_U8 ? 1 : 2;
  g.nch = d.channels;
  g.T = d.timepoints;
  int64_t dims[3] = {d.dims[0], d.dims[1], d.dims[2]};
  int64_t off = 0;
  for (int L = 0; L < g.levels; ++L) {
    for (int a = 0; a < 3; ++a) {
      g.nb[L][a] = (dims[a] + g.B - 1) / g.B;
      dims[a] = (dims[a] + 1) / 2;
    }
    g.off[L] = off;
    off += g.nb[L][0] * g.nb[L][1] * g.nb[L][2];
  }
  g.off[g.levels] = off;
  g.nodes = off;
  g.raw_bytes = (size_t)(g.B + 2) * (g.B + 2) * (g.B + 2) * g.esize;
  return g;
}

}  // namespace

struct sg_container {
  FILE* f = nullptr;
  std::string path;
  sg_volume_desc desc;
  Geometry g;
  bool writable = false, complete = false;
  std::map<int64_t, uint64_t> index;  // key (t, c, node) -> chunk header offset
  uint64_t end = 0;                   // append position
  uint64_t raw_total = 0, comp_total = 0;
  std::mutex m;                       // appends from several threads: write + index update

  int64_t key(int t, int c, int64_t node) const { return ((int64_t)t * g.nch + c) * g.nodes + node; }
};

namespace {

sg_status fail_io(const std::string& what) {
  set_error(what);
  return SG_ERR_IO;
}

bool read_at(FILE* f, uint64_t off, void* p, size_t n) {
  return fseeko(f, (off_t)off, SEEK_SET) == 0 && fread(p, 1, n, f) == n;
}

bool check_desc(const sg_volume_desc& d) {
  return d.dims[0] >= 1 && d.dims[1] >= 1 && d.dims[2] >= 1 && (d.dtype == SG_U8 || d.dtype == SG_U16) &&
         d.channels >= 1 && d.channels <= kMaxCh && d.timepoints >= 1 && d.brick_size >= 8 && d.brick_size <= 256 &&
         d.brick_size % 8 == 0 && d.lod_levels >= 1 && d.lod_levels <= kMaxLevels;
}

// Scans chunk headers from just after the file header; stops at the first
// chunk that is torn (short, bad magic or checksum) and returns the offset
// after the last complete one.
uint64_t scan_chunks(sg_container* k, uint64_t file_size) {
  uint64_t off = sizeof(FileHeader);
  std::vector<uint8_t> buf;
  while (off + sizeof(ChunkHeader) <= file_size) {
    ChunkHeader h;
    if (!read_at(k->f, off, &h, sizeof h) || h.magic != kChunkMagic) break;
    if (h.comp_bytes > lz4_bound(k->g.raw_bytes) || h.raw_bytes != k->g.raw_bytes) break;
    if (off + sizeof h + h.comp_bytes > file_size) break;
    buf.resize(h.comp_bytes);
    if (!read_at(k->f, off + sizeof h, buf.data(), h.comp_bytes) || checksum(buf.data(), h.comp_bytes) != h.checksum)
      break;
    if (h.level < 0 || h.level >= k->g.levels || h.t < 0 || h.t >= k->g.T || h.c < 0 || h.c >= k->g.nch) break;
    const int64_t node =
        k->g.off[h.level] + ((int64_t)h.bz * k->g.nb[h.level][1] + h.by) * k->g.nb[h.level][0] + h.bx;
    k->index[k->key(h.t, h.c, node)] = off;
    k->raw_total += h.raw_bytes;
    k->comp_total += h.comp_bytes;
    off += sizeof h + h.comp_bytes;
  }
  return off;
}

}  // namespace

extern "C" {

sg_status sg_container_create(const char* path, const sg_volume_desc* desc, sg_container** out) {
  return sg::guarded("sg_container_create", [&]() -> sg_status {
    if (!path || !desc || !out) {
      set_error("path, desc and out must not be NULL");
      return SG_ERR_INVALID_ARG;
    }
    *out = nullptr;
    if (!check_desc(*desc)) {
      set_error("invalid volume layout");
      return SG_ERR_INVALID_ARG;
    }
    sg_container* k = new (std::nothrow) sg_container();
    if (!k) {
      set_error("host allocation failed");
      return SG_ERR_OOM;
    }
    k->path = path;
    k->desc = *desc;
    k->g = geometry_of(*desc);
    k->f = fopen(path, "w+b");
    if (!k->f) {
      delete k;
      return fail_io(std::string("cannot create ") + path);
    }
    FileHeader h{kFileMagic, kVersion, *desc};
    if (fwrite(&h, sizeof h, 1, k->f) != 1 || fflush(k->f) != 0) {
      fclose(k->f);
      delete k;
      return fail_io("cannot write the container header");
    }
    k->writable = true;
    k->end = sizeof h;
    *out = k;
    return SG_OK;
  });
}

sg_status sg_container_open(const char* path, sg_container** out) {
  return sg::guarded("sg_container_open", [&]() -> sg_status {
    if (!path || !out) {
      set_error("path and out must not be NULL");
      return SG_ERR_INVALID_ARG;
    }
    *out = nullptr;
    sg_container* k = new (std::nothrow) sg_container();
    if (!k) {
      set_error("host allocation failed");
      return SG_ERR_OOM;
    }
    k->path = path;
    k->f = fopen(path, "r+b");
    if (!k->f) k->f = fopen(path, "rb");
    if (!k->f) {
      delete k;
      return fail_io(std::string("cannot open ") + path);
    }
    FileHeader h;
    if (!read_at(k->f, 0, &h, sizeof h) || h.magic != kFileMagic || h.version != kVersion || !check_desc(h.desc)) {
      fclose(k->f);
      delete k;
      return fail_io("not a brick container (bad header)");
    }
    k->desc = h.desc;
    k->g = geometry_of(h.desc);
    fseeko(k->f, 0, SEEK_END);
    const uint64_t size = (uint64_t)ftello(k->f);
    Footer ft;
    bool indexed = false;
    if (size >= sizeof(FileHeader) + sizeof ft && read_at(k->f, size - sizeof ft, &ft, sizeof ft) &&
        ft.magic == kIndexMagic && ft.version == kVersion && ft.index_offset + ft.chunks * 16 + sizeof ft == size) {
      std::vector<int64_t> rec(2 * ft.chunks);
      if (ft.chunks == 0 || read_at(k->f, ft.index_offset, rec.data(), rec.size() * sizeof(int64_t))) {
        for (uint64_t i = 0; i < ft.chunks; ++i) k->index[rec[2 * i]] = (uint64_t)rec[2 * i + 1];
        for (auto& e : k->index) {
          ChunkHeader ch;
          if (read_at(k->f, e.second, &ch, sizeof ch)) {
            k->raw_total += ch.raw_bytes;
            k->comp_total += ch.comp_bytes;
          }
        }
        k->complete = true;
        k->end = ft.index_offset;
        indexed = true;
      }
    }
    if (!indexed) {
      // an interrupted conversion: keep every complete chunk, cut off a torn
      // one, resume appending after them
      k->end = scan_chunks(k, size);
      fflush(k->f);
      if (k->end < size && ftruncate(fileno(k->f), (off_t)k->end) != 0) {
        fclose(k->f);
        delete k;
        return fail_io("cannot cut the torn chunk off the container");
      }
      k->writable = true;
    }
    *out = k;
    return SG_OK;
  });
}

sg_status sg_container_append(sg_container* k, int t, int c, int level, int bx, int by, int bz, const void* brick,
                              uint32_t vmin, uint32_t vmax) {
  return sg::guarded("sg_container_append", [&]() -> sg_status {
    if (!k || !brick) {
      set_error("container or brick NULL");
      return SG_ERR_INVALID_ARG;
    }
    if (!k->writable || k->complete) {
      set_error("sg_container_append: the container is finished (read only)");
      return SG_ERR_STATE;
    }
    if (t < 0 || t >= k->g.T || c < 0 || c >= k->g.nch || level < 0 || level >= k->g.levels || bx < 0 || by < 0 ||
        bz < 0 || bx >= k->g.nb[level][0] || by >= k->g.nb[level][1] || bz >= k->g.nb[level][2]) {
      set_error("sg_container_append: brick coordinates out of range");
      return SG_ERR_INVALID_ARG;
    }
    // compression runs outside the lock, so appends from several threads
    // compress in parallel and only the write is serialised
    std::vector<uint8_t> comp(lz4_bound(k->g.raw_bytes));
    const size_t cs = lz4_compress(static_cast<const uint8_t*>(brick), k->g.raw_bytes, comp.data());
    ChunkHeader h{kChunkMagic, t, c, level, bx, by, bz, (uint32_t)k->g.raw_bytes, (uint32_t)cs, vmin, vmax,
                  checksum(comp.data(), cs)};
    std::lock_guard<std::mutex> lock(k->m);
    if (k->complete) {
      set_error("sg_container_append: the container is finished (read only)");
      return SG_ERR_STATE;
    }
    if (fseeko(k->f, (off_t)k->end, SEEK_SET) != 0 || fwrite(&h, sizeof h, 1, k->f) != 1 ||
        fwrite(comp.data(), 1, cs, k->f) != cs || fflush(k->f) != 0)
      return fail_io("sg_container_append: write failed");
    const int64_t node = k->g.off[level] + ((int64_t)bz * k->g.nb[level][1] + by) * k->g.nb[level][0] + bx;
    k->index[k->key(t, c, node)] = k->end;
    k->end += sizeof h + cs;
    k->raw_total += k->g.raw_bytes;
    k->comp_total += cs;
    return SG_OK;
  });
}

sg_status sg_container_finish(sg_container* k) {
  return sg::guarded("sg_container_finish", [&]() -> sg_status {
    if (!k) {
      set_error("container NULL");
      return SG_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> lock(k->m);
    if (k->complete) return SG_OK;
    std::vector<int64_t> rec;
    rec.reserve(2 * k->index.size());
    for (auto& e : k->index) {
      rec.push_back(e.first);
      rec.push_back((int64_t)e.second);
    }
    Footer ft{kIndexMagic, kVersion, k->end, (uint64_t)k->index.size()};
    if (fseeko(k->f, (off_t)k->end, SEEK_SET) != 0 ||
        (!rec.empty() && fwrite(rec.data(), sizeof(int64_t), rec.size(), k->f) != rec.size()) ||
        fwrite(&ft, sizeof ft, 1, k->f) != 1 || fflush(k->f) != 0)
      return fail_io("sg_container_finish: write failed");
    k->complete = true;
    return SG_OK;
  });
}

sg_status sg_container_get_info(sg_container* k, sg_container_info* info) {
  if (!k || !info) {
    set_error("container or info NULL");
    return SG_ERR_INVALID_ARG;
  }
  memset(info, 0, sizeof *info);
  info->desc = k->desc;
  info->chunks = (int64_t)k->index.size();
  info->nodes = k->g.nodes;
  info->raw_bytes = k->raw_total;
  info->compressed_bytes = k->comp_total;
  info->complete = k->complete ? 1 : 0;
  return SG_OK;
}

sg_status sg_container_read(sg_container* k, int t, int c, int64_t node, void* out, uint32_t* minmax) {
  return sg::guarded("sg_container_read", [&]() -> sg_status {
    if (!k || !out) {
      set_error("container or output NULL");
      return SG_ERR_INVALID_ARG;
    }
    if (t < 0 || t >= k->g.T || c < 0 || c >= k->g.nch || node < 0 || node >= k->g.nodes) {
      set_error("sg_container_read: (t, c, node) out of range");
      return SG_ERR_INVALID_ARG;
    }
    auto it = k->index.find(k->key(t, c, node));
    if (it == k->index.end()) {
      set_error("sg_container_read: no chunk for this brick");
      return SG_ERR_NOT_RESIDENT;
    }
    return container_read_chunk(k, it->second, out, minmax, nullptr);
  });
}

sg_status sg_container_close(sg_container* k) {
  if (!k) return SG_OK;
  if (k->f) fclose(k->f);
  delete k;
  return SG_OK;
}

}  // extern "C"

namespace sg {

// Reads and decompresses the chunk whose header is at offset off; thread
// safe (positioned reads on the file descriptor, no shared file position).
sg_status container_read_chunk(sg_container* k, uint64_t off, void* out, uint32_t* minmax, uint32_t* comp_bytes) {
  ChunkHeader h;
  const int fd = fileno(k->f);
  if (pread(fd, &h, sizeof h, (off_t)off) != (ssize_t)sizeof h || h.magic != kChunkMagic ||
      h.raw_bytes != k->g.raw_bytes || h.comp_bytes > lz4_bound(k->g.raw_bytes)) {
    set_error("container: bad chunk header");
    return SG_ERR_IO;
  }
  std::vector<uint8_t> comp(h.comp_bytes);
  if (pread(fd, comp.data(), h.comp_bytes, (off_t)(off + sizeof h)) != (ssize_t)h.comp_bytes) {
    set_error("container: short chunk read");
    return SG_ERR_IO;
  }
  if (checksum(comp.data(), h.comp_bytes) != h.checksum ||
      !lz4_decompress(comp.data(), h.comp_bytes, static_cast<uint8_t*>(out), h.raw_bytes)) {
    set_error("container: corrupt chunk");
    return SG_ERR_IO;
  }
  if (minmax) {
    minmax[0] = h.vmin;
    minmax[1] = h.vmax;
  }
  if (comp_bytes) *comp_bytes = h.comp_bytes;
  return SG_OK;
}

const sg_volume_desc& container_desc(const sg_container* k) { return k->desc; }
uint64_t container_chunk_offset(const sg_container* k, int t, int c, int64_t node, bool* found) {
  auto it = k->index.find(k->key(t, c, node));
  *found = it != k->index.end();
  return *found ? it->second : 0;
}
size_t container_brick_bytes(const sg_container* k) { return k->g.raw_bytes; }
int64_t container_nodes(const sg_container* k) { return k->g.nodes; }

}  // namespace sg
