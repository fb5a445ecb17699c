// Host-memory brick cache between a container and a volume's GPU brick cache
// ("Volumetric Data Cashing": a CPU cache and a GPU cache, each keeping as
// many chunks as fit and dropping the least recently used, by timestamp).
// sg_stream_requests serves one selection's requests: coarse levels first,
// each brick from the host cache or, on a miss, read from the container and
// LZ4-decompressed by a pool of threads, then placed in the GPU cache by one
// list upload per channel. sg_stream_requests_async serves the requests the
// host cache already holds and hands the misses to background loader
// threads without waiting for the disk: until a brick arrives, the
// selection keeps rendering its resident ancestor ("Octree
// Representation"), so a frame never stalls on a read.
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <set>
#include <string>
#include <thread>
#include <utility>
#include <vector>

#include "internal.h"

using namespace sg;

struct sg_host_cache {
  sg_container* k = nullptr;
  uint8_t* arena = nullptr;
  bool pinned = false;
  size_t entry_bytes = 0;
  int64_t entries = 0;
  int threads = 1;
  uint64_t frame = 0;
  std::map<int64_t, int64_t> where;           // key (t, c, node) -> entry
  std::vector<int64_t> owner;                 // entry -> key or -1
  std::vector<uint64_t> stamp;                // entry -> frame of last use
  std::set<std::pair<uint64_t, int64_t>> lru;  // (stamp, entry) of occupied entries
  std::vector<int64_t> free_list;
  std::set<int64_t> failed;                    // keys whose chunk failed to read or decompress
  // background loading: an entry being loaded is in neither the LRU set nor
  // the free list (nothing evicts it) and counts as absent until collected
  std::vector<uint8_t> loading;                // entry -> 1 while its chunk is being loaded
  std::mutex mu;                               // guards jobs, done, stop, in_flight
  std::condition_variable cv_job, cv_done;
  std::deque<std::pair<int64_t, int64_t>> jobs;  // (entry, chunk offset) queued
  std::vector<std::pair<int64_t, uint32_t>> done;  // (entry, compressed bytes; 0 = failed) loaded, not collected
  int64_t in_flight = 0;                       // queued + being loaded
  bool stop = false;
  std::vector<std::thread> loaders;            // started on first use
  // the copies of recent sg_stream_requests_async calls may still be
  // reading entries, those stamped copies_frame or later: such an entry is
  // neither reused nor freed before this event (recorded after the last of
  // them, and covering the earlier ones) has passed
  cudaEvent_t ev_copies = nullptr;
  bool copies_pending = false;
  uint64_t copies_frame = 0;
};

extern "C" {

sg_status sg_host_cache_create(sg_container* k, uint64_t bytes, int pinned, int threads, sg_host_cache** out) {
  return sg::guarded("sg_host_cache_create", [&]() -> sg_status {
    if (!k || !out) {
      set_error("container and out must not be NULL");
      return SG_ERR_INVALID_ARG;
    }
    *out = nullptr;
    const size_t eb = container_brick_bytes(k);
    if (bytes < eb || threads < 1 || threads > 256) {
      set_error("host cache: at least one brick of bytes, 1..256 threads");
      return SG_ERR_INVALID_ARG;
    }
    sg_host_cache* hc = new (std::nothrow) sg_host_cache();
    if (!hc) {
      set_error("host allocation failed");
      return SG_ERR_OOM;
    }
    hc->k = k;
    hc->entry_bytes = eb;
    hc->entries = (int64_t)(bytes / eb);
    hc->threads = threads;
    const size_t total = (size_t)hc->entries * eb;
    if (pinned) {
      if (cudaHostAlloc(reinterpret_cast<void**>(&hc->arena), total, cudaHostAllocDefault) != cudaSuccess) {
        delete hc;
        set_error("host cache: page-locked allocation failed");
        return SG_ERR_OOM;
      }
      hc->pinned = true;
    } else {
      hc->arena = static_cast<uint8_t*>(malloc(total));
      if (!hc->arena) {
        delete hc;
        set_error("host cache: allocation failed");
        return SG_ERR_OOM;
      }
    }
    hc->owner.assign(hc->entries, -1);
    hc->stamp.assign(hc->entries, 0);
    hc->loading.assign(hc->entries, 0);
    for (int64_t i = hc->entries - 1; i >= 0; --i) hc->free_list.push_back(i);
    *out = hc;
    return SG_OK;
  });
}

sg_status sg_host_cache_destroy(sg_host_cache* hc) {
  if (!hc) return SG_OK;
  {
    std::lock_guard<std::mutex> g(hc->mu);
    hc->stop = true;
  }
  hc->cv_job.notify_all();
  for (auto& th : hc->loaders) th.join();
  host_cache_quiesce(hc);
  if (hc->ev_copies) cudaEventDestroy(hc->ev_copies);
  if (hc->pinned)
    cudaFreeHost(hc->arena);
  else
    free(hc->arena);
  delete hc;
  return SG_OK;
}

sg_status sg_host_cache_clear_failures(sg_host_cache* hc) {
  if (!hc) {
    set_error("cache NULL");
    return SG_ERR_INVALID_ARG;
  }
  hc->failed.clear();
  return SG_OK;
}

sg_status sg_host_cache_fetch(sg_host_cache* hc, int t, int c, int64_t node, const void** brick, int* hit) {
  return sg::guarded("sg_host_cache_fetch", [&]() -> sg_status {
    if (!hc || !brick) {
      set_error("cache or output NULL");
      return SG_ERR_INVALID_ARG;
    }
    host_cache_quiesce(hc);
    host_cache_drain(hc);
    ++hc->frame;
    std::vector<std::pair<int64_t, int64_t>> todo;  // (entry, chunk offset)
    int64_t entry = -1;
    sg_status st = host_cache_lookup(hc, t, c, node, &entry, hit, &todo);
    if (st != SG_OK) return st;
    if (!todo.empty()) {
      st = container_read_chunk(hc->k, (uint64_t)todo[0].second, hc->arena + (size_t)entry * hc->entry_bytes, nullptr,
                                nullptr);
      if (st != SG_OK) {
        host_cache_drop(hc, entry);
        return st;
      }
    }
    *brick = hc->arena + (size_t)entry * hc->entry_bytes;
    return SG_OK;
  });
}

}  // extern "C"

namespace sg {

// Finds or places (t, c, node) in the host cache, stamping it with the
// current frame (*hit: 1 held, 0 newly placed, 2 being loaded in the
// background). A new entry comes from the free list, else from the least
// recently used entry not used this frame; its chunk offset is queued in
// todo for loading. SG_ERR_NOT_RESIDENT: no chunk in the container;
// SG_ERR_OOM: every entry is in use this frame or being loaded.
sg_status host_cache_lookup(sg_host_cache* hc, int t, int c, int64_t node, int64_t* entry, int* hit,
                            std::vector<std::pair<int64_t, int64_t>>* todo) {
  const sg_volume_desc& d = container_desc(hc->k);
  const int64_t nodes = container_nodes(hc->k);
  const int64_t key = ((int64_t)t * d.channels + c) * nodes + node;
  auto it = hc->where.find(key);
  if (it != hc->where.end()) {
    const int64_t e = it->second;
    if (hc->loading[e]) {  // on its way: stays out of the LRU set until collected
      hc->stamp[e] = hc->frame;
      *entry = e;
      if (hit) *hit = 2;
      return SG_OK;
    }
    hc->lru.erase({hc->stamp[e], e});
    hc->stamp[e] = hc->frame;
    hc->lru.insert({hc->frame, e});
    *entry = e;
    if (hit) *hit = 1;
    return SG_OK;
  }
  bool found = false;
  const uint64_t off = container_chunk_offset(hc->k, t, c, node, &found);
  if (!found) {
    set_error("host cache: the container has no chunk for this brick");
    return SG_ERR_NOT_RESIDENT;
  }
  int64_t e;
  if (!hc->free_list.empty()) {
    e = hc->free_list.back();
    hc->free_list.pop_back();
  } else {
    auto lo = hc->lru.begin();
    if (lo == hc->lru.end() || lo->first >= hc->frame) {
      set_error("host cache: full of bricks used by the current frame");
      return SG_ERR_OOM;
    }
    // the entry may be the source of a copy still in flight
    if (hc->copies_pending && lo->first >= hc->copies_frame) host_cache_quiesce(hc);
    e = lo->second;
    hc->lru.erase(lo);
    hc->where.erase(hc->owner[e]);
  }
  hc->owner[e] = key;
  hc->where[key] = e;
  hc->stamp[e] = hc->frame;
  hc->lru.insert({hc->frame, e});
  todo->push_back({e, (int64_t)off});
  *entry = e;
  if (hit) *hit = 0;
  return SG_OK;
}

void host_cache_drop(sg_host_cache* hc, int64_t e) {
  hc->lru.erase({hc->stamp[e], e});
  hc->where.erase(hc->owner[e]);
  hc->owner[e] = -1;
  hc->loading[e] = 0;
  hc->free_list.push_back(e);
}

namespace {

// loader thread: reads + decompresses queued chunks into their entries
void loader_main(sg_host_cache* hc) {
  for (;;) {
    std::pair<int64_t, int64_t> job;
    {
      std::unique_lock<std::mutex> g(hc->mu);
      hc->cv_job.wait(g, [&] { return hc->stop || !hc->jobs.empty(); });
      if (hc->stop) return;
      job = hc->jobs.front();
      hc->jobs.pop_front();
    }
    uint32_t comp = 0;
    const sg_status st = container_read_chunk(hc->k, (uint64_t)job.second,
                                              hc->arena + (size_t)job.first * hc->entry_bytes, nullptr, &comp);
    {
      std::lock_guard<std::mutex> g(hc->mu);
      hc->done.push_back({job.first, st == SG_OK ? std::max<uint32_t>(comp, 1u) : 0u});
      --hc->in_flight;
    }
    hc->cv_done.notify_all();
  }
}

// queues the reads of newly placed entries on the loader threads
void host_cache_enqueue(sg_host_cache* hc, const std::vector<std::pair<int64_t, int64_t>>& todo) {
  if (todo.empty()) return;
  // out of the LRU set while loading (host_cache_lookup placed them there):
  // nothing may evict an entry a loader is writing; collect puts it back
  for (auto& j : todo) {
    hc->lru.erase({hc->stamp[j.first], j.first});
    hc->loading[j.first] = 1;
  }
  {
    std::lock_guard<std::mutex> g(hc->mu);
    for (auto& j : todo) hc->jobs.push_back(j);
    hc->in_flight += (int64_t)todo.size();
  }
  while ((int)hc->loaders.size() < hc->threads) {
    try {
      hc->loaders.emplace_back(loader_main, hc);
    } catch (...) {  // no thread to be had: fewer loaders (or none, below)
      break;
    }
  }
  if (hc->loaders.empty()) {
    // no loader could start: read the queue here, so that no wait can hang
    for (;;) {
      std::pair<int64_t, int64_t> job;
      {
        std::lock_guard<std::mutex> g(hc->mu);
        if (hc->jobs.empty()) break;
        job = hc->jobs.front();
        hc->jobs.pop_front();
      }
      uint32_t comp = 0;
      const sg_status st = container_read_chunk(hc->k, (uint64_t)job.second,
                                                hc->arena + (size_t)job.first * hc->entry_bytes, nullptr, &comp);
      std::lock_guard<std::mutex> g(hc->mu);
      hc->done.push_back({job.first, st == SG_OK ? std::max<uint32_t>(comp, 1u) : 0u});
      --hc->in_flight;
    }
    return;
  }
  hc->cv_job.notify_all();
}

}  // namespace

// Takes in the loads finished so far (waiting for all of them first if
// wait): a loaded entry joins the LRU set, a failed one is dropped and its
// key remembered. Adds the reads and bytes taken in to *reads, *bytes and
// the failures to *failed (each optional).
void host_cache_collect(sg_host_cache* hc, bool wait, int32_t* reads, uint64_t* bytes, int32_t* failed) {
  std::vector<std::pair<int64_t, uint32_t>> got;
  {
    std::unique_lock<std::mutex> g(hc->mu);
    if (wait) hc->cv_done.wait(g, [&] { return hc->in_flight == 0; });
    got.swap(hc->done);
  }
  for (auto& d : got) {
    const int64_t e = d.first;
    if (d.second) {
      hc->loading[e] = 0;
      hc->lru.insert({hc->stamp[e], e});
      if (reads) ++*reads;
      if (bytes) *bytes += d.second;
    } else {
      hc->failed.insert(hc->owner[e]);
      host_cache_drop(hc, e);
      if (failed) ++*failed;
    }
  }
}

void host_cache_drain(sg_host_cache* hc) { host_cache_collect(hc, true, nullptr, nullptr, nullptr); }

void host_cache_quiesce(sg_host_cache* hc) {
  if (hc->copies_pending) {
    cudaEventSynchronize(hc->ev_copies);
    hc->copies_pending = false;
  }
}

void host_cache_poll(sg_host_cache* hc) {
  if (hc->copies_pending && cudaEventQuery(hc->ev_copies) == cudaSuccess) hc->copies_pending = false;
}

}  // namespace sg

namespace {

sg_status stream_impl(sg_volume* v, int slot, sg_host_cache* hc, uint64_t max_bytes, sg_stream_stats* stats,
                      void* stream, bool async, const char* name) {
  NvtxRange nvtx_range(name);
  if (!v || !hc || slot < 0 || slot >= kMaxSlots) {
    set_error("volume/cache NULL or slot out of range");
    return SG_ERR_INVALID_ARG;
  }
  const sg_volume_desc& d = container_desc(hc->k);
  if (d.dims[0] != v->desc.dims[0] || d.dims[1] != v->desc.dims[1] || d.dims[2] != v->desc.dims[2] ||
      d.dtype != v->desc.dtype || d.brick_size != v->B || d.lod_levels != v->levels || d.channels != v->nch ||
      d.timepoints > v->T) {
    set_error(std::string(name) + ": the container's layout differs from the volume's");
    return SG_ERR_INVALID_ARG;
  }
  sg_stream_stats s0;
  memset(&s0, 0, sizeof s0);
  const SelSlot& sl = v->sel[slot];
  if (!sl.valid) {
    set_error(std::string(name) + ": slot was never selected");
    return SG_ERR_STATE;
  }
  const int t = sl.t;
  // entries that earlier calls' copies may still read: the blocking path
  // waits for those copies here, the asynchronous one only where it would
  // reuse such an entry (in host_cache_lookup)
  if (async)
    host_cache_poll(hc);
  else
    host_cache_quiesce(hc);
  std::vector<int32_t> req((size_t)v->nodes);
  int32_t nreq = 0;
  // read on a stream of its own, which waits for the selection alone and
  // not for copies already queued on the caller's stream
  cudaStream_t rs = side_stream(v);
  sg_status st = sg_read_selection(v, slot, nullptr, 0, nullptr, 0, req.data(), (int32_t)req.size(), &nreq,
                                   rs ? (void*)rs : stream);
  if (st != SG_OK) return st;
  req.resize((size_t)std::min<int64_t>(nreq, (int64_t)req.size()));
  s0.requested = (int32_t)req.size();
  // coarse levels first (a parent before its children), then node id
  auto level_of = [&](int32_t n) {
    int L = 0;
    while (L + 1 < v->levels && n >= v->geom[L + 1].off) ++L;
    return L;
  };
  std::stable_sort(req.begin(), req.end(), [&](int32_t a, int32_t b) {
    const int la = level_of(a), lb = level_of(b);
    return la != lb ? la > lb : a < b;
  });
  const uint64_t per_node = (uint64_t)hc->entry_bytes * v->nch;
  const size_t budget = per_node ? (size_t)std::min<uint64_t>(max_bytes / per_node, req.size()) : 0;
  const sg_volume_desc& kd = container_desc(hc->k);
  const int64_t knodes = container_nodes(hc->k);
  auto key_of = [&](int c, int32_t node) { return ((int64_t)t * kd.channels + c) * knodes + node; };
  std::vector<int32_t> nodes;
  std::vector<std::vector<const void*>> ptrs(v->nch);
  if (async) {
    // loads finished since the last call join the cache (failures are remembered)
    int32_t late_fail = 0;
    host_cache_collect(hc, false, &s0.disk_reads, &s0.disk_bytes, &late_fail);
    s0.failed += late_fail;
    ++hc->frame;
    // requests held in the host cache are uploaded (at most budget bricks);
    // misses are handed to the loaders (at most budget bricks a call)
    std::vector<std::pair<int64_t, int64_t>> todo;
    size_t loads = 0;
    bool full = false;
    for (size_t i = 0; i < req.size() && (nodes.size() < budget || (loads < budget && !full)); ++i) {
      const int32_t node = req[i];
      bool bad = false;
      for (int c = 0; c < v->nch && !bad; ++c) bad = hc->failed.count(key_of(c, node)) > 0;
      if (bad) {
        ++s0.failed;
        continue;
      }
      const bool may_load = loads < budget && !full;
      std::vector<int64_t> ent(v->nch);
      bool ok = true, pending = false;
      sg_status lst = SG_OK;
      const size_t todo_mark = todo.size();
      for (int c = 0; c < v->nch && ok; ++c) {
        if (!may_load && hc->where.find(key_of(c, node)) == hc->where.end()) {
          pending = true;  // would need a load this call has no budget for
          continue;
        }
        int hit = 0;
        lst = host_cache_lookup(hc, t, c, node, &ent[c], &hit, &todo);
        if (lst == SG_ERR_NOT_RESIDENT) {
          ++s0.missing;
          ok = false;
        } else if (lst == SG_ERR_OOM) {
          ok = false;
        } else if (lst != SG_OK) {
          return lst;
        } else if (hit == 1) {
          ++s0.host_hits;
        } else {
          pending = true;
        }
      }
      if (!ok) {
        while (todo.size() > todo_mark) {
          host_cache_drop(hc, todo.back().first);
          todo.pop_back();
        }
        if (lst == SG_ERR_OOM) full = true;
        continue;
      }
      if (todo.size() > todo_mark) ++loads;
      if (pending || nodes.size() >= budget) continue;
      nodes.push_back(node);
      for (int c = 0; c < v->nch; ++c) ptrs[c].push_back(hc->arena + (size_t)ent[c] * hc->entry_bytes);
    }
    host_cache_enqueue(hc, todo);
    s0.queued = (int32_t)todo.size();
    {
      std::lock_guard<std::mutex> g(hc->mu);
      s0.in_flight = (int32_t)hc->in_flight;
    }
  } else {
    host_cache_drain(hc);
    ++hc->frame;
    // place every (node, channel) of the budget in the host cache; a brick
    // whose chunk failed before is skipped without spending budget
    std::vector<std::pair<int64_t, int64_t>> todo;
    std::vector<size_t> todo_node;  // index into nodes of each queued read
    for (size_t i = 0; i < req.size() && nodes.size() < budget; ++i) {
      const int32_t node = req[i];
      bool bad = false;
      for (int c = 0; c < v->nch && !bad; ++c) bad = hc->failed.count(key_of(c, node)) > 0;
      if (bad) {
        ++s0.failed;
        continue;
      }
      std::vector<int64_t> ent(v->nch);
      bool ok = true;
      size_t todo_mark = todo.size();
      for (int c = 0; c < v->nch && ok; ++c) {
        int hit = 0;
        st = host_cache_lookup(hc, t, c, node, &ent[c], &hit, &todo);
        if (st == SG_ERR_NOT_RESIDENT) {
          ++s0.missing;
          ok = false;
        } else if (st == SG_ERR_OOM) {
          ok = false;
        } else if (st != SG_OK) {
          return st;
        } else if (hit) {
          ++s0.host_hits;
        }
      }
      if (!ok) {
        // undo the entries queued for this node; stop at a full cache
        while (todo.size() > todo_mark) {
          host_cache_drop(hc, todo.back().first);
          todo.pop_back();
        }
        if (st == SG_ERR_OOM) break;
        continue;
      }
      while (todo_node.size() < todo.size()) todo_node.push_back(nodes.size());
      nodes.push_back(node);
      for (int c = 0; c < v->nch; ++c) ptrs[c].push_back(hc->arena + (size_t)ent[c] * hc->entry_bytes);
    }
    // read + decompress the misses on a pool of threads
    std::atomic<size_t> next(0);
    std::vector<uint8_t> fail(todo.size(), 0);
    std::atomic<uint64_t> disk_bytes(0);
    auto work = [&]() {
      for (;;) {
        const size_t i = next.fetch_add(1);
        if (i >= todo.size()) return;
        uint32_t comp = 0;
        if (container_read_chunk(hc->k, (uint64_t)todo[i].second, hc->arena + (size_t)todo[i].first * hc->entry_bytes,
                                 nullptr, &comp) != SG_OK)
          fail[i] = 1;
        disk_bytes.fetch_add(comp);
      }
    };
    const int nt = (int)std::min<size_t>((size_t)hc->threads, todo.size());
    std::vector<std::thread> pool;
    for (int i = 1; i < nt; ++i) {
      try {
        pool.emplace_back(work);
      } catch (...) {  // no more threads: the calling thread reads the rest
        break;
      }
    }
    if (nt >= 1) work();
    for (auto& th : pool) th.join();
    // a failed chunk: its entry is dropped, its key remembered, and its brick
    // (every channel) left out of the upload, so it stays non-resident and
    // its parent keeps rendering; the other bricks are served
    int32_t nfail = 0;
    std::vector<uint8_t> drop(nodes.size(), 0);
    for (size_t i = 0; i < todo.size(); ++i)
      if (fail[i]) {
        const int64_t key = hc->owner[todo[i].first];
        hc->failed.insert(key);
        host_cache_drop(hc, todo[i].first);
        drop[todo_node[i]] = 1;
        ++nfail;
      }
    if (nfail) {
      size_t w = 0;
      for (size_t i = 0; i < nodes.size(); ++i) {
        if (drop[i]) {
          ++s0.failed;
          continue;
        }
        nodes[w] = nodes[i];
        for (int c = 0; c < v->nch; ++c) ptrs[c][w] = ptrs[c][i];
        ++w;
      }
      nodes.resize(w);
      for (int c = 0; c < v->nch; ++c) ptrs[c].resize(w);
    }
    s0.disk_reads = (int32_t)todo.size() - nfail;
    s0.disk_bytes = disk_bytes.load();
  }
  // one list upload per channel (the first places the slots)
  int32_t placed = (int32_t)nodes.size();
  for (int c = 0; c < v->nch && !nodes.empty(); ++c) {
    int32_t done = 0;
    // asynchronous: queued, not waited for (later selections wait on the device)
    st = async ? upload_list_nowait(v, t, c, placed, nodes.data(), ptrs[c].data(), &done, (cudaStream_t)stream)
               : sg_upload_brick_list(v, t, c, placed, nodes.data(), ptrs[c].data(), &done, stream);
    if (st != SG_OK) return st;
    placed = std::min(placed, done);
  }
  if (async && !nodes.empty()) {
    // the event, recorded after this call's copies, also covers copies of
    // earlier calls still pending (on whatever stream): the stream waits
    // for the previous event before the new one is recorded
    cudaStream_t s = (cudaStream_t)stream;
    if (!hc->ev_copies && cudaEventCreateWithFlags(&hc->ev_copies, cudaEventDisableTiming) != cudaSuccess) {
      cudaStreamSynchronize(s);  // no event to be had: wait here instead
    } else if ((!hc->copies_pending || cudaStreamWaitEvent(s, hc->ev_copies, 0) == cudaSuccess) &&
               cudaEventRecord(hc->ev_copies, s) == cudaSuccess) {
      if (!hc->copies_pending) hc->copies_frame = hc->frame;
      hc->copies_pending = true;
    } else {
      cudaStreamSynchronize(s);
      host_cache_quiesce(hc);
    }
  }
  s0.served = placed;
  s0.upload_bytes = (uint64_t)placed * per_node;
  if (stats) *stats = s0;
  if (s0.failed) {
    set_error(std::string(name) + ": " + std::to_string(s0.failed) +
              " requested bricks have a chunk that failed to read or decompress; the others were served");
    return SG_ERR_IO;
  }
  return SG_OK;
}

}  // namespace

extern "C" {

sg_status sg_stream_requests(sg_volume* v, int slot, sg_host_cache* hc, uint64_t max_bytes, sg_stream_stats* stats,
                             void* stream) {
  return sg::guarded("sg_stream_requests", [&]() -> sg_status {
    return stream_impl(v, slot, hc, max_bytes, stats, stream, false, "sg_stream_requests");
  });
}

sg_status sg_stream_requests_async(sg_volume* v, int slot, sg_host_cache* hc, uint64_t max_bytes,
                                   sg_stream_stats* stats, void* stream) {
  return sg::guarded("sg_stream_requests_async", [&]() -> sg_status {
    return stream_impl(v, slot, hc, max_bytes, stats, stream, true, "sg_stream_requests_async");
  });
}

sg_status sg_host_cache_prefetch(sg_host_cache* hc, int t, int c, const int64_t* nodes, int32_t n, int32_t* queued) {
  return sg::guarded("sg_host_cache_prefetch", [&]() -> sg_status {
    if (!hc || (n > 0 && !nodes) || n < 0) {
      set_error("sg_host_cache_prefetch: cache or nodes NULL, or n < 0");
      return SG_ERR_INVALID_ARG;
    }
    const sg_volume_desc& d = container_desc(hc->k);
    if (t < 0 || t >= d.timepoints || c < 0 || c >= d.channels) {
      set_error("sg_host_cache_prefetch: time point or channel out of range");
      return SG_ERR_INVALID_ARG;
    }
    host_cache_quiesce(hc);
    host_cache_collect(hc, false, nullptr, nullptr, nullptr);
    ++hc->frame;
    std::vector<std::pair<int64_t, int64_t>> todo;
    sg_status st = SG_OK;
    for (int32_t i = 0; i < n; ++i) {
      if (nodes[i] < 0 || nodes[i] >= container_nodes(hc->k)) {
        st = SG_ERR_INVALID_ARG;
        set_error("sg_host_cache_prefetch: node id out of range");
        break;
      }
      const int64_t key = ((int64_t)t * d.channels + c) * container_nodes(hc->k) + nodes[i];
      if (hc->failed.count(key)) continue;
      int64_t e = -1;
      int hit = 0;
      const sg_status s1 = host_cache_lookup(hc, t, c, nodes[i], &e, &hit, &todo);
      if (s1 == SG_ERR_NOT_RESIDENT) continue;
      if (s1 != SG_OK) {
        st = s1;
        break;
      }
    }
    host_cache_enqueue(hc, todo);
    if (queued) *queued = (int32_t)todo.size();
    return st;
  });
}

sg_status sg_host_cache_wait(sg_host_cache* hc, int32_t* failed) {
  if (!hc) {
    set_error("cache NULL");
    return SG_ERR_INVALID_ARG;
  }
  int32_t f = 0;
  host_cache_collect(hc, true, nullptr, nullptr, &f);
  if (failed) *failed = f;
  return SG_OK;
}

}  // extern "C"
