// The C ABI of libpgs.so (declared in include/pgs.h): argument checks, the
// workspace contract and dispatch by key type.  No entry point allocates device
// memory; all temporaries live in the caller's workspace.
#include <array>
#include <cstdio>
#include <mutex>
#include <new>
#include <vector>

#include "pgs_graph.cuh"
#include "pgs_host.cuh"

namespace pgs {
int sort_u32(const Shape&, const Options&, const void*, const uint32_t*, void*, uint32_t*, cudaStream_t);
int sort_u64(const Shape&, const Options&, const void*, const uint32_t*, void*, uint32_t*, cudaStream_t);
int sort_host_u32(const Shape&, const Options&, const void*, const uint32_t*, void*, uint32_t*, cudaStream_t);
int sort_host_u64(const Shape&, const Options&, const void*, const uint32_t*, void*, uint32_t*, cudaStream_t);
int fit_u32(uint64_t, uint32_t, const Options&, const void*, void*, float*, cudaStream_t);
int fit_u64(uint64_t, uint32_t, const Options&, const void*, void*, float*, cudaStream_t);

namespace {

// Host memory (pinned or pageable), not a device allocation.
bool is_host_pointer(const void* ptr) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeHost || a.type == cudaMemoryTypeUnregistered;
}

bool ranges_overlap(const void* a, const void* b, uint64_t bytes) {
  auto x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
  return x != y && x < y + bytes && y < x + bytes;
}

int sort_direct(const Shape& p, const Options& o, const void* ki, const uint32_t* vi, void* ko, uint32_t* vo,
                cudaStream_t st) {
  if (o.dtype == PGS_U64) return sort_u64(p, o, ki, vi, ko, vo, st);
  return sort_u32(p, o, ki, vi, ko, vo, st);
}

}  // namespace

// ---------------------------------------------------------------------------
// The graph cache behind launch_cached (declared in pgs_graph.cuh).
// ---------------------------------------------------------------------------

namespace {

constexpr size_t kGraphCacheSize = 16;
constexpr int kGraphMaxDevices = 64;

struct GraphEntry {
  GraphKey key{};
  cudaGraphExec_t exec = nullptr;
  bool failed = false;         // capture did not work for this key: run directly
  uint64_t used = 0;           // last use, for eviction
};

struct GraphCache {
  std::mutex mu;               // entries, clock, streams
  std::mutex capture_mu;       // one capture at a time (the capture streams are shared)
  std::vector<GraphEntry> entries;
  uint64_t clock = 0;
  std::array<cudaStream_t, kGraphMaxDevices> capture_stream{};
};

GraphCache& graph_cache() {
  static GraphCache* c = new GraphCache();          // never destroyed: graphs may outlive static teardown
  return *c;
}

}  // namespace

int launch_cached(const GraphKey& key_in, bool allow, cudaStream_t st, const std::function<int(cudaStream_t)>& run) {
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (!allow || cudaStreamIsCapturing(st, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone) {
    cudaGetLastError();
    return run(st);
  }
  int device = -1;
  if (cudaGetDevice(&device) != cudaSuccess || device < 0 || device >= kGraphMaxDevices) return PGS_ERR_CUDA;
  GraphKey key = key_in;
  key[key.size() - 1] = (uint64_t)device + 1;
  GraphCache& gc = graph_cache();
  cudaStream_t cs = nullptr;
  {
    std::lock_guard<std::mutex> lock(gc.mu);
    GraphEntry* e = nullptr;
    for (auto& x : gc.entries)
      if (x.key == key) e = &x;
    if (e == nullptr) {                               // first call: remember the key, run directly
      if (gc.entries.size() >= kGraphCacheSize) {
        size_t lru = 0;
        for (size_t i = 1; i < gc.entries.size(); ++i)
          if (gc.entries[i].used < gc.entries[lru].used) lru = i;
        if (gc.entries[lru].exec) cudaGraphExecDestroy(gc.entries[lru].exec);   // freed once idle
        gc.entries.erase(gc.entries.begin() + (long)lru);
      }
      GraphEntry ne;
      ne.key = key;
      ne.used = ++gc.clock;
      gc.entries.push_back(ne);
    } else {
      e->used = ++gc.clock;
      if (e->exec) return cudaGraphLaunch(e->exec, st) == cudaSuccess ? PGS_OK : PGS_ERR_CUDA;   // replay
      if (!e->failed) {
        if (!gc.capture_stream[device] &&
            cudaStreamCreateWithFlags(&gc.capture_stream[device], cudaStreamNonBlocking) != cudaSuccess)
          return PGS_ERR_CUDA;
        cs = gc.capture_stream[device];
      }
    }
  }
  if (cs == nullptr) return run(st);
  // Second call: capture (nothing runs), instantiate, launch.
  std::lock_guard<std::mutex> cap_lock(gc.capture_mu);
  cudaGraph_t g = nullptr;
  cudaGraphExec_t exec = nullptr;
  bool ok = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
  int rc = ok ? run(cs) : PGS_OK;
  if (ok) ok = cudaStreamEndCapture(cs, &g) == cudaSuccess && rc == PGS_OK && g != nullptr;
  if (ok) ok = cudaGraphInstantiate(&exec, g, 0) == cudaSuccess;
  if (g) cudaGraphDestroy(g);
  if (!ok) {
    cudaGetLastError();
    std::lock_guard<std::mutex> lock(gc.mu);
    for (auto& x : gc.entries)
      if (x.key == key) x.failed = true;
    return run(st);
  }
  std::lock_guard<std::mutex> lock(gc.mu);
  bool kept = false;
  for (auto& x : gc.entries)
    if (x.key == key && !x.exec) {
      x.exec = exec;
      kept = true;
    }
  const bool launched = cudaGraphLaunch(exec, st) == cudaSuccess;
  if (!kept) cudaGraphExecDestroy(exec);             // evicted meanwhile, or another thread won: freed once idle
  return launched ? PGS_OK : PGS_ERR_CUDA;
}

// ---------------------------------------------------------------------------
// The copy streams and events of host-buffer sorts (declared in pgs_host.cuh).
// ---------------------------------------------------------------------------

namespace {

constexpr size_t kHostCopiesCache = 16;

struct HostCopiesEntry {
  int device = -1;
  const void* workspace = nullptr;
  HostCopies hc;
  uint64_t used = 0;
};

struct HostCopiesCache {
  std::mutex mu;
  std::vector<HostCopiesEntry> entries;
  uint64_t clock = 0;
};

HostCopiesCache& host_copies_cache() {
  static HostCopiesCache* c = new HostCopiesCache();   // never destroyed: its streams may outlive static teardown
  return *c;
}

}  // namespace

int host_copies_for(const void* workspace, HostCopies* out) {
  int device = -1;
  PGS_CUDA(cudaGetDevice(&device));
  HostCopiesCache& hc = host_copies_cache();
  std::lock_guard<std::mutex> lock(hc.mu);
  for (auto& e : hc.entries)
    if (e.device == device && e.workspace == workspace) {
      e.used = ++hc.clock;
      *out = e.hc;
      return PGS_OK;
    }
  HostCopiesEntry ne;
  ne.device = device;
  ne.workspace = workspace;
  const int rc = ne.hc.create();
  if (rc != PGS_OK) {
    ne.hc.release();
    return rc;
  }
  if (hc.entries.size() >= kHostCopiesCache) {
    size_t lru = 0;
    for (size_t i = 1; i < hc.entries.size(); ++i)
      if (hc.entries[i].used < hc.entries[lru].used) lru = i;
    hc.entries[lru].hc.release();
    hc.entries.erase(hc.entries.begin() + (long)lru);
  }
  ne.used = ++hc.clock;
  hc.entries.push_back(ne);
  *out = ne.hc;
  return PGS_OK;
}

}  // namespace pgs

using namespace pgs;

extern "C" {

size_t pgs_workspace_bytes(uint64_t n, uint32_t P, const pgs_config* cfg) {
  Options o;
  if (read_options(cfg, &o) != PGS_OK || P == 0) return 0;
  Shape p = single_shape(n, P, true, o);
  if (p.Pmax > kMaxP) return 0;
  Buffers b;
  return carve(p, nullptr, &b);
}

int pgs_sort_copy(const void* keys_in, const uint32_t* vals_in, void* keys_out, uint32_t* vals_out,
                  uint64_t n, uint32_t P, void* stream, const pgs_config* cfg) {
  Options o;
  int rc = read_options(cfg, &o);
  if (rc) return rc;
  if (P == 0) return PGS_ERR_INVALID;
  if ((vals_in == nullptr) != (vals_out == nullptr)) return PGS_ERR_INVALID;
  if (n == 0) return PGS_OK;
  if (!keys_in || !keys_out) return PGS_ERR_INVALID;
  if (n >= (1ull << 40)) return PGS_ERR_UNSUPPORTED;
  const int w = key_bytes(o.dtype);
  if (ranges_overlap(keys_in, keys_out, n * (uint64_t)w)) return PGS_ERR_INVALID;
  if (vals_in && ranges_overlap(vals_in, vals_out, n * 4ull)) return PGS_ERR_INVALID;
  Shape p = single_shape(n, P, vals_in != nullptr, o);
  if (p.Pmax > kMaxP) return PGS_ERR_UNSUPPORTED;
  Buffers b;
  const size_t need = carve(p, nullptr, &b);
  if (!o.workspace || (reinterpret_cast<uintptr_t>(o.workspace) % kAlign) != 0 || o.workspace_bytes < need)
    return PGS_ERR_WORKSPACE;
  DeviceGuard dg;
  rc = dg.use_device_of(keys_out);
  if (rc) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  uint32_t eps_bits;
  std::memcpy(&eps_bits, &o.eps, sizeof(eps_bits));
  const GraphKey key{1, key_ptr(keys_in), key_ptr(vals_in), key_ptr(keys_out), key_ptr(vals_out), n, p.R,
                     (uint64_t)o.dtype, o.samples_per_run, eps_bits, (uint64_t)o.guaranteed,
                     (uint64_t)o.investigator, (uint64_t)o.exchange, (uint64_t)o.splitter_mode, key_ptr(o.workspace),
                     o.workspace_bytes, key_ptr(o.bucket_bounds), key_ptr(o.cuts), key_ptr(o.splitters),
                     key_ptr(o.stats), key_ptr(o.model), key_ptr(o.model_out), (uint64_t)o.tile_variant,
                     (uint64_t)o.merge_ways, o.spin_limit, (uint64_t)o.fault_inject};
  const bool allow = o.timer == nullptr && o.graph_cache == PGS_GRAPH_CACHE_AUTO;
  return launch_cached(key, allow, st, [&](cudaStream_t s) {
    return sort_direct(p, o, keys_in, vals_in, keys_out, vals_out, s);
  });
}

int pgs_sort(void* keys, uint32_t* vals, uint64_t n, uint32_t P, void* stream, const pgs_config* cfg) {
  return pgs_sort_copy(keys, vals, keys, vals, n, P, stream, cfg);
}

size_t pgs_host_workspace_bytes(uint64_t n, uint32_t P, const pgs_config* cfg) {
  Options o;
  if (read_options(cfg, &o) != PGS_OK || P == 0) return 0;
  Shape p = single_shape(n, P, true, o);
  if (p.Pmax > kMaxP) return 0;
  return host_layout(p).total;
}

int pgs_sort_host(const void* keys_in, const uint32_t* vals_in, void* keys_out, uint32_t* vals_out, uint64_t n,
                  uint32_t P, void* stream, const pgs_config* cfg) {
  Options o;
  int rc = read_options(cfg, &o);
  if (rc) return rc;
  if (P == 0) return PGS_ERR_INVALID;
  if ((vals_in == nullptr) != (vals_out == nullptr)) return PGS_ERR_INVALID;
  if (n == 0) return PGS_OK;
  if (!keys_in || !keys_out) return PGS_ERR_INVALID;
  if (n >= (1ull << 40)) return PGS_ERR_UNSUPPORTED;
  const int w = key_bytes(o.dtype);
  if (!is_host_pointer(keys_in) || !is_host_pointer(keys_out)) return PGS_ERR_INVALID;
  if (vals_in && (!is_host_pointer(vals_in) || !is_host_pointer(vals_out))) return PGS_ERR_INVALID;
  if (ranges_overlap(keys_in, keys_out, n * (uint64_t)w)) return PGS_ERR_INVALID;
  if (vals_in && ranges_overlap(vals_in, vals_out, n * 4ull)) return PGS_ERR_INVALID;
  Shape p = single_shape(n, P, vals_in != nullptr, o);
  if (p.Pmax > kMaxP) return PGS_ERR_UNSUPPORTED;
  const size_t need = host_layout(p).total;
  if (!o.workspace || (reinterpret_cast<uintptr_t>(o.workspace) % kAlign) != 0 || o.workspace_bytes < need)
    return PGS_ERR_WORKSPACE;
  DeviceGuard dg;
  rc = dg.use_device_of(o.workspace);
  if (rc) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (o.dtype == PGS_U64) return sort_host_u64(p, o, keys_in, vals_in, keys_out, vals_out, st);
  return sort_host_u32(p, o, keys_in, vals_in, keys_out, vals_out, st);
}

size_t pgs_fit_workspace_bytes(uint64_t m, uint32_t P, const pgs_config* cfg) {
  Options o;
  if (read_options(cfg, &o) != PGS_OK || P == 0) return 0;
  return fit_workspace(m, o, nullptr, nullptr);
}

int pgs_fit_splitters(const void* samples, uint64_t m, uint32_t P, void* stream, const pgs_config* cfg,
                      void* splitters_out, float* model_out) {
  Options o;
  int rc = read_options(cfg, &o);
  if (rc) return rc;
  if (P == 0) return PGS_ERR_INVALID;
  if (P == 1) return PGS_OK;                       // no splitters
  if (!samples || !splitters_out || m < P) return PGS_ERR_INVALID;
  if (m >= (1ull << 40)) return PGS_ERR_UNSUPPORTED;
  const size_t need = fit_workspace(m, o, nullptr, nullptr);
  if (!o.workspace || (reinterpret_cast<uintptr_t>(o.workspace) % kAlign) != 0 || o.workspace_bytes < need)
    return PGS_ERR_WORKSPACE;
  DeviceGuard dg;
  rc = dg.use_device_of(samples);
  if (rc) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (o.dtype == PGS_U64) return fit_u64(m, P, o, samples, splitters_out, model_out, st);
  return fit_u32(m, P, o, samples, splitters_out, model_out, st);
}

int pgs_get_stats(const void* stats_dev, pgs_stats* host_out, void* stream) {
  if (!stats_dev || !host_out) return PGS_ERR_INVALID;
  static_assert(sizeof(pgs_stats) == sizeof(DevStats), "pgs_stats layout");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (cudaMemcpyAsync(host_out, stats_dev, sizeof(pgs_stats), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return PGS_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return PGS_ERR_CUDA;
  if (host_out->error & kErrWaitTimeout) return PGS_ERR_TIMEOUT;
  if (host_out->error) return PGS_ERR_CUDA;
  return PGS_OK;
}

const char* pgs_strerror(int status) {
  switch (status) {
    case PGS_OK: return "ok";
    case PGS_ERR_INVALID: return "invalid argument";
    case PGS_ERR_WORKSPACE: return "workspace missing, misaligned or too small";
    case PGS_ERR_CUDA: return "CUDA error";
    case PGS_ERR_TIMEOUT: return "device-side wait timed out";
    case PGS_ERR_UNSUPPORTED: return "unsupported request";
    default: return "unknown status";
  }
}

const char* pgs_version(void) { return "0.1.0"; }

const char* pgs_last_error(void) { return last_error_buffer(); }

int pgs_timer_create(uint32_t capacity, pgs_timer** out) {
  if (!out || capacity == 0) return PGS_ERR_INVALID;
  *out = nullptr;
  pgs_timer* t = new (std::nothrow) pgs_timer;
  if (!t) return PGS_ERR_INVALID;
  t->ev = new (std::nothrow) cudaEvent_t[2ull * capacity];
  t->rec = new (std::nothrow) pgs_launch_record[capacity];
  if (!t->ev || !t->rec) {
    delete[] t->ev;
    delete[] t->rec;
    delete t;
    return PGS_ERR_INVALID;
  }
  for (uint64_t i = 0; i < 2ull * capacity; ++i) {
    cudaError_t e = cudaEventCreate(&t->ev[i]);
    if (e != cudaSuccess) {
      for (uint64_t j = 0; j < i; ++j) cudaEventDestroy(t->ev[j]);
      delete[] t->ev;
      delete[] t->rec;
      delete t;
      return record_cuda_error(e, "cudaEventCreate", __LINE__);
    }
  }
  t->cap = capacity;
  *out = t;
  return PGS_OK;
}

int pgs_timer_destroy(pgs_timer* t) {
  if (!t) return PGS_ERR_INVALID;
  for (uint64_t i = 0; i < 2ull * t->cap; ++i) cudaEventDestroy(t->ev[i]);
  delete[] t->ev;
  delete[] t->rec;
  delete t;
  return PGS_OK;
}

int pgs_timer_reset(pgs_timer* t) {
  if (!t) return PGS_ERR_INVALID;
  t->count = 0;
  t->dropped = 0;
  return PGS_OK;
}

int pgs_timer_read(pgs_timer* t, pgs_launch_record* out, uint32_t max, uint32_t* count, uint32_t* dropped) {
  if (!t || (max && !out)) return PGS_ERR_INVALID;
  for (uint32_t i = 0; i < t->count; ++i) {
    PGS_CUDA(cudaEventSynchronize(t->ev[2 * i + 1]));
    float ms = 0.0f;
    PGS_CUDA(cudaEventElapsedTime(&ms, t->ev[2 * i], t->ev[2 * i + 1]));
    t->rec[i].ms = ms;
    if (i < max) out[i] = t->rec[i];
  }
  if (count) *count = t->count;
  if (dropped) *dropped = t->dropped;
  return PGS_OK;
}

const char* pgs_kernel_name(uint32_t kernel) {
  static const char* names[PGS_KERNEL_COUNT] = {"block_sort", "merge", "partition", "pairs", "scan",
                                                "sample", "splitters", "cut_search", "investigator",
                                                "offsets", "scatter", "stats", "merge4"};
  return kernel < PGS_KERNEL_COUNT ? names[kernel] : "unknown";
}

}  // extern "C"
