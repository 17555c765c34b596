// Host orchestration of the load-balanced sample sort: the plan (pass counts,
// workspace layout) and the launch sequence of Section IV's six steps on one
// stream.  Nothing here synchronises the stream or allocates device memory.
#pragma once

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <functional>
#include <type_traits>
#include <vector>

#include "pgs.h"
#include "pgs_kernels.cuh"
#include "pgs_learned.cuh"

namespace pgs {

constexpr uint32_t kMaxP = 8192;               // cut matrices are P x (P+1)
// Sorts of at most this many keys (default: every size) launch their kernels
// as programmatic dependent launches: the next kernel is scheduled while its
// predecessor finishes.  Measured: a 2^20-key sort from direct launches 0.381
// -> 0.255 ms, from a captured graph 0.248 -> 0.239 ms; 2^28 keys 18.14 ->
// 17.93 ms direct, unchanged from a graph.
#ifndef PGS_PDL_MAX_KEYS
#define PGS_PDL_MAX_KEYS (~0ull)
#endif
constexpr uint64_t kPdlMaxKeys = PGS_PDL_MAX_KEYS;
constexpr uint64_t kSampleBufferBytes = 262144; // the 256 KB read buffer of Section IV-B
constexpr size_t kAlign = 256;

inline uint64_t ceil_div(uint64_t a, uint64_t b) { return (a + b - 1) / b; }
inline int ceil_log2(uint64_t x) {
  int k = 0;
  while ((1ull << k) < x) ++k;
  return k;
}

struct Options {
  int dtype = PGS_U32;
  uint32_t samples_per_run = 0;
  float eps = 0.05f;
  int guaranteed = 0;
  int investigator = PGS_INVESTIGATOR_RANK;
  int exchange = PGS_EXCHANGE_AUTO;
  int splitter_mode = PGS_SPLITTERS_SAMPLED;
  void* workspace = nullptr;
  uint64_t workspace_bytes = 0;
  uint64_t* bucket_bounds = nullptr;
  uint64_t* cuts = nullptr;
  void* splitters = nullptr;
  void* stats = nullptr;
  pgs_timer* timer = nullptr;
  const float* model = nullptr;
  float* model_out = nullptr;
  int tile_variant = 0;       // merge tile shape (see kMergeShapes)
  int merge_ways = 0;         // lists merged per pass: 4 (two tree levels), 2 (one level), 0 = by size
  int copy_back = PGS_COPY_BACK_AUTO;     // pgs_sort_host: by size, bucket groups after a host wait, or all at the end
  int graph_cache = PGS_GRAPH_CACHE_AUTO; // pgs_sort / pgs_sort_copy: replay repeated calls from a CUDA graph
  uint64_t spin_limit = 0;    // ns of %globaltimer a device-side wait may take; 0 = kWaitLimitNs
  int fault_inject = 0;       // testing only: PGS_FAULT_WAIT_TIMEOUT
};

// Validates and copies a (possibly NULL) pgs_config.  Returns PGS_OK or an error.
inline int read_options(const pgs_config* cfg, Options* o) {
  if (!cfg) return PGS_OK;
  o->dtype = cfg->dtype;
  o->samples_per_run = cfg->samples_per_run;
  o->eps = cfg->eps == 0.0f ? 0.05f : cfg->eps;
  o->guaranteed = cfg->guaranteed;
  o->investigator = cfg->investigator;
  o->exchange = cfg->exchange;
  o->splitter_mode = cfg->splitter_mode;
  o->workspace = cfg->workspace;
  o->workspace_bytes = cfg->workspace_bytes;
  o->bucket_bounds = cfg->bucket_bounds;
  o->cuts = cfg->cuts;
  o->splitters = cfg->splitters;
  o->stats = cfg->stats;
  o->timer = cfg->timer;
  o->model = cfg->model;
  o->model_out = cfg->model_out;
  o->tile_variant = cfg->tile_variant;
  o->merge_ways = cfg->merge_ways;
  o->copy_back = cfg->copy_back;
  o->graph_cache = cfg->graph_cache;
  o->spin_limit = cfg->spin_limit;
  o->fault_inject = cfg->fault_inject;
  if (o->dtype < PGS_U32 || o->dtype > PGS_F32) return PGS_ERR_INVALID;
  if (!(o->eps > 0.0f) || o->eps > 1.0f) return PGS_ERR_INVALID;
  if (o->investigator < 0 || o->investigator > 3) return PGS_ERR_INVALID;
  if (o->exchange < 0 || o->exchange > 2) return PGS_ERR_INVALID;
  if (o->splitter_mode < 0 || o->splitter_mode > 1) return PGS_ERR_INVALID;
  if (o->tile_variant < 0 || o->tile_variant >= PGS_TILE_VARIANTS) return PGS_ERR_INVALID;
  if (o->merge_ways != 0 && o->merge_ways != 2 && o->merge_ways != 4) return PGS_ERR_INVALID;
  if (o->copy_back != PGS_COPY_BACK_AUTO && o->copy_back != PGS_COPY_BACK_GROUPS &&
      o->copy_back != PGS_COPY_BACK_AT_END)
    return PGS_ERR_INVALID;
  if (o->graph_cache != PGS_GRAPH_CACHE_AUTO && o->graph_cache != PGS_GRAPH_CACHE_OFF) return PGS_ERR_INVALID;
  if (o->fault_inject != 0 && o->fault_inject != PGS_FAULT_WAIT_TIMEOUT) return PGS_ERR_INVALID;
  return PGS_OK;
}

inline int key_bytes(int dtype) { return dtype == PGS_U64 ? 8 : 4; }

// Bump allocator over the caller's workspace (or a dry run that only measures).
struct Carver {
  char* base;
  size_t used = 0;
  explicit Carver(void* b) : base(static_cast<char*>(b)) {}
  template <typename T> T* take(uint64_t count) {
    used = (used + kAlign - 1) / kAlign * kAlign;
    T* p = base ? reinterpret_cast<T*>(base + used) : nullptr;
    used += std::max<uint64_t>(count, 1) * sizeof(T);
    return p;
  }
};

// Host-side scalars of a batch of sort instances (a single sort is a batch of one).
struct Shape {
  uint32_t I = 1;            // instances
  uint32_t R = 1;            // runs = buckets, sum of P_i
  uint32_t Pmax = 1;         // largest P_i
  uint64_t n = 0;            // keys in all instances
  uint64_t Q = 1;            // bucket segments, sum of P_i^2
  uint64_t MAT = 2;          // entries of the P x (P+1) matrices, sum of P_i (P_i + 1)
  uint64_t S = 0;            // samples of all runs
  uint64_t maxlen = 0;       // longest run
  uint64_t s = 0;            // samples per run of a single sort (reported in the stats)
  int w = 4;                 // key bytes
  bool vals = false;
  bool learned = false;      // learned-CDF splitters (single sorts only)
  bool scatter = false;      // step 5 as its own pass (else fused into step 6's first round)
  bool four = false;         // four-way rounds (two tree levels per pass)
  uint64_t max_quads = 1;
  uint64_t max_tiles4 = 1;   // tiles of the largest four-way round
  int run_rounds = 0;        // merge rounds growing block-sorted tiles into runs (step 1)
  int bucket_rounds = 0;     // merge rounds of steps 3 and 6: ceil(log2 Pmax)
  uint64_t max_pairs = 1;
  uint64_t max_tiles = 1;
  uint64_t scan_len = 1;
  int passes = 0;            // full passes over the keys
  uint32_t pre_rounds = 0;   // step 6 rounds planned with the bucket offsets (single small sorts)
  uint64_t pre_stride = 0;   // jobs per pre-planned round, at most
};

// Keys from which merge_ways 0 uses four-way passes: below it the sort is
// bound by its launches and the four-way round's extra planning launches (the
// index-sample merge, the co-ranks) cost more than the passes they save
// (measured on u32 and u64 keys at 2^20 .. 2^26: pairwise 1-4 % faster up to
// 2^22 keys, four-way 5-16 % faster from 2^24).
constexpr uint64_t kFourWayMinKeys = 1ull << 23;
// Cut searches by one warp per slot up to this many (run, splitter) slots:
// 12.5 -> 6.0 us at 256 slots, but 0.04 -> 0.49 ms at 2^20 slots.
constexpr uint64_t kCutWarpMaxSlots = 4096;

inline bool use_four_way(uint64_t n, const Options& o) {
  return o.merge_ways == 4 || (o.merge_ways == 0 && n >= kFourWayMinKeys);
}

inline uint64_t samples_per_run(uint32_t P, int w, const Options& o) {
  uint64_t s = o.samples_per_run ? o.samples_per_run
                                 : std::max<uint64_t>(1, kSampleBufferBytes / ((uint64_t)P * w));
  if (o.guaranteed) {
    uint64_t g = (uint64_t)std::ceil((double)P / (double)o.eps);
    s = std::max(s, g);
  }
  return s;
}

// Completes a Shape whose I, R, Pmax, n, Q, MAT, S, maxlen, w and vals are set.
inline void finish_shape(Shape& sh) {
  uint64_t w = kTile;
  sh.run_rounds = 0;
  while (w < sh.maxlen) { w *= 2; ++sh.run_rounds; }
  sh.bucket_rounds = sh.Pmax > 1 ? ceil_log2(sh.Pmax) : 0;
  uint64_t mp = std::max<uint64_t>(sh.R, sh.Q);
  if (sh.run_rounds > 0) mp = std::max<uint64_t>(mp, (uint64_t)sh.R * ceil_div(sh.maxlen, 2ull * kTile));
  sh.max_pairs = std::max<uint64_t>(mp, 1);
  sh.max_quads = std::max<uint64_t>(sh.Q, 1);
  if (sh.run_rounds > 1) sh.max_quads = std::max<uint64_t>(sh.max_quads, (uint64_t)sh.R * ceil_div(sh.maxlen, 4ull * kTile));
  if (sh.four) sh.max_pairs = std::max<uint64_t>(sh.max_pairs, 2 * sh.max_quads);   // the index-sample merges
  sh.max_tiles = ceil_div(std::max<uint64_t>(sh.n, 1), kMergeMinTile) + sh.max_pairs + 1;
  sh.max_tiles4 = ceil_div(ceil_div(std::max<uint64_t>(sh.n, 1), kIdxStride) + sh.max_quads, kMerge4MinQ) +
                  sh.max_quads + 1;
  sh.scan_len = std::max<uint64_t>(std::max<uint64_t>(sh.max_pairs, sh.Q), sh.max_quads);
  // Step 6 planned by the offsets kernel: one instance, pairwise rounds, the
  // offsets in one CTA and every round small at any tile shape (a round has
  // at most ceil(n / tile) + Q tiles).
  sh.pre_rounds = 0;
  sh.pre_stride = ceil_div(std::max<uint64_t>(sh.n, 1), kMergeMinTile) + sh.Q;
  if (sh.I == 1 && !sh.four && sh.Pmax > 1 && sh.Q <= kSizesMax && sh.Q <= kPlanMaxPairs &&
      sh.pre_stride <= kPlanMaxTiles)
    sh.pre_rounds = (uint32_t)sh.bucket_rounds;
  auto passes_for = [&](int levels) { return sh.four ? levels / 2 + levels % 2 : levels; };
  int bucket_passes = 0;
  if (sh.Pmax > 1) bucket_passes = sh.scatter ? 1 + passes_for(sh.bucket_rounds) : 1 + passes_for(sh.bucket_rounds - 1);
  sh.passes = 1 + passes_for(sh.run_rounds) + bucket_passes;
}

// A single sort of n keys on P_req logical partitions.
inline Shape single_shape(uint64_t n, uint32_t P_req, bool vals, const Options& o) {
  Shape sh;
  sh.n = n;
  sh.w = key_bytes(o.dtype);
  sh.vals = vals;
  const uint32_t P = (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(P_req, n));
  sh.I = 1;
  sh.R = P;
  sh.Pmax = P;
  sh.Q = (uint64_t)P * P;
  sh.MAT = (uint64_t)P * (P + 1);
  sh.maxlen = ceil_div(n, P);
  sh.s = P > 1 ? samples_per_run(P, sh.w, o) : 0;
  sh.S = P > 1 ? (sh.s >= sh.maxlen ? n : (uint64_t)P * sh.s) : 0;
  sh.learned = o.splitter_mode == PGS_SPLITTERS_LEARNED && P > 1;
  sh.scatter = o.exchange == PGS_EXCHANGE_SCATTER;
  sh.four = use_four_way(n, o);
  finish_shape(sh);
  return sh;
}

// Device buffers inside the workspace.
struct Buffers {
  void* alt_k; uint32_t* alt_v;
  void* samp_a; void* samp_b; void* spl;
  uint64_t *lb, *cnt, *cut, *sizes, *seg_src, *off, *e;
  uint64_t *samp_counts, *samp_off;
  Pair* pairs; uint64_t *tcount, *tbegin;
  TileSplit* split;
  TileJob* jobs;             // the same storage as split: a round uses one or the other
  TileJob* pre_jobs;         // step 6 rounds planned with the bucket offsets (sh.pre_rounds x sh.pre_stride)
  uint64_t* pre_tbegin;      // their tile-count scans (sh.pre_rounds x (Q + 1))
  Pair* pre_pairs; uint64_t* pre_tcount; uint64_t* pre_offs;   // each planning CTA's scratch
  void* kidx;                // key index of the last pass: the key at every 64th position
  Quad* quads; uint64_t *tcount4, *tbegin4; Split4* splits4; void* xs;   // four-way rounds
  uint64_t max_tiles4 = 0;
  uint64_t max_tiles = 0;    // entries of split / jobs
  uint64_t *scan_sums, *scan_sums2;
  uint64_t* first_seg;
  // batch tables
  uint64_t* koff; uint32_t* Pt; uint32_t* R0; uint64_t* mat; uint64_t* seg; uint64_t* st;
  uint64_t* run_off; uint32_t* run_inst;
  uint32_t* err;
  float* max_ratio;
  // learned splitters
  MlpState* mlp; float* mlp_part; float* model; uint64_t* cutL; uint64_t* eL;
  uint32_t* fallback; float* learned_ratio;
  Geo geo(const Shape& sh) const {
    return Geo{koff, Pt, R0, mat, seg, st, run_off, run_inst, sh.I, sh.R};
  }
};

// Lays the buffers out in the workspace (base may be NULL to only measure).
// The tables come first so that a batch can upload them with one copy.
inline size_t carve(const Shape& sh, void* base, Buffers* b, size_t* tables_bytes = nullptr) {
  Carver c(base);
  b->koff = c.take<uint64_t>(sh.I + 1);
  b->Pt = c.take<uint32_t>(sh.I);
  b->R0 = c.take<uint32_t>(sh.I + 1);
  b->mat = c.take<uint64_t>(sh.I + 1);
  b->seg = c.take<uint64_t>(sh.I + 1);
  b->st = c.take<uint64_t>(sh.I);
  b->run_off = c.take<uint64_t>(sh.R + 1);
  b->run_inst = c.take<uint32_t>(sh.R);
  if (tables_bytes) *tables_bytes = c.used;
  b->alt_k = c.take<char>(sh.n * sh.w);
  b->alt_v = sh.vals ? c.take<uint32_t>(sh.n) : nullptr;
  b->samp_a = c.take<char>(sh.S * sh.w);
  b->samp_b = c.take<char>(sh.S * sh.w);
  b->spl = c.take<char>((uint64_t)sh.R * sh.w);
  b->lb = c.take<uint64_t>(sh.MAT);
  b->cnt = c.take<uint64_t>(sh.MAT);
  b->cut = c.take<uint64_t>(sh.MAT);
  b->sizes = c.take<uint64_t>(sh.Q);
  b->seg_src = c.take<uint64_t>(sh.Q);
  b->off = c.take<uint64_t>(sh.Q + 1);
  b->e = c.take<uint64_t>((uint64_t)sh.R + sh.I);
  b->samp_counts = c.take<uint64_t>(sh.R);
  b->samp_off = c.take<uint64_t>(sh.R + 1);
  b->pairs = c.take<Pair>(sh.max_pairs);
  b->tcount = c.take<uint64_t>(sh.max_pairs);
  b->tbegin = c.take<uint64_t>(sh.max_pairs + 1);
  b->split = c.take<TileSplit>(sh.max_tiles);
  b->jobs = reinterpret_cast<TileJob*>(b->split);
  b->max_tiles = sh.max_tiles;
  b->pre_jobs = sh.pre_rounds ? c.take<TileJob>((uint64_t)sh.pre_rounds * sh.pre_stride) : nullptr;
  b->pre_tbegin = sh.pre_rounds ? c.take<uint64_t>((uint64_t)sh.pre_rounds * (sh.Q + 1)) : nullptr;
  b->pre_pairs = sh.pre_rounds ? c.take<Pair>((uint64_t)sh.pre_rounds * sh.Q) : nullptr;
  b->pre_tcount = sh.pre_rounds ? c.take<uint64_t>((uint64_t)sh.pre_rounds * sh.Q) : nullptr;
  b->pre_offs = sh.pre_rounds ? c.take<uint64_t>((uint64_t)sh.pre_rounds * (sh.Q + 1)) : nullptr;
  b->kidx = c.take<char>(ceil_div(std::max<uint64_t>(sh.n, 1), kIdxStride) * sh.w);
  if (sh.four) {
    b->quads = c.take<Quad>(sh.max_quads);
    b->tcount4 = c.take<uint64_t>(sh.max_quads);
    b->tbegin4 = c.take<uint64_t>(sh.max_quads + 1);
    b->splits4 = c.take<Split4>(sh.max_tiles4);
    b->max_tiles4 = sh.max_tiles4;
    b->xs = c.take<char>(ceil_div(std::max<uint64_t>(sh.n, 1), kIdxStride) * sh.w);
  } else {
    b->quads = nullptr;
    b->tcount4 = b->tbegin4 = nullptr;
    b->splits4 = nullptr;
    b->xs = nullptr;
  }
  const uint64_t chunks = ceil_div(sh.scan_len, kScanChunk);
  b->scan_sums = c.take<uint64_t>(chunks + 1);
  b->scan_sums2 = c.take<uint64_t>(chunks + 1);
  b->first_seg = c.take<uint64_t>(ceil_div(std::max<uint64_t>(sh.n, 1), kScatterTile));
  b->err = c.take<uint32_t>(1);
  b->max_ratio = c.take<float>(1);
  b->mlp = nullptr;
  b->mlp_part = nullptr;
  b->model = nullptr;
  b->cutL = b->eL = nullptr;
  b->fallback = nullptr;
  b->learned_ratio = nullptr;
  if (sh.learned) {
    b->mlp = c.take<MlpState>(1);
    b->mlp_part = c.take<float>(ceil_div(std::max<uint64_t>(sh.S, 1), kMlpBatch) * (kMlpW + 1));
    b->model = c.take<float>(kMlpWords);
    b->cutL = c.take<uint64_t>(sh.MAT);
    b->eL = c.take<uint64_t>(sh.R + 1);
    b->fallback = c.take<uint32_t>(1);
    b->learned_ratio = c.take<float>(1);
  }
  return c.used;
}

// ---------------------------------------------------------------------------
// Launch helpers
// ---------------------------------------------------------------------------

// The last failure of this thread, for pgs_last_error().
inline char* last_error_buffer() {
  static thread_local char buf[256] = "";
  return buf;
}
inline int record_cuda_error(cudaError_t e, const char* where, int line) {
  snprintf(last_error_buffer(), 256, "%s (line %d): %s", where, line, cudaGetErrorString(e));
  return PGS_ERR_CUDA;
}

#define PGS_CUDA(call)                                                    \
  do {                                                                    \
    cudaError_t e_ = (call);                                              \
    if (e_ != cudaSuccess) return record_cuda_error(e_, #call, __LINE__); \
  } while (0)

#define PGS_TRY(expr)            \
  do {                           \
    int rc_ = (expr);            \
    if (rc_ != PGS_OK) return rc_; \
  } while (0)

// Makes the device that owns a call's memory current for the rest of the call
// and gives the caller back its own current device on every return path.
struct DeviceGuard {
  int saved = -1;
  bool changed = false;
  DeviceGuard() {
    if (cudaGetDevice(&saved) != cudaSuccess) {
      cudaGetLastError();
      saved = -1;
    }
  }
  DeviceGuard(const DeviceGuard&) = delete;
  DeviceGuard& operator=(const DeviceGuard&) = delete;
  // Device memory (or managed memory) only: the device it lives on.
  static int device_of(const void* ptr, int* dev) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
      cudaGetLastError();
      return PGS_ERR_INVALID;
    }
    if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged) return PGS_ERR_INVALID;
    *dev = a.device;
    return PGS_OK;
  }
  int use(int dev) {
    if (dev == saved && !changed) return PGS_OK;
    cudaError_t e = cudaSetDevice(dev);
    if (e != cudaSuccess) return record_cuda_error(e, "cudaSetDevice", __LINE__);
    changed = dev != saved;
    return PGS_OK;
  }
  // Makes the device of `ptr` current; PGS_ERR_INVALID if it is not device memory.
  int use_device_of(const void* ptr) {
    int dev = -1;
    PGS_TRY(device_of(ptr, &dev));
    return use(dev);
  }
  ~DeviceGuard() {
    if (changed && saved >= 0) cudaSetDevice(saved);
  }
};

inline unsigned grid_for(uint64_t threads, unsigned block) {
  return (unsigned)std::max<uint64_t>(1, ceil_div(threads, block));
}

}  // namespace pgs

// Caller-owned record of launch times (the per-step breakdown of Fig. 5(b)).
struct pgs_timer {
  uint32_t cap = 0;
  uint32_t count = 0;
  uint32_t dropped = 0;
  cudaEvent_t* ev = nullptr;        // 2 * cap events
  pgs_launch_record* rec = nullptr;  // cap records
};

namespace pgs {

// Launch context: the stream, the optional timer and the launch count.
struct Ctx {
  cudaStream_t st = nullptr;
  pgs_timer* timer = nullptr;
  uint32_t launches = 0;
  int variant = 0;            // merge tile shape
  uint64_t wait_ns = 0;       // limit of every bounded device-side wait (0: kWaitLimitNs)
  int inject_timeout = 0;     // testing only: the next merge launch's tile 0 waits for copies never issued
  bool pdl = false;           // launch with programmatic dependent launch (small sorts)
};

// Launch `k` on `st`; with `pdl`, as a programmatic dependent launch: the grid
// may be scheduled while its predecessor in the stream finishes, and every
// pipeline kernel starts with pdl_enter(), which waits for the predecessor's
// completion and memory before touching any data (so only the launch and
// dispatch latency overlap).
template <typename... KArgs, typename... Args>
inline void klaunch(cudaStream_t st, bool pdl, void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem,
                    Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  if (pdl) {
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
  }
  cudaLaunchKernelEx(&cfg, k, static_cast<KArgs>(args)...);
}

// Run `f` (which launches exactly one kernel on c.st), check the launch, count
// it and, with a timer, bracket it with events.
template <typename F>
inline int launch(Ctx& c, uint32_t kind, uint32_t step, uint64_t bytes, F&& f) {
  pgs_timer* t = c.timer;
  const bool rec = t && t->count < t->cap;
  if (t && !rec) ++t->dropped;
  if (rec) PGS_CUDA(cudaEventRecord(t->ev[2 * t->count], c.st));
  f();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return record_cuda_error(e, pgs_kernel_name(kind), (int)kind);
  ++c.launches;
  if (rec) {
    PGS_CUDA(cudaEventRecord(t->ev[2 * t->count + 1], c.st));
    pgs_launch_record& r = t->rec[t->count++];
    r.kernel = kind;
    r.step = step;
    r.bytes = bytes;
    r.ms = 0.0f;
    r.reserved = 0;
  }
  return PGS_OK;
}

// out[0..m] = exclusive scan of in[0..m) with the total in out[m].
inline int scan_u64(Ctx& c, const uint64_t* in, uint64_t* out, uint64_t m, uint64_t* sums, uint64_t* sums2,
                    uint32_t step) {
  if (m == 0) {
    PGS_CUDA(cudaMemsetAsync(out, 0, sizeof(uint64_t), c.st));
    return PGS_OK;
  }
  const uint64_t chunks = ceil_div(m, kScanChunk);
  const uint64_t bytes = 16 * m;
  if (chunks == 1)
    return launch(c, PGS_KERNEL_SCAN, step, bytes, [&] { klaunch(c.st, c.pdl, k_scan_chunks, 1, kScanNT, 0, in, m, out, nullptr); });
  if (chunks > (uint64_t)kScanChunk) return PGS_ERR_UNSUPPORTED;
  PGS_TRY(launch(c, PGS_KERNEL_SCAN, step, 8 * m,
                 [&] { klaunch(c.st, c.pdl, k_scan_reduce, (unsigned)chunks, kScanNT, 0, in, m, sums); }));
  PGS_TRY(launch(c, PGS_KERNEL_SCAN, step, 16 * chunks,
                 [&] { klaunch(c.st, c.pdl, k_scan_chunks, 1, kScanNT, 0, sums, chunks, sums2, nullptr); }));
  return launch(c, PGS_KERNEL_SCAN, step, bytes,
                [&] { klaunch(c.st, c.pdl, k_scan_chunks, (unsigned)chunks, kScanNT, 0, in, m, out, sums2); });
}

// Merge tile shapes the tuner chooses from (threads x outputs per thread);
// variant 0 is the default.
struct MergeShape { int nt, vt; };
constexpr MergeShape kMergeShapes[PGS_TILE_VARIANTS] = {{128, 17}, {256, 13}, {128, 9}, {64, 17}};

template <typename K, bool V, int NT, int VT>
inline int set_merge_attr() {
  PGS_CUDA(cudaFuncSetAttribute(k_merge_tile<K, V, NT, VT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)Merge2Layout<K, V, NT, VT>::bytes));
  return PGS_OK;
}

// Opt in to more than 48 KB of dynamic shared memory (set on every call: the
// attribute belongs to the current device, and the call costs microseconds).
template <typename K, bool V>
inline int set_smem_attrs() {
  PGS_CUDA(cudaFuncSetAttribute(k_block_sort<K, V>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)sizeof(BlockSortSmem<K>)));
  PGS_TRY((set_merge_attr<K, V, kMergeShapes[0].nt, kMergeShapes[0].vt>()));
  PGS_TRY((set_merge_attr<K, V, kMergeShapes[1].nt, kMergeShapes[1].vt>()));
  PGS_TRY((set_merge_attr<K, V, kMergeShapes[2].nt, kMergeShapes[2].vt>()));
  PGS_TRY((set_merge_attr<K, V, kMergeShapes[3].nt, kMergeShapes[3].vt>()));
  constexpr int NT4 = merge4_nt<K>(), VT4 = merge4_vt<K>();
  PGS_CUDA(cudaFuncSetAttribute(k_merge4<K, V, NT4, VT4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)Merge4Layout<K, V, NT4, VT4>::bytes));
  static_assert(merge4_max_tile(merge4_q<K>()) <= (uint32_t)(merge4_nt<K>() * merge4_vt<K>()),
                "four-way tiles fit the CTA");
  PGS_CUDA(cudaFuncSetAttribute(k_scatter<K, V>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)sizeof(ScatterSmem<K>)));
  PGS_CUDA(cudaFuncSetAttribute(k_mlp_grad<K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)sizeof(MlpGradSmem)));
  return PGS_OK;
}

template <typename K, bool V, int NT, int VT>
inline void launch_merge_tile(const K* ks, const uint32_t* vs, K* kd, uint32_t* vd, uint64_t tiles,
                              const Buffers& b, bool jobs, const TileJob* table, const InlinePairs& ip,
                              const uint64_t* total, int f32_out, K* idx_out, uint64_t wait_ns, int inject,
                              cudaStream_t st, bool pdl) {
  klaunch(st, pdl, k_merge_tile<K, V, NT, VT>, (unsigned)tiles, NT, Merge2Layout<K, V, NT, VT>::bytes, ks, vs, kd, vd,
          jobs ? nullptr : b.split, jobs && ip.kind == 0 ? table : nullptr, ip, total, f32_out, b.err, idx_out,
          wait_ns, inject);
}

// One pairwise merge round over pairs already described in b.pairs / b.tcount
// (tile counts of the chosen tile shape).  `len` keys take part; every one of
// them is read and written once.  idx_in: the key index of ks (NULL: none);
// idx_out: where the round writes the key index of kd (NULL: not written).
// live_pairs: an upper bound on the slots that can hold a non-empty pair (the
// grid covers ceil(len / tile) tiles plus one partial tile per such pair;
// empty CTAs beyond the round's total cost launch time).  inl (single sorts'
// run and sample rounds): the same pairs as gen, described by their offsets
// table, for a small round's merge CTAs to work out themselves; inl_max_pair
// bounds the keys of any one pair.  pre (step 6 of a single small sort): the
// round's jobs and tile-count scan, already planned by the offsets kernel.
struct PrePlanned { const TileJob* jobs; const uint64_t* tbegin; };

template <typename K, bool V, typename Gen>
inline int merge_round(Ctx& c, const Gen& gen, const K* ks, const uint32_t* vs, K* kd, uint32_t* vd, uint64_t npairs,
                       uint64_t len, const Buffers& b, int f32_out, uint32_t step, const K* idx_in = nullptr,
                       K* idx_out = nullptr, uint64_t live_pairs = ~0ull, const InlinePairs* inl = nullptr,
                       uint64_t inl_max_pair = 0, const PrePlanned* pre = nullptr) {
  const MergeShape ms = kMergeShapes[c.variant];
  const uint32_t tile = (uint32_t)(ms.nt * ms.vt);
  uint64_t tiles_ub = ceil_div(len, tile) + std::min(npairs, live_pairs);
  const bool small = npairs <= kPlanMaxPairs && tiles_ub <= kPlanMaxTiles;
  InlinePairs ip{};
  const TileJob* table = b.jobs;
  const uint64_t* total = b.tbegin + npairs;
  if (pre) {
    if (!small) return PGS_ERR_CUDA;                     // plan bug: pre-planned rounds are small
    table = pre->jobs;
    total = pre->tbegin + npairs;
  } else if (small && inl) {
    // No planning launch: grid = pair slots x the most tiles a pair can need.
    ip = *inl;
    ip.cm = (uint32_t)std::max<uint64_t>(1, ceil_div(inl_max_pair, tile));
    const uint64_t slots = ip.kind == kRunPairs ? (uint64_t)ip.n_lists * ip.spr : ceil_div(ip.n_lists, 2ull * ip.step);
    tiles_ub = slots * ip.cm;
  } else if (small) {
    // A small round: descriptors, their scan and one job per tile in one CTA;
    // each merge CTA then finds its own splits.
    PGS_TRY(launch(c, PGS_KERNEL_PARTITION, step, 48 * tiles_ub + 56 * npairs, [&] {
      klaunch(c.st, c.pdl, k_plan_jobs<Gen>, 1, kPlanNT, 0, gen, b.pairs, b.tcount, b.tbegin, npairs, b.jobs,
              b.max_tiles, tile, b.err);
    }));
  } else {
    if (!std::is_same<Gen, GenNone>::value)
      PGS_TRY(launch(c, PGS_KERNEL_PAIRS, step, 48 * npairs, [&] {
        klaunch(c.st, c.pdl, k_pairs<Gen>, grid_for(npairs, 256), 256, 0, gen, npairs);
      }));
    PGS_TRY(scan_u64(c, b.tcount, b.tbegin, npairs, b.scan_sums, b.scan_sums2, step));
    PGS_TRY(launch(c, PGS_KERNEL_PARTITION, step, 48 * ceil_div(len, tile), [&] {
      klaunch(c.st, c.pdl, k_partition_split<K>, grid_for(tiles_ub, 256), 256, 0, ks, b.pairs, b.tbegin, npairs,
              b.split, tile, idx_in, b.err);
    }));
  }
  const uint64_t bytes = 2 * len * (sizeof(K) + (V ? 4 : 0));
  const int inject = c.inject_timeout;
  c.inject_timeout = 0;                                   // injected into one launch only
  return launch(c, PGS_KERNEL_MERGE, step, bytes, [&] {
    switch (c.variant) {
#define PGS_MERGE_SHAPE(i) kMergeShapes[i].nt, kMergeShapes[i].vt
#define PGS_MERGE_ARGS ks, vs, kd, vd, tiles_ub, b, small, table, ip, total, f32_out, idx_out, c.wait_ns, inject, c.st, \
                       c.pdl
      case 1: launch_merge_tile<K, V, PGS_MERGE_SHAPE(1)>(PGS_MERGE_ARGS); break;
      case 2: launch_merge_tile<K, V, PGS_MERGE_SHAPE(2)>(PGS_MERGE_ARGS); break;
      case 3: launch_merge_tile<K, V, PGS_MERGE_SHAPE(3)>(PGS_MERGE_ARGS); break;
      default: launch_merge_tile<K, V, PGS_MERGE_SHAPE(0)>(PGS_MERGE_ARGS); break;
#undef PGS_MERGE_ARGS
#undef PGS_MERGE_SHAPE
    }
  });
}

// One four-way round over the quads that the caller's quads kernel described
// in b.quads / b.tcount4, with the index-sample pairs in b.pairs / b.tcount
// (tile counts at the current merge tile shape).  idx_in: the key index of ks
// (required); idx_out: where the round writes the key index of kd (NULL: not
// written).  live_quads bounds the quads that can be non-empty.
template <typename K, bool V>
inline int merge4_round(Ctx& c, const K* ks, const uint32_t* vs, K* kd, uint32_t* vd, uint64_t nquads,
                        uint64_t len, const Buffers& b, int f32_out, uint32_t step, const K* idx_in, K* idx_out,
                        uint64_t live_quads = ~0ull) {
  const uint64_t nq_live = std::min(nquads, live_quads);
  const uint64_t samples = ceil_div(len, kIdxStride) + nq_live;   // index samples of the round, at most
  K* xs = static_cast<K*>(b.xs);
  // X' = merge(I_0, I_1) and Y' = merge(I_2, I_3) of every quad (keys only).
  const int inject = c.inject_timeout;
  c.inject_timeout = 0;
  PGS_TRY((merge_round<K, false>(c, GenNone{}, idx_in, nullptr, xs, nullptr, 2 * nquads, samples, b, 0, step,
                                 nullptr, nullptr, 2 * nq_live)));
  PGS_TRY(scan_u64(c, b.tcount4, b.tbegin4, nquads, b.scan_sums, b.scan_sums2, step));
  const uint64_t tiles_ub = ceil_div(samples, merge4_q<K>()) + nq_live + 1;   // <= sh.max_tiles4
  if (tiles_ub > b.max_tiles4) return PGS_ERR_CUDA;                        // plan bug: never expected
  PGS_TRY(launch(c, PGS_KERNEL_PARTITION, step, 48 * tiles_ub, [&] {
    klaunch(c.st, c.pdl, k_corank4<K>, grid_for(tiles_ub, 256), 256, 0, ks, idx_in, xs, b.quads, b.tbegin4, nquads, b.splits4,
                                                            tiles_ub, merge4_q<K>(), b.err);
  }));
  const uint64_t bytes = 2 * len * (sizeof(K) + (V ? 4 : 0));
  constexpr int NT4 = merge4_nt<K>(), VT4 = merge4_vt<K>();
  constexpr size_t smem = Merge4Layout<K, V, NT4, VT4>::bytes;
  return launch(c, PGS_KERNEL_MERGE4, step, bytes, [&] {
    klaunch(c.st, c.pdl, k_merge4<K, V, NT4, VT4>, (unsigned)tiles_ub, NT4, smem, 
        ks, vs, kd, vd, b.splits4, b.quads, b.tbegin4 + nquads, tiles_ub, f32_out, b.err, idx_out, c.wait_ns, inject);
  });
}

// Learned splitters (single sort, P > 1): the model (trained on the sorted
// sample `sorted` or the caller's), the learned cuts (a bisection of each run
// per bucket), and the judge's choice between them and the sampled cuts
// already in b.cut / b.e.
template <typename K>
int learned_cuts(const Shape& sh, const Options& o, const K* sorted, const K* runs, Ctx& c, const Buffers& b) {
  cudaStream_t st = c.st;
  const uint32_t P = sh.R;
  const uint64_t S = sh.S;
  if (!o.model && P > kLearnedMaxP) {                   // beyond the model's capacity: no training
    return launch(c, PGS_KERNEL_SPLITTERS, 3, 8, [&] {
      klaunch(st, c.pdl, k_learned_skip, 1, 256, 0, b.fallback, b.learned_ratio, o.model_out);
    });
  }
  if (o.model) {
    PGS_TRY(launch(c, PGS_KERNEL_SPLITTERS, 3, 8 * kMlpWords, [&] {
      klaunch(st, c.pdl, k_mlp_validate, 1, 256, 0, o.model, b.model);
    }));
  } else {
    PGS_TRY(launch(c, PGS_KERNEL_SPLITTERS, 3, 16 * kMlpW, [&] { klaunch(st, c.pdl, k_mlp_init<K>, 1, 256, 0, sorted, S, b.mlp); }));
    const uint32_t nparts = (uint32_t)ceil_div(S, kMlpBatch);
    for (uint32_t step = 1; step <= (uint32_t)kMlpSteps; ++step) {
      PGS_TRY(launch(c, PGS_KERNEL_SPLITTERS, 3, S * sizeof(K), [&] {
        klaunch(st, c.pdl, k_mlp_grad<K>, nparts, kMlpBatch, sizeof(MlpGradSmem), sorted, S, b.mlp, b.mlp_part);
      }));
      PGS_TRY(launch(c, PGS_KERNEL_SPLITTERS, 3, 4ull * nparts * (kMlpW + 1), [&] {
        klaunch(st, c.pdl, k_mlp_adam, (unsigned)ceil_div(kMlpW + 1, kAdamParams), kAdamParams * kAdamWarps, 0, 
            b.mlp_part, nparts, b.mlp, step, S);
      }));
    }
    PGS_TRY(launch(c, PGS_KERNEL_SPLITTERS, 3, 16 * kMlpW, [&] { klaunch(st, c.pdl, k_mlp_finalize, 1, 256, 0, b.mlp, b.model); }));
  }
  if (o.model_out) {
    PGS_CUDA(cudaMemcpyAsync(o.model_out, b.model, 4ull * kMlpWords, cudaMemcpyDeviceToDevice, st));
  }
  // K11: the learned cut matrix, one bisection of a sorted run per (run, bucket).
  PGS_TRY(launch(c, PGS_KERNEL_SAMPLE, 4, 8 * sh.MAT * (uint64_t)ceil_log2(std::max<uint64_t>(sh.maxlen, 2)), [&] {
    klaunch(st, c.pdl, k_learned_search<K>, grid_for(sh.MAT, kLearnedSearchNT), kLearnedSearchNT, 0, runs, b.run_off, P,
                                                                                         b.model, b.cutL);
  }));
  PGS_TRY(launch(c, PGS_KERNEL_INVESTIGATOR, 4, 8 * sh.MAT, [&] {
    klaunch(st, c.pdl, k_learned_colsum, grid_for(P + 1, 256), 256, 0, b.cutL, P, b.eL);
  }));
  PGS_TRY(launch(c, PGS_KERNEL_INVESTIGATOR, 4, 8 * (uint64_t)P, [&] {
    klaunch(st, c.pdl, k_learned_judge, 1, 256, 0, b.eL, P, sh.n, o.eps, b.model, b.fallback, b.learned_ratio);
  }));
  return launch(c, PGS_KERNEL_INVESTIGATOR, 4, 16 * sh.MAT, [&] {
    klaunch(st, c.pdl, k_learned_select, grid_for(sh.MAT, 256), 256, 0, b.cutL, b.eL, P, b.fallback, b.cut, b.e);
  });
}

template <typename K, bool V>
int set_all_smem_attrs() {
  PGS_TRY((set_smem_attrs<K, V>()));
  return set_smem_attrs<K, false>();          // the sample sort runs keys only
}

// Run r's first key, computed as the device computes it (run_start).
inline uint64_t host_run_start(uint64_t r, uint64_t n, uint64_t P) { return (r * n) / P; }

// Host-buffer sorts: the input reaches the device in groups of whole runs on a
// copy stream; group g's copy records ev[g], and its step-1 work waits for
// that event only, so later groups copy while earlier ones sort.
// The output leaves the same way: step 6 runs bucket group by bucket group
// (their bounds read back once step 4 has fixed them), and group g's keys are
// copied to the host while group g + 1 merges.
constexpr uint32_t kHostGroups = 8;
// With copy_back AUTO, below this many keys a host-buffer sort copies in and
// out in one piece and never waits on the host: the groups' extra copies,
// events and the host's read of the bucket bounds cost more than the overlap
// they buy.  Measured (two calls in flight / one call, Gkeys/s): 2^22 u32
// keys 9.35 / 5.42 in one piece against 5.25 / 4.08 in groups, 2^24 u32
// 11.15 / 6.97 against 8.16 / 6.26, 2^26 u32 12.45 / 7.27 against 12.91 /
// 8.90 (u64 alike).
#ifndef PGS_HOST_GROUP_MIN_LOG2
#define PGS_HOST_GROUP_MIN_LOG2 25
#endif
constexpr uint64_t kHostGroupMinKeys = 1ull << PGS_HOST_GROUP_MIN_LOG2;
struct HostGroups {
  uint32_t groups = 0;                 // 0: the input is already on the device
  uint32_t r0[kHostGroups + 1] = {};   // runs [r0[g], r0[g+1]) form group g
  cudaEvent_t ev[kHostGroups] = {};
  // Issues group g's copy to the device on cs and records ev[g].  A copy from
  // pageable memory may hold the host until it is done, so group g + 1's copy
  // is issued after group g's sort is enqueued: the GPU sorts while the host
  // waits.  (Pinned copies return at once; the order changes nothing for them.)
  std::function<int(uint32_t)> copy_in;
  uint32_t out_groups = 0;             // 0: the caller copies the output
  cudaStream_t cs = nullptr;           // copy stream
  void* hk_out = nullptr;              // host outputs
  uint32_t* hv_out = nullptr;
  cudaEvent_t ev_out[kHostGroups] = {};
  cudaEvent_t done = nullptr;          // recorded on cs after the last output copy
};

// One sort's launch sequence, step by step (Section IV).  The keys move
// between the caller's output and the workspace's alternate buffer on every
// full pass; `left` counts the passes still to come, and the pass that leaves
// none writes the caller's output, with float keys back in their own bits.
// No attribute or allocation calls: the sequence can be captured into a CUDA
// graph once set_all_smem_attrs has run on the device.
template <typename K, bool V>
struct Pipeline {
  const Shape& sh;
  const Options& o;
  Ctx& c;
  const Buffers& b;
  const Geo g;
  const K* kin;
  const uint32_t* vin;
  K* kout;
  uint32_t* vout;
  cudaStream_t st;
  int f32;
  uint64_t kv;                                         // bytes per key/payload pair
  uint32_t mtile;                                      // outputs per merge tile
  K* cur_k;
  K* oth_k;
  uint32_t* cur_v;
  uint32_t* oth_v;
  int left;
  int k0 = 0;                                          // bucket rounds already done by step 5
  bool idx_ok = false;                                 // b.kidx indexes cur_k (written by its pass)

  struct Saved {
    K* ck;
    K* ok;
    uint32_t* cv;
    uint32_t* ov;
    int left;
    bool idx_ok;
  };

  Pipeline(const Shape& sh_, const Options& o_, const K* kin_, const uint32_t* vin_, K* kout_, uint32_t* vout_,
           Ctx& c_, const Buffers& b_)
      : sh(sh_), o(o_), c(c_), b(b_), g(b_.geo(sh_)), kin(kin_), vin(vin_), kout(kout_), vout(vout_), st(c_.st) {
    c.variant = o.tile_variant;
    c.wait_ns = o.spin_limit;
    c.inject_timeout = o.fault_inject == PGS_FAULT_WAIT_TIMEOUT;
    c.pdl = sh.n <= kPdlMaxKeys;
    f32 = o.dtype == PGS_F32;
    kv = sizeof(K) + (V ? 4 : 0);
    mtile = (uint32_t)(kMergeShapes[c.variant].nt * kMergeShapes[c.variant].vt);
    // Ping-pong so that the last pass lands in kout.
    const int after_block = sh.passes - 1;
    cur_k = (after_block % 2 == 0) ? kout : static_cast<K*>(b.alt_k);
    oth_k = (cur_k == kout) ? static_cast<K*>(b.alt_k) : kout;
    cur_v = V ? ((after_block % 2 == 0) ? vout : b.alt_v) : nullptr;
    oth_v = V ? ((cur_v == vout) ? b.alt_v : vout) : nullptr;
    left = after_block;
  }

  Saved save() const { return Saved{cur_k, oth_k, cur_v, oth_v, left, idx_ok}; }
  void restore(const Saved& s) {
    cur_k = s.ck;
    oth_k = s.ok;
    cur_v = s.cv;
    oth_v = s.ov;
    left = s.left;
    idx_ok = s.idx_ok;
  }
  void flip() {
    std::swap(cur_k, oth_k);
    std::swap(cur_v, oth_v);
  }
  int f32_out() const { return left == 0 ? f32 : 0; }   // float bits back on the last pass
  // Slots of a bucket round that can hold a non-empty pair: in a bucket of p
  // segments only the ceil(p / (2 step)) slots j with j % (2 step) == 0 do,
  // and summed over the buckets in Qg slots (at most sh.R of them) that is at
  // most Qg / (2 step) + sh.R.  (A four-way round at `step` has its quads at
  // j % (4 step) == 0: the same bound at 2 step.)
  uint64_t bucket_live_pairs(uint64_t Qg, uint32_t step) const {
    return ceil_div(Qg, 2ull * step) + sh.R;
  }
  // Step 6 round r (step 2^r) as the offsets kernel planned it.
  PrePlanned pre_planned(uint32_t r) const {
    return PrePlanned{b.pre_jobs + (uint64_t)r * sh.pre_stride, b.pre_tbegin + (uint64_t)r * (sh.Q + 1)};
  }
  // The key index: read while it describes the round's input; written by
  // every merge pass but the last (whose output no partition searches).
  const K* idx_in() const { return idx_ok ? static_cast<const K*>(b.kidx) : nullptr; }
  K* idx_out() const { return left > 0 ? static_cast<K*>(b.kidx) : nullptr; }
  // A four-way round of the quads in b.quads from cur to oth (left already
  // counts it).  Its tile boundaries come from the key index of cur, which
  // every pass but the last writes for the next.
  int quad_round(uint64_t nquads, uint64_t len, uint32_t step, uint64_t live_quads = ~0ull) {
    if (!idx_ok) return PGS_ERR_CUDA;                   // plan bug: no index for this round
    K* io = idx_out();
    PGS_TRY((merge4_round<K, V>(c, cur_k, cur_v, oth_k, oth_v, nquads, len, b, f32_out(), step,
                                static_cast<const K*>(b.kidx), io, live_quads)));
    idx_ok = io != nullptr;
    return PGS_OK;
  }
  // A pairwise round of the pairs in b.pairs from cur to oth (left already counts it).
  template <typename Gen>
  int pair_round(const Gen& gen, uint64_t npairs, uint64_t len, uint32_t step, uint64_t live_pairs = ~0ull,
                 const InlinePairs* inl = nullptr, uint64_t inl_max_pair = 0, const PrePlanned* pre = nullptr) {
    K* io = idx_out();
    PGS_TRY((merge_round<K, V>(c, gen, cur_k, cur_v, oth_k, oth_v, npairs, len, b, f32_out(), step, idx_in(), io,
                               live_pairs, inl, inl_max_pair, pre)));
    idx_ok = io != nullptr;
    return PGS_OK;
  }

  // Step 1 for runs [r0, r0 + Rg) holding len keys: block sort of kTile tiles,
  // then the balanced merge tree (Fig. 2) until each run is one list: two
  // levels per pass (four-way rounds) while two remain, else a pairwise round.
  int sort_runs(uint32_t r0, uint32_t Rg, uint64_t len) {
    const uint32_t tiles_per_run = (uint32_t)std::max<uint64_t>(1, ceil_div(sh.maxlen, kTile));
    const uint64_t* ro = b.run_off + r0;
    K* io = idx_out();
    PGS_TRY(launch(c, PGS_KERNEL_BLOCK_SORT, 1, 2 * len * kv, [&] {
      klaunch(st, c.pdl, k_block_sort<K, V>, (unsigned)((uint64_t)Rg * tiles_per_run), kNT, sizeof(BlockSortSmem<K>), 
          kin, vin, cur_k, cur_v, ro, tiles_per_run, f32, f32_out(), io);
    }));
    idx_ok = io != nullptr;
    uint64_t w = kTile;
    int levels = sh.run_rounds;
    while (levels > 0) {
      --left;
      if (sh.four && levels >= 2) {
        const uint64_t cmax = ceil_div(sh.maxlen, 4 * w);
        const uint64_t nq = cmax * Rg;
        PGS_TRY(launch(c, PGS_KERNEL_PAIRS, 1, 112 * nq, [&] {
          klaunch(st, c.pdl, k_quads4_runs, grid_for(nq, 256), 256, 0, b.quads, b.tcount4, b.pairs, b.tcount, ro, Rg, w, cmax,
                                                           merge4_q<K>(), mtile);
        }));
        PGS_TRY(quad_round(nq, len, 1));
        w *= 4;
        levels -= 2;
      } else {
        const uint64_t cmax = ceil_div(sh.maxlen, 2 * w);
        const uint64_t np = cmax * Rg;
        const InlinePairs inl{ro, w, kRunPairs, Rg, (uint32_t)cmax, 0, 0};
        PGS_TRY(pair_round(GenRuns{b.pairs, b.tcount, ro, Rg, w, cmax, mtile}, np, len, 1, ~0ull,
                           sh.I == 1 ? &inl : nullptr, 2 * w));
        w *= 2;
        levels -= 1;
      }
      flip();
    }
    return PGS_OK;
  }

  // Step 1 for every run; with host groups, group by group as their copies
  // land (group g + 1's copy is issued once group g's sort is enqueued).
  int local_sort(const HostGroups* hg) {
    if (hg == nullptr || hg->groups == 0) return sort_runs(0, sh.R, sh.n);
    const Saved s0 = save();
    PGS_TRY(hg->copy_in(0));
    for (uint32_t gi = 0; gi < hg->groups; ++gi) {
      restore(s0);
      const uint32_t r0 = hg->r0[gi], r1 = hg->r0[gi + 1];
      PGS_CUDA(cudaStreamWaitEvent(st, hg->ev[gi], 0));
      PGS_TRY(sort_runs(r0, r1 - r0, host_run_start(r1, sh.n, sh.R) - host_run_start(r0, sh.n, sh.R)));
      if (gi + 1 < hg->groups) PGS_TRY(hg->copy_in(gi + 1));
    }
    return PGS_OK;
  }

  // Step 2: regular samples of every sorted run, gathered in (run, position)
  // order.  Step 3: the Master sorts the samples (merging each instance's P
  // sorted sample lists with the Fig. 2 schedule) and picks every (S/P)-th one.
  // Returns the sorted samples.
  int sample_and_splitters(K** sorted_sample) {
    const uint32_t R = sh.R;
    K* sa = static_cast<K*>(b.samp_a);
    K* sb = static_cast<K*>(b.samp_b);
    const bool single = sh.I == 1 && sh.s > 0;
    if (single) {
      PGS_TRY(launch(c, PGS_KERNEL_SAMPLE, 2, 2 * sh.S * sizeof(K) + 16 * (uint64_t)R, [&] {
        klaunch(st, c.pdl, k_sample_single<K>, grid_for(std::max<uint64_t>(sh.S, R + 1), 256), 256, 0, cur_k,
                b.run_off, R, sh.s, sh.s >= sh.maxlen, b.samp_off, sa, sh.S);
      }));
    } else {
      PGS_TRY(launch(c, PGS_KERNEL_SAMPLE, 2, 16 * (uint64_t)R, [&] {
        klaunch(st, c.pdl, k_sample_counts, grid_for(R, 256), 256, 0, g, b.samp_counts);
      }));
      PGS_TRY(scan_u64(c, b.samp_counts, b.samp_off, R, b.scan_sums, b.scan_sums2, 2));
      PGS_TRY(launch(c, PGS_KERNEL_SAMPLE, 2, 2 * sh.S * sizeof(K), [&] {
        klaunch(st, c.pdl, k_sample<K>, grid_for(sh.S, 256), 256, 0, cur_k, g, b.samp_off, sa, sh.S);
      }));
    }
    for (int k = 0; k < sh.bucket_rounds; ++k) {
      const uint32_t step = 1u << k;
      // A single sort's runs hold at most s samples each.
      const InlinePairs inl{b.samp_off, 0, kListPairs, R, 0, step, 0};
      const uint64_t max_pair = std::min<uint64_t>(2ull * step, R) * std::max<uint64_t>(sh.s, 1);
      PGS_TRY((merge_round<K, false>(c, GenSampleLists{b.pairs, b.tcount, g, b.samp_off, step, mtile}, sa, nullptr,
                                     sb, nullptr, R, sh.S, b, 0, 3, nullptr, nullptr, ~0ull,
                                     single ? &inl : nullptr, max_pair)));
      std::swap(sa, sb);
    }
    *sorted_sample = sa;                                  // the pick of every (S/P)-th is fused into cuts()
    return PGS_OK;
  }

  // Step 4: binary search of every splitter in every run, then the
  // investigator (Section IV-B); LEARNED mode adds the model's cuts and its
  // judge.  Then the receive offset of every (bucket, run) segment (IV-C).
  int cuts(const K* sorted_sample) {
    const uint32_t R = sh.R;
    PGS_TRY(launch(c, PGS_KERNEL_CUT_SEARCH, 4, 16 * sh.Q + 2 * (uint64_t)R * sizeof(K), [&] {
      K* spl = static_cast<K*>(b.spl);
      K* user = static_cast<K*>(o.splitters);
      if (sh.Q <= kCutWarpMaxSlots)
        klaunch(st, c.pdl, k_cut_search<K, true>, grid_for(32 * sh.Q, 256), 256, 0, cur_k, g, sh.Q, sorted_sample,
                b.samp_off, spl, user, f32, b.lb, b.cnt, b.cut, b.e);
      else
        klaunch(st, c.pdl, k_cut_search<K, false>, grid_for(sh.Q, 256), 256, 0, cur_k, g, sh.Q, sorted_sample,
                b.samp_off, spl, user, f32, b.lb, b.cnt, b.cut, b.e);
    }));
    PGS_TRY(launch(c, PGS_KERNEL_INVESTIGATOR, 4, 24 * sh.MAT, [&] {
      klaunch(st, c.pdl, k_investigator<K>, R, 256, 0, b.lb, b.cnt, static_cast<const K*>(b.spl), g, o.investigator, b.cut,
                                           b.e);
    }));
    if (sh.learned) PGS_TRY((learned_cuts<K>(sh, o, sorted_sample, cur_k, c, b)));
    if (sh.Q <= kSizesMax) {
      PrePlan pp{b.pre_pairs, b.pre_tcount, b.pre_tbegin, b.pre_jobs, b.pre_offs, sh.pre_stride, sh.pre_rounds,
                 mtile, sh.scatter ? 1 : 0};
      return launch(c, PGS_KERNEL_OFFSETS, 5, 40 * sh.Q + 48 * sh.pre_stride * sh.pre_rounds, [&] {
        klaunch(st, c.pdl, k_bucket_offsets, std::max<uint32_t>(1, sh.pre_rounds), kSizesNT, 0, g, sh.Q, b.cut,
                b.sizes, b.seg_src, b.off, pp, b.err);
      });
    }
    PGS_TRY(launch(c, PGS_KERNEL_OFFSETS, 5, 32 * sh.Q, [&] {
      klaunch(st, c.pdl, k_bucket_sizes, grid_for(sh.Q, 256), 256, 0, g, sh.Q, b.cut, b.sizes, b.seg_src);
    }));
    return scan_u64(c, b.sizes, b.off, sh.Q, b.scan_sums, b.scan_sums2, 5);
  }

  // Step 5.  SCATTER: the exchange as an in-HBM scatter into bucket-major
  // order.  Otherwise fused with step 6: the first merge round of every bucket
  // reads its two segments where the sorted runs hold them and writes the
  // merged pair to its place in bucket-major order (all buckets at once: the
  // runs' buffer is free only after every bucket has read its segments).
  int exchange() {
    const uint64_t n = sh.n;
    if (sh.scatter) {
      const uint64_t stiles = ceil_div(n, kScatterTile);
      PGS_TRY(launch(c, PGS_KERNEL_OFFSETS, 5, 8 * stiles, [&] {
        klaunch(st, c.pdl, k_scatter_part, grid_for(stiles, 256), 256, 0, b.off, sh.Q, n, b.first_seg);
      }));
      --left;
      PGS_TRY(launch(c, PGS_KERNEL_SCATTER, 5, 2 * n * kv, [&] {
        klaunch(st, c.pdl, k_scatter<K, V>, (unsigned)stiles, kScatterNT, sizeof(ScatterSmem<K>), 
            cur_k, cur_v, oth_k, oth_v, b.off, b.seg_src, b.first_seg, n, sh.Q, f32_out(), b.err, idx_out());
      }));
      idx_ok = idx_out() != nullptr;
      flip();
      k0 = 0;
      return PGS_OK;
    }
    --left;
    const PrePlanned pre0 = pre_planned(0);
    PGS_TRY(pair_round(GenFused{b.pairs, b.tcount, g, b.off, b.seg_src, 0, mtile}, sh.Q, n, 6,
                       bucket_live_pairs(sh.Q, 1), nullptr, 0, sh.pre_rounds ? &pre0 : nullptr));
    flip();
    k0 = 1;
    return PGS_OK;
  }

  // Step 6 for the buckets of segment slots [q0, q0 + Qg), len keys, already
  // in bucket-major order: every bucket merges its P segments with the Fig. 2
  // schedule, two levels per pass while two remain.
  int merge_buckets(uint64_t q0, uint64_t Qg, uint64_t len) {
    int levels = sh.bucket_rounds - k0;
    uint32_t step = 1u << k0;
    while (levels > 0) {
      --left;
      if (sh.four && levels >= 2) {
        PGS_TRY(launch(c, PGS_KERNEL_PAIRS, 6, 112 * Qg, [&] {
          klaunch(st, c.pdl, k_quads4_buckets, grid_for(Qg, 256), 256, 0, b.quads, b.tcount4, b.pairs, b.tcount, g, b.off, q0,
                                                              Qg, step, merge4_q<K>(), mtile);
        }));
        PGS_TRY(quad_round(Qg, len, 6, bucket_live_pairs(Qg, 2 * step)));
        step *= 4;
        levels -= 2;
      } else {
        // The offsets kernel planned the round if it covers every bucket.
        const PrePlanned pre = pre_planned((uint32_t)ceil_log2(step));
        const bool use_pre = sh.pre_rounds && q0 == 0 && Qg == sh.Q;
        PGS_TRY(pair_round(GenBucketLists{b.pairs, b.tcount, g, b.off, q0, step, mtile}, Qg, len, 6,
                           bucket_live_pairs(Qg, step), nullptr, 0, use_pre ? &pre : nullptr));
        step *= 2;
        levels -= 1;
      }
      flip();
    }
    return PGS_OK;
  }

  // Step 6 of a host-buffer sort of one instance: the bucket bounds come back
  // once (the host waits for steps 1-5 here), then the rounds run bucket group
  // by bucket group; a group's range is final when its last round ends, no
  // later group writes inside it, and its copy to the host starts right away.
  int merge_buckets_to_host(const HostGroups& hg) {
    const uint32_t R = sh.R;
    std::vector<uint64_t> e(R + 1);
    uint32_t err = 0;
    PGS_CUDA(cudaMemcpyAsync(e.data(), b.e, (R + 1) * sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
    PGS_CUDA(cudaMemcpyAsync(&err, b.err, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    PGS_CUDA(cudaStreamSynchronize(st));
    // The bounds size the copies to the caller's host buffers: after a failed
    // kernel they may be anything, so nothing is copied back.
    if (err & kErrWaitTimeout) return PGS_ERR_TIMEOUT;
    if (err) return PGS_ERR_CUDA;
    bool ok = e[0] == 0 && e[R] == sh.n;
    for (uint32_t r = 0; r < R && ok; ++r) ok = e[r] <= e[r + 1];
    if (!ok) return PGS_ERR_CUDA;
    const Saved s0 = save();
    // Group g's copy back is issued once group g + 1's merges are enqueued (a
    // copy to pageable memory may hold the host until it is done).
    auto copy_out = [&](uint32_t gi) -> int {
      const uint64_t b0 = ((uint64_t)gi * R) / hg.out_groups, b1 = ((uint64_t)(gi + 1) * R) / hg.out_groups;
      const uint64_t lo = e[b0], hi = e[b1];
      PGS_CUDA(cudaStreamWaitEvent(hg.cs, hg.ev_out[gi], 0));
      if (hi > lo) {
        PGS_CUDA(cudaMemcpyAsync(static_cast<K*>(hg.hk_out) + lo, kout + lo, (hi - lo) * sizeof(K),
                                 cudaMemcpyDeviceToHost, hg.cs));
        if (V) PGS_CUDA(cudaMemcpyAsync(hg.hv_out + lo, vout + lo, (hi - lo) * 4, cudaMemcpyDeviceToHost, hg.cs));
      }
      return PGS_OK;
    };
    for (uint32_t gi = 0; gi < hg.out_groups; ++gi) {
      restore(s0);
      const uint64_t b0 = ((uint64_t)gi * R) / hg.out_groups, b1 = ((uint64_t)(gi + 1) * R) / hg.out_groups;
      const uint64_t lo = e[b0], hi = e[b1];
      if (b1 > b0) PGS_TRY(merge_buckets(b0 * R, (b1 - b0) * R, hi - lo));
      PGS_CUDA(cudaEventRecord(hg.ev_out[gi], st));
      if (gi > 0) PGS_TRY(copy_out(gi - 1));
    }
    if (hg.out_groups > 0) PGS_TRY(copy_out(hg.out_groups - 1));
    PGS_CUDA(cudaEventRecord(hg.done, hg.cs));
    PGS_CUDA(cudaStreamWaitEvent(st, hg.done, 0));
    return PGS_OK;
  }

  // P = 1 for every instance: the sorted runs are the buckets.
  int single_bucket() {
    return launch(c, PGS_KERNEL_INVESTIGATOR, 4, 24 * (uint64_t)sh.R, [&] {
      klaunch(st, c.pdl, k_cut_edges, grid_for(sh.R, 256), 256, 0, g, b.cut, b.e);
    });
  }

  // The plan and the launches must agree; then the cut matrix and Table II's loads.
  int finish() {
    if (left != 0 || cur_k != kout) return PGS_ERR_CUDA;   // plan/launch mismatch: never expected
    if (o.cuts && sh.I == 1) {
      PGS_CUDA(cudaMemcpyAsync(o.cuts, b.cut, sizeof(uint64_t) * sh.MAT, cudaMemcpyDeviceToDevice, st));
    }
    const uint32_t launches = c.launches + 1;             // including the statistics kernel
    return launch(c, PGS_KERNEL_STATS, 0, 8 * ((uint64_t)sh.R + sh.I), [&] {
      klaunch(st, c.pdl, k_stats, 1, 256, 0, g, b.e, sh.n, (uint32_t)std::min<uint64_t>(sh.s, 0xFFFFFFFFu),
                                 sh.learned ? PGS_SPLITTERS_LEARNED : PGS_SPLITTERS_SAMPLED, (uint32_t)sh.passes,
                                 launches, b.err, b.fallback, b.learned_ratio, static_cast<DevStats*>(o.stats),
                                 o.bucket_bounds, b.max_ratio);
    });
  }
};

template <typename K, bool V>
int run_pipeline(const Shape& sh, const Options& o, const K* kin, const uint32_t* vin, K* kout, uint32_t* vout,
                 Ctx& c, const Buffers& b, const HostGroups* hg = nullptr) {
  Pipeline<K, V> p(sh, o, kin, vin, kout, vout, c, b);
  PGS_CUDA(cudaMemsetAsync(b.err, 0, sizeof(uint32_t), c.st));
  PGS_TRY(p.local_sort(hg));                                  // step 1
  if (sh.Pmax > 1) {
    K* sample = nullptr;
    PGS_TRY(p.sample_and_splitters(&sample));                 // steps 2-3
    PGS_TRY(p.cuts(sample));                                  // step 4, offsets of step 5
    PGS_TRY(p.exchange());                                    // step 5 (or fused with step 6's first round)
    if (hg && hg->out_groups)
      PGS_TRY(p.merge_buckets_to_host(*hg));                  // step 6, copied back group by group
    else
      PGS_TRY(p.merge_buckets(0, sh.Q, sh.n));                // step 6
  } else {
    PGS_TRY(p.single_bucket());
  }
  return p.finish();
}

// A single sort: build the batch-of-one tables on the device, then the pipeline.
template <typename K, bool V>
int run_sort(const Shape& sh, const Options& o, const K* kin, const uint32_t* vin, K* kout, uint32_t* vout,
             cudaStream_t st) {
  PGS_TRY((set_all_smem_attrs<K, V>()));
  Ctx c;
  c.st = st;
  c.timer = o.timer;
  c.pdl = sh.n <= kPdlMaxKeys;
  Buffers b;
  carve(sh, o.workspace, &b);
  const uint32_t P = sh.R;
  PGS_TRY(launch(c, PGS_KERNEL_OFFSETS, 0, 16 * (uint64_t)(P + 1), [&] {
    klaunch(st, c.pdl, k_tables_single, grid_for(P + 1, 256), 256, 0, b.koff, b.Pt, b.R0, b.mat, b.seg, b.st, b.run_off,
                                                          b.run_inst, sh.n, P, sh.s);
  }));
  return run_pipeline<K, V>(sh, o, kin, vin, kout, vout, c, b);
}

// ---------------------------------------------------------------------------
// pgs_sort_host: a single sort of host-resident keys and payloads.  The device
// copies of input and output follow the sort's own buffers in the workspace.
// ---------------------------------------------------------------------------

struct HostLayout {
  size_t kin = 0, vin = 0, kout = 0, vout = 0, total = 0;
};

inline HostLayout host_layout(const Shape& sh) {
  Buffers b;
  const size_t used = carve(sh, nullptr, &b);
  auto al = [](size_t x) { return (x + kAlign - 1) / kAlign * kAlign; };
  const size_t kb = (size_t)sh.n * sh.w, vb = sh.vals ? (size_t)sh.n * 4 : 0;
  HostLayout L;
  L.kin = al(used);
  L.vin = al(L.kin + kb);
  L.kout = al(L.vin + vb);
  L.vout = al(L.kout + kb);
  L.total = L.vout + vb;
  return L;
}

// Copy stream and events of host-buffer sorts.  They belong to the
// (device, workspace) pair a call uses and are kept for later calls with the
// same pair (two calls sharing a workspace must not overlap anyway), so a
// call creates no stream or event once its pair has been seen.
struct HostCopies {
  cudaStream_t cs = nullptr;
  cudaEvent_t start = nullptr;
  cudaEvent_t ev[kHostGroups] = {};
  cudaEvent_t ev_out[kHostGroups] = {};
  cudaEvent_t done = nullptr;
  void release() {                 // the runtime frees each object once its pending work has finished
    for (uint32_t g = 0; g < kHostGroups; ++g) {
      if (ev[g]) cudaEventDestroy(ev[g]);
      if (ev_out[g]) cudaEventDestroy(ev_out[g]);
      ev[g] = ev_out[g] = nullptr;
    }
    if (done) cudaEventDestroy(done);
    if (start) cudaEventDestroy(start);
    if (cs) cudaStreamDestroy(cs);
    done = start = nullptr;
    cs = nullptr;
  }
  int create() {
    PGS_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    PGS_CUDA(cudaEventCreateWithFlags(&start, cudaEventDisableTiming));
    for (uint32_t g = 0; g < kHostGroups; ++g) {
      PGS_CUDA(cudaEventCreateWithFlags(&ev[g], cudaEventDisableTiming));
      PGS_CUDA(cudaEventCreateWithFlags(&ev_out[g], cudaEventDisableTiming));
    }
    PGS_CUDA(cudaEventCreateWithFlags(&done, cudaEventDisableTiming));
    return PGS_OK;
  }
};

// Process-wide cache of HostCopies (16 pairs, least recently used out).
// Defined once, in the C ABI's translation unit.
int host_copies_for(const void* workspace, HostCopies* out);

template <typename K, bool V>
int run_sort_host(const Shape& sh, const Options& o, const K* hk, const uint32_t* hv, K* hko, uint32_t* hvo,
                  cudaStream_t st) {
  PGS_TRY((set_all_smem_attrs<K, V>()));
  Ctx c;
  c.st = st;
  c.timer = o.timer;
  Buffers b;
  carve(sh, o.workspace, &b);
  const HostLayout L = host_layout(sh);
  char* ws = static_cast<char*>(o.workspace);
  K* dki = reinterpret_cast<K*>(ws + L.kin);
  K* dko = reinterpret_cast<K*>(ws + L.kout);
  uint32_t* dvi = V ? reinterpret_cast<uint32_t*>(ws + L.vin) : nullptr;
  uint32_t* dvo = V ? reinterpret_cast<uint32_t*>(ws + L.vout) : nullptr;
  const uint64_t n = sh.n;
  const uint32_t R = sh.R;
  HostCopies hc;
  PGS_TRY(host_copies_for(o.workspace, &hc));
  HostGroups hg;
  const bool whole = o.copy_back == PGS_COPY_BACK_AUTO && n < kHostGroupMinKeys;
  hg.groups = whole ? 1 : std::min<uint32_t>(kHostGroups, R);
  for (uint32_t g = 0; g <= hg.groups; ++g) hg.r0[g] = (uint32_t)(((uint64_t)g * R) / hg.groups);
  // Bucket groups copied back during step 6 (P = 1 has no step 6; AT_END
  // copies everything after it and never waits on the host).
  hg.out_groups = (!whole && R > 1 && o.copy_back != PGS_COPY_BACK_AT_END) ? std::min<uint32_t>(kHostGroups, R) : 0;
  for (uint32_t g = 0; g < kHostGroups; ++g) {
    hg.ev[g] = hc.ev[g];
    hg.ev_out[g] = hc.ev_out[g];
  }
  hg.done = hc.done;
  hg.cs = hc.cs;
  hg.hk_out = hko;
  hg.hv_out = hvo;
  // The copies may overwrite the workspace only after earlier work on `st`.
  PGS_CUDA(cudaEventRecord(hc.start, st));
  PGS_CUDA(cudaStreamWaitEvent(hc.cs, hc.start, 0));
  hg.copy_in = [&](uint32_t g) -> int {
    const uint64_t e0 = host_run_start(hg.r0[g], n, R), e1 = host_run_start(hg.r0[g + 1], n, R);
    if (e1 > e0) {
      PGS_CUDA(cudaMemcpyAsync(dki + e0, hk + e0, (e1 - e0) * sizeof(K), cudaMemcpyHostToDevice, hc.cs));
      if (V) PGS_CUDA(cudaMemcpyAsync(dvi + e0, hv + e0, (e1 - e0) * 4, cudaMemcpyHostToDevice, hc.cs));
    }
    PGS_CUDA(cudaEventRecord(hg.ev[g], hc.cs));
    return PGS_OK;
  };
  PGS_TRY(launch(c, PGS_KERNEL_OFFSETS, 0, 16 * (uint64_t)(R + 1), [&] {
    klaunch(st, c.pdl, k_tables_single, grid_for(R + 1, 256), 256, 0, b.koff, b.Pt, b.R0, b.mat, b.seg, b.st, b.run_off,
                                                          b.run_inst, n, R, sh.s);
  }));
  PGS_TRY((run_pipeline<K, V>(sh, o, dki, dvi, dko, dvo, c, b, &hg)));
  if (hg.out_groups == 0) {                              // no bucket groups: one copy after step 6
    PGS_CUDA(cudaMemcpyAsync(hko, dko, n * sizeof(K), cudaMemcpyDeviceToHost, st));
    if (V) PGS_CUDA(cudaMemcpyAsync(hvo, dvo, n * 4, cudaMemcpyDeviceToHost, st));
  }
  return PGS_OK;
}

// ---------------------------------------------------------------------------
// pgs_fit_splitters: step 3 on a caller-given sample.  The sample is sorted as
// one run (a single sort with P = 1, keys only) into a buffer after the sort's
// own workspace, then every (m/P)-th key is picked.
// ---------------------------------------------------------------------------

struct FitLayout {
  size_t sorted = 0, ordered = 0, mlp = 0, part = 0, total = 0;
};

// The fit's workspace: a single sort of the sample (P = 1, keys only), the
// sorted sample, and for LEARNED mode its order-form copy and the trainer state.
inline size_t fit_workspace(uint64_t m, const Options& o, Shape* sh_out, FitLayout* lay_out) {
  Options inner = o;
  inner.splitter_mode = PGS_SPLITTERS_SAMPLED;
  Shape sh = single_shape(m, 1, false, inner);
  Buffers b;
  Carver c(nullptr);
  c.used = carve(sh, nullptr, &b);
  FitLayout lay;
  const uint64_t mm = std::max<uint64_t>(m, 1);
  c.take<char>(0);
  lay.sorted = (c.used + kAlign - 1) / kAlign * kAlign;
  c.used = lay.sorted + mm * key_bytes(o.dtype);
  if (o.splitter_mode == PGS_SPLITTERS_LEARNED) {
    lay.ordered = (c.used + kAlign - 1) / kAlign * kAlign;
    c.used = lay.ordered + mm * key_bytes(o.dtype);
    lay.mlp = (c.used + kAlign - 1) / kAlign * kAlign;
    c.used = lay.mlp + sizeof(MlpState);
    lay.part = (c.used + kAlign - 1) / kAlign * kAlign;
    c.used = lay.part + ceil_div(mm, kMlpBatch) * (kMlpW + 1) * sizeof(float);
  }
  lay.total = c.used;
  if (sh_out) *sh_out = sh;
  if (lay_out) *lay_out = lay;
  return lay.total;
}

template <typename K>
int run_fit(uint64_t m, uint32_t P, const Options& o, const K* samples, K* splitters_out, float* model_out,
            cudaStream_t st) {
  Shape sh;
  FitLayout lay;
  fit_workspace(m, o, &sh, &lay);
  Options inner = o;
  inner.splitter_mode = PGS_SPLITTERS_SAMPLED;
  inner.bucket_bounds = nullptr;
  inner.cuts = nullptr;
  inner.splitters = nullptr;
  inner.stats = nullptr;
  char* ws = static_cast<char*>(o.workspace);
  K* sorted = reinterpret_cast<K*>(ws + lay.sorted);
  PGS_TRY((run_sort<K, false>(sh, inner, samples, nullptr, sorted, nullptr, st)));
  Ctx c;
  c.st = st;
  c.timer = o.timer;
  // The inner sort already returned the caller's bit patterns: no transform here.
  PGS_TRY(launch(c, PGS_KERNEL_SPLITTERS, 3, 2 * (uint64_t)P * sizeof(K), [&] {
    klaunch(st, c.pdl, k_pick_splitters_flat<K>, grid_for(P, 256), 256, 0, sorted, m, P, splitters_out, 0);
  }));
  if (o.splitter_mode != PGS_SPLITTERS_LEARNED || !model_out) return PGS_OK;
  // K10 on the sorted sample, in order form.
  K* ordered = reinterpret_cast<K*>(ws + lay.ordered);
  MlpState* mlp = reinterpret_cast<MlpState*>(ws + lay.mlp);
  float* part = reinterpret_cast<float*>(ws + lay.part);
  PGS_TRY(launch(c, PGS_KERNEL_SAMPLE, 3, 2 * m * sizeof(K), [&] {
    klaunch(st, c.pdl, k_to_order<K>, grid_for(m, 256), 256, 0, sorted, ordered, m, o.dtype == PGS_F32);
  }));
  PGS_TRY(launch(c, PGS_KERNEL_SPLITTERS, 3, 16 * kMlpW, [&] { klaunch(st, c.pdl, k_mlp_init<K>, 1, 256, 0, ordered, m, mlp); }));
  const uint32_t nparts = (uint32_t)ceil_div(m, kMlpBatch);
  for (uint32_t step = 1; step <= (uint32_t)kMlpSteps; ++step) {
    PGS_TRY(launch(c, PGS_KERNEL_SPLITTERS, 3, m * sizeof(K), [&] {
      klaunch(st, c.pdl, k_mlp_grad<K>, nparts, kMlpBatch, sizeof(MlpGradSmem), ordered, m, mlp, part);
    }));
    PGS_TRY(launch(c, PGS_KERNEL_SPLITTERS, 3, 4ull * nparts * (kMlpW + 1), [&] {
      klaunch(st, c.pdl, k_mlp_adam, (unsigned)ceil_div(kMlpW + 1, kAdamParams), kAdamParams * kAdamWarps, 0, 
          part, nparts, mlp, step, m);
    }));
  }
  return launch(c, PGS_KERNEL_SPLITTERS, 3, 16 * kMlpW, [&] { klaunch(st, c.pdl, k_mlp_finalize, 1, 256, 0, mlp, model_out); });
}

}  // namespace pgs
