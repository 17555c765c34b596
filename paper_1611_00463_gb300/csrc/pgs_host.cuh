// Host orchestration of the load-balanced sample sort: the plan (pass counts,
// workspace layout) and the launch sequence of Section IV's six steps on one
// stream.  Nothing here synchronises the stream or allocates device memory.
#pragma once

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>

#include "pgs.h"
#include "pgs_kernels.cuh"

namespace pgs {

constexpr uint32_t kMaxP = 8192;               // cut matrices are P x (P+1)
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
  if (o->dtype < PGS_U32 || o->dtype > PGS_F32) return PGS_ERR_INVALID;
  if (!(o->eps > 0.0f) || o->eps > 1.0f) return PGS_ERR_INVALID;
  if (o->investigator < 0 || o->investigator > 2) return PGS_ERR_INVALID;
  if (o->exchange < 0 || o->exchange > 2) return PGS_ERR_INVALID;
  if (o->splitter_mode < 0 || o->splitter_mode > 1) return PGS_ERR_INVALID;
  if (o->exchange == PGS_EXCHANGE_FUSED) return PGS_ERR_UNSUPPORTED;
  if (o->splitter_mode == PGS_SPLITTERS_LEARNED) return PGS_ERR_UNSUPPORTED;
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

struct Plan {
  uint64_t n = 0;
  uint32_t P = 1;                 // effective partitions
  int w = 4;                      // key bytes
  bool vals = false;
  uint64_t s = 1;                 // samples per run
  bool all_samples = false;       // s >= every run length: every key is a sample
  uint64_t S = 0;                 // total samples
  uint64_t nmax = 0;              // longest run
  int run_rounds = 0;             // merge rounds to grow block-sorted tiles into runs
  int bucket_rounds = 0;          // merge rounds of step 6 (ceil(log2 P))
  uint64_t max_pairs = 1;
  uint64_t max_tiles = 1;
  uint64_t scan_len = 1;          // longest array scanned
  int passes = 0;                 // full passes over the keys
};

inline uint64_t samples_per_run(uint32_t P, int w, const Options& o) {
  uint64_t s = o.samples_per_run ? o.samples_per_run
                                 : std::max<uint64_t>(1, kSampleBufferBytes / ((uint64_t)P * w));
  if (o.guaranteed) {
    uint64_t g = (uint64_t)std::ceil((double)P / (double)o.eps);
    s = std::max(s, g);
  }
  return s;
}

inline Plan make_plan(uint64_t n, uint32_t P_req, bool vals, const Options& o) {
  Plan p;
  p.n = n;
  p.w = key_bytes(o.dtype);
  p.vals = vals;
  p.P = (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(P_req, n));
  const uint32_t P = p.P;
  p.nmax = ceil_div(n, P);
  const uint64_t nmin = n / P;
  p.s = samples_per_run(P, p.w, o);
  p.all_samples = p.s >= p.nmax;
  p.S = p.all_samples ? n : (uint64_t)P * p.s;
  (void)nmin;
  uint64_t w = kTile;
  while (w < p.nmax) { w *= 2; ++p.run_rounds; }
  p.bucket_rounds = P > 1 ? ceil_log2(P) : 0;
  // Largest number of pairs in any round.
  uint64_t mp = 1;
  for (int k = 0; k < p.run_rounds; ++k)
    mp = std::max<uint64_t>(mp, (uint64_t)P * ceil_div(p.nmax, 2ull * ((uint64_t)kTile << k)));
  for (int k = 0; k < p.bucket_rounds; ++k) {
    uint64_t per = ceil_div(P, 2ull << k);
    mp = std::max<uint64_t>(mp, (uint64_t)P * per);
  }
  p.max_pairs = mp;
  p.max_tiles = ceil_div(std::max<uint64_t>(n, 1), kTile) + mp + 1;
  p.scan_len = std::max<uint64_t>(mp, (uint64_t)P * P);
  p.passes = 1 + p.run_rounds + (P > 1 ? 1 + p.bucket_rounds : 0);
  return p;
}

// Device buffers inside the workspace.
struct Buffers {
  void* alt_k; uint32_t* alt_v;
  void* samp_a; void* samp_b; void* spl;
  uint64_t *lb, *cnt, *cut, *sizes, *off, *e, *sample_off;
  Pair* pairs; uint64_t *tcount, *tbegin;
  uint32_t* tile_pair; uint64_t* part;
  uint64_t *scan_sums, *scan_sums2;
  uint64_t* first_seg;
  DevStats* stats; uint32_t* err;
};

inline size_t carve(const Plan& p, void* base, Buffers* b) {
  Carver c(base);
  const uint64_t P = p.P;
  b->alt_k = c.take<char>(p.n * p.w);
  b->alt_v = p.vals ? c.take<uint32_t>(p.n) : nullptr;
  b->samp_a = c.take<char>(p.S * p.w);
  b->samp_b = c.take<char>(p.S * p.w);
  b->spl = c.take<char>(P * p.w);
  b->lb = c.take<uint64_t>(P * (P + 1));
  b->cnt = c.take<uint64_t>(P * (P + 1));
  b->cut = c.take<uint64_t>(P * (P + 1));
  b->sizes = c.take<uint64_t>(P * P);
  b->off = c.take<uint64_t>(P * P + 1);
  b->e = c.take<uint64_t>(P + 1);
  b->sample_off = c.take<uint64_t>(P + 1);
  b->pairs = c.take<Pair>(p.max_pairs);
  b->tcount = c.take<uint64_t>(p.max_pairs);
  b->tbegin = c.take<uint64_t>(p.max_pairs + 1);
  b->tile_pair = c.take<uint32_t>(p.max_tiles);
  b->part = c.take<uint64_t>(p.max_tiles + 1);
  const uint64_t chunks = ceil_div(p.scan_len, kScanChunk);
  b->scan_sums = c.take<uint64_t>(chunks + 1);
  b->scan_sums2 = c.take<uint64_t>(chunks + 1);
  b->first_seg = c.take<uint64_t>(ceil_div(std::max<uint64_t>(p.n, 1), kScatterTile));
  b->stats = c.take<DevStats>(1);
  b->err = c.take<uint32_t>(1);
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
};

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
    return launch(c, PGS_KERNEL_SCAN, step, bytes, [&] { k_scan_chunks<<<1, kScanNT, 0, c.st>>>(in, m, out, nullptr); });
  if (chunks > (uint64_t)kScanChunk) return PGS_ERR_UNSUPPORTED;
  PGS_TRY(launch(c, PGS_KERNEL_SCAN, step, 8 * m,
                 [&] { k_scan_reduce<<<(unsigned)chunks, kScanNT, 0, c.st>>>(in, m, sums); }));
  PGS_TRY(launch(c, PGS_KERNEL_SCAN, step, 16 * chunks,
                 [&] { k_scan_chunks<<<1, kScanNT, 0, c.st>>>(sums, chunks, sums2, nullptr); }));
  return launch(c, PGS_KERNEL_SCAN, step, bytes,
                [&] { k_scan_chunks<<<(unsigned)chunks, kScanNT, 0, c.st>>>(in, m, out, sums2); });
}

// Opt in to more than 48 KB of dynamic shared memory (set on every call: the
// attribute belongs to the current device, and the call costs microseconds).
template <typename K, bool V>
inline int set_smem_attrs() {
  PGS_CUDA(cudaFuncSetAttribute(k_block_sort<K, V>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)sizeof(BlockSortSmem<K>)));
  PGS_CUDA(cudaFuncSetAttribute(k_merge<K, V>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)sizeof(MergeSmem<K>)));
  PGS_CUDA(cudaFuncSetAttribute(k_scatter<K, V>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)sizeof(ScatterSmem<K>)));
  return PGS_OK;
}

// One pairwise merge round over pairs already described in b.pairs / b.tcount.
// `len` keys take part; every one of them is read and written once.
template <typename K, bool V>
inline int merge_round(Ctx& c, const K* ks, const uint32_t* vs, K* kd, uint32_t* vd, uint64_t npairs,
                       uint64_t len, const Buffers& b, int f32_out, uint32_t step) {
  PGS_TRY(scan_u64(c, b.tcount, b.tbegin, npairs, b.scan_sums, b.scan_sums2, step));
  const uint64_t tiles_ub = ceil_div(len, kTile) + npairs;
  PGS_TRY(launch(c, PGS_KERNEL_PARTITION, step, 24 * ceil_div(len, kTile), [&] {
    k_partition<K><<<grid_for(tiles_ub, 256), 256, 0, c.st>>>(ks, b.pairs, b.tbegin, npairs, b.tile_pair, b.part);
  }));
  const uint64_t bytes = 2 * len * (sizeof(K) + (V ? 4 : 0));
  return launch(c, PGS_KERNEL_MERGE, step, bytes, [&] {
    k_merge<K, V><<<(unsigned)tiles_ub, kNT, sizeof(MergeSmem<K>), c.st>>>(ks, vs, kd, vd, b.pairs, b.tbegin,
                                                                          npairs, b.tile_pair, b.part, f32_out);
  });
}

// ---------------------------------------------------------------------------
// The sort: Section IV, steps 1-6.
// ---------------------------------------------------------------------------

template <typename K, bool V>
int run_sort(const Plan& p, const Options& o, const K* kin, const uint32_t* vin, K* kout,
             uint32_t* vout, cudaStream_t st) {
  PGS_TRY((set_smem_attrs<K, V>()));
  PGS_TRY((set_smem_attrs<K, false>()));     // the sample sort runs keys only
  Ctx c;
  c.st = st;
  c.timer = o.timer;
  Buffers b;
  carve(p, o.workspace, &b);
  const uint64_t n = p.n;
  const uint32_t P = p.P;
  const int f32 = o.dtype == PGS_F32;
  const uint64_t kv = sizeof(K) + (V ? 4 : 0);       // bytes per key/payload pair

  // Ping-pong so that the last pass lands in kout.
  const int after_block = p.passes - 1;
  K* cur_k = (after_block % 2 == 0) ? kout : static_cast<K*>(b.alt_k);
  K* oth_k = (cur_k == kout) ? static_cast<K*>(b.alt_k) : kout;
  uint32_t* cur_v = V ? ((after_block % 2 == 0) ? vout : b.alt_v) : nullptr;
  uint32_t* oth_v = V ? ((cur_v == vout) ? b.alt_v : vout) : nullptr;
  int left = after_block;

  // Step 1: local sort of every run.  Block sort of kTile tiles ...
  const uint32_t tiles_per_run = (uint32_t)ceil_div(p.nmax, kTile);
  PGS_TRY(launch(c, PGS_KERNEL_BLOCK_SORT, 1, 2 * n * kv, [&] {
    k_block_sort<K, V><<<(unsigned)((uint64_t)P * tiles_per_run), kNT, sizeof(BlockSortSmem<K>), st>>>(
        kin, vin, cur_k, cur_v, n, P, tiles_per_run, f32, left == 0 ? f32 : 0);
  }));
  // ... then balanced pairwise merge rounds (Fig. 2) until each run is one list.
  for (int k = 0; k < p.run_rounds; ++k) {
    const uint64_t w = (uint64_t)kTile << k;
    const uint64_t ppr = ceil_div(p.nmax, 2 * w);
    const uint64_t np = ppr * P;
    PGS_TRY(launch(c, PGS_KERNEL_PAIRS, 1, 32 * np, [&] {
      k_pairs_runs<<<grid_for(np, 256), 256, 0, st>>>(b.pairs, b.tcount, n, P, w, ppr);
    }));
    --left;
    PGS_TRY((merge_round<K, V>(c, cur_k, cur_v, oth_k, oth_v, np, n, b, left == 0 ? f32 : 0, 1)));
    std::swap(cur_k, oth_k);
    std::swap(cur_v, oth_v);
  }

  if (P > 1) {
    // Step 2: regular samples of every sorted run, gathered in (run, position) order.
    K* sa = static_cast<K*>(b.samp_a);
    K* sb = static_cast<K*>(b.samp_b);
    PGS_TRY(launch(c, PGS_KERNEL_SAMPLE, 2, 2 * p.S * sizeof(K), [&] {
      k_sample<K><<<grid_for(p.S, 256), 256, 0, st>>>(cur_k, n, P, p.s, p.all_samples, sa, p.S);
    }));
    PGS_TRY(launch(c, PGS_KERNEL_SAMPLE, 2, 8 * (P + 1), [&] {
      k_sample_offsets<<<grid_for(P + 1, 256), 256, 0, st>>>(b.sample_off, n, P, p.s, p.all_samples);
    }));
    // Step 3: the Master sorts the samples (merging the P sorted sample lists
    // with the Fig. 2 schedule) and picks every (S/P)-th one.
    for (int k = 0; k < p.bucket_rounds; ++k) {
      const uint32_t step = 1u << k;
      const uint64_t np = ceil_div(P, 2ull * step);
      PGS_TRY(launch(c, PGS_KERNEL_PAIRS, 3, 32 * np, [&] {
        k_pairs_lists<<<grid_for(np, 256), 256, 0, st>>>(b.pairs, b.tcount, b.sample_off, 0, 1, P, step, np);
      }));
      PGS_TRY((merge_round<K, false>(c, sa, nullptr, sb, nullptr, np, p.S, b, 0, 3)));
      std::swap(sa, sb);
    }
    PGS_TRY(launch(c, PGS_KERNEL_SPLITTERS, 3, 2 * (uint64_t)P * sizeof(K), [&] {
      k_pick_splitters<K><<<grid_for(P - 1, 256), 256, 0, st>>>(sa, p.S, P, static_cast<K*>(b.spl),
                                                                static_cast<K*>(o.splitters), f32);
    }));
    // Step 4: binary search of every splitter in every run, then the investigator.
    PGS_TRY(launch(c, PGS_KERNEL_CUT_SEARCH, 4, 16 * (uint64_t)P * P, [&] {
      k_cut_search<K><<<grid_for((uint64_t)P * (P - 1), 256), 256, 0, st>>>(
          cur_k, n, P, static_cast<const K*>(b.spl), b.lb, b.cnt);
    }));
    PGS_TRY(launch(c, PGS_KERNEL_INVESTIGATOR, 4, 16 * (uint64_t)P, [&] {
      k_cut_edges<<<grid_for(P, 256), 256, 0, st>>>(b.cut, b.e, n, P);
    }));
    PGS_TRY(launch(c, PGS_KERNEL_INVESTIGATOR, 4, 24 * (uint64_t)P * P, [&] {
      k_investigator<K><<<P - 1, 256, 0, st>>>(b.lb, b.cnt, static_cast<const K*>(b.spl), n, P, o.investigator,
                                               b.cut, b.e);
    }));
    // Section IV-C: receive offsets of every (run, bucket) segment.
    PGS_TRY(launch(c, PGS_KERNEL_OFFSETS, 5, 16 * (uint64_t)P * P, [&] {
      k_bucket_sizes<<<grid_for((uint64_t)P * P, 256), 256, 0, st>>>(b.cut, P, b.sizes);
    }));
    PGS_TRY(scan_u64(c, b.sizes, b.off, (uint64_t)P * P, b.scan_sums, b.scan_sums2, 5));
    // Step 5: the exchange, as an in-HBM scatter into bucket-major order.
    const uint64_t stiles = ceil_div(n, kScatterTile);
    PGS_TRY(launch(c, PGS_KERNEL_OFFSETS, 5, 8 * stiles, [&] {
      k_scatter_part<<<grid_for(stiles, 256), 256, 0, st>>>(b.off, (uint64_t)P * P, n, b.first_seg);
    }));
    --left;
    PGS_TRY(launch(c, PGS_KERNEL_SCATTER, 5, 2 * n * kv, [&] {
      k_scatter<K, V><<<(unsigned)stiles, kScatterNT, sizeof(ScatterSmem<K>), st>>>(
          cur_k, cur_v, oth_k, oth_v, b.off, b.cut, b.first_seg, n, P, left == 0 ? f32 : 0);
    }));
    std::swap(cur_k, oth_k);
    std::swap(cur_v, oth_v);
    // Step 6: every bucket merges its P segments with the Fig. 2 schedule.
    for (int k = 0; k < p.bucket_rounds; ++k) {
      const uint32_t step = 1u << k;
      const uint64_t per = ceil_div(P, 2ull * step);
      const uint64_t np = per * P;
      PGS_TRY(launch(c, PGS_KERNEL_PAIRS, 6, 32 * np, [&] {
        k_pairs_lists<<<grid_for(np, 256), 256, 0, st>>>(b.pairs, b.tcount, b.off, P, P, P, step, per);
      }));
      --left;
      PGS_TRY((merge_round<K, V>(c, cur_k, cur_v, oth_k, oth_v, np, n, b, left == 0 ? f32 : 0, 6)));
      std::swap(cur_k, oth_k);
      std::swap(cur_v, oth_v);
    }
  } else {
    PGS_TRY(launch(c, PGS_KERNEL_INVESTIGATOR, 4, 32, [&] { k_cut_edges<<<1, 32, 0, st>>>(b.cut, b.e, n, P); }));
  }
  if (left != 0 || cur_k != kout) return PGS_ERR_CUDA;   // plan/launch mismatch: never expected

  if (o.cuts) {
    PGS_CUDA(cudaMemcpyAsync(o.cuts, b.cut, sizeof(uint64_t) * (uint64_t)P * (P + 1),
                             cudaMemcpyDeviceToDevice, st));
  }
  PGS_CUDA(cudaMemsetAsync(b.err, 0, sizeof(uint32_t), st));
  const uint32_t launches = c.launches + 1;             // including the statistics kernel
  return launch(c, PGS_KERNEL_STATS, 0, 8 * (uint64_t)(P + 1), [&] {
    k_stats<<<1, 256, 0, st>>>(b.e, n, P, (uint32_t)std::min<uint64_t>(p.s, 0xFFFFFFFFu), PGS_SPLITTERS_SAMPLED,
                               (uint32_t)p.passes, launches, b.err, static_cast<DevStats*>(o.stats),
                               o.bucket_bounds);
  });
}

// ---------------------------------------------------------------------------
// pgs_fit_splitters: step 3 on a caller-given sample.
// ---------------------------------------------------------------------------

struct FitPlan {
  uint64_t m = 0;
  uint32_t P = 1;
  int w = 4;
  int rounds = 0;
  uint64_t max_pairs = 1, max_tiles = 1;
};

inline FitPlan make_fit_plan(uint64_t m, uint32_t P, const Options& o) {
  FitPlan f;
  f.m = m;
  f.P = P;
  f.w = key_bytes(o.dtype);
  uint64_t w = kTile;
  while (w < m) { w *= 2; ++f.rounds; }
  f.max_pairs = std::max<uint64_t>(1, ceil_div(m, 2ull * kTile));
  f.max_tiles = ceil_div(std::max<uint64_t>(m, 1), kTile) + f.max_pairs + 1;
  return f;
}

inline size_t carve_fit(const FitPlan& f, void* base, void** a, void** bb, Buffers* b) {
  Carver c(base);
  *a = c.take<char>(f.m * f.w);
  *bb = c.take<char>(f.m * f.w);
  b->pairs = c.take<Pair>(f.max_pairs);
  b->tcount = c.take<uint64_t>(f.max_pairs);
  b->tbegin = c.take<uint64_t>(f.max_pairs + 1);
  b->tile_pair = c.take<uint32_t>(f.max_tiles);
  b->part = c.take<uint64_t>(f.max_tiles + 1);
  const uint64_t chunks = ceil_div(f.max_pairs, kScanChunk);
  b->scan_sums = c.take<uint64_t>(chunks + 1);
  b->scan_sums2 = c.take<uint64_t>(chunks + 1);
  return c.used;
}

template <typename K>
int run_fit(const FitPlan& f, const Options& o, const K* samples, K* splitters_out, cudaStream_t st) {
  PGS_TRY((set_smem_attrs<K, false>()));
  Ctx c;
  c.st = st;
  c.timer = o.timer;
  Buffers b;
  void *va, *vb;
  carve_fit(f, o.workspace, &va, &vb, &b);
  K* a = static_cast<K*>(va);
  K* bb = static_cast<K*>(vb);
  const int f32 = o.dtype == PGS_F32;
  // Sort the sample as one run: block sort, then pairwise merge rounds.
  const uint32_t tiles = (uint32_t)ceil_div(f.m, kTile);
  PGS_TRY(launch(c, PGS_KERNEL_BLOCK_SORT, 3, 2 * f.m * sizeof(K), [&] {
    k_block_sort<K, false><<<tiles, kNT, sizeof(BlockSortSmem<K>), st>>>(samples, nullptr, a, nullptr, f.m, 1,
                                                                         tiles, f32, 0);
  }));
  for (int k = 0; k < f.rounds; ++k) {
    const uint64_t w = (uint64_t)kTile << k;
    const uint64_t np = ceil_div(f.m, 2 * w);
    PGS_TRY(launch(c, PGS_KERNEL_PAIRS, 3, 32 * np, [&] {
      k_pairs_runs<<<grid_for(np, 256), 256, 0, st>>>(b.pairs, b.tcount, f.m, 1, w, np);
    }));
    PGS_TRY((merge_round<K, false>(c, a, nullptr, bb, nullptr, np, f.m, b, 0, 3)));
    std::swap(a, bb);
  }
  return launch(c, PGS_KERNEL_SPLITTERS, 3, 2 * (uint64_t)f.P * sizeof(K), [&] {
    k_pick_splitters<K><<<grid_for(f.P, 256), 256, 0, st>>>(a, f.m, f.P, bb, splitters_out, f32);
  });
}

}  // namespace pgs
