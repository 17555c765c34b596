// Batched sort: the host plan of a batch of instances, the upload of its
// tables, and the launch of the whole pipeline for every instance at once.
#include <atomic>
#include <cstring>
#include <new>
#include <vector>

#include "pgs_graph.cuh"
#include "pgs_host.cuh"

namespace pgs {
int batch_attrs_u32(bool vals);
int batch_attrs_u64(bool vals);
int batch_u32(const Shape&, const Options&, const void*, const uint32_t*, void*, uint32_t*, cudaStream_t);
int batch_u64(const Shape&, const Options&, const void*, const uint32_t*, void*, uint32_t*, cudaStream_t);
int fill_random_u32(void*, uint32_t*, uint64_t, uint64_t, cudaStream_t);
int fill_random_u64(void*, uint32_t*, uint64_t, uint64_t, cudaStream_t);
}  // namespace pgs

using namespace pgs;

struct pgs_batch {
  uint64_t id = 0;            // unique per plan (a freed plan's address may come back)
  Shape sh;
  Options o;
  std::vector<char> tables;   // the table region of the workspace, laid out by carve()
  size_t tables_bytes = 0;
  size_t ws_bytes = 0;
  int variant = 0;            // merge tile shape chosen by pgs_batch_tune
};

extern "C" {

uint32_t pgs_batch_auto_partitions(uint64_t n) {
  if (n < (1ull << 16)) return 1;
  uint32_t k = 0;
  while ((n >> (16 + k + 1)) != 0) ++k;               // floor(log2(n / 2^16))
  return k >= 8 ? 256u : (1u << k);
}

int pgs_batch_create(const uint64_t* offsets, uint32_t num, const uint32_t* P, int with_vals,
                     const pgs_config* cfg, pgs_batch** out) {
  if (!out) return PGS_ERR_INVALID;
  *out = nullptr;
  if (!offsets || num == 0 || offsets[0] != 0) return PGS_ERR_INVALID;
  Options o;
  int rc = read_options(cfg, &o);
  if (rc) return rc;
  if (o.splitter_mode == PGS_SPLITTERS_LEARNED) return PGS_ERR_UNSUPPORTED;   // single sorts only
  pgs_batch* bt = new (std::nothrow) pgs_batch;
  static std::atomic<uint64_t> next_id{1};
  if (bt) bt->id = next_id.fetch_add(1);
  if (!bt) return PGS_ERR_INVALID;
  bt->o = o;
  Shape& sh = bt->sh;
  sh.I = num;
  sh.w = key_bytes(o.dtype);
  sh.vals = with_vals != 0;
  sh.n = offsets[num];
  std::vector<uint64_t> koff(num + 1), mat(num + 1), seg(num + 1), st(num);
  std::vector<uint32_t> Pv(num), R0(num + 1);
  uint64_t R = 0, Q = 0, MAT = 0, S = 0, maxlen = 0;
  uint32_t Pmax = 1;
  for (uint32_t i = 0; i < num; ++i) {
    if (offsets[i + 1] < offsets[i]) { delete bt; return PGS_ERR_INVALID; }
    const uint64_t ni = offsets[i + 1] - offsets[i];
    uint64_t Pi = P ? P[i] : pgs_batch_auto_partitions(ni);
    if (Pi == 0) { delete bt; return PGS_ERR_INVALID; }
    Pi = std::max<uint64_t>(1, std::min<uint64_t>(Pi, ni));
    if (Pi > kMaxP) { delete bt; return PGS_ERR_UNSUPPORTED; }
    koff[i] = offsets[i];
    Pv[i] = (uint32_t)Pi;
    R0[i] = (uint32_t)R;
    mat[i] = MAT;
    seg[i] = Q;
    st[i] = Pi > 1 ? samples_per_run((uint32_t)Pi, sh.w, o) : 0;
    for (uint64_t r = 0; r < Pi; ++r) {
      const uint64_t len = ((r + 1) * ni) / Pi - (r * ni) / Pi;
      maxlen = std::max(maxlen, len);
      S += std::min(st[i], len);
    }
    R += Pi;
    Q += Pi * Pi;
    MAT += Pi * (Pi + 1);
    Pmax = std::max<uint32_t>(Pmax, (uint32_t)Pi);
    if (R > 0xFFFFFFF0ull) { delete bt; return PGS_ERR_UNSUPPORTED; }
  }
  koff[num] = offsets[num];
  R0[num] = (uint32_t)R;
  mat[num] = MAT;
  seg[num] = Q;
  sh.R = (uint32_t)R;
  sh.Pmax = Pmax;
  sh.Q = Q;
  sh.MAT = MAT;
  sh.S = S;
  sh.maxlen = maxlen;
  sh.s = 0;
  sh.scatter = o.exchange == PGS_EXCHANGE_SCATTER;
  sh.four = use_four_way(sh.n, o);
  finish_shape(sh);

  std::vector<uint64_t> run_off(R + 1);
  std::vector<uint32_t> run_inst(R);
  for (uint32_t i = 0; i < num; ++i) {
    const uint64_t ni = koff[i + 1] - koff[i];
    for (uint64_t r = 0; r < Pv[i]; ++r) {
      run_off[R0[i] + r] = koff[i] + (r * ni) / Pv[i];
      run_inst[R0[i] + r] = i;
    }
  }
  run_off[R] = koff[num];

  // Lay the tables out exactly where carve() puts them in a workspace.
  Buffers b;
  bt->ws_bytes = carve(sh, nullptr, &b, &bt->tables_bytes);
  bt->tables.assign(bt->tables_bytes, 0);
  carve(sh, bt->tables.data(), &b);
  std::memcpy(b.koff, koff.data(), koff.size() * sizeof(uint64_t));
  std::memcpy(b.Pt, Pv.data(), Pv.size() * sizeof(uint32_t));
  std::memcpy(b.R0, R0.data(), R0.size() * sizeof(uint32_t));
  std::memcpy(b.mat, mat.data(), mat.size() * sizeof(uint64_t));
  std::memcpy(b.seg, seg.data(), seg.size() * sizeof(uint64_t));
  std::memcpy(b.st, st.data(), st.size() * sizeof(uint64_t));
  std::memcpy(b.run_off, run_off.data(), run_off.size() * sizeof(uint64_t));
  std::memcpy(b.run_inst, run_inst.data(), run_inst.size() * sizeof(uint32_t));
  *out = bt;
  return PGS_OK;
}

size_t pgs_batch_workspace_bytes(const pgs_batch* bt) { return bt ? bt->ws_bytes : 0; }

int pgs_batch_upload(pgs_batch* bt, void* workspace, uint64_t workspace_bytes, void* stream) {
  if (!bt) return PGS_ERR_INVALID;
  if (!workspace || (reinterpret_cast<uintptr_t>(workspace) % kAlign) != 0 || workspace_bytes < bt->ws_bytes)
    return PGS_ERR_WORKSPACE;
  DeviceGuard dg;
  PGS_TRY(dg.use_device_of(workspace));
  PGS_TRY(bt->o.dtype == PGS_U64 ? batch_attrs_u64(bt->sh.vals) : batch_attrs_u32(bt->sh.vals));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  PGS_CUDA(cudaMemcpyAsync(workspace, bt->tables.data(), bt->tables_bytes, cudaMemcpyHostToDevice, st));
  PGS_CUDA(cudaStreamSynchronize(st));
  return PGS_OK;
}

int pgs_sort_batched_copy(pgs_batch* bt, const void* keys_in, const uint32_t* vals_in, void* keys_out,
                          uint32_t* vals_out, void* stream, const pgs_config* cfg) {
  if (!bt) return PGS_ERR_INVALID;
  Options o;
  int rc = read_options(cfg, &o);
  if (rc) return rc;
  if (o.dtype != bt->o.dtype) return PGS_ERR_INVALID;
  if (o.splitter_mode == PGS_SPLITTERS_LEARNED) return PGS_ERR_UNSUPPORTED;
  if ((vals_in != nullptr) != bt->sh.vals || (vals_out != nullptr) != bt->sh.vals) return PGS_ERR_INVALID;
  if (bt->sh.n == 0) return PGS_OK;
  if (!keys_in || !keys_out) return PGS_ERR_INVALID;
  if (!o.workspace || (reinterpret_cast<uintptr_t>(o.workspace) % kAlign) != 0 || o.workspace_bytes < bt->ws_bytes)
    return PGS_ERR_WORKSPACE;
  DeviceGuard dg;
  PGS_TRY(dg.use_device_of(o.workspace));                   // the device the batch's tables were uploaded to
  // Batch options: the sampling settings fixed at create time; the per-call
  // outputs of a single sort are not written for a batch.
  Options run = bt->o;
  run.workspace = o.workspace;
  run.workspace_bytes = o.workspace_bytes;
  run.stats = o.stats;
  run.timer = o.timer;
  run.investigator = o.investigator;
  run.tile_variant = o.tile_variant ? o.tile_variant : bt->variant;
  run.bucket_bounds = nullptr;
  run.cuts = nullptr;
  run.splitters = nullptr;
  run.spin_limit = o.spin_limit;
  run.fault_inject = o.fault_inject;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // Repeated identical calls replay a captured graph (pgs_graph_cache): the
  // key holds the plan, the buffers (the workspace holds the uploaded tables)
  // and the per-call options.
  const GraphKey key{2, bt->id, key_ptr(keys_in), key_ptr(vals_in), key_ptr(keys_out), key_ptr(vals_out),
                     key_ptr(run.workspace), run.workspace_bytes, key_ptr(run.stats), (uint64_t)run.investigator,
                     (uint64_t)run.tile_variant, (uint64_t)run.dtype, run.spin_limit, (uint64_t)run.fault_inject};
  const bool allow = o.timer == nullptr && o.graph_cache == PGS_GRAPH_CACHE_AUTO;
  const Shape& sh = bt->sh;
  return launch_cached(key, allow, st, [&](cudaStream_t s) {
    if (o.dtype == PGS_U64) return batch_u64(sh, run, keys_in, vals_in, keys_out, vals_out, s);
    return batch_u32(sh, run, keys_in, vals_in, keys_out, vals_out, s);
  });
}

int pgs_sort_batched(pgs_batch* bt, void* keys, uint32_t* vals, void* stream, const pgs_config* cfg) {
  return pgs_sort_batched_copy(bt, keys, vals, keys, vals, stream, cfg);
}

int pgs_batch_tune(pgs_batch* bt, void* scratch_keys, uint32_t* scratch_vals, void* stream, const pgs_config* cfg,
                   uint32_t* chosen, float* ms_out) {
  if (!bt) return PGS_ERR_INVALID;
  if (bt->sh.n && !scratch_keys) return PGS_ERR_INVALID;
  if ((scratch_vals != nullptr) != bt->sh.vals) return PGS_ERR_INVALID;
  DeviceGuard dg;
  if (bt->sh.n) PGS_TRY(dg.use_device_of(scratch_keys));     // the events belong to the sorting device
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaEvent_t e0, e1;
  PGS_CUDA(cudaEventCreate(&e0));
  if (cudaError_t e = cudaEventCreate(&e1); e != cudaSuccess) {
    cudaEventDestroy(e0);
    return record_cuda_error(e, "cudaEventCreate", __LINE__);
  }
  float best = 0.0f;
  int best_v = 0;
  int rc = PGS_OK;
  for (int v = 0; v < PGS_TILE_VARIANTS && rc == PGS_OK; ++v) {
    pgs_config c = cfg ? *cfg : pgs_config{};
    c.tile_variant = v;
    c.graph_cache = PGS_GRAPH_CACHE_OFF;                    // time the launches, not a capture
    float ms = 0.0f;
    for (int rep = 0; rep < 2 && rc == PGS_OK; ++rep) {      // first run warms up
      rc = bt->o.dtype == PGS_U64 ? fill_random_u64(scratch_keys, scratch_vals, bt->sh.n, 0x5EED + rep, st)
                                  : fill_random_u32(scratch_keys, scratch_vals, bt->sh.n, 0x5EED + rep, st);
      if (rc) break;
      if (cudaEventRecord(e0, st) != cudaSuccess) { rc = PGS_ERR_CUDA; break; }
      rc = pgs_sort_batched(bt, scratch_keys, scratch_vals, stream, &c);
      if (rc) break;
      if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
          cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) rc = PGS_ERR_CUDA;
    }
    if (ms_out) ms_out[v] = ms;
    if (rc == PGS_OK && (v == 0 || ms < best)) {
      best = ms;
      best_v = v;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  bt->variant = best_v;
  if (chosen) *chosen = (uint32_t)best_v;
  return PGS_OK;
}

int pgs_batch_destroy(pgs_batch* bt) {
  if (!bt) return PGS_ERR_INVALID;
  delete bt;
  return PGS_OK;
}

}  // extern "C"
