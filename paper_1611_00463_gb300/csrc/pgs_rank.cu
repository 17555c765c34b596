// The C ABI of the sharded sort's rank steps (declared in include/pgs.h):
// Section IV's steps 2, 4 and 6 for one of G ranks, the investigator over all
// ranks' counts, and the merge of received segments.  The caller runs step 1
// with pgs_sort_copy, step 3 with pgs_fit_splitters and moves the data
// between ranks (samples, counts, segments) with its own collectives.
#include "pgs_rank.cuh"

namespace pgs {
int merge_lists_u32(const Shape&, const Options&, const void*, const uint32_t*, void*, uint32_t*, const uint64_t*,
                    uint32_t, cudaStream_t);
int merge_lists_u64(const Shape&, const Options&, const void*, const uint32_t*, void*, uint32_t*, const uint64_t*,
                    uint32_t, cudaStream_t);
}  // namespace pgs

using namespace pgs;

namespace {

bool overlap(const void* a, const void* b, uint64_t bytes) {
  auto x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
  return x < y + bytes && y < x + bytes;
}

}  // namespace

extern "C" {

uint64_t pgs_samples_per_run(uint32_t P, const pgs_config* cfg) {
  Options o;
  if (read_options(cfg, &o) != PGS_OK || P == 0) return 0;
  return P > 1 ? samples_per_run(P, key_bytes(o.dtype), o) : 0;
}

int pgs_rank_samples(const void* sorted, uint64_t n, uint32_t s, void* samples_out, void* stream,
                     const pgs_config* cfg) {
  Options o;
  int rc = read_options(cfg, &o);
  if (rc) return rc;
  if (s == 0) return PGS_ERR_INVALID;
  if (n == 0) return PGS_OK;
  if (!sorted || !samples_out) return PGS_ERR_INVALID;
  DeviceGuard dg;
  PGS_TRY(dg.use_device_of(sorted));
  const uint64_t sr = std::min<uint64_t>(s, n);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (o.dtype == PGS_U64)
    k_rank_samples<uint64_t><<<grid_for(sr, 256), 256, 0, st>>>(static_cast<const uint64_t*>(sorted), n, sr,
                                                                static_cast<uint64_t*>(samples_out));
  else
    k_rank_samples<uint32_t><<<grid_for(sr, 256), 256, 0, st>>>(static_cast<const uint32_t*>(sorted), n, sr,
                                                                static_cast<uint32_t*>(samples_out));
  PGS_CUDA(cudaGetLastError());
  return PGS_OK;
}

int pgs_rank_counts(const void* sorted, uint64_t n, const void* splitters, uint32_t G, uint64_t* counts_out,
                    void* stream, const pgs_config* cfg) {
  Options o;
  int rc = read_options(cfg, &o);
  if (rc) return rc;
  if (G == 0 || G > kMaxP) return G == 0 ? PGS_ERR_INVALID : PGS_ERR_UNSUPPORTED;
  if (G == 1) return PGS_OK;                            // no splitters
  if (!splitters || !counts_out || (n > 0 && !sorted)) return PGS_ERR_INVALID;
  DeviceGuard dg;
  PGS_TRY(dg.use_device_of(counts_out));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int f32 = o.dtype == PGS_F32;
  if (o.dtype == PGS_U64)
    k_rank_counts<uint64_t><<<grid_for(G - 1, 256), 256, 0, st>>>(static_cast<const uint64_t*>(sorted), n,
                                                                  static_cast<const uint64_t*>(splitters), G,
                                                                  counts_out, 0);
  else
    k_rank_counts<uint32_t><<<grid_for(G - 1, 256), 256, 0, st>>>(static_cast<const uint32_t*>(sorted), n,
                                                                  static_cast<const uint32_t*>(splitters), G,
                                                                  counts_out, f32);
  PGS_CUDA(cudaGetLastError());
  return PGS_OK;
}

size_t pgs_rank_cuts_workspace_bytes(uint32_t G, const pgs_config* cfg) {
  Options o;
  if (read_options(cfg, &o) != PGS_OK || G == 0 || G > kMaxP) return 0;
  return rank_cuts_layout(G, key_bytes(o.dtype)).total;
}

int pgs_rank_cuts(const uint64_t* counts_all, const uint64_t* shard_sizes, uint32_t G, const void* splitters,
                  uint64_t* cut_out, uint64_t* bounds_out, void* stream, const pgs_config* cfg) {
  Options o;
  int rc = read_options(cfg, &o);
  if (rc) return rc;
  if (G == 0) return PGS_ERR_INVALID;
  if (G > kMaxP) return PGS_ERR_UNSUPPORTED;
  if (!shard_sizes || !cut_out || !bounds_out || (G > 1 && (!counts_all || !splitters))) return PGS_ERR_INVALID;
  uint64_t N = 0;
  for (uint32_t r = 0; r < G; ++r) N += shard_sizes[r];
  if (N >= (1ull << 40)) return PGS_ERR_UNSUPPORTED;
  const size_t need = rank_cuts_layout(G, key_bytes(o.dtype)).total;
  if (!o.workspace || (reinterpret_cast<uintptr_t>(o.workspace) % kAlign) != 0 || o.workspace_bytes < need)
    return PGS_ERR_WORKSPACE;
  DeviceGuard dg;
  PGS_TRY(dg.use_device_of(cut_out));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (o.dtype == PGS_U64)
    return run_rank_cuts<uint64_t>(counts_all, shard_sizes, G, static_cast<const uint64_t*>(splitters), cut_out,
                                   bounds_out, o, st);
  return run_rank_cuts<uint32_t>(counts_all, shard_sizes, G, static_cast<const uint32_t*>(splitters), cut_out,
                                 bounds_out, o, st);
}

size_t pgs_merge_workspace_bytes(uint64_t n, uint32_t k, const pgs_config* cfg) {
  Options o;
  if (read_options(cfg, &o) != PGS_OK || k == 0 || k > kMaxP) return 0;
  Shape sh = merge_shape(n, k, true, o);
  Buffers b;
  return carve(sh, nullptr, &b);
}

int pgs_merge_lists(const void* keys_in, const uint32_t* vals_in, const uint64_t* offsets, uint32_t k, void* keys_out,
                    uint32_t* vals_out, void* stream, const pgs_config* cfg) {
  Options o;
  int rc = read_options(cfg, &o);
  if (rc) return rc;
  if (k == 0 || !offsets) return PGS_ERR_INVALID;
  if (k > kMaxP) return PGS_ERR_UNSUPPORTED;
  if ((vals_in == nullptr) != (vals_out == nullptr)) return PGS_ERR_INVALID;
  if (offsets[0] != 0) return PGS_ERR_INVALID;
  for (uint32_t j = 0; j < k; ++j)
    if (offsets[j + 1] < offsets[j]) return PGS_ERR_INVALID;
  const uint64_t n = offsets[k];
  if (n == 0) return PGS_OK;
  if (!keys_in || !keys_out) return PGS_ERR_INVALID;
  if (n >= (1ull << 40)) return PGS_ERR_UNSUPPORTED;
  const int w = key_bytes(o.dtype);
  if (overlap(keys_in, keys_out, n * (uint64_t)w)) return PGS_ERR_INVALID;
  if (vals_in && overlap(vals_in, vals_out, n * 4ull)) return PGS_ERR_INVALID;
  Shape sh = merge_shape(n, k, vals_in != nullptr, o);
  Buffers b;
  const size_t need = carve(sh, nullptr, &b);
  if (!o.workspace || (reinterpret_cast<uintptr_t>(o.workspace) % kAlign) != 0 || o.workspace_bytes < need)
    return PGS_ERR_WORKSPACE;
  DeviceGuard dg;
  PGS_TRY(dg.use_device_of(keys_out));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (o.dtype == PGS_U64) return merge_lists_u64(sh, o, keys_in, vals_in, keys_out, vals_out, offsets, k, st);
  return merge_lists_u32(sh, o, keys_in, vals_in, keys_out, vals_out, offsets, k, st);
}

}  // extern "C"
