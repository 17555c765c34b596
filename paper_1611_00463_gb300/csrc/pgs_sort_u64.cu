// 64-bit keys of the sort pipeline.
#include "pgs_rank.cuh"

namespace pgs {

int sort_u64(const Shape& p, const Options& o, const void* kin, const uint32_t* vin, void* kout,
             uint32_t* vout, cudaStream_t st) {
  auto ki = static_cast<const uint64_t*>(kin);
  auto ko = static_cast<uint64_t*>(kout);
  if (vin) return run_sort<uint64_t, true>(p, o, ki, vin, ko, vout, st);
  return run_sort<uint64_t, false>(p, o, ki, nullptr, ko, nullptr, st);
}

int sort_host_u64(const Shape& p, const Options& o, const void* kin, const uint32_t* vin, void* kout,
                  uint32_t* vout, cudaStream_t st) {
  auto ki = static_cast<const uint64_t*>(kin);
  auto ko = static_cast<uint64_t*>(kout);
  if (vin) return run_sort_host<uint64_t, true>(p, o, ki, vin, ko, vout, st);
  return run_sort_host<uint64_t, false>(p, o, ki, nullptr, ko, nullptr, st);
}

int fit_u64(uint64_t m, uint32_t P, const Options& o, const void* samples, void* out, float* model_out,
            cudaStream_t st) {
  return run_fit<uint64_t>(m, P, o, static_cast<const uint64_t*>(samples), static_cast<uint64_t*>(out), model_out, st);
}

int batch_attrs_u64(bool vals) {
  return vals ? set_all_smem_attrs<uint64_t, true>() : set_all_smem_attrs<uint64_t, false>();
}

int batch_u64(const Shape& sh, const Options& o, const void* kin, const uint32_t* vin, void* kout,
             uint32_t* vout, cudaStream_t st) {
  Ctx c;
  c.st = st;
  c.timer = o.timer;
  Buffers b;
  carve(sh, o.workspace, &b);
  auto ki = static_cast<const uint64_t*>(kin);
  auto ko = static_cast<uint64_t*>(kout);
  if (vin) return run_pipeline<uint64_t, true>(sh, o, ki, vin, ko, vout, c, b);
  return run_pipeline<uint64_t, false>(sh, o, ki, nullptr, ko, nullptr, c, b);
}

int fill_random_u64(void* keys, uint32_t* vals, uint64_t n, uint64_t seed, cudaStream_t st) {
  k_fill_random<uint64_t><<<grid_for(n, 256), 256, 0, st>>>(static_cast<uint64_t*>(keys), vals, n, seed);
  PGS_CUDA(cudaGetLastError());
  return PGS_OK;
}

int merge_lists_u64(const Shape& sh, const Options& o, const void* kin, const uint32_t* vin, void* kout,
                    uint32_t* vout, const uint64_t* off, uint32_t k, cudaStream_t st) {
  auto ki = static_cast<const uint64_t*>(kin);
  auto ko = static_cast<uint64_t*>(kout);
  if (vin) return run_merge_lists<uint64_t, true>(sh, o, ki, vin, ko, vout, off, k, st);
  return run_merge_lists<uint64_t, false>(sh, o, ki, nullptr, ko, nullptr, off, k, st);
}

}  // namespace pgs
