// 64-bit keys of the sort pipeline.
#include "pgs_host.cuh"

namespace pgs {

int sort_u64(const Plan& p, const Options& o, const void* kin, const uint32_t* vin, void* kout,
             uint32_t* vout, cudaStream_t st) {
  auto ki = static_cast<const uint64_t*>(kin);
  auto ko = static_cast<uint64_t*>(kout);
  if (vin) return run_sort<uint64_t, true>(p, o, ki, vin, ko, vout, st);
  return run_sort<uint64_t, false>(p, o, ki, nullptr, ko, nullptr, st);
}

int fit_u64(const FitPlan& f, const Options& o, const void* samples, void* out, cudaStream_t st) {
  return run_fit<uint64_t>(f, o, static_cast<const uint64_t*>(samples), static_cast<uint64_t*>(out), st);
}

}  // namespace pgs
