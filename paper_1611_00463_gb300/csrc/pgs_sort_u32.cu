// 32-bit keys (uint32 and float32 in totalOrder form) of the sort pipeline.
#include "pgs_host.cuh"

namespace pgs {

int sort_u32(const Plan& p, const Options& o, const void* kin, const uint32_t* vin, void* kout,
             uint32_t* vout, cudaStream_t st) {
  auto ki = static_cast<const uint32_t*>(kin);
  auto ko = static_cast<uint32_t*>(kout);
  if (vin) return run_sort<uint32_t, true>(p, o, ki, vin, ko, vout, st);
  return run_sort<uint32_t, false>(p, o, ki, nullptr, ko, nullptr, st);
}

int fit_u32(const FitPlan& f, const Options& o, const void* samples, void* out, cudaStream_t st) {
  return run_fit<uint32_t>(f, o, static_cast<const uint32_t*>(samples), static_cast<uint32_t*>(out), st);
}

}  // namespace pgs
