// pgs_sort_static: the in-place sort for callers that cannot allocate device
// memory.  Some callers run where cudaMalloc is off limits: inside a custom
// allocator or memory-pool callback, in a plug-in whose host application owns
// every device allocation, or on a path that must never block on the driver's
// allocator.  For them the temporary storage lives in one file-scope device
// array, so the call allocates nothing.
//
// The array is PGS_STATIC_SCRATCH_BYTES (8 MiB) on every GPU that loads the
// library, held until the process exits; it bounds the request to
// n <= PGS_STATIC_MAX_KEYS keys on P <= PGS_STATIC_MAX_P partitions.  All calls
// share it and it keeps the last call's contents (the pipeline writes every
// byte it reads, so nothing has to start at zero); two calls whose work
// overlaps on the GPU (different streams, or different host threads) race on it.
#include <algorithm>
#include <mutex>

#include "pgs_host.cuh"

static __device__ __align__(256) unsigned char g_pgs_static_scratch[PGS_STATIC_SCRATCH_BYTES];

namespace pgs {
int sort_u32(const Shape&, const Options&, const void*, const uint32_t*, void*, uint32_t*, cudaStream_t);
int sort_u64(const Shape&, const Options&, const void*, const uint32_t*, void*, uint32_t*, cudaStream_t);

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device.  Host code only
// holds a host-side stand-in for the symbol, so the address is looked up once
// per device, with that device current, and cached.
int scratch_address(int device, void** out) {
  if (device < 0 || device >= kMaxDevices) return PGS_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_addr[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_pgs_static_scratch);
    if (e != cudaSuccess || !p) return record_cuda_error(e, "cudaGetSymbolAddress", __LINE__);
    g_scratch_addr[device] = p;
  }
  *out = g_scratch_addr[device];
  return PGS_OK;
}

}  // namespace
}  // namespace pgs

using namespace pgs;

extern "C" int pgs_sort_static(void* keys, uint32_t* vals, uint64_t n, uint32_t P, void* stream,
                               const pgs_config* cfg) {
  Options o;
  int rc = read_options(cfg, &o);
  if (rc) return rc;
  if (o.workspace) return PGS_ERR_INVALID;          // the scratch is the library's own
  if (P == 0) return PGS_ERR_INVALID;
  if (n == 0) return PGS_OK;
  if (!keys) return PGS_ERR_INVALID;
  const uint64_t P_eff = std::max<uint64_t>(1, std::min<uint64_t>(P, n));   // the clamp every sort applies
  if (n > PGS_STATIC_MAX_KEYS || P_eff > PGS_STATIC_MAX_P) return PGS_ERR_UNSUPPORTED;
  Shape p = single_shape(n, P, vals != nullptr, o);
  Buffers b;
  const size_t need = carve(p, nullptr, &b);
  if (need > PGS_STATIC_SCRATCH_BYTES) return PGS_ERR_UNSUPPORTED;   // never within the limits (tested)

  DeviceGuard dg;
  int device = -1;
  rc = DeviceGuard::device_of(keys, &device);
  if (rc) return rc;
  rc = dg.use(device);
  if (rc) return rc;
  void* scratch = nullptr;
  rc = scratch_address(device, &scratch);
  if (rc) return rc;
  o.workspace = scratch;
  o.workspace_bytes = PGS_STATIC_SCRATCH_BYTES;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (o.dtype == PGS_U64) return sort_u64(p, o, keys, vals, keys, vals, st);
  return sort_u32(p, o, keys, vals, keys, vals, st);
}
