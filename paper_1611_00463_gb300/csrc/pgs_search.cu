// Lookups on the sorted output (Section IV-C: the library lets its users
// binary-search the sorted data and find every entry's previous processor and
// index).  C ABI: pgs_search, pgs_provenance (declared in include/pgs.h).
#include "pgs_host.cuh"

namespace pgs {
namespace {

constexpr int kSearchNT = 256;

// Last b in [0, P) with e[b] <= pos, for pos < e[P] (the bucket holding pos).
__device__ __forceinline__ uint32_t bucket_holding(const uint64_t* __restrict__ e, uint32_t P, uint64_t pos) {
  if (pos >= e[P]) return P;
  uint32_t a = 0, z = P;                                // e[a] <= pos < e[z]
  while (z - a > 1) {
    const uint32_t mid = (a + z) >> 1;
    if (e[mid] <= pos) a = mid; else z = mid;
  }
  return a;
}

// One thread per query: lower (RIGHT = false) or upper bound of the query in
// the sorted keys, by key order (float32 by totalOrder of its bits).
template <typename K, bool RIGHT>
__global__ void __launch_bounds__(kSearchNT)
k_search(const K* __restrict__ keys, uint64_t n, const K* __restrict__ queries, uint64_t m, int f32,
         const uint64_t* __restrict__ e, uint32_t P, uint64_t* __restrict__ pos_out, uint32_t* __restrict__ bucket_out) {
  const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (i >= m) return;
  const K v = to_order<K>(queries[i], f32);
  uint64_t lo = 0, hi = n;
  while (lo < hi) {
    const uint64_t mid = lo + ((hi - lo) >> 1);
    const K k = to_order<K>(__ldg(keys + mid), f32);
    if (RIGHT ? !(v < k) : (k < v)) lo = mid + 1; else hi = mid;
  }
  pos_out[i] = lo;
  if (bucket_out) bucket_out[i] = bucket_holding(e, P, lo);
}

// Indexed search: a compact copy of every kStride-th key (1/64 of the array,
// small enough to stay in L2) is bisected first, then the query's block of
// kStride keys in the array itself.  A plain bisection of a large array misses
// in L2 on most of its lower levels (measured: about 16 DRAM sectors a query);
// this one touches one or two DRAM lines a query.
constexpr uint64_t kStride = 64;

template <typename K>
__global__ void __launch_bounds__(kSearchNT)
k_search_index(const K* __restrict__ keys, uint64_t n, int f32, K* __restrict__ index, uint64_t I) {
  const uint64_t j = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (j < I) index[j] = to_order<K>(keys[j * kStride], f32);
}

template <typename K, bool RIGHT>
__global__ void __launch_bounds__(kSearchNT)
k_search_indexed(const K* __restrict__ keys, uint64_t n, const K* __restrict__ index, uint64_t I,
                 const K* __restrict__ queries, uint64_t m, int f32, const uint64_t* __restrict__ e, uint32_t P,
                 uint64_t* __restrict__ pos_out, uint32_t* __restrict__ bucket_out) {
  const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (i >= m) return;
  const K v = to_order<K>(queries[i], f32);
  // j* = number of index entries 1..I-1 ordered before v (RIGHT: not after v);
  // every key up to position j* kStride is then before v and the key at
  // (j* + 1) kStride is not, so the answer lies in [j* kStride, (j* + 1) kStride].
  uint64_t a = 1, z = I;
  while (a < z) {
    const uint64_t mid = (a + z) >> 1;
    const K k = __ldg(index + mid);
    if (RIGHT ? !(v < k) : (k < v)) a = mid + 1; else z = mid;
  }
  uint64_t lo = (a - 1) * kStride, hi = umin(a * kStride, n);
  while (lo < hi) {
    const uint64_t mid = lo + ((hi - lo) >> 1);
    const K k = to_order<K>(__ldg(keys + mid), f32);
    if (RIGHT ? !(v < k) : (k < v)) lo = mid + 1; else hi = mid;
  }
  pos_out[i] = lo;
  if (bucket_out) bucket_out[i] = bucket_holding(e, P, lo);
}

// Run r of the floor split holds input positions [floor(r n / P), floor((r+1) n / P)).
__global__ void __launch_bounds__(kSearchNT)
k_provenance(const uint32_t* __restrict__ vals, uint64_t m, uint64_t n, uint64_t P, uint32_t* __restrict__ run_out,
             uint64_t* __restrict__ index_out) {
  const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (i >= m) return;
  const uint64_t v = vals[i];
  uint64_t r;
  if (v >= n) {
    r = P;                                              // not an input position
  } else {
    // Largest r with floor(r n / P) <= v is ceil((v + 1) P / n) - 1; then check.
    r = (uint64_t)(((unsigned __int128)(v + 1) * P + n - 1) / n) - 1;
    if (r >= P) r = P - 1;
    while (r > 0 && run_start(r, n, P) > v) --r;
    while (r + 1 < P && run_start(r + 1, n, P) <= v) ++r;
  }
  if (run_out) run_out[i] = (uint32_t)r;
  if (index_out) index_out[i] = v - (r < P ? run_start(r, n, P) : n);
}

bool on_device(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Bytes of workspace the indexed search uses for n keys of w bytes (0: none).
inline size_t search_index_bytes(uint64_t n, int w) {
  return n >= kStride * 1024 ? (size_t)ceil_div(n, kStride) * w : 0;
}

template <typename K>
int launch_search(const K* keys, uint64_t n, const K* q, uint64_t m, int side, int f32, const uint64_t* e,
                  uint32_t P, uint64_t* pos, uint32_t* bucket, void* ws, size_t ws_bytes, cudaStream_t st) {
  const size_t need = search_index_bytes(n, sizeof(K));
  if (need && ws && ws_bytes >= need) {
    K* index = static_cast<K*>(ws);
    const uint64_t I = ceil_div(n, kStride);
    k_search_index<K><<<(unsigned)ceil_div(I, kSearchNT), kSearchNT, 0, st>>>(keys, n, f32, index, I);
    const unsigned grid = (unsigned)ceil_div(m, kSearchNT);
    if (side)
      k_search_indexed<K, true><<<grid, kSearchNT, 0, st>>>(keys, n, index, I, q, m, f32, e, P, pos, bucket);
    else
      k_search_indexed<K, false><<<grid, kSearchNT, 0, st>>>(keys, n, index, I, q, m, f32, e, P, pos, bucket);
    PGS_CUDA(cudaGetLastError());
    return PGS_OK;
  }
  const unsigned grid = (unsigned)ceil_div(m, kSearchNT);
  if (side)
    k_search<K, true><<<grid, kSearchNT, 0, st>>>(keys, n, q, m, f32, e, P, pos, bucket);
  else
    k_search<K, false><<<grid, kSearchNT, 0, st>>>(keys, n, q, m, f32, e, P, pos, bucket);
  PGS_CUDA(cudaGetLastError());
  return PGS_OK;
}

}  // namespace
}  // namespace pgs

using namespace pgs;

extern "C" {

int pgs_search(const void* keys, uint64_t n, const void* queries, uint64_t m, int side,
               const uint64_t* bucket_bounds, uint32_t P, uint64_t* pos_out, uint32_t* bucket_out, void* stream,
               const pgs_config* cfg) {
  Options o;
  int rc = read_options(cfg, &o);
  if (rc) return rc;
  if (side != 0 && side != 1) return PGS_ERR_INVALID;
  if ((bucket_bounds == nullptr) != (bucket_out == nullptr)) return PGS_ERR_INVALID;
  if (bucket_bounds && P == 0) return PGS_ERR_INVALID;
  if (m == 0) return PGS_OK;
  if (!queries || !pos_out || (n > 0 && !keys)) return PGS_ERR_INVALID;
  if (n >= (1ull << 40) || m >= (1ull << 40)) return PGS_ERR_UNSUPPORTED;
  if (!on_device(queries) || !on_device(pos_out) || (n > 0 && !on_device(keys)) ||
      (bucket_bounds && (!on_device(bucket_bounds) || !on_device(bucket_out))))
    return PGS_ERR_INVALID;
  if (ceil_div(m, kSearchNT) > 0x7FFFFFFFull) return PGS_ERR_UNSUPPORTED;
  DeviceGuard dg;
  PGS_TRY(dg.use_device_of(pos_out));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int f32 = o.dtype == PGS_F32;
  if (o.workspace && (!on_device(o.workspace) || (reinterpret_cast<uintptr_t>(o.workspace) % kAlign) != 0))
    return PGS_ERR_WORKSPACE;
  if (o.dtype == PGS_U64)
    return launch_search<uint64_t>(static_cast<const uint64_t*>(keys), n, static_cast<const uint64_t*>(queries), m,
                                   side, 0, bucket_bounds, P, pos_out, bucket_out, o.workspace, o.workspace_bytes,
                                   st);
  return launch_search<uint32_t>(static_cast<const uint32_t*>(keys), n, static_cast<const uint32_t*>(queries), m,
                                 side, f32, bucket_bounds, P, pos_out, bucket_out, o.workspace, o.workspace_bytes,
                                 st);
}

size_t pgs_search_workspace_bytes(uint64_t n, const pgs_config* cfg) {
  Options o;
  if (read_options(cfg, &o) != PGS_OK) return 0;
  return search_index_bytes(n, key_bytes(o.dtype));
}

int pgs_provenance(const uint32_t* vals, uint64_t m, uint64_t n, uint32_t P, uint32_t* run_out,
                   uint64_t* index_out, void* stream) {
  if (P == 0) return PGS_ERR_INVALID;
  if (m == 0) return PGS_OK;
  if (!vals || (!run_out && !index_out)) return PGS_ERR_INVALID;
  if (n >= (1ull << 40) || m >= (1ull << 40)) return PGS_ERR_UNSUPPORTED;
  if (!on_device(vals) || (run_out && !on_device(run_out)) || (index_out && !on_device(index_out)))
    return PGS_ERR_INVALID;
  if (ceil_div(m, kSearchNT) > 0x7FFFFFFFull) return PGS_ERR_UNSUPPORTED;
  DeviceGuard dg;
  PGS_TRY(dg.use_device_of(vals));
  const uint64_t Peff = n == 0 ? 1 : std::max<uint64_t>(1, std::min<uint64_t>(P, n));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  k_provenance<<<(unsigned)ceil_div(m, kSearchNT), kSearchNT, 0, st>>>(vals, m, n, Peff, run_out, index_out);
  PGS_CUDA(cudaGetLastError());
  return PGS_OK;
}

}  // extern "C"
