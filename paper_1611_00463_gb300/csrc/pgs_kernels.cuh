// Device code of the GB300 load-balanced sample sort (arXiv 1611.00463, Section IV).
//
// Keys travel through the pipeline as unsigned integers in "order form": integer
// keys as they are, float32 keys as their IEEE 754 totalOrder image (the first
// kernel converts, the last one converts back).  Payloads are uint32.  Arrays
// are structure-of-arrays in HBM: keys[n] and vals[n].
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "pgs_ptx.cuh"

namespace pgs {

constexpr int kNT = 256;             // threads per CTA of the sort and merge kernels
constexpr int kVT = 17;              // items per thread; odd, so blocked smem access is conflict free
constexpr int kTile = kNT * kVT;     // 4352 keys per block-sort tile and per merge tile
constexpr int kMergeMinTile = 64 * 17;            // smallest merge tile of the tunable shapes
constexpr int kMerge4NT = 256;                    // four-way rounds: threads per CTA
constexpr int kMerge4VT = 9;                      // outputs per thread at most; a chunk holds <= 2304
constexpr int kMerge4Cut = kMerge4NT * kMerge4VT / 2;   // X and Y are cut every 1152 elements
constexpr int kScanNT = 1024;
constexpr int kScanVT = 8;
constexpr int kScanChunk = kScanNT * kScanVT;
constexpr int kScatterNT = 256;
constexpr int kScatterVT = 16;
constexpr int kScatterTile = kScatterNT * kScatterVT;
constexpr int kScatterWindow = 1024;  // bucket segments staged per scatter CTA

struct Pair {                         // one pairwise merge: A = [a, a+na), B = [b, b+nb) -> [out, out+na+nb)
  uint64_t a, na, b, nb, out;
};

// Batch geometry: device tables describing I sort instances laid end to end.
// Instance i owns keys [koff[i], koff[i+1]) split into P[i] runs (the paper's
// processors); its runs, and its buckets, are the global indices
// [R0[i], R0[i] + P[i]).  Its P x (P+1) matrices (lb, cnt, cut) start at
// mat[i]; its P x P bucket segments (bucket-major) start at seg[i]; its
// bucket vector e (P+1 entries) starts at R0[i] + i.  A single sort is a
// batch of one.
struct Geo {
  const uint64_t* koff;      // I+1
  const uint32_t* P;         // I
  const uint32_t* R0;        // I+1
  const uint64_t* mat;       // I+1
  const uint64_t* seg;       // I+1
  const uint64_t* s;         // I: samples per run (0 for an instance with one run)
  const uint64_t* run_off;   // R+1: first key of every run
  const uint32_t* run_inst;  // R: instance of every run
  uint32_t I, R;
};

// Index of the last entry of a sorted table t[0..n] with t[k] <= x.
template <typename T>
__device__ __forceinline__ uint32_t last_le(const T* t, uint32_t n, T x) {
  uint32_t lo = 0, hi = n;                  // invariant t[lo] <= x < t[hi] (t[n] > x assumed)
  while (hi - lo > 1) {
    uint32_t mid = (lo + hi) >> 1;
    if (t[mid] <= x) lo = mid; else hi = mid;
  }
  return lo;
}

// ---------------------------------------------------------------------------
// Key order
// ---------------------------------------------------------------------------

template <typename K> __device__ __forceinline__ K key_max();
template <> __device__ __forceinline__ uint32_t key_max<uint32_t>() { return 0xFFFFFFFFu; }
template <> __device__ __forceinline__ uint64_t key_max<uint64_t>() { return 0xFFFFFFFFFFFFFFFFull; }

// IEEE 754 totalOrder: negative patterns flip every bit, non-negative ones set the sign.
__device__ __forceinline__ uint32_t f32_to_order(uint32_t b) {
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ uint32_t order_to_f32(uint32_t o) {
  return (o & 0x80000000u) ? (o & 0x7FFFFFFFu) : ~o;
}
template <typename K> __device__ __forceinline__ K to_order(K k, int f32) { return k; }
template <> __device__ __forceinline__ uint32_t to_order<uint32_t>(uint32_t k, int f32) {
  return f32 ? f32_to_order(k) : k;
}
template <typename K> __device__ __forceinline__ K from_order(K k, int f32) { return k; }
template <> __device__ __forceinline__ uint32_t from_order<uint32_t>(uint32_t k, int f32) {
  return f32 ? order_to_f32(k) : k;
}

__device__ __forceinline__ uint64_t umin(uint64_t a, uint64_t b) { return a < b ? a : b; }
__device__ __forceinline__ uint64_t umax(uint64_t a, uint64_t b) { return a > b ? a : b; }

// Run r of the logical partition owns [floor(r n / P), floor((r+1) n / P)).
__device__ __forceinline__ uint64_t run_start(uint64_t r, uint64_t n, uint64_t P) {
  return (r * n) / P;
}

// ---------------------------------------------------------------------------
// Merge path (stable: on equal keys list A comes first)
// ---------------------------------------------------------------------------

// Number of A items among the first `diag` outputs of merge(A, B).
template <typename K, typename I>
__device__ __forceinline__ I merge_path(const K* a, I na, const K* b, I nb, I diag) {
  I lo = diag > nb ? diag - nb : 0;
  I hi = diag < na ? diag : na;
  while (lo < hi) {
    I mid = (lo + hi) >> 1;
    if (a[mid] <= b[diag - 1 - mid]) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// Merge VT items of two sorted ranges of one smem array, A = [ai, a_end) and
// B = [bi, b_end), into registers (ties take A, so the merge is stable);
// pos[] receives the smem index of each item.  One shared-memory read per
// item: the next key of whichever list advanced.  That read may land one slot
// past a range's end; the caller keeps that slot inside the array, and the
// index tests, not the key read there, decide.
template <typename K, int VT>
__device__ __forceinline__ void serial_merge(const K* s, int ai, int a_end, int bi, int b_end,
                                             K (&key)[VT], int (&pos)[VT]) {
  K ak = s[ai];
  K bk = s[bi];
#pragma unroll
  for (int j = 0; j < VT; ++j) {
    const bool take_b = (bi < b_end) && ((ai >= a_end) || (bk < ak));
    key[j] = take_b ? bk : ak;
    pos[j] = take_b ? bi : ai;
    if (take_b) ++bi; else ++ai;
    const K nx = s[take_b ? bi : ai];
    if (take_b) bk = nx; else ak = nx;
  }
}

// ---------------------------------------------------------------------------
// K1: block sort.  One CTA sorts one tile of one run, stably.
// Step 1 of Section IV / Section IV-A: every thread sorts its own VT keys
// (odd-even transposition: only strictly smaller keys move left, so it is
// stable), then the sorted thread lists are merged pairwise in rounds, list
// 2i+1 into list 2i, exactly the balanced schedule of Fig. 2, in shared memory.
// ---------------------------------------------------------------------------

// Key index of a merge pass's output: entry e holds the (order-mapped) key at
// global position 64 e.  Every merge kernel that writes a tile of sorted
// output [g0, g0 + cnt) also writes the entries whose positions fall inside
// it, so after the pass the index covers all of the output; the next round's
// partition bisects it before touching the keys themselves.  (The block sort
// writes none: its lists, one tile each, are short enough to bisect directly.)
constexpr uint64_t kIdxStride = 64;

template <typename K>
__device__ __forceinline__ void write_key_index(K* kidx, const K* tile, uint64_t g0, int cnt) {
  const uint64_t first = (g0 + kIdxStride - 1) / kIdxStride;
  const uint64_t last = (g0 + (uint64_t)cnt + kIdxStride - 1) / kIdxStride;
  for (uint64_t e = first + threadIdx.x; e < last; e += blockDim.x) kidx[e] = tile[e * kIdxStride - g0];
}

template <typename K>
struct BlockSortSmem {
  K keys[kTile + 1];      // + one slot the serial merge may read past the last list
  uint16_t ids[kTile + 8];
  uint32_t vals[kTile];
};

template <typename K, bool VALS>
__global__ void __launch_bounds__(kNT)
k_block_sort(const K* __restrict__ kin, const uint32_t* __restrict__ vin, K* kout, uint32_t* vout,
             const uint64_t* __restrict__ run_off, uint32_t tiles_per_run, int f32_in, int f32_out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  BlockSortSmem<K>& sm = *reinterpret_cast<BlockSortSmem<K>*>(smem_raw);
  const int tid = threadIdx.x;
  const uint64_t r = blockIdx.x / tiles_per_run;
  const uint64_t t = blockIdx.x % tiles_per_run;
  const uint64_t rs = run_off[r], re = run_off[r + 1];
  const uint64_t g0 = rs + t * kTile;
  if (g0 >= re) return;
  const int cnt = (int)umin(kTile, re - g0);

#pragma unroll
  for (int i = 0; i < kVT; ++i) {
    int idx = i * kNT + tid;
    sm.keys[idx] = idx < cnt ? to_order<K>(kin[g0 + idx], f32_in) : key_max<K>();
    if (VALS) sm.vals[idx] = idx < cnt ? vin[g0 + idx] : 0u;
  }
  if (tid == 0) sm.keys[kTile] = key_max<K>();
  __syncthreads();

  K key[kVT];
  int pos[kVT];
#pragma unroll
  for (int j = 0; j < kVT; ++j) {
    key[j] = sm.keys[tid * kVT + j];
    pos[j] = tid * kVT + j;
  }
  // Thread-level stable sort.
#pragma unroll
  for (int i = 0; i < kVT; ++i) {
#pragma unroll
    for (int j = i & 1; j < kVT - 1; j += 2) {
      if (key[j + 1] < key[j]) {
        K tk = key[j]; key[j] = key[j + 1]; key[j + 1] = tk;
        int tp = pos[j]; pos[j] = pos[j + 1]; pos[j + 1] = tp;
      }
    }
  }
  // Pairwise merge rounds (Fig. 2): coop threads share one merged list.  While
  // a list pair lies inside one warp (coop <= 32) a warp barrier is enough: a
  // thread only reads slots of its own group, besides the one slot past its
  // B list, whose key is never used.
#pragma unroll 1
  for (int coop = 2; coop <= kNT; coop *= 2) {
    if (coop <= 64) __syncwarp(); else __syncthreads();    // last round's reads stayed in coop/2 threads
#pragma unroll
    for (int j = 0; j < kVT; ++j) {
      sm.keys[tid * kVT + j] = key[j];
      sm.ids[tid * kVT + j] = (uint16_t)pos[j];
    }
    if (coop <= 32) __syncwarp(); else __syncthreads();
    const int half = (coop / 2) * kVT;
    const int start = (tid & ~(coop - 1)) * kVT;
    const int diag = (tid & (coop - 1)) * kVT;
    const int a = merge_path<K, int>(sm.keys + start, half, sm.keys + start + half, half, diag);
    int spos[kVT];
    serial_merge<K, kVT>(sm.keys, start + a, start + half, start + half + (diag - a), start + 2 * half,
                         key, spos);
#pragma unroll
    for (int j = 0; j < kVT; ++j) pos[j] = sm.ids[spos[j]];
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < kVT; ++j) {
    sm.keys[tid * kVT + j] = key[j];
    sm.ids[tid * kVT + j] = (uint16_t)pos[j];
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < kVT; ++i) {
    int idx = i * kNT + tid;
    if (idx < cnt) {
      kout[g0 + idx] = from_order<K>(sm.keys[idx], f32_out);
      if (VALS) vout[g0 + idx] = sm.vals[sm.ids[idx]];
    }
  }
}

// ---------------------------------------------------------------------------
// Pair descriptors for one merge round, and the tile bookkeeping.
// ---------------------------------------------------------------------------

// Contiguous pair [lo, mid) + [mid, hi) -> [lo, hi).
__device__ __forceinline__ void put_pair(Pair* pairs, uint64_t* tcount, uint64_t p, uint64_t lo, uint64_t mid,
                                         uint64_t hi, uint32_t tile) {
  pairs[p] = Pair{lo, mid - lo, mid, hi - mid, lo};
  tcount[p] = (hi - lo + tile - 1) / tile;
}

// Run formation (step 1): inside every run, blocks [j 2w, j 2w + w) and
// [j 2w + w, (j+1) 2w) merge; a run that is already one list is copied.
// Index space: run x pair slot (cmax slots per run, unused slots are empty).
static __global__ void k_pairs_runs(Pair* pairs, uint64_t* tcount, const uint64_t* __restrict__ run_off,
                                    uint32_t R, uint64_t w, uint64_t cmax, uint32_t tile) {
  uint64_t p = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (p >= (uint64_t)R * cmax) return;
  uint64_t r = p / cmax, j = p % cmax;
  uint64_t rs = run_off[r], re = run_off[r + 1];
  uint64_t lo = umin(rs + j * 2 * w, re);
  if (j > 0 && lo >= re) lo = re;                     // empty slot
  uint64_t mid = umin(lo + w, re);
  uint64_t hi = umin(lo + 2 * w, re);
  put_pair(pairs, tcount, p, lo, mid, hi, tile);
}

// The Fig. 2 schedule over the P lists of one group: round `step` merges list
// group [j, j+step) with [j+step, j+2 step) for j a multiple of 2 step.  Lists
// of group g are [tbl[g0 + j], tbl[g0 + j + 1]); the index space is one slot
// per list (slots that do not start a pair are empty).
//  - samples (step 3): one group per instance, lists = its runs' samples,
//    tbl = sample offsets indexed by global run, slot = global run;
//  - buckets (step 6): one group per bucket, lists = its P segments,
//    tbl = segment offsets (bucket-major), slot = global segment.
static __global__ void k_pairs_sample_lists(Pair* pairs, uint64_t* tcount, Geo g,
                                            const uint64_t* __restrict__ samp_off, uint32_t step, uint32_t tile) {
  uint64_t p = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (p >= g.R) return;
  const uint32_t i = g.run_inst[p];
  const uint32_t r0 = g.R0[i], P = g.P[i];
  const uint32_t j = (uint32_t)p - r0;
  const uint64_t end = samp_off[r0 + P];
  if (j % (2 * step) != 0) {
    put_pair(pairs, tcount, p, end, end, end, tile);
    return;
  }
  put_pair(pairs, tcount, p, samp_off[r0 + j], samp_off[r0 + min(j + step, P)],
           samp_off[r0 + min(j + 2 * step, P)], tile);
}

// Slots [q0, q0 + Q) take part (whole buckets); slot q0 + t writes pair t.
static __global__ void k_pairs_bucket_lists(Pair* pairs, uint64_t* tcount, Geo g, const uint64_t* __restrict__ off,
                                            uint64_t q0, uint64_t Q, uint32_t step, uint32_t tile) {
  const uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (t >= Q) return;
  const uint64_t q = q0 + t;
  const uint32_t i = last_le<uint64_t>(g.seg, g.I, q);
  const uint64_t P = g.P[i];
  const uint64_t local = q - g.seg[i];
  const uint64_t b = local / P, j = local % P;
  const uint64_t base = g.seg[i] + b * P;           // first segment of bucket b
  if (j % (2 * step) != 0) {
    const uint64_t end = off[base + P];
    put_pair(pairs, tcount, t, end, end, end, tile);
    return;
  }
  put_pair(pairs, tcount, t, off[base + j], off[base + umin(j + step, P)], off[base + umin(j + 2 * step, P)],
           tile);
}

// Step 5 fused into the first round of step 6: segment j of bucket b (j even)
// merges with segment j+1 straight from the sorted runs, where the exchange
// would have copied them from, into the pair's place in bucket-major order.
// Slots [q0, q0 + Q) take part (whole buckets); slot q0 + t writes pair t.
static __global__ void k_pairs_fused(Pair* pairs, uint64_t* tcount, Geo g, const uint64_t* __restrict__ off,
                                     const uint64_t* __restrict__ seg_src, uint64_t q0, uint64_t Q, uint32_t tile) {
  const uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (t >= Q) return;
  const uint64_t q = q0 + t;
  const uint32_t i = last_le<uint64_t>(g.seg, g.I, q);
  const uint64_t P = g.P[i];
  const uint64_t j = (q - g.seg[i]) % P;
  if (j % 2 != 0) {
    pairs[t] = Pair{0, 0, 0, 0, 0};
    tcount[t] = 0;
    return;
  }
  const uint64_t na = off[q + 1] - off[q];
  const uint64_t nb = j + 1 < P ? off[q + 2] - off[q + 1] : 0;
  pairs[t] = Pair{seg_src[q], na, j + 1 < P ? seg_src[q + 1] : 0, nb, off[q]};
  tcount[t] = (na + nb + tile - 1) / tile;
}

// ---------------------------------------------------------------------------
// K2/K8: merge-path merge of one round (Section IV-A's pairwise merge; used for
// step 1's run formation, step 3's sample sort and step 6's bucket merge).
// Every CTA produces one tile of MT = NT x VT outputs of one pair: its two
// input ranges arrive in shared memory by bulk asynchronous copy (one thread
// issues them, an mbarrier counts the bytes), every thread merges VT outputs
// into registers, and once all threads are done the tile is staged in the
// input buffer it came from and leaves with 16-byte vector stores.  Reusing
// the input buffer halves the shared memory a CTA holds, so more CTAs share an
// SM and more copies are in flight (about 10 % faster than a separate output
// staging area at every tile shape).  With kidx set, the thread whose outputs
// cover a global position 64 e also writes key index entry e for the next
// round's partition.
// ---------------------------------------------------------------------------

template <typename K, bool VALS, int NT, int VT>
struct Merge2Layout {
  static constexpr int T = NT * VT;
  static constexpr size_t kin = 16;                                   // after the mbarrier
  static constexpr size_t vin = kin + (size_t)T * sizeof(K) + 64;     // 64: two 16-byte widenings
  static constexpr size_t bytes = vin + (VALS ? (size_t)T * 4 + 64 : 0);
  static_assert(T % 4 == 0, "staging offsets stay 16-byte aligned");
};

// A global range widened to 16-byte boundaries for a bulk copy.
struct Span16 {
  const char* base;
  uint32_t bytes;   // multiple of 16 (0 for an empty range)
  uint32_t skip;    // elements between base and the range's first element
};

template <typename T>
__device__ __forceinline__ Span16 widen16(const T* p, uint32_t count) {
  if (count == 0) return Span16{reinterpret_cast<const char*>(p), 0u, 0u};
  const uintptr_t a = reinterpret_cast<uintptr_t>(p);
  const uintptr_t lo = a & ~uintptr_t(15);
  const uintptr_t hi = (a + (uintptr_t)count * sizeof(T) + 15) & ~uintptr_t(15);
  return Span16{reinterpret_cast<const char*>(lo), (uint32_t)(hi - lo), (uint32_t)((a - lo) / sizeof(T))};
}

// Store cnt elements from shared memory to global memory with 16-byte vector
// stores where the destination allows it (unaligned head and tail element-wise).
template <typename T, int NT>
__device__ __forceinline__ void store_tile_vec(T* g, const T* s, int cnt) {
  constexpr int E = 16 / sizeof(T);
  const int tid = threadIdx.x;
  const uintptr_t addr = reinterpret_cast<uintptr_t>(g);
  int head = (int)(((16 - (addr & 15)) & 15) / sizeof(T));
  if (head > cnt) head = cnt;
  if (tid < head) g[tid] = s[tid];
  const int body = (cnt - head) / E;
  uint4* gb = reinterpret_cast<uint4*>(g + head);
  const T* sb = s + head;
  for (int c = tid; c < body; c += NT) {
    union { T e[E]; uint4 v; } u;
#pragma unroll
    for (int k = 0; k < E; ++k) u.e[k] = sb[c * E + k];
    gb[c] = u.v;
  }
  for (int i = head + body * E + tid; i < cnt; i += NT) g[i] = s[i];
}

// The partition kernel writes, per merge tile, where the tile's A and B ranges
// start and where its output goes, plus the ends of its pair (one merge-path
// search per tile, all tiles in parallel); a merge CTA reads its split and the
// next one together and knows both of its ranges after one dependent load.

struct TileSplit {
  uint64_t a, b, out;     // first A element, first B element, first output element
  uint64_t a_end, b_end;  // end of the pair's A list and of its B list
  uint64_t pair;          // index of the pair the tile belongs to
};

// Merge path of a and b at diagonal d, searched only inside [lo, hi], which
// must hold the answer.
template <typename K>
__device__ __forceinline__ uint64_t merge_path_in(const K* a, const K* b, uint64_t d, uint64_t lo, uint64_t hi) {
  while (lo < hi) {
    const uint64_t mid = (lo + hi) >> 1;
    if (a[mid] <= b[d - 1 - mid]) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ int64_t ceil_div64(int64_t t) {            // ceil(t / 64) for any sign
  return t >= 0 ? (t + (int64_t)kIdxStride - 1) / (int64_t)kIdxStride : -((-t) / (int64_t)kIdxStride);
}

// Merge path through the key index.  A' = A[oa + 64 i] and B' = B[ob + 64 j]
// are the keys of A and B at global multiples of 64 (contiguous index
// entries).  If c keys of B' are below A'[i], the keys of B below it number
// between ob + 64 (c - 1) + 1 and ob + 64 c (none past B[ob + 64 c], all up to
// B[ob + 64 (c - 1)]; for c = 0 at most ob), so the output position of A'[i]
// in merge(A, B) lies in [o + 64 p - 63, o + 64 p], where p = i + c is its
// position in merge(A', B') and o = oa + ob.  With t = d - o: every A' item
// among the first ceil(t / 64) outputs of the sample merge comes before
// output d, and the first A' item not among the first ceil((t + 63) / 64)
// comes at or after it.  So the split lies in a window of at most 127
// positions between the two, where the plain bisection finishes.  The two
// sample diagonals differ by at most one: one sample merge path and one
// comparison give both.
template <typename K>
__device__ __forceinline__ uint64_t merge_path_indexed(const K* src, const K* __restrict__ kidx, const Pair& pr,
                                                       uint64_t d) {
  const uint64_t na = pr.na, nb = pr.nb;
  uint64_t lo = d > nb ? d - nb : 0, hi = d < na ? d : na;
  const uint64_t ea = (pr.a + kIdxStride - 1) / kIdxStride, eb = (pr.b + kIdxStride - 1) / kIdxStride;
  const uint64_t ca = (pr.a + na + kIdxStride - 1) / kIdxStride - ea;
  const uint64_t cb = (pr.b + nb + kIdxStride - 1) / kIdxStride - eb;
  const uint64_t oa = ea * kIdxStride - pr.a, ob = eb * kIdxStride - pr.b;
  const int64_t t = (int64_t)d - (int64_t)(oa + ob);
  const int64_t cmax = (int64_t)(ca + cb);
  const int64_t dl = min(max(ceil_div64(t), (int64_t)0), cmax);
  const int64_t dh = min(max(ceil_div64(t + (int64_t)kIdxStride - 1), (int64_t)0), cmax);
  const K* ia = kidx + ea;
  const K* ib = kidx + eb;
  const uint64_t D = (uint64_t)dl;
  const uint64_t alo = merge_path<K, uint64_t>(ia, ca, ib, cb, D);
  uint64_t ahi = alo;
  if (dh > dl && alo < ca && (D - alo >= cb || ia[alo] <= ib[D - alo])) ahi = alo + 1;
  if (alo >= 1) lo = max(lo, oa + kIdxStride * (alo - 1) + 1);
  if (ahi < ca) hi = min(hi, oa + kIdxStride * ahi);
  return merge_path_in<K>(src + pr.a, src + pr.b, d, lo, hi);
}

// Lists shorter than this bisect the keys directly.
constexpr uint64_t kIdxMinList = 1024;

// The last p in [0, n) with t[p] <= i, for t non-decreasing with t[0] = 0 <= i:
// gallop from the guess g to a bracket, then bisect it.  Tiles spread nearly
// evenly over the pairs, so the guess i n / t[n] is usually a few pairs off
// and the search takes a few loads instead of log2(n).
__device__ __forceinline__ uint64_t last_le_from(const uint64_t* __restrict__ t, uint64_t n, uint64_t i,
                                                 uint64_t g) {
  uint64_t lo, hi;                                  // t[lo] <= i, and hi == n or t[hi] > i
  if (t[g] <= i) {
    lo = g;
    for (uint64_t step = 1;; step <<= 1) {
      const uint64_t nx = lo + step;
      if (nx >= n) { hi = n; break; }
      if (t[nx] > i) { hi = nx; break; }
      lo = nx;
    }
  } else {
    hi = g;
    for (uint64_t step = 1;; step <<= 1) {
      if (hi <= step) { lo = 0; break; }
      const uint64_t nx = hi - step;
      if (t[nx] <= i) { lo = nx; break; }
      hi = nx;
    }
  }
  while (hi - lo > 1) {
    const uint64_t mid = (lo + hi) >> 1;
    if (t[mid] <= i) lo = mid; else hi = mid;
  }
  return lo;
}

template <typename K>
__global__ void k_partition_split(const K* __restrict__ src, const Pair* __restrict__ pairs,
                                  const uint64_t* __restrict__ tbegin, uint64_t npairs, TileSplit* split,
                                  uint32_t tile, const K* __restrict__ kidx, const uint32_t* err) {
  if (poisoned(err)) return;
  uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  uint64_t total = tbegin[npairs];
  if (i >= total) return;
  const uint64_t guess = (uint64_t)(((unsigned __int128)i * npairs) / total);   // < npairs as i < total
  const uint64_t lo = last_le_from(tbegin, npairs, i, guess);                 // the tile's pair
  const Pair pr = pairs[lo];
  const uint64_t d0 = (i - tbegin[lo]) * tile;
  const uint64_t a0 = (kidx && pr.na >= kIdxMinList && pr.nb >= kIdxMinList)
                          ? merge_path_indexed<K>(src, kidx, pr, d0)
                          : merge_path<K, uint64_t>(src + pr.a, pr.na, src + pr.b, pr.nb, d0);
  split[i] = TileSplit{pr.a + a0, pr.b + (d0 - a0), pr.out + d0, pr.a + pr.na, pr.b + pr.nb, lo};
}

// CTAs per SM the merge tile is compiled for (0: the compiler's choice).
// With 4-byte keys a tile holds half the bytes, so more tiles must be in
// flight per SM to cover HBM latency: for the default 128 x 17 tile the
// register cap for 10 CTAs (48 registers, a few bytes of spill in the set-up
// thread) is measured 2 % faster on f32 keys and 1 % on u32 keys than the 9
// CTAs that the compiler's 55 registers allow.
template <typename K, int NT, int VT>
constexpr int merge_min_blocks() { return (sizeof(K) == 4 && NT == 128 && VT == 17) ? 10 : 0; }

template <typename K, bool VALS, int NT, int VT>
__global__ void __launch_bounds__(NT, (merge_min_blocks<K, NT, VT>()))
k_merge_tile(const K* __restrict__ ksrc, const uint32_t* __restrict__ vsrc, K* __restrict__ kdst,
             uint32_t* __restrict__ vdst, const TileSplit* __restrict__ split, const uint64_t* __restrict__ total_ptr,
             int f32_out, uint32_t* err, K* __restrict__ kidx, uint64_t wait_ns, int inject_timeout) {
  using L = Merge2Layout<K, VALS, NT, VT>;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);
  K* s_kin = reinterpret_cast<K*>(smem_raw + L::kin);
  uint32_t* s_vin = reinterpret_cast<uint32_t*>(smem_raw + L::vin);
  __shared__ uint32_t s_na, s_nb;
  __shared__ uint64_t s_a, s_b, s_out;

  const uint64_t tile = blockIdx.x;
  const int tid = threadIdx.x;
  if (tid == 0) {
    const uint64_t total = *total_ptr;
    uint32_t na = 0, nb = 0;
    TileSplit t{};
    if (tile < total && !poisoned(err)) {
      t = split[tile];
      bool same = false;
      TileSplit nx{};
      if (tile + 1 < total) {
        nx = split[tile + 1];
        same = nx.pair == t.pair;
      }
      const uint64_t a_hi = same ? nx.a : t.a_end, b_hi = same ? nx.b : t.b_end;
      if (a_hi < t.a || b_hi < t.b || (a_hi - t.a) + (b_hi - t.b) > (uint64_t)L::T) {
        atomicOr(err, kErrBadTile);                     // inconsistent split: skip the tile, never copy
        t = TileSplit{};
      } else {
        na = (uint32_t)(a_hi - t.a);
        nb = (uint32_t)(b_hi - t.b);
      }
      const Span16 ka = widen16(ksrc + t.a, na), kb = widen16(ksrc + t.b, nb);
      Span16 va{nullptr, 0, 0}, vb{nullptr, 0, 0};
      if (VALS) {
        va = widen16(vsrc + t.a, na);
        vb = widen16(vsrc + t.b, nb);
      }
      mbar_init(bar, 1);
      fence_barrier_init();
      mbar_arrive_expect_tx(bar, ka.bytes + kb.bytes + va.bytes + vb.bytes);
      // Fault injection (testing only): tile 0 announces its bytes but issues
      // no copy, so nothing is in flight and its wait runs out.
      if (!(inject_timeout && tile == 0)) {
        if (ka.bytes) bulk_load(s_kin, ka.base, ka.bytes, bar);
        if (kb.bytes) bulk_load(reinterpret_cast<char*>(s_kin) + ka.bytes, kb.base, kb.bytes, bar);
        if (VALS) {
          if (va.bytes) bulk_load(s_vin, va.base, va.bytes, bar);
          if (vb.bytes) bulk_load(reinterpret_cast<char*>(s_vin) + va.bytes, vb.base, vb.bytes, bar);
        }
      }
    }
    s_na = na;
    s_nb = nb;
    s_a = t.a;
    s_b = t.b;
    s_out = t.out;
  }
  __syncthreads();
  const int na = (int)s_na, nb = (int)s_nb, cnt = na + nb;
  if (cnt == 0) return;                                 // tile beyond the round's total
  const uint64_t ga = s_a, gb = s_b;
  const Span16 ka = widen16(ksrc + ga, na), kb = widen16(ksrc + gb, nb);
  const K* sa = s_kin + ka.skip;
  const K* sb = reinterpret_cast<const K*>(reinterpret_cast<const char*>(s_kin) + ka.bytes) + kb.skip;
  const uint32_t* sva = nullptr;
  const uint32_t* svb = nullptr;
  if (VALS) {
    const Span16 va = widen16(vsrc + ga, na), vb = widen16(vsrc + gb, nb);
    sva = s_vin + va.skip;
    svb = reinterpret_cast<const uint32_t*>(reinterpret_cast<const char*>(s_vin) + va.bytes) + vb.skip;
  }
  if (!mbar_wait(bar, 0, wait_ns)) {                   // gave up: flag it, let copies in flight land, leave
    if (tid == 0) atomicOr(err, kErrWaitTimeout);
    mbar_wait(bar, 0, wait_ns);
    return;
  }
  const int diag = min(tid * VT, cnt);
  const int mine = min(VT, cnt - diag);
  int ai = merge_path<K, int>(sa, na, sb, nb, diag);
  int bi = diag - ai;
  // One shared-memory read per output for the key (the list that advanced) and
  // one for the payload.  A key read may land one slot past A's end (inside
  // B's copy) or past B's end (inside the 64-byte slack of the key buffer);
  // the index tests decide, never that key.
  K ak = sa[ai];
  K bk = sb[bi];
  K ok[VT];
  uint32_t ov[VT];
#pragma unroll
  for (int j = 0; j < VT; ++j) {
    if (j < mine) {
      const bool take_b = (bi < nb) && ((ai >= na) || (bk < ak));
      ok[j] = from_order<K>(take_b ? bk : ak, f32_out);
      if (VALS) ov[j] = *(take_b ? svb + bi : sva + ai);
      if (take_b) ++bi; else ++ai;
      const K nx = *(take_b ? sb + bi : sa + ai);
      if (take_b) bk = nx; else ak = nx;
    }
  }
  __syncthreads();                                      // every thread is done reading the inputs
  K* s_kout = s_kin;                                    // 16-byte aligned staging, cnt <= T items
  uint32_t* s_vout = s_vin;
#pragma unroll
  for (int j = 0; j < VT; ++j) {
    if (j < mine) {
      s_kout[diag + j] = ok[j];
      if (VALS) s_vout[diag + j] = ov[j];
    }
  }
  static_assert(VT < kIdxStride, "at most one index entry per thread");
  if (kidx) {
    const int j0 = (int)((0u - (uint32_t)s_out - (uint32_t)diag) & (uint32_t)(kIdxStride - 1));
    if (j0 < mine) kidx[(s_out + (uint64_t)(diag + j0)) / kIdxStride] = s_kout[diag + j0];
  }
  __syncthreads();
  store_tile_vec<K, NT>(kdst + s_out, s_kout, cnt);
  if (VALS) store_tile_vec<uint32_t, NT>(vdst + s_out, s_vout, cnt);
}

// ---------------------------------------------------------------------------
// Four-way merge round: two levels of the Fig. 2 tree in one pass over HBM.
// Lists A, B, C, D (in stable order) merge into X = merge(A, B), Y = merge(C,
// D), then merge(X, Y).  The output is cut into chunks at every T-th element
// of X and of Y (the way step 4 cuts runs at splitters): an X cut at X
// position m takes the merge-path split of (A, B) at m, and its value's
// lower bounds in C and D (equal keys of C and D come after it); a Y cut
// takes the split of (C, D) and upper bounds in A and B.  Sorted by stable
// rank, consecutive cuts bound a chunk with at most T elements of X and at
// most T of Y, split exactly; a CTA merges the chunk's four pieces in shared
// memory (A+B and C+D, then X+Y) and stores it.
// ---------------------------------------------------------------------------

struct Quad {                 // four lists in stable order -> [out, out + sum n)
  uint64_t s[4];              // first element of each list
  uint64_t n[4];              // list lengths
  uint64_t out;
};

struct Cut4 {                 // a chunk boundary: its stable rank in the quad, the four list positions
  uint64_t rank;
  uint64_t p[4];
  uint64_t quad;
};

__device__ __forceinline__ uint64_t quad_cuts(const Quad& q, uint32_t T) {
  const uint64_t nx = q.n[0] + q.n[1], ny = q.n[2] + q.n[3];
  if (nx + ny == 0) return 0;
  const uint64_t cx = nx ? (nx + T - 1) / T - 1 : 0;
  const uint64_t cy = ny ? (ny + T - 1) / T - 1 : 0;
  return 1 + cx + cy;                                   // the start, X cuts, Y cuts
}

__device__ __forceinline__ void put_quad(Quad* quads, uint64_t* ccount, uint64_t p, const uint64_t b[5],
                                         uint64_t out, uint32_t T) {
  Quad q;
  for (int i = 0; i < 4; ++i) {
    q.s[i] = b[i];
    q.n[i] = b[i + 1] - b[i];
  }
  q.out = out;
  quads[p] = q;
  ccount[p] = quad_cuts(q, T);
}

// Run formation: blocks [j 4w + i w, j 4w + (i+1) w) of every run, i = 0..3.
static __global__ void k_quads_runs(Quad* quads, uint64_t* ccount, const uint64_t* __restrict__ run_off, uint32_t R,
                                    uint64_t w, uint64_t cmax, uint32_t T) {
  uint64_t p = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (p >= (uint64_t)R * cmax) return;
  const uint64_t r = p / cmax, j = p % cmax;
  const uint64_t rs = run_off[r], re = run_off[r + 1];
  uint64_t b[5];
  for (int i = 0; i < 5; ++i) b[i] = umin(rs + j * 4 * w + i * w, re);
  put_quad(quads, ccount, p, b, b[0], T);
}

// Bucket merge: groups of `step` segments; group g of a bucket starts at
// segment 4 g step (slot = global segment index; other slots empty).
static __global__ void k_quads_buckets(Quad* quads, uint64_t* ccount, Geo g, const uint64_t* __restrict__ off,
                                       uint64_t q0, uint64_t Q, uint32_t step, uint32_t T) {
  const uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (t >= Q) return;
  const uint64_t q = q0 + t;
  const uint32_t i = last_le<uint64_t>(g.seg, g.I, q);
  const uint64_t P = g.P[i];
  const uint64_t local = q - g.seg[i];
  const uint64_t bk = local / P, j = local % P;
  const uint64_t base = g.seg[i] + bk * P;
  uint64_t b[5];
  if (j % (4ull * step) != 0) {
    for (int k = 0; k < 5; ++k) b[k] = off[base + P];
  } else {
    for (int k = 0; k < 5; ++k) b[k] = off[base + umin(j + (uint64_t)k * step, P)];
  }
  put_quad(quads, ccount, t, b, b[0], T);
}

template <typename K>
__device__ __forceinline__ uint64_t lower_bound_g(const K* x, uint64_t n, K v) {
  uint64_t lo = 0, hi = n;
  while (lo < hi) { uint64_t mid = (lo + hi) >> 1; if (x[mid] < v) lo = mid + 1; else hi = mid; }
  return lo;
}
template <typename K>
__device__ __forceinline__ uint64_t upper_bound_g(const K* x, uint64_t n, K v) {
  uint64_t lo = 0, hi = n;
  while (lo < hi) { uint64_t mid = (lo + hi) >> 1; if (x[mid] <= v) lo = mid + 1; else hi = mid; }
  return lo;
}

// One thread per cut (unsorted): local index 0 is the quad start, 1..cx the
// X cuts at X positions T, 2T, ..., then the Y cuts.
template <typename K>
__global__ void k_cuts4(const K* __restrict__ src, const Quad* __restrict__ quads, const uint64_t* __restrict__ coff,
                        uint64_t nquads, Cut4* cuts, uint32_t T, const uint32_t* err) {
  if (poisoned(err)) return;
  const uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (t >= coff[nquads]) return;
  const uint64_t qi = last_le<uint64_t>(coff, (uint32_t)nquads, t);
  const Quad q = quads[qi];
  const uint64_t l = t - coff[qi];
  const uint64_t nx = q.n[0] + q.n[1];
  const uint64_t cx = nx ? (nx + T - 1) / T - 1 : 0;
  const K* A = src + q.s[0];
  const K* B = src + q.s[1];
  const K* C = src + q.s[2];
  const K* D = src + q.s[3];
  Cut4 c;
  c.quad = qi;
  if (l == 0) {
    c.rank = 0;
    c.p[0] = c.p[1] = c.p[2] = c.p[3] = 0;
  } else if (l <= cx) {
    const uint64_t m = l * T;
    const uint64_t a = merge_path<K, uint64_t>(A, q.n[0], B, q.n[1], m);
    const uint64_t b = m - a;
    const bool from_a = a < q.n[0] && (b >= q.n[1] || A[a] <= B[b]);
    const K v = from_a ? A[a] : B[b];
    c.p[0] = a;
    c.p[1] = b;
    c.p[2] = lower_bound_g<K>(C, q.n[2], v);
    c.p[3] = lower_bound_g<K>(D, q.n[3], v);
    c.rank = m + c.p[2] + c.p[3];
  } else {
    const uint64_t m = (l - cx) * T;
    const uint64_t cc = merge_path<K, uint64_t>(C, q.n[2], D, q.n[3], m);
    const uint64_t d = m - cc;
    const bool from_c = cc < q.n[2] && (d >= q.n[3] || C[cc] <= D[d]);
    const K v = from_c ? C[cc] : D[d];
    c.p[2] = cc;
    c.p[3] = d;
    c.p[0] = upper_bound_g<K>(A, q.n[0], v);
    c.p[1] = upper_bound_g<K>(B, q.n[1], v);
    c.rank = m + c.p[0] + c.p[1];
  }
  cuts[t] = c;
}

// Sort the cuts of every quad by rank: X cuts and Y cuts are each in rank
// order already, so a cut's place is its own index plus the number of the
// other side's cuts of smaller rank (ranks are distinct: they are the stable
// ranks of distinct elements).
static __global__ void k_cuts4_sort(const Cut4* __restrict__ in, const Quad* __restrict__ quads,
                                    const uint64_t* __restrict__ coff, uint64_t nquads, Cut4* out, uint32_t T,
                                    const uint32_t* err) {
  if (poisoned(err)) return;
  const uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (t >= coff[nquads]) return;
  const Cut4 c = in[t];
  const uint64_t qi = c.quad;
  const uint64_t base = coff[qi];
  const uint64_t l = t - base;
  if (l == 0) {
    out[base] = c;
    return;
  }
  const Quad q = quads[qi];
  const uint64_t nx = q.n[0] + q.n[1];
  const uint64_t cx = nx ? (nx + T - 1) / T - 1 : 0;
  const uint64_t ncut = coff[qi + 1] - base;
  const uint64_t cy = ncut - 1 - cx;
  // Other side: X cuts at [base+1, base+1+cx), Y cuts at [base+1+cx, base+ncut).
  const bool is_x = l <= cx;
  const Cut4* other = in + base + 1 + (is_x ? cx : 0);
  const uint64_t no = is_x ? cy : cx;
  uint64_t lo = 0, hi = no;                            // other cuts with rank < c.rank
  while (lo < hi) { uint64_t mid = (lo + hi) >> 1; if (other[mid].rank < c.rank) lo = mid + 1; else hi = mid; }
  const uint64_t own = is_x ? l - 1 : l - 1 - cx;
  out[base + 1 + own + lo] = c;
}

struct Chunk4 {               // one chunk of a four-way round: the four source ranges and the output start
  uint64_t s[4];
  uint32_t n[4];
  uint64_t out;
};

// Chunk t spans sorted cuts t and t+1 (or the quad's end).  A chunk whose
// pieces would not be ranges of their lists or would not fit max_chunk
// elements (impossible for sorted lists) is emptied and flagged.
static __global__ void k_chunks4(const Cut4* __restrict__ cuts, const Quad* __restrict__ quads,
                                 const uint64_t* __restrict__ coff, uint64_t nquads, Chunk4* chunks,
                                 uint32_t max_chunk, uint32_t* err) {
  if (poisoned(err)) return;
  const uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (t >= coff[nquads]) return;
  const Cut4 lo = cuts[t];
  const Quad q = quads[lo.quad];
  const bool last = t + 1 >= coff[lo.quad + 1];
  Chunk4 c;
  uint64_t sum = 0;
  bool bad = false;
  for (int i = 0; i < 4; ++i) {
    const uint64_t hi = last ? q.n[i] : cuts[t + 1].p[i];
    bad = bad || hi < lo.p[i] || hi > q.n[i];
    c.s[i] = q.s[i] + lo.p[i];
    c.n[i] = (uint32_t)(hi - lo.p[i]);
    sum += hi - lo.p[i];
  }
  if (bad || sum > max_chunk) {
    atomicOr(err, kErrBadTile);
    for (int i = 0; i < 4; ++i) { c.s[i] = q.s[i]; c.n[i] = 0; }
  }
  c.out = q.out + lo.rank;
  chunks[t] = c;
}

template <typename K, bool VALS, int NT, int VT>
struct Merge4Layout {
  static constexpr int M = NT * VT;                                   // largest chunk (2 T)
  static constexpr size_t kin = 16;
  static constexpr size_t vin = kin + (size_t)M * sizeof(K) + 128;
  static constexpr size_t kmid = vin + (VALS ? (size_t)M * 4 + 128 : 0);
  static constexpr size_t vmid = kmid + (size_t)M * sizeof(K);
  static constexpr size_t bytes = vmid + (VALS ? (size_t)M * 4 : 0);
  static_assert(M % 4 == 0, "16-byte aligned staging");
};

// Merge VT outputs of merge(a[0..na), b[0..nb)) starting at output `diag` into
// out[diag..]; payloads follow their keys (source payload arrays va, vb).
template <typename K, bool VALS, int VT>
__device__ __forceinline__ void merge_into(const K* a, const uint32_t* va, int na, const K* b, const uint32_t* vb,
                                           int nb, int diag, int count, K* out, uint32_t* vout, int f32_out) {
  if (count <= 0) return;
  int ai = merge_path<K, int>(a, na, b, nb, diag);
  int bi = diag - ai;
  K ak = ai < na ? a[ai] : key_max<K>();
  K bk = bi < nb ? b[bi] : key_max<K>();
#pragma unroll
  for (int j = 0; j < VT; ++j) {
    if (j < count) {
      const bool take_a = (bi >= nb) || (ai < na && ak <= bk);
      out[diag + j] = from_order<K>(take_a ? ak : bk, f32_out);
      if (VALS) vout[diag + j] = take_a ? va[ai] : vb[bi];
      if (take_a) {
        ++ai;
        ak = ai < na ? a[ai] : key_max<K>();
      } else {
        ++bi;
        bk = bi < nb ? b[bi] : key_max<K>();
      }
    }
  }
}

template <typename K, bool VALS, int NT, int VT>
__global__ void __launch_bounds__(NT)
k_merge4(const K* __restrict__ ksrc, const uint32_t* __restrict__ vsrc, K* __restrict__ kdst,
         uint32_t* __restrict__ vdst, const Chunk4* __restrict__ chunks, const uint64_t* __restrict__ total,
         int f32_out, uint32_t* err, K* __restrict__ kidx, uint64_t wait_ns) {
  using L = Merge4Layout<K, VALS, NT, VT>;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);
  char* s_kin = reinterpret_cast<char*>(smem_raw + L::kin);
  char* s_vin = reinterpret_cast<char*>(smem_raw + L::vin);
  K* s_kmid = reinterpret_cast<K*>(smem_raw + L::kmid);
  uint32_t* s_vmid = reinterpret_cast<uint32_t*>(smem_raw + L::vmid);
  __shared__ uint64_t s_lo[4], s_cnt[4], s_out;
  __shared__ uint32_t s_off_k[4], s_off_v[4];
  const uint64_t t = blockIdx.x;
  const int tid = threadIdx.x;
  if (tid == 0) {
    if (t < *total && !poisoned(err)) {
      const Chunk4 ch = chunks[t];
      uint32_t kbytes = 0, vbytes = 0;
      Span16 ks[4], vs[4];
      for (int i = 0; i < 4; ++i) {
        s_lo[i] = ch.s[i];
        s_cnt[i] = ch.n[i];
        ks[i] = widen16(ksrc + s_lo[i], (uint32_t)s_cnt[i]);
        s_off_k[i] = kbytes + ks[i].skip * (uint32_t)sizeof(K);
        kbytes += ks[i].bytes;
        if (VALS) {
          vs[i] = widen16(vsrc + s_lo[i], (uint32_t)s_cnt[i]);
          s_off_v[i] = vbytes + vs[i].skip * 4u;
          vbytes += vs[i].bytes;
        }
      }
      s_out = ch.out;
      mbar_init(bar, 1);
      fence_barrier_init();
      mbar_arrive_expect_tx(bar, kbytes + vbytes);
      uint32_t ko = 0, vo = 0;
      for (int i = 0; i < 4; ++i) {
        if (ks[i].bytes) bulk_load(s_kin + ko, ks[i].base, ks[i].bytes, bar);
        ko += ks[i].bytes;
        if (VALS) {
          if (vs[i].bytes) bulk_load(s_vin + vo, vs[i].base, vs[i].bytes, bar);
          vo += vs[i].bytes;
        }
      }
    } else {
      for (int i = 0; i < 4; ++i) s_cnt[i] = 0;
    }
  }
  __syncthreads();
  const int na = (int)s_cnt[0], nb = (int)s_cnt[1], nc = (int)s_cnt[2], nd = (int)s_cnt[3];
  const int nx = na + nb, ny = nc + nd, cnt = nx + ny;
  if (cnt == 0) return;
  if (!mbar_wait(bar, 0, wait_ns)) {
    if (tid == 0) atomicOr(err, kErrWaitTimeout);
    mbar_wait(bar, 0, wait_ns);
    return;
  }
  const K* A = reinterpret_cast<const K*>(s_kin + s_off_k[0]);
  const K* B = reinterpret_cast<const K*>(s_kin + s_off_k[1]);
  const K* C = reinterpret_cast<const K*>(s_kin + s_off_k[2]);
  const K* D = reinterpret_cast<const K*>(s_kin + s_off_k[3]);
  const uint32_t* vA = VALS ? reinterpret_cast<const uint32_t*>(s_vin + s_off_v[0]) : nullptr;
  const uint32_t* vB = VALS ? reinterpret_cast<const uint32_t*>(s_vin + s_off_v[1]) : nullptr;
  const uint32_t* vC = VALS ? reinterpret_cast<const uint32_t*>(s_vin + s_off_v[2]) : nullptr;
  const uint32_t* vD = VALS ? reinterpret_cast<const uint32_t*>(s_vin + s_off_v[3]) : nullptr;
  // Every thread takes an equal share of the chunk (odd, so blocked staging
  // writes stay conflict free), whatever the chunk's size.
  const int per = ((cnt + NT - 1) / NT) | 1;
  // Level 1: X = merge(A, B) into mid[0, nx), Y = merge(C, D) into mid[nx, cnt).
  {
    const int d0 = min(tid * per, cnt), d1 = min(d0 + per, cnt);
    if (d0 < nx) merge_into<K, VALS, VT>(A, vA, na, B, vB, nb, d0, min(d1, nx) - d0, s_kmid, s_vmid, 0);
    if (d1 > nx) {
      const int y0 = max(d0, nx) - nx;
      merge_into<K, VALS, VT>(C, vC, nc, D, vD, nd, y0, d1 - max(d0, nx), s_kmid + nx,
                              VALS ? s_vmid + nx : nullptr, 0);
    }
  }
  __syncthreads();
  // Level 2: merge(X, Y) into the (now free) input staging.
  K* s_kout = reinterpret_cast<K*>(s_kin);
  uint32_t* s_vout = reinterpret_cast<uint32_t*>(s_vin);
  {
    const int d0 = min(tid * per, cnt);
    merge_into<K, VALS, VT>(s_kmid, s_vmid, nx, s_kmid + nx, VALS ? s_vmid + nx : nullptr, ny, d0,
                            min(per, cnt - d0), s_kout, s_vout, f32_out);
  }
  __syncthreads();
  store_tile_vec<K, NT>(kdst + s_out, s_kout, cnt);
  if (VALS) store_tile_vec<uint32_t, NT>(vdst + s_out, s_vout, cnt);
  if (kidx) write_key_index(kidx, s_kout, s_out, cnt);
}

// ---------------------------------------------------------------------------
// Device-wide exclusive scan of uint64 (reduce, scan of chunk sums, scan).
// out[i] = sum_{j<i} in[j] for i in [0, m]; out[m] is the total.
// ---------------------------------------------------------------------------

// Exclusive scan across the CTA (blockDim.x a multiple of 32, at most 1024);
// every thread also gets the CTA total.  Ends with a barrier, so it may be
// called back to back.
__device__ __forceinline__ uint64_t block_exclusive_scan(uint64_t x, uint64_t* total) {
  __shared__ uint64_t warp_sums[33];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint64_t inc = x;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    uint64_t y = __shfl_up_sync(0xFFFFFFFFu, inc, d);
    if (lane >= d) inc += y;
  }
  if (lane == 31) warp_sums[warp] = inc;
  __syncthreads();
  const int nw = blockDim.x >> 5;
  if (warp == 0) {
    uint64_t v = lane < nw ? warp_sums[lane] : 0;
    uint64_t vi = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      uint64_t y = __shfl_up_sync(0xFFFFFFFFu, vi, d);
      if (lane >= d) vi += y;
    }
    if (lane < nw) warp_sums[lane] = vi - v;
    if (lane == 31) warp_sums[32] = vi;
  }
  __syncthreads();
  uint64_t res = warp_sums[warp] + inc - x;
  uint64_t tot = warp_sums[32];
  __syncthreads();
  if (total) *total = tot;
  return res;
}

static __global__ void __launch_bounds__(kScanNT)
k_scan_reduce(const uint64_t* __restrict__ in, uint64_t m, uint64_t* __restrict__ sums) {
  uint64_t base = blockIdx.x * (uint64_t)kScanChunk;
  uint64_t acc = 0;
#pragma unroll
  for (int i = 0; i < kScanVT; ++i) {
    uint64_t idx = base + i * kScanNT + threadIdx.x;
    if (idx < m) acc += in[idx];
  }
  uint64_t tot;
  block_exclusive_scan(acc, &tot);
  if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

// Scan chunk blockIdx.x of `in` with a starting offset (offsets[blockIdx.x] or 0).
static __global__ void __launch_bounds__(kScanNT)
k_scan_chunks(const uint64_t* __restrict__ in, uint64_t m, uint64_t* __restrict__ out,
              const uint64_t* __restrict__ offsets) {
  uint64_t base = blockIdx.x * (uint64_t)kScanChunk;
  uint64_t carry = offsets ? offsets[blockIdx.x] : 0;
  uint64_t v[kScanVT];
  uint64_t acc = 0;
#pragma unroll
  for (int i = 0; i < kScanVT; ++i) {             // blocked: thread t owns [t VT, t VT + VT)
    uint64_t idx = base + (uint64_t)threadIdx.x * kScanVT + i;
    v[i] = idx < m ? in[idx] : 0;
    acc += v[i];
  }
  uint64_t tot;
  uint64_t pre = block_exclusive_scan(acc, &tot) + carry;
#pragma unroll
  for (int i = 0; i < kScanVT; ++i) {
    uint64_t idx = base + (uint64_t)threadIdx.x * kScanVT + i;
    if (idx < m) out[idx] = pre;
    pre += v[i];
  }
  uint64_t end = base + kScanChunk;
  if (threadIdx.x == 0 && end >= m && base <= m) out[m] = carry + tot;
}

// ---------------------------------------------------------------------------
// Tables of a single sort of n keys on P runs (a batch of one).
// ---------------------------------------------------------------------------

static __global__ void k_tables_single(uint64_t* koff, uint32_t* Pt, uint32_t* R0, uint64_t* mat, uint64_t* seg,
                                       uint64_t* st, uint64_t* run_off, uint32_t* run_inst, uint64_t n, uint32_t P,
                                       uint64_t s) {
  uint64_t r = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (r > P) return;
  run_off[r] = run_start(r, n, P);
  if (r < P) run_inst[r] = 0;
  if (r == 0) {
    koff[0] = 0; koff[1] = n;
    Pt[0] = P;
    R0[0] = 0; R0[1] = P;
    mat[0] = 0; mat[1] = (uint64_t)P * (P + 1);
    seg[0] = 0; seg[1] = (uint64_t)P * P;
    st[0] = P > 1 ? s : 0;
  }
}

// ---------------------------------------------------------------------------
// K3: regular samples (step 2 of Section IV).
// Run r is cut into s_r = min(s, n_r) equal blocks; the last key of each block
// is sampled, local position floor((i+1) n_r / s_r) - 1.  Samples are written
// in (run, position) order, so each run's samples are sorted.
// ---------------------------------------------------------------------------

// Samples per run, s_r = min(s, n_r) (the scan of these gives every run's first sample).
static __global__ void k_sample_counts(Geo g, uint64_t* counts) {
  uint64_t r = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (r >= g.R) return;
  counts[r] = umin(g.s[g.run_inst[r]], g.run_off[r + 1] - g.run_off[r]);
}

template <typename K>
__global__ void k_sample(const K* __restrict__ runs, Geo g, const uint64_t* __restrict__ samp_off,
                         K* __restrict__ samples, uint64_t S) {
  uint64_t j = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (j >= S) return;
  const uint32_t r = last_le<uint64_t>(samp_off, g.R, j);
  const uint64_t i = j - samp_off[r], sr = samp_off[r + 1] - samp_off[r];
  const uint64_t rs = g.run_off[r], nr = g.run_off[r + 1] - rs;
  const uint64_t pos = (uint64_t)(((unsigned __int128)(i + 1) * nr) / sr) - 1;   // exact for any s_r, n_r
  samples[j] = runs[rs + pos];
}

// Step 3 of Section IV: with S_i samples, t_b = sorted sample at index
// floor(b S_i / P_i) - 1, b = 1..P_i-1.  t is indexed by global run (slot b of
// instance i is R0[i] + b; slot 0 unused).
template <typename K>
__global__ void k_pick_splitters(const K* __restrict__ sorted, Geo g, const uint64_t* __restrict__ samp_off, K* t,
                                 K* user_out, int f32) {
  uint64_t beta = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (beta >= g.R) return;
  const uint32_t i = g.run_inst[beta];
  const uint32_t r0 = g.R0[i];
  const uint64_t b = beta - r0, P = g.P[i];
  if (b == 0) return;
  const uint64_t s0 = samp_off[r0], S = samp_off[r0 + P] - s0;
  const K v = sorted[s0 + (b * S) / P - 1];
  t[beta] = v;
  if (user_out && g.I == 1) user_out[b - 1] = from_order<K>(v, f32);
}

// The same pick on one sorted sample of m keys: out[b-1] = sorted[floor(b m / P) - 1].
template <typename K>
__global__ void k_pick_splitters_flat(const K* __restrict__ sorted, uint64_t m, uint32_t P, K* out, int f32) {
  uint64_t b = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x + 1;
  if (b >= P) return;
  out[b - 1] = from_order<K>(sorted[(b * m) / P - 1], f32);
}

// ---------------------------------------------------------------------------
// K5: cut search + investigator (step 4 of Section IV, Section IV-B).
// ---------------------------------------------------------------------------

// lb[r][b] = #{x in run r : x < t_b}, cnt[r][b] = #{x in run r : x == t_b},
// b = 1..P-1, for every run of every instance (index space: the P x P
// segments; entries with b = 0 do nothing).
template <typename K>
__global__ void k_cut_search(const K* __restrict__ runs, Geo g, uint64_t Q, const K* __restrict__ t,
                             uint64_t* lb, uint64_t* cnt) {
  uint64_t q = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (q >= Q) return;
  const uint32_t i = last_le<uint64_t>(g.seg, g.I, q);
  const uint64_t P = g.P[i];
  const uint64_t local = q - g.seg[i];
  const uint64_t rl = local / P, b = local % P;
  if (b == 0) return;
  const uint32_t r0 = g.R0[i];
  const uint64_t rs = g.run_off[r0 + rl], nr = g.run_off[r0 + rl + 1] - rs;
  const K* x = runs + rs;
  const K v = t[r0 + b];
  uint64_t lo = 0, hi = nr;
  while (lo < hi) { uint64_t mid = (lo + hi) >> 1; if (x[mid] < v) lo = mid + 1; else hi = mid; }
  const uint64_t l = lo;
  hi = nr;
  while (lo < hi) { uint64_t mid = (lo + hi) >> 1; if (x[mid] <= v) lo = mid + 1; else hi = mid; }
  const uint64_t at = g.mat[i] + rl * (P + 1) + b;
  lb[at] = l;
  cnt[at] = lo - l;
}

// One CTA per splitter b = 1..P_i-1 of every instance (CTAs of slot b = 0
// exit).  L_b = sum_r lb, G_b = sum_r cnt, pre[r] = sum_{r'<r} cnt.  The
// variant picks e_b, then every run cuts cut[r][b] = lb + clamp(e_b - L_b -
// pre[r], 0, cnt): the keys equal to t_b are handed out in stable order (run,
// position) until e_b ranks are reached.
template <typename K>
__global__ void __launch_bounds__(256)
k_investigator(const uint64_t* __restrict__ lb, const uint64_t* __restrict__ cnt, const K* __restrict__ t, Geo g,
               int variant, uint64_t* cut, uint64_t* e) {
  const uint32_t beta = blockIdx.x;
  const uint32_t i = g.run_inst[beta];
  const uint32_t r0 = g.R0[i];
  const uint64_t b = beta - r0, P = g.P[i];
  if (b == 0) return;
  const uint64_t n = g.koff[i + 1] - g.koff[i];
  const uint64_t W = P + 1;
  const uint64_t* lbi = lb + g.mat[i];
  const uint64_t* cnti = cnt + g.mat[i];
  uint64_t* cuti = cut + g.mat[i];
  __shared__ uint64_t sh_L, sh_e, sh_g0, sh_k;
  // Group of equal splitters containing t_b: slots [g0, g0 + k) of 1..P-1.
  auto group = [&](uint64_t& g0, uint64_t& k) {
    const K* ti = t + r0;
    const K v = ti[b];
    uint64_t lo = 1, hi = P;
    while (lo < hi) { uint64_t m = (lo + hi) >> 1; if (ti[m] < v) lo = m + 1; else hi = m; }
    g0 = lo;
    hi = P;
    while (lo < hi) { uint64_t m = (lo + hi) >> 1; if (ti[m] <= v) lo = m + 1; else hi = m; }
    k = lo - g0;
  };
  if (variant == 3) {
    // The text's literal rule: every run divides its own range of a duplicated
    // value into k equal parts; e_b is the sum of the runs' cuts.
    if (threadIdx.x == 0) {
      uint64_t g0, k;
      group(g0, k);
      sh_g0 = g0;
      sh_k = k;
    }
    __syncthreads();
    const uint64_t j = b - sh_g0, k = sh_k;
    uint64_t part = 0;
    for (uint64_t r = threadIdx.x; r < P; r += blockDim.x) {
      const uint64_t c = lbi[r * W + b] + (cnti[r * W + b] * (j + 1)) / k;
      cuti[r * W + b] = c;
      part += c;
    }
    uint64_t total;
    block_exclusive_scan(part, &total);
    if (threadIdx.x == 0) e[r0 + i + b] = total;
    return;
  }
  uint64_t ls = 0, gs = 0;
  for (uint64_t r = threadIdx.x; r < P; r += blockDim.x) {
    ls += lbi[r * W + b];
    gs += cnti[r * W + b];
  }
  uint64_t Lb, Gb;
  block_exclusive_scan(ls, &Lb);
  block_exclusive_scan(gs, &Gb);
  if (threadIdx.x == 0) {
    const uint64_t target = (b * n) / P;
    uint64_t eb;
    if (variant == 0) {
      eb = umin(umax(target, Lb), Lb + Gb);
    } else if (variant == 2) {
      eb = Lb + Gb;
    } else {
      uint64_t g0, k;
      group(g0, k);
      eb = Lb + (Gb * (b - g0 + 1)) / k;
    }
    sh_L = Lb;
    sh_e = eb;
    e[r0 + i + b] = eb;
  }
  __syncthreads();
  const uint64_t L = sh_L, eb = sh_e;
  uint64_t carry = 0;
  for (uint64_t rb = 0; rb < P; rb += blockDim.x) {
    const uint64_t r = rb + threadIdx.x;
    const uint64_t c = r < P ? cnti[r * W + b] : 0;
    uint64_t chunk;
    const uint64_t pre = block_exclusive_scan(c, &chunk) + carry;
    if (r < P) {
      const uint64_t want = eb - L;                 // >= 0: L <= e_b in every variant
      const uint64_t take = want > pre ? umin(want - pre, c) : 0;
      cuti[r * W + b] = lbi[r * W + b] + take;
    }
    carry += chunk;
  }
}

// cut[r][0] = 0, cut[r][P] = n_r for every run; e[0] = 0, e[P] = n_i.
static __global__ void k_cut_edges(Geo g, uint64_t* cut, uint64_t* e) {
  uint64_t r = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (r >= g.R) return;
  const uint32_t i = g.run_inst[r];
  const uint32_t r0 = g.R0[i];
  const uint64_t P = g.P[i], rl = r - r0;
  uint64_t* row = cut + g.mat[i] + rl * (P + 1);
  row[0] = 0;
  row[P] = g.run_off[r + 1] - g.run_off[r];
  if (rl == 0) {
    e[r0 + i] = 0;
    e[r0 + i + P] = g.koff[i + 1] - g.koff[i];
  }
}

// Segments (bucket b, run r) of every instance, bucket-major: their sizes
// cut[r][b+1] - cut[r][b] and the global position where they start.
static __global__ void k_bucket_sizes(Geo g, uint64_t Q, const uint64_t* __restrict__ cut, uint64_t* sizes,
                                      uint64_t* src) {
  uint64_t q = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (q >= Q) return;
  const uint32_t i = last_le<uint64_t>(g.seg, g.I, q);
  const uint64_t P = g.P[i];
  const uint64_t local = q - g.seg[i];
  const uint64_t b = local / P, rl = local % P;
  const uint64_t* c = cut + g.mat[i] + rl * (P + 1);
  sizes[q] = c[b + 1] - c[b];
  src[q] = g.run_off[g.R0[i] + rl] + c[b];
}

// ---------------------------------------------------------------------------
// K7: the exchange (step 5 of Section IV, Section IV-C) as an in-HBM scatter.
// Segment q = b P + r (bucket-major) moves from run r's sorted positions
// [cut[r][b], cut[r][b+1]) to [off[q], off[q+1]).  The copy is tiled by
// destination: each CTA stages kScatterTile outputs in shared memory and
// stores them back contiguously.
// ---------------------------------------------------------------------------

static __global__ void k_scatter_part(const uint64_t* __restrict__ off, uint64_t Q, uint64_t n,
                               uint64_t* first_seg) {
  uint64_t tile = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  uint64_t o = tile * kScatterTile;
  if (o >= n) return;
  uint64_t lo = 0, hi = Q;                        // last q with off[q] <= o
  while (hi - lo > 1) {
    uint64_t mid = (lo + hi) >> 1;
    if (off[mid] <= o) lo = mid; else hi = mid;
  }
  first_seg[tile] = lo;
}

template <typename K>
struct ScatterSmem {
  uint64_t off[kScatterWindow + 1];
  uint64_t src[kScatterWindow];
  K keys[kScatterTile];
  uint32_t vals[kScatterTile];
};

template <typename K, bool VALS>
__global__ void __launch_bounds__(kScatterNT)
k_scatter(const K* __restrict__ ksrc, const uint32_t* __restrict__ vsrc, K* __restrict__ kdst,
          uint32_t* __restrict__ vdst, const uint64_t* __restrict__ off, const uint64_t* __restrict__ seg_src,
          const uint64_t* __restrict__ first_seg, uint64_t n, uint64_t Q, int f32_out, const uint32_t* err) {
  if (poisoned(err)) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  ScatterSmem<K>& sm = *reinterpret_cast<ScatterSmem<K>*>(smem_raw);
  const uint64_t o = blockIdx.x * (uint64_t)kScatterTile;
  const int cnt = (int)umin(kScatterTile, n - o);
  const uint64_t q0 = first_seg[blockIdx.x];
  const int wn = (int)umin(kScatterWindow, Q - q0);
  for (int i = threadIdx.x; i <= wn; i += blockDim.x) sm.off[i] = off[q0 + i];
  for (int i = threadIdx.x; i < wn; i += blockDim.x) sm.src[i] = seg_src[q0 + i];
  __syncthreads();
  // Warp w copies positions [o + w 32 VT, ...) 32 at a time; lane l walks its segment forward.
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int base = warp * 32 * kScatterVT;
  int lo = 0, hi = wn;
  uint64_t gp = o + base + lane;
  while (hi - lo > 1) { int mid = (lo + hi) >> 1; if (sm.off[mid] <= gp) lo = mid; else hi = mid; }
  int q = lo;
  for (int k = 0; k < kScatterVT; ++k) {
    const int p = base + k * 32 + lane;
    if (p >= cnt) break;
    gp = o + p;
    uint64_t s;
    while (q < wn && sm.off[q + 1] <= gp) ++q;
    if (q < wn) {
      s = sm.src[q] + (gp - sm.off[q]);
    } else {                                         // beyond the staged window: search globally
      uint64_t glo = q0 + wn, ghi = Q;
      while (ghi - glo > 1) {
        uint64_t mid = (glo + ghi) >> 1;
        if (off[mid] <= gp) glo = mid; else ghi = mid;
      }
      s = seg_src[glo] + (gp - off[glo]);
    }
    sm.keys[p] = ksrc[s];
    if (VALS) sm.vals[p] = vsrc[s];
  }
  __syncthreads();
  for (int p = threadIdx.x; p < cnt; p += blockDim.x) sm.keys[p] = from_order<K>(sm.keys[p], f32_out);
  __syncthreads();
  store_tile_vec<K, kScatterNT>(kdst + o, sm.keys, cnt);
  if (VALS) store_tile_vec<uint32_t, kScatterNT>(vdst + o, sm.vals, cnt);
}

// Pseudo-random keys (splitmix64 of the position and a seed) and index
// payloads, for timing runs of the tuner.
template <typename K>
__global__ void k_fill_random(K* keys, uint32_t* vals, uint64_t n, uint64_t seed) {
  const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint64_t z = (i + 1) * 0x9E3779B97F4A7C15ull + seed;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  keys[i] = (K)z;
  if (vals) vals[i] = (uint32_t)i;
}

// ---------------------------------------------------------------------------
// K9: load statistics (Table II: each processor's share after the sort).
// ---------------------------------------------------------------------------

struct DevStats {                     // layout of pgs_stats
  uint64_t n;
  uint32_t P, s;
  uint64_t max_bucket, min_bucket;
  uint32_t splitter_mode, fallback, error, passes;
  uint32_t launches;
  float max_over_mean;
  float learned_over_mean;
  uint32_t reserved;
};

// Bucket sizes e_{b+1} - e_b over all buckets of all instances: the largest,
// the smallest, and the largest ratio to its instance's mean n_i / P_i.
static __global__ void __launch_bounds__(256)
k_stats(Geo g, const uint64_t* __restrict__ e, uint64_t n_total, uint32_t s, uint32_t mode, uint32_t passes,
        uint32_t launches, const uint32_t* err_word, const uint32_t* fallback_word,
        const float* learned_ratio, DevStats* st, uint64_t* user_bounds, float* max_ratio_out) {
  __shared__ uint64_t smax[256], smin[256];
  __shared__ float sratio[256];
  uint64_t mx = 0, mn = ~0ull;
  float ratio = 0.0f;
  for (uint32_t beta = threadIdx.x; beta < g.R; beta += blockDim.x) {
    const uint32_t i = g.run_inst[beta];
    const uint32_t b = beta - g.R0[i];
    const uint64_t sz = e[g.R0[i] + i + b + 1] - e[g.R0[i] + i + b];
    mx = umax(mx, sz);
    mn = umin(mn, sz);
    const uint64_t ni = g.koff[i + 1] - g.koff[i];
    if (ni) ratio = fmaxf(ratio, (float)((double)sz * g.P[i] / (double)ni));
  }
  smax[threadIdx.x] = mx;
  smin[threadIdx.x] = mn;
  sratio[threadIdx.x] = ratio;
  __syncthreads();
  for (int d = 128; d > 0; d >>= 1) {
    if (threadIdx.x < d) {
      smax[threadIdx.x] = umax(smax[threadIdx.x], smax[threadIdx.x + d]);
      smin[threadIdx.x] = umin(smin[threadIdx.x], smin[threadIdx.x + d]);
      sratio[threadIdx.x] = fmaxf(sratio[threadIdx.x], sratio[threadIdx.x + d]);
    }
    __syncthreads();
  }
  if (user_bounds && g.I == 1)
    for (uint32_t b = threadIdx.x; b <= g.P[0]; b += blockDim.x) user_bounds[b] = e[b];
  if (threadIdx.x == 0) {
    if (max_ratio_out) *max_ratio_out = sratio[0];
    if (st) {
      st->n = n_total;
      st->P = g.I == 1 ? g.P[0] : g.R;
      st->s = s;
      st->max_bucket = smax[0];
      st->min_bucket = g.R ? smin[0] : 0;
      st->splitter_mode = mode;
      st->fallback = fallback_word ? *fallback_word : 0;
      st->error = err_word ? *err_word : 0;
      st->passes = passes;
      st->launches = launches;
      st->max_over_mean = sratio[0];
      st->learned_over_mean = learned_ratio ? *learned_ratio : 0.0f;
      st->reserved = 0;
    }
  }
}

}  // namespace pgs
