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
#ifndef PGS_BLOCK_VT
#define PGS_BLOCK_VT 17
#endif
constexpr int kVT = PGS_BLOCK_VT;    // items per thread; odd, so blocked smem access is conflict free
constexpr int kTile = kNT * kVT;     // 4352 keys per block-sort tile and per merge tile
constexpr int kMergeMinTile = 64 * 17;            // smallest merge tile of the tunable shapes
// Four-way rounds, per key width: threads per CTA, outputs per thread at most
// (odd, so the blocked staging is free of bank conflicts) and CTAs per SM to
// compile for.  Measured per pass (ms; 2^27 u64 keys, 2^28 u32 keys):
// 8-byte keys 128 x 19 0.748, 128 x 17 0.752, 128 x 25 0.761, 256 x 17 0.779,
// 128 x 21 0.796, 128 x 33 0.823 (the whole 2^28-key u64 sort 17.79 ms with
// 128 x 19 against 17.86 with 128 x 17); 4-byte keys 256 x 17 1.133-1.136,
// 128 x 21 1.168, 256 x 15 1.182, 128 x 17 1.188, 128 x 25 1.188,
// 256 x 21 1.246, 256 x 13 1.248, 128 x 33 1.257, 256 x 19 1.283.
// (PGS_MERGE4_NT / _VT / _MIN_BLOCKS set one shape for both widths, for such
// sweeps.)
template <int W> struct Merge4Shape;
#ifdef PGS_MERGE4_NT
template <int W> struct Merge4Shape {
  static constexpr int NT = PGS_MERGE4_NT, VT = PGS_MERGE4_VT, MIN_BLOCKS = PGS_MERGE4_MIN_BLOCKS;
};
#else
template <> struct Merge4Shape<8> { static constexpr int NT = 128, VT = 19, MIN_BLOCKS = 6; };
template <> struct Merge4Shape<4> { static constexpr int NT = 256, VT = 17, MIN_BLOCKS = 3; };
#endif
template <typename K> constexpr int merge4_nt() { return Merge4Shape<(int)sizeof(K)>::NT; }
template <typename K> constexpr int merge4_vt() { return Merge4Shape<(int)sizeof(K)>::VT; }
// Index samples per tile: tiles hold at most 64 Q + 4 x 63 <= NT x VT outputs.
template <typename K> constexpr uint32_t merge4_q() { return (merge4_nt<K>() * merge4_vt<K>() - 4 * 63) / 64; }
// The smallest Q of any key width (workspace bounds that hold for all of them).
constexpr uint32_t kMerge4MinQ = merge4_q<uint64_t>() < merge4_q<uint32_t>() ? merge4_q<uint64_t>()
                                                                              : merge4_q<uint32_t>();
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
// partition bisects it before touching the keys themselves, and a four-way
// round places its tile boundaries with it.  The block sort and the exchange
// write it too.
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
             const uint64_t* __restrict__ run_off, uint32_t tiles_per_run, int f32_in, int f32_out,
             K* __restrict__ kidx) {
  pdl_enter();
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
  if (kidx) write_key_index(kidx, sm.keys, g0, cnt);
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

// Pair descriptors of one pairwise round.  A generator writes slot p of the
// round's pair table (pairs[p], and its tile count at merge tile `tile`);
// k_pairs runs one generator over all slots, and k_plan_jobs (below) runs it
// inside the single CTA that also scans a small round and writes its tile jobs.

// Run formation (step 1): inside every run, blocks [j 2w, j 2w + w) and
// [j 2w + w, (j+1) 2w) merge; a run that is already one list is copied.
// Index space: run x pair slot (cmax slots per run, unused slots are empty).
struct GenRuns {
  Pair* pairs; uint64_t* tcount; const uint64_t* run_off; uint32_t R; uint64_t w, cmax; uint32_t tile;
  __device__ void operator()(uint64_t p) const {
    const uint64_t r = p / cmax, j = p % cmax;
    const uint64_t rs = run_off[r], re = run_off[r + 1];
    uint64_t lo = umin(rs + j * 2 * w, re);
    if (j > 0 && lo >= re) lo = re;                   // empty slot
    const uint64_t mid = umin(lo + w, re);
    const uint64_t hi = umin(lo + 2 * w, re);
    put_pair(pairs, tcount, p, lo, mid, hi, tile);
  }
};

// The Fig. 2 schedule over the P lists of one group: round `step` merges list
// group [j, j+step) with [j+step, j+2 step) for j a multiple of 2 step.  Lists
// of group g are [tbl[g0 + j], tbl[g0 + j + 1]); the index space is one slot
// per list (slots that do not start a pair are empty).
//  - samples (step 3): one group per instance, lists = its runs' samples,
//    tbl = sample offsets indexed by global run, slot = global run;
//  - buckets (step 6): one group per bucket, lists = its P segments,
//    tbl = segment offsets (bucket-major), slot = global segment.
struct GenSampleLists {
  Pair* pairs; uint64_t* tcount; Geo g; const uint64_t* samp_off; uint32_t step; uint32_t tile;
  __device__ void operator()(uint64_t p) const {
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
};

// Slots [q0, q0 + Q) take part (whole buckets); slot q0 + t writes pair t.
struct GenBucketLists {
  Pair* pairs; uint64_t* tcount; Geo g; const uint64_t* off; uint64_t q0; uint32_t step; uint32_t tile;
  __device__ void operator()(uint64_t t) const {
    const uint64_t q = q0 + t;
    const uint32_t i = last_le<uint64_t>(g.seg, g.I, q);
    const uint64_t P = g.P[i];
    const uint64_t local = q - g.seg[i];
    const uint64_t b = local / P, j = local % P;
    const uint64_t base = g.seg[i] + b * P;         // first segment of bucket b
    if (j % (2 * step) != 0) {
      const uint64_t end = off[base + P];
      put_pair(pairs, tcount, t, end, end, end, tile);
      return;
    }
    put_pair(pairs, tcount, t, off[base + j], off[base + umin(j + step, P)], off[base + umin(j + 2 * step, P)],
             tile);
  }
};

// Step 5 fused into the first round of step 6: segment j of bucket b (j even)
// merges with segment j+1 straight from the sorted runs, where the exchange
// would have copied them from, into the pair's place in bucket-major order.
// Slots [q0, q0 + Q) take part (whole buckets); slot q0 + t writes pair t.
struct GenFused {
  Pair* pairs; uint64_t* tcount; Geo g; const uint64_t* off; const uint64_t* seg_src; uint64_t q0; uint32_t tile;
  __device__ void operator()(uint64_t t) const {
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
};

// The pair table is already written (the four-way round's index-sample pairs).
struct GenNone {
  __device__ void operator()(uint64_t) const {}
};

template <typename Gen>
__global__ void k_pairs(Gen gen, uint64_t npairs) {
  pdl_enter();
  const uint64_t p = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (p < npairs) gen(p);
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

// Staging offset for a tile that will leave for global address g: element i
// of the tile is staged at s[pad + i], where pad (< 16 / sizeof(T)) makes the
// first 16-byte-aligned global element land on a 16-byte-aligned shared slot
// (s itself 16-byte aligned), so the aligned body can leave by one bulk store.
template <typename T>
__device__ __forceinline__ int stage_pad(const T* g) {
  constexpr int E = 16 / sizeof(T);
  const int head = (int)(((16 - (reinterpret_cast<uintptr_t>(g) & 15)) & 15) / sizeof(T));
  return (E - head) % E;
}

// Store cnt staged elements s[0, cnt) (s = the staging base plus stage_pad(g))
// to g: the unaligned head and tail element by element, the 16-byte-aligned
// body by one bulk store issued by thread 0.  Call after every thread has
// staged its elements, run fence_proxy_async_smem() and passed a barrier;
// thread 0 then commits and waits for the bulk reads before leaving.
template <typename T, int NT>
__device__ __forceinline__ void store_tile_bulk(T* g, const T* s, int cnt) {
  constexpr int E = 16 / sizeof(T);
  const int tid = threadIdx.x;
  int head = (int)(((16 - (reinterpret_cast<uintptr_t>(g) & 15)) & 15) / sizeof(T));
  if (head > cnt) head = cnt;
  const int body = ((cnt - head) / E) * E;
  if (tid < head) g[tid] = s[tid];
  for (int i = head + body + tid; i < cnt; i += NT) g[i] = s[i];
  if (tid == 0 && body > 0) bulk_store(g + head, s + head, (uint32_t)(body * sizeof(T)));
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

// A merge tile described by its pair and its first diagonal only: the merge
// CTA finds the splits at both ends itself (warp_merge_path).  Small rounds
// use it, so that their planning launch does no search.
struct TileJob {
  uint64_t a, na, b, nb;  // the pair's A and B lists
  uint64_t out;           // where the pair's output starts
  uint64_t d0;            // the tile's first output within the pair
};
static_assert(sizeof(TileJob) == sizeof(TileSplit), "jobs and splits share a buffer");

// Pairs that a merge CTA of a single sort's small round works out itself from
// an offsets table, so the round needs no planning launch.  CTA v takes tile
// v % cm of pair slot v / cm (cm: the most tiles any pair can need):
//  - kind kRunPairs: run formation, slot = run r x pair j (spr slots per run),
//    blocks [j 2w, j 2w + w) and [j 2w + w, (j+1) 2w) of run [off[r], off[r+1]);
//  - kind kListPairs: the Fig. 2 schedule over lists [off[j], off[j+1]),
//    j < n_lists, at `step`: slot k merges list group [2 step k, 2 step k + step)
//    with [2 step k + step, 2 step (k+1)).
// The output of a pair starts where its first list does.
constexpr uint32_t kRunPairs = 1, kListPairs = 2;
struct InlinePairs {
  const uint64_t* off;
  uint64_t w;
  uint32_t kind, n_lists, spr, step, cm;
};

__device__ __forceinline__ bool inline_job(const InlinePairs& ip, uint64_t v, uint64_t T, TileJob& jb) {
  const uint64_t slot = v / ip.cm, k = v % ip.cm;
  uint64_t lo, mid, hi;
  if (ip.kind == kRunPairs) {
    const uint64_t r = slot / ip.spr, j = slot % ip.spr;
    if (r >= ip.n_lists) return false;
    const uint64_t rs = ip.off[r], re = ip.off[r + 1];
    lo = umin(rs + j * 2 * ip.w, re);
    mid = umin(lo + ip.w, re);
    hi = umin(lo + 2 * ip.w, re);
  } else {
    const uint64_t j = slot * 2 * ip.step;
    if (j >= ip.n_lists) return false;
    lo = ip.off[j];
    mid = ip.off[umin(j + ip.step, ip.n_lists)];
    hi = ip.off[umin(j + 2 * ip.step, ip.n_lists)];
  }
  if (k * T >= hi - lo) return false;
  jb = TileJob{lo, mid - lo, mid, hi - mid, lo, k * T};
  return true;
}

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

// The first index in [lo, hi) whose test fails, for a test that holds on a
// prefix of [lo, hi) (hi if it holds everywhere), found by one warp: each
// step the 32 lanes evaluate 32 evenly spaced candidates at once, so a range
// of m candidates takes about log_33(m) dependent steps instead of log_2(m).
// Every lane of the warp must call it with the same range and test; every
// lane gets the answer.
template <typename Test>
__device__ __forceinline__ uint64_t warp_partition_point(uint64_t lo, uint64_t hi, const Test& test) {
  const uint32_t lane = threadIdx.x & 31u;
  while (hi > lo) {
    const uint64_t span = hi - lo;
    const bool last = span <= 32;
    // candidates strictly increasing in the lane, all inside [lo, hi)
    const uint64_t m = last ? lo + lane : lo + ((uint64_t)(lane + 1) * span) / 33;
    const bool holds = (!last || lane < span) && test(m);
    const int c = __popc(__ballot_sync(0xFFFFFFFFu, holds));   // the test holds on a prefix of the lanes
    if (last) return lo + (uint64_t)c;
    const uint64_t below = __shfl_sync(0xFFFFFFFFu, m, c > 0 ? c - 1 : 0);
    const uint64_t above = __shfl_sync(0xFFFFFFFFu, m, c < 32 ? c : 31);
    if (c > 0) lo = below + 1;
    if (c < 32) hi = above;
  }
  return lo;
}

// merge_path by one warp (the same test, so the same answer).
template <typename K>
__device__ __forceinline__ uint64_t warp_merge_path(const K* a, uint64_t na, const K* b, uint64_t nb, uint64_t d) {
  return warp_partition_point(d > nb ? d - nb : 0, d < na ? d : na,
                              [&](uint64_t m) { return a[m] <= b[d - 1 - m]; });
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

// The split of merge tile i of a round: its pair (a gallop from the guess
// i npairs / total through the tile-count scan), then one merge-path search,
// through the key index when both lists are long.
template <typename K>
__device__ __forceinline__ void partition_tile(uint64_t i, uint64_t total, const K* __restrict__ src,
                                               const Pair* __restrict__ pairs, const uint64_t* __restrict__ tbegin,
                                               uint64_t npairs, TileSplit* split, uint32_t tile,
                                               const K* __restrict__ kidx) {
  const uint64_t guess = (uint64_t)(((unsigned __int128)i * npairs) / total);   // < npairs as i < total
  const uint64_t lo = last_le_from(tbegin, npairs, i, guess);                 // the tile's pair
  const Pair pr = pairs[lo];
  const uint64_t d0 = (i - tbegin[lo]) * tile;
  const uint64_t a0 = (kidx && pr.na >= kIdxMinList && pr.nb >= kIdxMinList)
                          ? merge_path_indexed<K>(src, kidx, pr, d0)
                          : merge_path<K, uint64_t>(src + pr.a, pr.na, src + pr.b, pr.nb, d0);
  split[i] = TileSplit{pr.a + a0, pr.b + (d0 - a0), pr.out + d0, pr.a + pr.na, pr.b + pr.nb, lo};
}

template <typename K>
__global__ void k_partition_split(const K* __restrict__ src, const Pair* __restrict__ pairs,
                                  const uint64_t* __restrict__ tbegin, uint64_t npairs, TileSplit* split,
                                  uint32_t tile, const K* __restrict__ kidx, const uint32_t* err) {
  pdl_enter();
  if (poisoned(err)) return;
  const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  const uint64_t total = tbegin[npairs];
  if (i >= total) return;
  partition_tile<K>(i, total, src, pairs, tbegin, npairs, split, tile, kidx);
}

// A small round planned by one CTA: the pair table (gen), its tile counts'
// exclusive scan into tbegin, and one job per tile (its pair and first
// diagonal; the merge CTA searches its own splits).  For rounds of at most
// kPlanMaxPairs pairs and kPlanMaxTiles tiles, where separate launches for
// the table, the scan and the splits would cost more than the work.  (With
// 8192 tiles a 2^24-key pairwise sort was measured 6-7 % slower than with the
// separate partition kernel; 4096 covers the pairwise rounds of sorts up to
// about 2^23 keys, and larger sorts merge four ways.)
constexpr int kPlanNT = 1024;
constexpr int kPlanVT = 8;
constexpr uint64_t kPlanMaxPairs = (uint64_t)kPlanNT * kPlanVT;
constexpr uint64_t kPlanMaxTiles = 4096;             // larger rounds plan faster with the partition kernel

// One round's plan by the whole CTA (kPlanNT threads) into a job table of
// cap entries (cap <= kPlanMaxTiles); ends with a barrier.
template <typename Gen>
__device__ __forceinline__ void plan_round(const Gen& gen, const Pair* pairs, const uint64_t* tcount, uint64_t* tbegin,
                                           uint64_t npairs, TileJob* jobs, uint64_t cap, uint32_t tile,
                                           uint32_t* err) {
  __shared__ uint16_t s_tb[kPlanMaxPairs + 1];         // tbegin, while the total fits kPlanMaxTiles
  const int tid = threadIdx.x;
  for (uint64_t p = tid; p < npairs; p += kPlanNT) gen(p);
  __syncthreads();                                    // the CTA's global writes are visible to itself
  uint64_t v[kPlanVT];
  uint64_t acc = 0;
#pragma unroll
  for (int k = 0; k < kPlanVT; ++k) {                 // blocked: thread t owns slots [t VT, t VT + VT)
    const uint64_t idx = (uint64_t)tid * kPlanVT + k;
    v[k] = idx < npairs ? tcount[idx] : 0;
    acc += v[k];
  }
  uint64_t total;
  uint64_t pre = block_exclusive_scan(acc, &total);
  if (total > cap) {                                  // the host's bound did not hold: never expected
    if (tid == 0) {
      atomicOr(err, kErrBadTile);
      tbegin[npairs] = 0;                             // no tiles: the round's merge CTAs all leave
    }
    __syncthreads();
    return;
  }
#pragma unroll
  for (int k = 0; k < kPlanVT; ++k) {
    const uint64_t idx = (uint64_t)tid * kPlanVT + k;
    if (idx < npairs) {
      tbegin[idx] = pre;
      s_tb[idx] = (uint16_t)pre;
    }
    pre += v[k];
  }
  if (tid == 0) {
    tbegin[npairs] = total;
    s_tb[npairs] = (uint16_t)total;
  }
  __syncthreads();
  for (uint32_t t = tid; t < total; t += kPlanNT) {
    uint32_t lo = 0, hi = (uint32_t)npairs;             // the last slot whose first tile is <= t
    while (hi - lo > 1) {
      const uint32_t mid = (lo + hi) >> 1;
      if (s_tb[mid] <= t) lo = mid; else hi = mid;
    }
    const Pair pr = pairs[lo];
    jobs[t] = TileJob{pr.a, pr.na, pr.b, pr.nb, pr.out, (uint64_t)(t - s_tb[lo]) * tile};
  }
  __syncthreads();                                    // pairs and s_tb are free for the next round
}

template <typename Gen>
__global__ void __launch_bounds__(kPlanNT)
k_plan_jobs(Gen gen, const Pair* pairs, const uint64_t* tcount, uint64_t* tbegin, uint64_t npairs, TileJob* jobs,
            uint64_t cap, uint32_t tile, uint32_t* err) {
  pdl_enter();
  if (cta_poisoned(err)) return;
  plan_round(gen, pairs, tcount, tbegin, npairs, jobs, umin(cap, kPlanMaxTiles), tile, err);
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
             uint32_t* __restrict__ vdst, const TileSplit* __restrict__ split, const TileJob* __restrict__ jobs,
             InlinePairs ip, const uint64_t* __restrict__ total_ptr, int f32_out, uint32_t* err,
             K* __restrict__ kidx, uint64_t wait_ns, int inject_timeout) {
  pdl_enter();
  using L = Merge2Layout<K, VALS, NT, VT>;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);
  K* s_kin = reinterpret_cast<K*>(smem_raw + L::kin);
  uint32_t* s_vin = reinterpret_cast<uint32_t*>(smem_raw + L::vin);
  __shared__ uint32_t s_na, s_nb;
  __shared__ uint64_t s_a, s_b, s_out;
  __shared__ uint64_t s_cut[2];                         // job mode: A items before the tile's two ends
  __shared__ int s_found[2];

  const uint64_t tile = blockIdx.x;
  const int tid = threadIdx.x;
  static_assert(NT >= 64, "job mode searches with two warps");
  const bool job_mode = jobs != nullptr || ip.kind != 0;
  TileJob jb{};
  if (job_mode) {
    // Warp 0 finds the split at the tile's first diagonal, warp 1 at its end.
    // A warp that saw no failed kernel reads a job table the plan wrote for
    // this round (the error word only ever gains bits).
    if (tid < 64) {
      const int w = tid >> 5;
      bool live = !poisoned(err);
      if (live) {
        if (ip.kind != 0) live = inline_job(ip, tile, (uint64_t)L::T, jb);
        else if (tile < *total_ptr) jb = jobs[tile];
        else live = false;
      }
      live = __all_sync(0xFFFFFFFFu, live);             // the warp searches together or not at all
      if (live) {
        const uint64_t n = jb.na + jb.nb;
        const uint64_t d = w == 0 ? jb.d0 : umin(jb.d0 + (uint64_t)L::T, n);
        const uint64_t cut = warp_merge_path<K>(ksrc + jb.a, jb.na, ksrc + jb.b, jb.nb, d);
        if ((tid & 31) == 0) s_cut[w] = cut;
      }
      if ((tid & 31) == 0) s_found[w] = live ? 1 : 0;
    }
    __syncthreads();
  }
  if (tid == 0) {
    const uint64_t total = job_mode ? 0 : *total_ptr;
    uint32_t na = 0, nb = 0;
    TileSplit t{};
    const bool live = job_mode ? (s_found[0] && s_found[1]) : (tile < total && !poisoned(err));
    if (live) {
      uint64_t a_hi, b_hi;
      if (job_mode) {                                   // thread 0 holds warp 0's job
        const uint64_t d1 = umin(jb.d0 + (uint64_t)L::T, jb.na + jb.nb);
        t = TileSplit{jb.a + s_cut[0], jb.b + (jb.d0 - s_cut[0]), jb.out + jb.d0, 0, 0, 0};
        a_hi = jb.a + s_cut[1];
        b_hi = jb.b + (d1 - s_cut[1]);
      } else {
        t = split[tile];
        bool same = false;
        TileSplit nx{};
        if (tile + 1 < total) {
          nx = split[tile + 1];
          same = nx.pair == t.pair;
        }
        a_hi = same ? nx.a : t.a_end;
        b_hi = same ? nx.b : t.b_end;
      }
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
  // Staged over the (now free) input buffers, shifted so that the tile's
  // 16-byte-aligned body leaves by bulk store (cnt + pad <= T + 3 items).
  K* s_kout = s_kin + stage_pad(kdst + s_out);
  uint32_t* s_vout = VALS ? s_vin + stage_pad(vdst + s_out) : nullptr;
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
  fence_proxy_async_smem();                             // the staging is read by the bulk copy engine
  __syncthreads();
  store_tile_bulk<K, NT>(kdst + s_out, s_kout, cnt);
  if (VALS) store_tile_bulk<uint32_t, NT>(vdst + s_out, s_vout, cnt);
  if (tid == 0) {
    bulk_commit();
    bulk_wait_read();
  }
}

// ---------------------------------------------------------------------------
// Four-way merge round: two levels of the Fig. 2 tree in one pass over HBM.
// A quad is four adjacent lists L0..L3 (A, B, C, D, in stable order) that
// merge into X = merge(A, B), Y = merge(C, D), then merge(X, Y); ties go to
// the earlier list, so the output is the stable four-way merge, ordered by
// (key, list, position).
//
// Tiles with exact co-ranks.  The key index holds the keys at the global
// positions 64 e of the round's input, so list j's index entries I_j are the
// keys at its local positions o_j + 64 k (o_j < 64), and a quad's entries are
// contiguous.  A small pairwise round over the index merges I_0 with I_1 into
// X' and I_2 with I_3 into Y'; merging X' and Y' would order every index
// sample of the quad by (key, list, position).  A tile boundary sits just
// before the sample s at every Q-th position q of that order.  Let kappa_j be
// the number of list-j samples before s and v its key: the boundary's co-rank
// in s's own list is s's position o + 64 kappa, in an earlier list the number
// of keys <= v, in a later one the number of keys < v.  The samples fix each
// of those to a window of at most 64 positions, (o_j + 64 kappa_j - 64,
// o_j + 64 kappa_j], finished by a short bisection of the keys.  Summing over
// the lists, a boundary's output rank lies in [sum_j o_j + 64 q - 189,
// sum_j o_j + 64 q], so a tile between two boundaries Q samples apart holds
// 64 Q - 189 to 64 Q + 189 outputs, and the first and last tiles of a quad at
// most 64 Q + 252 (tests/test_corank4.py checks all of it by brute force).
// ---------------------------------------------------------------------------

struct Quad {                 // four adjacent lists in stable order -> [out, out + sum n)
  uint64_t s[4];              // first element of each list (global position in the round's input)
  uint64_t n[4];              // list lengths
  uint64_t out;
};

// A tile boundary: the four lists' first positions (global) and the output
// position they start at, and the quad they belong to.
struct Split4 {
  uint64_t p[4];
  uint64_t out;
  uint64_t quad;
};

// The largest tile the boundaries can make for Q samples per tile: 64 Q + 4 x 63.
constexpr uint32_t merge4_max_tile(uint32_t Q) { return 64u * Q + 4u * 63u; }

__device__ __forceinline__ uint64_t idx_entry(uint64_t pos) { return (pos + kIdxStride - 1) / kIdxStride; }

// Describes quad p (lists [b[i], b[i+1]), output at b[0]) for the round: the
// quad, its tile count ceil(M / Q) for its M index samples (0 for an empty
// quad, 1 for a non-empty quad with no sample), and the two pairs of the
// index-sample merge, slots 2p (I_0 + I_1 -> X') and 2p + 1 (I_2 + I_3 -> Y'),
// in index-entry coordinates, with their tile counts at merge tile `mtile`.
__device__ __forceinline__ void put_quad4(Quad* quads, uint64_t* tcount4, Pair* spairs, uint64_t* stcount,
                                          uint64_t p, const uint64_t b[5], uint32_t Q, uint32_t mtile) {
  Quad q;
  uint64_t E[5];
  for (int i = 0; i < 5; ++i) E[i] = idx_entry(b[i]);
  for (int i = 0; i < 4; ++i) {
    q.s[i] = b[i];
    q.n[i] = b[i + 1] - b[i];
  }
  q.out = b[0];
  quads[p] = q;
  const uint64_t M = E[4] - E[0];
  tcount4[p] = b[4] == b[0] ? 0 : (M == 0 ? 1 : (M + Q - 1) / Q);
  spairs[2 * p] = Pair{E[0], E[1] - E[0], E[1], E[2] - E[1], E[0]};
  spairs[2 * p + 1] = Pair{E[2], E[3] - E[2], E[3], E[4] - E[3], E[2]};
  stcount[2 * p] = (E[2] - E[0] + mtile - 1) / mtile;
  stcount[2 * p + 1] = (E[4] - E[2] + mtile - 1) / mtile;
}

// Run formation: blocks [j 4w + i w, j 4w + (i+1) w) of every run, i = 0..3.
static __global__ void k_quads4_runs(Quad* quads, uint64_t* tcount4, Pair* spairs, uint64_t* stcount,
                                     const uint64_t* __restrict__ run_off, uint32_t R, uint64_t w, uint64_t cmax,
                                     uint32_t Q, uint32_t mtile) {
  pdl_enter();
  uint64_t p = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (p >= (uint64_t)R * cmax) return;
  const uint64_t r = p / cmax, j = p % cmax;
  const uint64_t rs = run_off[r], re = run_off[r + 1];
  uint64_t b[5];
  for (int i = 0; i < 5; ++i) b[i] = umin(rs + j * 4 * w + i * w, re);
  put_quad4(quads, tcount4, spairs, stcount, p, b, Q, mtile);
}

// Bucket merge: groups of `step` segments; group g of a bucket starts at
// segment 4 g step (slot = global segment index q0 + t; other slots empty).
static __global__ void k_quads4_buckets(Quad* quads, uint64_t* tcount4, Pair* spairs, uint64_t* stcount, Geo g,
                                        const uint64_t* __restrict__ off, uint64_t q0, uint64_t Qg, uint32_t step,
                                        uint32_t Q, uint32_t mtile) {
  pdl_enter();
  const uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (t >= Qg) return;
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
  put_quad4(quads, tcount4, spairs, stcount, t, b, Q, mtile);
}

// One thread per tile: the tile's first boundary.  Tile j of a quad starts
// just before the sample at position j Q of the quad's sample order (j = 0:
// the quad's start).  kidx: the index of the round's input; xs: X' and Y' at
// the quad's index entries [E_0, E_2) and [E_2, E_4).
template <typename K>
__global__ void k_corank4(const K* __restrict__ src, const K* __restrict__ kidx, const K* __restrict__ xs,
                          const Quad* __restrict__ quads, const uint64_t* __restrict__ tbegin4, uint64_t nquads,
                          Split4* splits, uint64_t cap, uint32_t Q, uint32_t* err) {
  pdl_enter();
  if (poisoned(err)) return;
  const uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  const uint64_t total = tbegin4[nquads];
  if (t == 0 && total > cap) atomicOr(err, kErrBadTile);   // more tiles than the grid and buffer hold
  if (t >= total || t >= cap) return;
  const uint64_t guess = (uint64_t)(((unsigned __int128)t * nquads) / total);
  const uint64_t qi = last_le_from(tbegin4, nquads, t, guess);
  const Quad q = quads[qi];
  const uint64_t j = t - tbegin4[qi];
  Split4 sp;
  sp.quad = qi;
  uint64_t c[4] = {0, 0, 0, 0};
  if (j > 0) {
    uint64_t E[5], m[4], o[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) E[i] = idx_entry(q.s[i]);
    E[4] = idx_entry(q.s[3] + q.n[3]);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      m[i] = E[i + 1] - E[i];
      o[i] = E[i] * kIdxStride - q.s[i];
    }
    const uint64_t qpos = j * (uint64_t)Q;                 // < E[4] - E[0] by the tile count
    const K* X = xs + E[0];
    const K* Y = xs + E[2];
    const uint64_t nx = E[2] - E[0], ny = E[4] - E[2];
    const uint64_t x = merge_path<K, uint64_t>(X, nx, Y, ny, qpos);
    const uint64_t y = qpos - x;
    const K* I0 = kidx + E[0];
    const K* I1 = kidx + E[1];
    const K* I2 = kidx + E[2];
    const K* I3 = kidx + E[3];
    const uint64_t a = merge_path<K, uint64_t>(I0, m[0], I1, m[1], x);
    const uint64_t cc = merge_path<K, uint64_t>(I2, m[2], I3, m[3], y);
    const uint64_t kap[4] = {a, x - a, cc, y - cc};
    // The sample at position qpos: X'[x] or Y'[y], and the list it came from.
    const bool from_x = x < nx && (y >= ny || X[x] <= Y[y]);
    int own;
    K v;
    if (from_x) {
      v = X[x];
      own = (a < m[0] && (x - a >= m[1] || I0[a] <= I1[x - a])) ? 0 : 1;
    } else {
      v = Y[y];
      own = (cc < m[2] && (y - cc >= m[3] || I2[cc] <= I3[y - cc])) ? 2 : 3;
    }
    // Co-ranks: exact in s's own list; a bisection of a window of <= 64 keys
    // in the others (all three in lockstep, so their loads overlap).
    uint64_t lo[4], hi[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      if (i == own) {
        lo[i] = hi[i] = o[i] + kIdxStride * kap[i];
      } else {
        lo[i] = kap[i] ? o[i] + kIdxStride * (kap[i] - 1) + 1 : 0;
        hi[i] = kap[i] < m[i] ? o[i] + kIdxStride * kap[i] : q.n[i];
      }
    }
#pragma unroll 1
    for (int it = 0; it < 7; ++it) {                       // windows of <= 64 keys: 7 halvings end them
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        if (lo[i] < hi[i]) {
          const uint64_t mid = (lo[i] + hi[i]) >> 1;
          const K kv = src[q.s[i] + mid];
          const bool before = i < own ? (kv <= v) : (kv < v);
          if (before) lo[i] = mid + 1; else hi[i] = mid;
        }
      }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) c[i] = lo[i];
  }
  uint64_t sum = 0;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    sp.p[i] = q.s[i] + c[i];
    sum += c[i];
  }
  sp.out = q.out + sum;
  splits[t] = sp;
}

template <typename K, bool VALS, int NT, int VT>
struct Merge4Layout {
  static constexpr int C = NT * VT;                                   // outputs per tile at most
  static constexpr size_t kin = 16;                                   // after the mbarrier
  // Four pieces, each widened by up to 15 bytes on either side, plus the key
  // one slot past the last piece that a serial merge may read.
  static constexpr size_t vin = kin + (size_t)C * sizeof(K) + 4 * 32 + 16;
  static constexpr size_t bytes = vin + (VALS ? (size_t)C * 4 + 4 * 32 + 16 : 0);
  static_assert(C % 4 == 0, "16-byte aligned staging");
};

// One CTA per tile of a four-way round: the tile's four pieces arrive by bulk
// copy; every thread merges VT outputs of [X | Y] (level 1: A with B, C with
// D) into registers, the CTA writes X and Y compactly over its input staging,
// every thread merges VT outputs of merge(X, Y) (level 2), and the tile is
// staged once more in place and leaves with 16-byte stores.  A thread whose
// level-1 outputs straddle the end of X switches from the (A, B) merge to the
// (C, D) merge in mid-loop.
// CTAs per SM the four-way tile is compiled for (with 8-byte keys and
// payloads the compiler's own choice of registers would hold 128 x 17 to 5).
template <typename K, bool VALS>
constexpr int merge4_min_blocks() { return Merge4Shape<(int)sizeof(K)>::MIN_BLOCKS; }

template <typename K, bool VALS, int NT, int VT>
__global__ void __launch_bounds__(NT, (merge4_min_blocks<K, VALS>()))
k_merge4(const K* __restrict__ ksrc, const uint32_t* __restrict__ vsrc, K* __restrict__ kdst,
         uint32_t* __restrict__ vdst, const Split4* __restrict__ splits, const Quad* __restrict__ quads,
         const uint64_t* __restrict__ total_ptr, uint64_t cap, int f32_out, uint32_t* err, K* __restrict__ kidx,
         uint64_t wait_ns, int inject_timeout) {
  pdl_enter();
  using L = Merge4Layout<K, VALS, NT, VT>;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);
  K* sk = reinterpret_cast<K*>(smem_raw + L::kin);
  uint32_t* sv = reinterpret_cast<uint32_t*>(smem_raw + L::vin);
  __shared__ int s_n[4], s_ko[4], s_vo[4];                // piece lengths; element offsets in sk and sv
  __shared__ uint64_t s_out;
  const uint64_t tile = blockIdx.x;
  const int tid = threadIdx.x;
  if (tid == 0) {
    const uint64_t total = umin(*total_ptr, cap);
    int n[4] = {0, 0, 0, 0};
    uint64_t p0[4] = {0, 0, 0, 0};
    if (tile < total && !poisoned(err)) {
      const Split4 lo = splits[tile];
      uint64_t p1[4];
      if (tile + 1 < total && splits[tile + 1].quad == lo.quad) {
        const Split4 hi = splits[tile + 1];
        for (int i = 0; i < 4; ++i) p1[i] = hi.p[i];
      } else {
        const Quad q = quads[lo.quad];
        for (int i = 0; i < 4; ++i) p1[i] = q.s[i] + q.n[i];
      }
      uint64_t sum = 0;
      bool bad = false;
      for (int i = 0; i < 4; ++i) {
        bad = bad || p1[i] < lo.p[i];
        sum += p1[i] - lo.p[i];
      }
      if (bad || sum > (uint64_t)L::C) {
        atomicOr(err, kErrBadTile);                     // inconsistent boundaries: skip, never copy
      } else {
        for (int i = 0; i < 4; ++i) {
          p0[i] = lo.p[i];
          n[i] = (int)(p1[i] - lo.p[i]);
        }
        s_out = lo.out;
      }
    }
    uint32_t kbytes = 0, vbytes = 0;
    Span16 ks[4], vs[4];
    for (int i = 0; i < 4; ++i) {
      ks[i] = widen16(ksrc + p0[i], (uint32_t)n[i]);
      s_ko[i] = (int)((kbytes / sizeof(K)) + ks[i].skip);
      kbytes += ks[i].bytes;
      if (VALS) {
        vs[i] = widen16(vsrc + p0[i], (uint32_t)n[i]);
        s_vo[i] = (int)(vbytes / 4 + vs[i].skip);
        vbytes += vs[i].bytes;
      }
      s_n[i] = n[i];
    }
    if (n[0] + n[1] + n[2] + n[3] > 0) {
      mbar_init(bar, 1);
      fence_barrier_init();
      mbar_arrive_expect_tx(bar, kbytes + vbytes);
      // Fault injection (testing only): tile 0 announces its bytes but issues
      // no copy, so nothing is in flight and its wait runs out.
      if (!(inject_timeout && tile == 0)) {
        uint32_t ko = 0, vo = 0;
        for (int i = 0; i < 4; ++i) {
          if (ks[i].bytes) bulk_load(reinterpret_cast<char*>(sk) + ko, ks[i].base, ks[i].bytes, bar);
          ko += ks[i].bytes;
          if (VALS) {
            if (vs[i].bytes) bulk_load(reinterpret_cast<char*>(sv) + vo, vs[i].base, vs[i].bytes, bar);
            vo += vs[i].bytes;
          }
        }
      }
    }
  }
  __syncthreads();
  const int na = s_n[0], nb = s_n[1], nc = s_n[2], nd = s_n[3];
  const int nx = na + nb, cnt = nx + nc + nd;
  if (cnt == 0) return;                                 // tile beyond the round's total, or skipped
  if (!mbar_wait(bar, 0, wait_ns)) {                    // gave up: flag it, let copies in flight land, leave
    if (tid == 0) atomicOr(err, kErrWaitTimeout);
    mbar_wait(bar, 0, wait_ns);
    return;
  }
  const int d0 = min(tid * VT, cnt);
  const int mine = min(VT, cnt - d0);
  K ok[VT];
  uint32_t ov[VT];
  // Level 1: outputs [d0, d0 + mine) of [X | Y].  The merge state indexes the
  // staged keys; dva / dvb map a key slot of the current A / B piece to its
  // payload slot.  A read one slot past a piece lands in the next piece or the
  // slack after the last one; the index tests decide, never that key.
  {
    const int cx = max(0, min(mine, nx - d0));          // outputs taken from X
    int ai, a_end, bi, b_end, dva, dvb;
    auto start = [&](int pa, int la, int pb, int lb, int diag, int via, int vib) {
      const int s = merge_path<K, int>(sk + pa, la, sk + pb, lb, diag);
      ai = pa + s;
      a_end = pa + la;
      bi = pb + (diag - s);
      b_end = pb + lb;
      dva = via - pa;
      dvb = vib - pb;
    };
    if (cx > 0) start(s_ko[0], na, s_ko[1], nb, d0, s_vo[0], s_vo[1]);
    else start(s_ko[2], nc, s_ko[3], nd, d0 - nx, s_vo[2], s_vo[3]);
    K ak = sk[ai];
    K bk = sk[bi];
#pragma unroll
    for (int j = 0; j < VT; ++j) {
      if (j < mine) {
        if (j == cx && j > 0) {                         // this thread's outputs cross from X into Y
          start(s_ko[2], nc, s_ko[3], nd, 0, s_vo[2], s_vo[3]);
          ak = sk[ai];
          bk = sk[bi];
        }
        const bool take_b = (bi < b_end) && ((ai >= a_end) || (bk < ak));
        ok[j] = take_b ? bk : ak;
        if (VALS) ov[j] = sv[take_b ? bi + dvb : ai + dva];
        if (take_b) ++bi; else ++ai;
        const K nx_key = sk[take_b ? bi : ai];
        if (take_b) bk = nx_key; else ak = nx_key;
      }
    }
  }
  __syncthreads();                                      // every thread is done reading the pieces
#pragma unroll
  for (int j = 0; j < VT; ++j) {
    if (j < mine) {
      sk[d0 + j] = ok[j];
      if (VALS) sv[d0 + j] = ov[j];
    }
  }
  __syncthreads();
  // Level 2: outputs [d0, d0 + mine) of merge(X, Y); X = sk[0, nx), Y = sk[nx, cnt).
  {
    const int s = merge_path<K, int>(sk, nx, sk + nx, cnt - nx, d0);
    int ai = s, bi = nx + (d0 - s);
    K ak = sk[ai];
    K bk = sk[bi];
#pragma unroll
    for (int j = 0; j < VT; ++j) {
      if (j < mine) {
        const bool take_b = (bi < cnt) && ((ai >= nx) || (bk < ak));
        ok[j] = take_b ? bk : ak;
        if (VALS) ov[j] = sv[take_b ? bi : ai];
        if (take_b) ++bi; else ++ai;
        const K nx_key = sk[take_b ? bi : ai];
        if (take_b) bk = nx_key; else ak = nx_key;
      }
    }
  }
  __syncthreads();
  K* ko = sk + stage_pad(kdst + s_out);                 // staging shifted for the bulk store
  uint32_t* vo = VALS ? sv + stage_pad(vdst + s_out) : nullptr;
#pragma unroll
  for (int j = 0; j < VT; ++j) {
    if (j < mine) {
      ko[d0 + j] = from_order<K>(ok[j], f32_out);
      if (VALS) vo[d0 + j] = ov[j];
    }
  }
  static_assert(VT < kIdxStride, "at most one index entry per thread");
  if (kidx) {
    const int j0 = (int)((0u - (uint32_t)s_out - (uint32_t)d0) & (uint32_t)(kIdxStride - 1));
    if (j0 < mine) kidx[(s_out + (uint64_t)(d0 + j0)) / kIdxStride] = ko[d0 + j0];   // no index on the last pass
  }
  fence_proxy_async_smem();
  __syncthreads();
  store_tile_bulk<K, NT>(kdst + s_out, ko, cnt);
  if (VALS) store_tile_bulk<uint32_t, NT>(vdst + s_out, vo, cnt);
  if (tid == 0) {
    bulk_commit();
    bulk_wait_read();
  }
}

// ---------------------------------------------------------------------------
// Device-wide exclusive scan of uint64 (reduce, scan of chunk sums, scan).
// out[i] = sum_{j<i} in[j] for i in [0, m]; out[m] is the total.
// ---------------------------------------------------------------------------

static __global__ void __launch_bounds__(kScanNT)
k_scan_reduce(const uint64_t* __restrict__ in, uint64_t m, uint64_t* __restrict__ sums) {
  pdl_enter();
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
  pdl_enter();
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
  pdl_enter();
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
  pdl_enter();
  uint64_t r = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (r >= g.R) return;
  counts[r] = umin(g.s[g.run_inst[r]], g.run_off[r + 1] - g.run_off[r]);
}

template <typename K>
__global__ void k_sample(const K* __restrict__ runs, Geo g, const uint64_t* __restrict__ samp_off,
                         K* __restrict__ samples, uint64_t S) {
  pdl_enter();
  uint64_t j = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (j >= S) return;
  const uint32_t r = last_le<uint64_t>(samp_off, g.R, j);
  const uint64_t i = j - samp_off[r], sr = samp_off[r + 1] - samp_off[r];
  const uint64_t rs = g.run_off[r], nr = g.run_off[r + 1] - rs;
  const uint64_t pos = (uint64_t)(((unsigned __int128)(i + 1) * nr) / sr) - 1;   // exact for any s_r, n_r
  samples[j] = runs[rs + pos];
}

// Step 2 of a single sort in one launch.  Run r gives min(s, n_r) samples,
// and its length n_r is floor(n / P) or ceil(n / P): with s < ceil(n / P)
// every run gives s (s <= floor(n / P)) and its samples start at r s; with
// s >= ceil(n / P) every key is a sample and they start at run_off[r].  The
// positions are k_sample's.  Thread j < S writes sample j, thread r <= R
// writes samp_off[r].
template <typename K>
__global__ void k_sample_single(const K* __restrict__ runs, const uint64_t* __restrict__ run_off, uint32_t R,
                                uint64_t s, bool all_keys, uint64_t* __restrict__ samp_off, K* __restrict__ samples,
                                uint64_t S) {
  pdl_enter();
  const uint64_t j = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (j <= R) samp_off[j] = all_keys ? run_off[j] : j * s;
  if (j >= S) return;
  if (all_keys) {
    samples[j] = runs[j];
    return;
  }
  const uint64_t r = j / s, i = j % s;
  const uint64_t rs = run_off[r], nr = run_off[r + 1] - rs;
  const uint64_t pos = (uint64_t)(((unsigned __int128)(i + 1) * nr) / s) - 1;
  samples[j] = runs[rs + pos];
}

// Step 3's pick on one sorted sample of m keys: out[b-1] = sorted[floor(b m / P) - 1], b = 1..P-1.
template <typename K>
__global__ void k_pick_splitters_flat(const K* __restrict__ sorted, uint64_t m, uint32_t P, K* out, int f32) {
  pdl_enter();
  uint64_t b = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x + 1;
  if (b >= P) return;
  out[b - 1] = from_order<K>(sorted[(b * m) / P - 1], f32);
}

// ---------------------------------------------------------------------------
// K5: cut search + investigator (step 4 of Section IV, Section IV-B).
// ---------------------------------------------------------------------------

// lb[r][b] = #{x in run r : x < t_b}, cnt[r][b] = #{x in run r : x == t_b},
// b = 1..P-1, for every run of every instance; index space: the P x P
// segments, one warp or one thread each (two searches).  Step 3's pick
// is fused in: every warp reads its t_b from the sorted sample, and run 0's
// warps store it (and the caller's copy of a single sort's splitters).  The
// slots b = 0 write run r's fixed cuts cut[r][0] = 0 and cut[r][P] = n_r, and
// run 0's also e[0] = 0 and e[P] = n_i.  t is indexed by global run (slot b
// of instance i is R0[i] + b; slot 0 unused).
// The first index in [lo, hi) whose test fails (test true on a prefix), by
// one thread's bisection.
template <typename Test>
__device__ __forceinline__ uint64_t partition_point(uint64_t lo, uint64_t hi, const Test& test) {
  while (lo < hi) {
    const uint64_t mid = (lo + hi) >> 1;
    if (test(mid)) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// WARP: one warp per slot with warp_partition_point (few slots: the searches'
// dependent loads bound the time); else one thread per slot with bisection
// (many slots: a warp's 32 searches share its load instructions).
template <typename K, bool WARP>
__global__ void k_cut_search(const K* __restrict__ runs, Geo g, uint64_t Q, const K* __restrict__ sorted,
                             const uint64_t* __restrict__ samp_off, K* t, K* user_out, int f32, uint64_t* lb,
                             uint64_t* cnt, uint64_t* cut, uint64_t* e) {
  pdl_enter();
  const uint64_t gt = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  const uint64_t q = WARP ? gt >> 5 : gt;
  if (q >= Q) return;
  const bool lead = WARP ? (threadIdx.x & 31u) == 0 : true;
  const uint32_t i = last_le<uint64_t>(g.seg, g.I, q);
  const uint64_t P = g.P[i];
  const uint64_t local = q - g.seg[i];
  const uint64_t rl = local / P, b = local % P;
  const uint32_t r0 = g.R0[i];
  const uint64_t rs = g.run_off[r0 + rl], nr = g.run_off[r0 + rl + 1] - rs;
  if (b == 0) {                                       // the fixed cuts of run rl: 0 and n_r
    if (lead) {
      uint64_t* row = cut + g.mat[i] + rl * (P + 1);
      row[0] = 0;
      row[P] = nr;
      if (rl == 0) {
        e[r0 + i] = 0;
        e[r0 + i + P] = g.koff[i + 1] - g.koff[i];
      }
    }
    return;
  }
  // Step 3's pick: t_b = the sorted sample at floor(b S / P) - 1.
  const uint64_t s0 = samp_off[r0], S = samp_off[r0 + P] - s0;
  const K v = sorted[s0 + (b * S) / P - 1];
  if (rl == 0 && lead) {
    t[r0 + b] = v;
    if (user_out && g.I == 1) user_out[b - 1] = from_order<K>(v, f32);
  }
  const K* x = runs + rs;
  auto below = [&](uint64_t m) { return x[m] < v; };
  auto not_above = [&](uint64_t m) { return x[m] <= v; };
  const uint64_t l = WARP ? warp_partition_point(0, nr, below) : partition_point(0, nr, below);
  const uint64_t u = WARP ? warp_partition_point(l, nr, not_above) : partition_point(l, nr, not_above);
  if (lead) {
    const uint64_t at = g.mat[i] + rl * (P + 1) + b;
    lb[at] = l;
    cnt[at] = u - l;
  }
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
  pdl_enter();
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
  pdl_enter();
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
__device__ __forceinline__ uint64_t segment_size(const Geo& g, uint64_t q, const uint64_t* __restrict__ cut,
                                                 uint64_t* src) {
  const uint32_t i = last_le<uint64_t>(g.seg, g.I, q);
  const uint64_t P = g.P[i];
  const uint64_t local = q - g.seg[i];
  const uint64_t b = local / P, rl = local % P;
  const uint64_t* c = cut + g.mat[i] + rl * (P + 1);
  if (src) src[q] = g.run_off[g.R0[i] + rl] + c[b];
  return c[b + 1] - c[b];
}

static __global__ void k_bucket_sizes(Geo g, uint64_t Q, const uint64_t* __restrict__ cut, uint64_t* sizes,
                                      uint64_t* src) {
  pdl_enter();
  uint64_t q = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (q >= Q) return;
  sizes[q] = segment_size(g, q, cut, src);
}

// The same sizes and their exclusive scan (the receive offsets, off[Q] = n)
// in one CTA, for at most kSizesMax segments (beyond, the CTA's dependent
// loads cost more than a second launch: 47 us for 16384 segments).  With
// pp.rounds > 0 (a single sort whose bucket rounds are all small) the kernel
// also plans every round of step 6 as k_plan_jobs would, one CTA per round:
// CTA r recomputes the offsets (CTA 0 stores them), keeps its copy in
// pp.offs + r (Q + 1) and plans round r (step 2^r; round 0 fused with the
// exchange unless pp.scatter) into pp.jobs + r pp.stride and pp.tbegin +
// r (Q + 1), with its own pair scratch, so those rounds need no planning
// launch and no CTA waits for another.
constexpr int kSizesNT = 1024, kSizesVT = 4;
constexpr uint64_t kSizesMax = (uint64_t)kSizesNT * kSizesVT;
static_assert(kSizesNT == kPlanNT, "the offsets CTAs also plan rounds");

struct PrePlan {
  Pair* pairs; uint64_t* tcount; uint64_t* tbegin; TileJob* jobs; uint64_t* offs;
  uint64_t stride; uint32_t rounds, tile; int scatter;
};

static __global__ void __launch_bounds__(kSizesNT)
k_bucket_offsets(Geo g, uint64_t Q, const uint64_t* __restrict__ cut, uint64_t* sizes, uint64_t* src,
                 uint64_t* off, PrePlan pp, uint32_t* err) {
  pdl_enter();
  __shared__ int s_skip;
  const uint32_t r = blockIdx.x;
  const bool store = r == 0;
  const uint64_t q0 = (uint64_t)threadIdx.x * kSizesVT;   // blocked: thread t owns [t VT, t VT + VT)
  uint64_t v[kSizesVT];
  uint64_t acc = 0;
#pragma unroll
  for (int k = 0; k < kSizesVT; ++k) {
    v[k] = q0 + k < Q ? segment_size(g, q0 + k, cut, store ? src : nullptr) : 0;
    acc += v[k];
  }
  uint64_t total;
  uint64_t pre = block_exclusive_scan(acc, &total);
  uint64_t* my_off = r == 0 ? off : pp.offs + (uint64_t)r * (Q + 1);
#pragma unroll
  for (int k = 0; k < kSizesVT; ++k) {
    if (q0 + k < Q) {
      if (store) sizes[q0 + k] = v[k];
      my_off[q0 + k] = pre;
    }
    pre += v[k];
  }
  if (threadIdx.x == 0) {
    my_off[Q] = total;
    s_skip = poisoned(err);                           // one decision for the whole CTA
  }
  if (pp.rounds == 0) return;
  __syncthreads();                                    // the offsets (and src) are visible to the CTA
  if (s_skip) return;                                 // a kernel failed: no plan (its merges leave)
  Pair* pairs = pp.pairs + (uint64_t)r * Q;
  uint64_t* tcount = pp.tcount + (uint64_t)r * Q;
  uint64_t* tb = pp.tbegin + (uint64_t)r * (Q + 1);
  TileJob* jobs = pp.jobs + (uint64_t)r * pp.stride;
  const uint64_t cap = umin(pp.stride, kPlanMaxTiles);
  if (r == 0 && !pp.scatter)
    plan_round(GenFused{pairs, tcount, g, my_off, src, 0, pp.tile}, pairs, tcount, tb, Q, jobs, cap, pp.tile, err);
  else
    plan_round(GenBucketLists{pairs, tcount, g, my_off, 0, 1u << r, pp.tile}, pairs, tcount, tb, Q, jobs, cap,
               pp.tile, err);
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
  pdl_enter();
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
          const uint64_t* __restrict__ first_seg, uint64_t n, uint64_t Q, int f32_out, const uint32_t* err,
          K* __restrict__ kidx) {
  pdl_enter();
  if (cta_poisoned(err)) return;
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
  if (kidx) {                                        // order-form keys, before any conversion
    write_key_index(kidx, sm.keys, o, cnt);
    __syncthreads();
  }
  for (int p = threadIdx.x; p < cnt; p += blockDim.x) sm.keys[p] = from_order<K>(sm.keys[p], f32_out);
  __syncthreads();
  store_tile_vec<K, kScatterNT>(kdst + o, sm.keys, cnt);
  if (VALS) store_tile_vec<uint32_t, kScatterNT>(vdst + o, sm.vals, cnt);
}

// Pseudo-random keys (splitmix64 of the position and a seed) and index
// payloads, for timing runs of the tuner.
template <typename K>
__global__ void k_fill_random(K* keys, uint32_t* vals, uint64_t n, uint64_t seed) {
  pdl_enter();
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
  pdl_enter();
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
