// Device code of the GB300 load-balanced sample sort (arXiv 1611.00463, Section IV).
//
// Keys travel through the pipeline as unsigned integers in "order form": integer
// keys as they are, float32 keys as their IEEE 754 totalOrder image (the first
// kernel converts, the last one converts back).  Payloads are uint32.  Arrays
// are structure-of-arrays in HBM: keys[n] and vals[n].
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace pgs {

constexpr int kNT = 256;             // threads per CTA of the sort and merge kernels
constexpr int kVT = 17;              // items per thread; odd, so blocked smem access is conflict free
constexpr int kTile = kNT * kVT;     // 4352 keys per block-sort tile and per merge tile
constexpr int kScanNT = 1024;
constexpr int kScanVT = 8;
constexpr int kScanChunk = kScanNT * kScanVT;
constexpr int kScatterNT = 256;
constexpr int kScatterVT = 16;
constexpr int kScatterTile = kScatterNT * kScatterVT;
constexpr int kScatterWindow = 1024;  // bucket segments staged per scatter CTA

struct Pair {                         // one pairwise merge: [lo, mid) + [mid, hi) -> [lo, hi)
  uint64_t lo, mid, hi;
};

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

// Merge up to `count` items of two sorted ranges of one smem array, A = [ai, a_end)
// and B = [bi, b_end), into registers.  pos[] receives the smem index of each item.
template <typename K, int VT>
__device__ __forceinline__ void serial_merge(const K* s, int ai, int a_end, int bi, int b_end,
                                             int count, K (&key)[VT], int (&pos)[VT]) {
  K ak = ai < a_end ? s[ai] : key_max<K>();
  K bk = bi < b_end ? s[bi] : key_max<K>();
#pragma unroll
  for (int j = 0; j < VT; ++j) {
    if (j < count) {
      bool take_a = (bi >= b_end) || (ai < a_end && ak <= bk);
      key[j] = take_a ? ak : bk;
      pos[j] = take_a ? ai : bi;
      if (take_a) {
        ++ai;
        ak = ai < a_end ? s[ai] : key_max<K>();
      } else {
        ++bi;
        bk = bi < b_end ? s[bi] : key_max<K>();
      }
    }
  }
}

// ---------------------------------------------------------------------------
// K1: block sort.  One CTA sorts one tile of one run, stably.
// Step 1 of Section IV / Section IV-A: every thread sorts its own VT keys
// (odd-even transposition: only strictly smaller keys move left, so it is
// stable), then the sorted thread lists are merged pairwise in rounds, list
// 2i+1 into list 2i, exactly the balanced schedule of Fig. 2, in shared memory.
// ---------------------------------------------------------------------------

template <typename K>
struct BlockSortSmem {
  K keys[kTile];
  uint16_t ids[kTile];
  uint32_t vals[kTile];
};

template <typename K, bool VALS>
__global__ void __launch_bounds__(kNT)
k_block_sort(const K* __restrict__ kin, const uint32_t* __restrict__ vin, K* kout, uint32_t* vout,
             uint64_t n, uint32_t P, uint32_t tiles_per_run, int f32_in, int f32_out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  BlockSortSmem<K>& sm = *reinterpret_cast<BlockSortSmem<K>*>(smem_raw);
  const int tid = threadIdx.x;
  const uint64_t r = blockIdx.x / tiles_per_run;
  const uint64_t t = blockIdx.x % tiles_per_run;
  const uint64_t rs = run_start(r, n, P), re = run_start(r + 1, n, P);
  const uint64_t g0 = rs + t * kTile;
  if (g0 >= re) return;
  const int cnt = (int)umin(kTile, re - g0);

#pragma unroll
  for (int i = 0; i < kVT; ++i) {
    int idx = i * kNT + tid;
    sm.keys[idx] = idx < cnt ? to_order<K>(kin[g0 + idx], f32_in) : key_max<K>();
    if (VALS) sm.vals[idx] = idx < cnt ? vin[g0 + idx] : 0u;
  }
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
  // Pairwise merge rounds (Fig. 2): coop threads share one merged list.
  for (int coop = 2; coop <= kNT; coop *= 2) {
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kVT; ++j) {
      sm.keys[tid * kVT + j] = key[j];
      sm.ids[tid * kVT + j] = (uint16_t)pos[j];
    }
    __syncthreads();
    const int half = (coop / 2) * kVT;
    const int start = (tid & ~(coop - 1)) * kVT;
    const int diag = (tid & (coop - 1)) * kVT;
    const int a = merge_path<K, int>(sm.keys + start, half, sm.keys + start + half, half, diag);
    int spos[kVT];
    serial_merge<K, kVT>(sm.keys, start + a, start + half, start + half + (diag - a), start + 2 * half,
                         kVT, key, spos);
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

// Run formation: inside every run, blocks [j 2w, j 2w + w) and [j 2w + w, (j+1) 2w) merge.
static __global__ void k_pairs_runs(Pair* pairs, uint64_t* tcount, uint64_t n, uint32_t P, uint64_t w,
                             uint64_t pairs_per_run) {
  uint64_t p = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (p >= pairs_per_run * P) return;
  uint64_t r = p / pairs_per_run, j = p % pairs_per_run;
  uint64_t rs = run_start(r, n, P), re = run_start(r + 1, n, P);
  uint64_t lo = umin(rs + j * 2 * w, re);
  uint64_t mid = umin(lo + w, re);
  uint64_t hi = umin(lo + 2 * w, re);
  pairs[p] = Pair{lo, mid, hi};
  tcount[p] = (hi - lo + kTile - 1) / kTile;
}

// Lists given by an offset table: segment g has L lists, list i = [tbl[g*stride + i],
// tbl[g*stride + i + 1]).  Round `step` merges group [i, i+step) with [i+step, i+2 step).
static __global__ void k_pairs_lists(Pair* pairs, uint64_t* tcount, const uint64_t* tbl, uint64_t stride,
                              uint32_t segs, uint32_t L, uint32_t step, uint64_t pairs_per_seg) {
  uint64_t p = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (p >= pairs_per_seg * segs) return;
  uint64_t g = p / pairs_per_seg, j = p % pairs_per_seg;
  const uint64_t* o = tbl + g * stride;
  uint64_t i0 = j * 2ull * step;
  uint64_t lo = o[umin(i0, L)];
  uint64_t mid = o[umin(i0 + step, L)];
  uint64_t hi = o[umin(i0 + 2ull * step, L)];
  pairs[p] = Pair{lo, mid, hi};
  tcount[p] = (hi - lo + kTile - 1) / kTile;
}

// One thread per merge tile: find its pair, then the merge-path split at the
// tile's first output.  Splits are computed up front so every merge CTA starts
// with its two ranges known and moves equal output work.
template <typename K>
__global__ void k_partition(const K* __restrict__ src, const Pair* __restrict__ pairs,
                            const uint64_t* __restrict__ tbegin, uint64_t npairs,
                            uint32_t* tile_pair, uint64_t* part) {
  uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  uint64_t total = tbegin[npairs];
  if (i >= total) return;
  uint64_t lo = 0, hi = npairs;                     // last p with tbegin[p] <= i
  while (hi - lo > 1) {
    uint64_t mid = (lo + hi) >> 1;
    if (tbegin[mid] <= i) lo = mid; else hi = mid;
  }
  uint64_t p = lo;
  Pair pr = pairs[p];
  uint64_t diag = (i - tbegin[p]) * kTile;
  uint64_t na = pr.mid - pr.lo, nb = pr.hi - pr.mid;
  tile_pair[i] = (uint32_t)p;
  part[i] = merge_path<K, uint64_t>(src + pr.lo, na, src + pr.mid, nb, diag);
}

// ---------------------------------------------------------------------------
// K2/K8: merge-path merge.  Each CTA produces kTile outputs of one pair.
// ---------------------------------------------------------------------------

template <typename K>
struct MergeSmem {
  K keys[kTile];
  uint32_t vals[kTile];
};

template <typename K, bool VALS>
__global__ void __launch_bounds__(kNT)
k_merge(const K* __restrict__ ksrc, const uint32_t* __restrict__ vsrc, K* __restrict__ kdst,
        uint32_t* __restrict__ vdst, const Pair* __restrict__ pairs, const uint64_t* __restrict__ tbegin,
        uint64_t npairs, const uint32_t* __restrict__ tile_pair, const uint64_t* __restrict__ part,
        int f32_out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  MergeSmem<K>& sm = *reinterpret_cast<MergeSmem<K>*>(smem_raw);
  const uint64_t tile = blockIdx.x;
  if (tile >= tbegin[npairs]) return;
  const int tid = threadIdx.x;
  const uint32_t p = tile_pair[tile];
  const Pair pr = pairs[p];
  const uint64_t na_all = pr.mid - pr.lo, total = pr.hi - pr.lo;
  const uint64_t d0 = (tile - tbegin[p]) * kTile;
  const uint64_t d1 = umin(d0 + kTile, total);
  const uint64_t a0 = part[tile];
  const uint64_t a1 = (d1 == total) ? na_all : part[tile + 1];
  const int na = (int)(a1 - a0);
  const int cnt = (int)(d1 - d0);
  const K* ka = ksrc + pr.lo + a0;
  const K* kb = ksrc + pr.mid + (d0 - a0);
#pragma unroll
  for (int i = 0; i < kVT; ++i) {
    int idx = i * kNT + tid;
    if (idx < cnt) sm.keys[idx] = idx < na ? ka[idx] : kb[idx - na];
  }
  if (VALS) {
    const uint32_t* va = vsrc + pr.lo + a0;
    const uint32_t* vb = vsrc + pr.mid + (d0 - a0);
#pragma unroll
    for (int i = 0; i < kVT; ++i) {
      int idx = i * kNT + tid;
      if (idx < cnt) sm.vals[idx] = idx < na ? va[idx] : vb[idx - na];
    }
  }
  __syncthreads();
  const int diag = min(tid * kVT, cnt);
  const int a = merge_path<K, int>(sm.keys, na, sm.keys + na, cnt - na, diag);
  K key[kVT];
  int pos[kVT];
  const int mine = min(kVT, cnt - diag);
  serial_merge<K, kVT>(sm.keys, a, na, na + (diag - a), cnt, mine, key, pos);
  uint32_t val[kVT];
  if (VALS) {
#pragma unroll
    for (int j = 0; j < kVT; ++j)
      if (j < mine) val[j] = sm.vals[pos[j]];
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < kVT; ++j) {
    if (j < mine) {
      sm.keys[diag + j] = key[j];
      if (VALS) sm.vals[diag + j] = val[j];
    }
  }
  __syncthreads();
  K* ko = kdst + pr.lo + d0;
  uint32_t* vo = vdst + pr.lo + d0;
#pragma unroll
  for (int i = 0; i < kVT; ++i) {
    int idx = i * kNT + tid;
    if (idx < cnt) {
      ko[idx] = from_order<K>(sm.keys[idx], f32_out);
      if (VALS) vo[idx] = sm.vals[idx];
    }
  }
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
// K3: regular samples (step 2 of Section IV).
// Run r is cut into s_r = min(s, n_r) equal blocks; the last key of each block
// is sampled, local position floor((i+1) n_r / s_r) - 1.  Samples are written
// in (run, position) order, each run's samples sorted.
// ---------------------------------------------------------------------------

template <typename K>
__global__ void k_sample(const K* __restrict__ runs, uint64_t n, uint32_t P, uint64_t s,
                         int all, K* __restrict__ samples, uint64_t S) {
  uint64_t j = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (j >= S) return;
  if (all) {                        // s >= every run length: every key is a sample
    samples[j] = runs[j];
    return;
  }
  uint64_t r = j / s, i = j % s;
  uint64_t rs = run_start(r, n, P), nr = run_start(r + 1, n, P) - rs;
  uint64_t pos = (uint64_t)(((unsigned __int128)(i + 1) * nr) / s) - 1;   // exact for any s, n_r
  samples[j] = runs[rs + pos];
}

// Offsets of the per-run sample lists: r s, or the run starts when all keys are samples.
static __global__ void k_sample_offsets(uint64_t* off, uint64_t n, uint32_t P, uint64_t s, int all) {
  uint64_t r = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (r > P) return;
  off[r] = all ? run_start(r, n, P) : r * s;
}

// Step 3 of Section IV: t_b = sorted sample at index floor(b S / P) - 1, b = 1..P-1.
template <typename K>
__global__ void k_pick_splitters(const K* __restrict__ sorted, uint64_t S, uint32_t P, K* t,
                                 K* user_out, int f32) {
  uint64_t b = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x + 1;
  if (b >= P) return;
  K v = sorted[(b * S) / P - 1];
  t[b - 1] = v;
  if (user_out) user_out[b - 1] = from_order<K>(v, f32);
}

// ---------------------------------------------------------------------------
// K5: cut search + investigator (step 4 of Section IV, Section IV-B).
// ---------------------------------------------------------------------------

// lb[r][b] = #{x in run r : x < t_b}, cnt[r][b] = #{x in run r : x == t_b}; b = 1..P-1.
template <typename K>
__global__ void k_cut_search(const K* __restrict__ runs, uint64_t n, uint32_t P,
                             const K* __restrict__ t, uint64_t* lb, uint64_t* cnt) {
  uint64_t q = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  uint64_t Pm1 = P - 1;
  if (q >= (uint64_t)P * Pm1) return;
  uint64_t r = q / Pm1, b = q % Pm1 + 1;
  uint64_t rs = run_start(r, n, P), nr = run_start(r + 1, n, P) - rs;
  const K* x = runs + rs;
  K v = t[b - 1];
  uint64_t lo = 0, hi = nr;
  while (lo < hi) { uint64_t mid = (lo + hi) >> 1; if (x[mid] < v) lo = mid + 1; else hi = mid; }
  uint64_t l = lo;
  hi = nr;
  while (lo < hi) { uint64_t mid = (lo + hi) >> 1; if (x[mid] <= v) lo = mid + 1; else hi = mid; }
  lb[r * (P + 1) + b] = l;
  cnt[r * (P + 1) + b] = lo - l;
}

// One CTA per splitter b = 1..P-1.  L_b = sum_r lb, G_b = sum_r cnt,
// pre[r] = sum_{r'<r} cnt.  The variant picks e_b, then every run cuts
// cut[r][b] = lb + clamp(e_b - L_b - pre[r], 0, cnt): the keys equal to t_b
// are handed out in stable order (run, position) until e_b ranks are reached.
template <typename K>
__global__ void __launch_bounds__(256)
k_investigator(const uint64_t* __restrict__ lb, const uint64_t* __restrict__ cnt,
               const K* __restrict__ t, uint64_t n, uint32_t P, int variant,
               uint64_t* cut, uint64_t* e) {
  const uint64_t b = blockIdx.x + 1;
  const uint64_t W = P + 1;
  __shared__ uint64_t sh_L, sh_e;
  // L_b and G_b.
  uint64_t ls = 0, gs = 0;
  for (uint64_t r = threadIdx.x; r < P; r += blockDim.x) {
    ls += lb[r * W + b];
    gs += cnt[r * W + b];
  }
  uint64_t Lb, Gb;
  block_exclusive_scan(ls, &Lb);
  block_exclusive_scan(gs, &Gb);
  if (threadIdx.x == 0) {
    uint64_t target = (b * n) / P;
    uint64_t eb;
    if (variant == 0) {
      eb = umin(umax(target, Lb), Lb + Gb);
    } else if (variant == 2) {
      eb = Lb + Gb;
    } else {
      // Group of equal splitters containing t_b: [g0, g1) in splitter index (0-based).
      K v = t[b - 1];
      uint64_t lo = 0, hi = P - 1;
      while (lo < hi) { uint64_t m = (lo + hi) >> 1; if (t[m] < v) lo = m + 1; else hi = m; }
      uint64_t g0 = lo;
      hi = P - 1;
      while (lo < hi) { uint64_t m = (lo + hi) >> 1; if (t[m] <= v) lo = m + 1; else hi = m; }
      uint64_t k = lo - g0, i = (b - 1) - g0;
      eb = Lb + (Gb * (i + 1)) / k;
    }
    sh_L = Lb;
    sh_e = eb;
    e[b] = eb;
  }
  __syncthreads();
  const uint64_t L = sh_L, eb = sh_e;
  uint64_t carry = 0;
  for (uint64_t r0 = 0; r0 < P; r0 += blockDim.x) {
    uint64_t r = r0 + threadIdx.x;
    uint64_t c = r < P ? cnt[r * W + b] : 0;
    uint64_t chunk;
    uint64_t pre = block_exclusive_scan(c, &chunk) + carry;
    if (r < P) {
      uint64_t want = eb - L;                        // >= 0: L <= e_b in every variant
      uint64_t take = want > pre ? umin(want - pre, c) : 0;
      cut[r * W + b] = lb[r * W + b] + take;
    }
    carry += chunk;
  }
}

// cut[r][0] = 0, cut[r][P] = n_r, e[0] = 0, e[P] = n.
static __global__ void k_cut_edges(uint64_t* cut, uint64_t* e, uint64_t n, uint32_t P) {
  uint64_t r = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (r == 0) { e[0] = 0; e[P] = n; }
  if (r >= P) return;
  cut[r * (P + 1)] = 0;
  cut[r * (P + 1) + P] = run_start(r + 1, n, P) - run_start(r, n, P);
}

// Sizes of the P x P segments in bucket-major order: size[b P + r] = cut[r][b+1] - cut[r][b].
static __global__ void k_bucket_sizes(const uint64_t* __restrict__ cut, uint32_t P, uint64_t* sizes) {
  uint64_t q = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (q >= (uint64_t)P * P) return;
  uint64_t b = q / P, r = q % P;
  const uint64_t* c = cut + r * (P + 1);
  sizes[q] = c[b + 1] - c[b];
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
          uint32_t* __restrict__ vdst, const uint64_t* __restrict__ off, const uint64_t* __restrict__ cut,
          const uint64_t* __restrict__ first_seg, uint64_t n, uint32_t P, int f32_out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  ScatterSmem<K>& sm = *reinterpret_cast<ScatterSmem<K>*>(smem_raw);
  const uint64_t Q = (uint64_t)P * P;
  const uint64_t o = blockIdx.x * (uint64_t)kScatterTile;
  const int cnt = (int)umin(kScatterTile, n - o);
  const uint64_t q0 = first_seg[blockIdx.x];
  const int wn = (int)umin(kScatterWindow, Q - q0);
  for (int i = threadIdx.x; i <= wn; i += blockDim.x) sm.off[i] = off[q0 + i];
  for (int i = threadIdx.x; i < wn; i += blockDim.x) {
    uint64_t q = q0 + i, b = q / P, r = q % P;
    sm.src[i] = run_start(r, n, P) + cut[r * (P + 1) + b];
  }
  __syncthreads();
  // Warp w copies positions [o + w 32 VT, ...) 32 at a time; lane l walks its segment forward.
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int base = warp * 32 * kScatterVT;
  int p0 = base + lane;
  // Locate the first segment of this lane inside the staged window.
  int lo = 0, hi = wn;
  uint64_t gp = o + p0;
  while (hi - lo > 1) { int mid = (lo + hi) >> 1; if (sm.off[mid] <= gp) lo = mid; else hi = mid; }
  int q = lo;
  for (int k = 0; k < kScatterVT; ++k) {
    int p = base + k * 32 + lane;
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
      uint64_t b = glo / P, r = glo % P;
      s = run_start(r, n, P) + cut[r * (P + 1) + b] + (gp - off[glo]);
    }
    sm.keys[p] = ksrc[s];
    if (VALS) sm.vals[p] = vsrc[s];
  }
  __syncthreads();
  for (int p = threadIdx.x; p < cnt; p += blockDim.x) {
    kdst[o + p] = from_order<K>(sm.keys[p], f32_out);
    if (VALS) vdst[o + p] = sm.vals[p];
  }
}

// ---------------------------------------------------------------------------
// K9: load statistics (Table II: each processor's share after the sort).
// ---------------------------------------------------------------------------

struct DevStats {                     // layout of pgs_stats
  uint64_t n;
  uint32_t P, s;
  uint64_t max_bucket, min_bucket;
  uint32_t splitter_mode, fallback, error, passes;
  uint32_t launches, reserved;
};

static __global__ void __launch_bounds__(256)
k_stats(const uint64_t* __restrict__ e, uint64_t n, uint32_t P, uint32_t s, uint32_t mode,
        uint32_t passes, uint32_t launches, uint32_t* err_word, DevStats* st, uint64_t* user_bounds) {
  __shared__ uint64_t smax[256], smin[256];
  uint64_t mx = 0, mn = ~0ull;
  for (uint32_t b = threadIdx.x; b < P; b += blockDim.x) {
    uint64_t sz = e[b + 1] - e[b];
    mx = umax(mx, sz);
    mn = umin(mn, sz);
  }
  smax[threadIdx.x] = mx;
  smin[threadIdx.x] = mn;
  __syncthreads();
  for (int d = 128; d > 0; d >>= 1) {
    if (threadIdx.x < d) {
      smax[threadIdx.x] = umax(smax[threadIdx.x], smax[threadIdx.x + d]);
      smin[threadIdx.x] = umin(smin[threadIdx.x], smin[threadIdx.x + d]);
    }
    __syncthreads();
  }
  if (user_bounds)
    for (uint32_t b = threadIdx.x; b <= P; b += blockDim.x) user_bounds[b] = e[b];
  if (threadIdx.x == 0 && st) {
    st->n = n;
    st->P = P;
    st->s = s;
    st->max_bucket = smax[0];
    st->min_bucket = P ? smin[0] : 0;
    st->splitter_mode = mode;
    st->fallback = 0;
    st->error = err_word ? *err_word : 0;
    st->passes = passes;
    st->launches = launches;
    st->reserved = 0;
  }
}

}  // namespace pgs
