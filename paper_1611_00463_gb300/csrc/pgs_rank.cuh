// The sort of one global array spread over G ranks (processes, one GPU
// each), step by step as Section IV runs it on the paper's processors.  The
// library gives each rank its steps; the caller moves the data between them
// with its own collectives (an all-gather of samples, an all-gather of
// counts, an all-to-all of segments):
//   1. local sort of the rank's shard (pgs_sort_copy, any P);
//   2. regular samples of the sorted shard            (k_rank_samples);
//   3. splitters from all ranks' samples              (pgs_fit_splitters);
//   4. per-splitter counts in the sorted shard         (k_rank_counts), then,
//      from every rank's counts, the investigator's cut matrix and bucket
//      bounds, the same on every rank                  (run_rank_cuts);
//   5. the exchange: rank r sends its sorted positions [cut[r][b],
//      cut[r][b+1]) to rank b (the caller's all-to-all);
//   6. the merge of the G received sorted segments     (run_merge_lists).
#pragma once

#include <vector>

#include "pgs_host.cuh"

namespace pgs {

// Step 2 on one rank: sr = min(s, n) samples of its sorted keys, at local
// positions floor((i+1) n / sr) - 1 (the caller's bit patterns).
template <typename K>
__global__ void k_rank_samples(const K* __restrict__ sorted, uint64_t n, uint64_t sr, K* out) {
  pdl_enter();
  const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (i >= sr) return;
  out[i] = sorted[(uint64_t)(((unsigned __int128)(i + 1) * n) / sr) - 1];
}

// Step 4 on one rank: for b = 1..G-1, lb = #{keys < t_b} and cnt = #{keys ==
// t_b} in key order; out = [lb_1..lb_{G-1}, cnt_1..cnt_{G-1}].
template <typename K>
__global__ void k_rank_counts(const K* __restrict__ sorted, uint64_t n, const K* __restrict__ spl, uint32_t G,
                              uint64_t* out, int f32) {
  pdl_enter();
  const uint64_t b = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x + 1;
  if (b >= G) return;
  const K v = to_order<K>(spl[b - 1], f32);
  uint64_t lo = 0, hi = n;
  while (lo < hi) {
    const uint64_t mid = (lo + hi) >> 1;
    if (to_order<K>(sorted[mid], f32) < v) lo = mid + 1; else hi = mid;
  }
  const uint64_t l = lo;
  hi = n;
  while (lo < hi) {
    const uint64_t mid = (lo + hi) >> 1;
    if (to_order<K>(sorted[mid], f32) <= v) lo = mid + 1; else hi = mid;
  }
  out[b - 1] = l;
  out[G - 1 + b - 1] = lo - l;
}

// Every rank's counts (row r as k_rank_counts writes it) into the G x (G+1)
// lb / cnt matrices of the investigator (entries b = 1..G-1 of each row).
static __global__ void k_rank_unpack(const uint64_t* __restrict__ counts_all, uint32_t G, uint64_t* lb,
                                     uint64_t* cnt) {
  pdl_enter();
  const uint64_t q = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (q >= (uint64_t)G * (G - 1)) return;
  const uint64_t r = q / (G - 1), b = q % (G - 1) + 1;
  const uint64_t* row = counts_all + r * 2 * (G - 1);
  lb[r * (G + 1) + b] = row[b - 1];
  cnt[r * (G + 1) + b] = row[G - 1 + b - 1];
}

// The splitters in order form at slots 1..G-1 (slot 0 unused), as the
// investigator reads them.
template <typename K>
__global__ void k_rank_splitters(const K* __restrict__ spl, uint32_t G, K* t, int f32) {
  pdl_enter();
  const uint64_t b = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x + 1;
  if (b >= G) return;
  t[b] = to_order<K>(spl[b - 1], f32);
}

// Device scratch of the investigator over G ranks.
struct RankCutsLayout {
  size_t koff, Pt, R0, mat, seg, st, run_off, run_inst, lb, cnt, t, total;
};

inline RankCutsLayout rank_cuts_layout(uint32_t G, int w) {
  Carver c(nullptr);
  RankCutsLayout L;
  auto at = [&](uint64_t bytes) {
    c.used = (c.used + kAlign - 1) / kAlign * kAlign;
    const size_t off = c.used;
    c.used += std::max<uint64_t>(bytes, 1);
    return off;
  };
  const uint64_t MAT = (uint64_t)G * (G + 1);
  L.koff = at(16);
  L.Pt = at(4);
  L.R0 = at(8);
  L.mat = at(16);
  L.seg = at(16);
  L.st = at(8);
  L.run_off = at(8ull * (G + 1));
  L.run_inst = at(4ull * G);
  L.lb = at(8 * MAT);
  L.cnt = at(8 * MAT);
  L.t = at((uint64_t)w * G);
  L.total = c.used;
  return L;
}

// The investigator (Section IV-B) over every rank's counts: the tables of one
// instance of G runs whose sizes are the shard sizes, then the same kernels
// as the single-GPU sort.  cut_out: G x (G+1); e_out: G+1 (device).
template <typename K>
int run_rank_cuts(const uint64_t* counts_all, const uint64_t* host_sizes, uint32_t G, const K* spl, uint64_t* cut_out,
                  uint64_t* e_out, const Options& o, cudaStream_t st) {
  const RankCutsLayout L = rank_cuts_layout(G, (int)sizeof(K));
  char* ws = static_cast<char*>(o.workspace);
  std::vector<uint64_t> run_off(G + 1, 0);
  for (uint32_t r = 0; r < G; ++r) run_off[r + 1] = run_off[r] + host_sizes[r];
  const uint64_t N = run_off[G];
  const uint64_t koff[2] = {0, N}, mat[2] = {0, (uint64_t)G * (G + 1)}, seg[2] = {0, (uint64_t)G * G}, s0[1] = {0};
  const uint32_t Pt[1] = {G}, R0[2] = {0, G};
  std::vector<uint32_t> run_inst(G, 0);
  // Pageable host sources: each copy is staged before the call returns.
  PGS_CUDA(cudaMemcpyAsync(ws + L.koff, koff, sizeof(koff), cudaMemcpyHostToDevice, st));
  PGS_CUDA(cudaMemcpyAsync(ws + L.Pt, Pt, sizeof(Pt), cudaMemcpyHostToDevice, st));
  PGS_CUDA(cudaMemcpyAsync(ws + L.R0, R0, sizeof(R0), cudaMemcpyHostToDevice, st));
  PGS_CUDA(cudaMemcpyAsync(ws + L.mat, mat, sizeof(mat), cudaMemcpyHostToDevice, st));
  PGS_CUDA(cudaMemcpyAsync(ws + L.seg, seg, sizeof(seg), cudaMemcpyHostToDevice, st));
  PGS_CUDA(cudaMemcpyAsync(ws + L.st, s0, sizeof(s0), cudaMemcpyHostToDevice, st));
  PGS_CUDA(cudaMemcpyAsync(ws + L.run_off, run_off.data(), 8ull * (G + 1), cudaMemcpyHostToDevice, st));
  PGS_CUDA(cudaMemcpyAsync(ws + L.run_inst, run_inst.data(), 4ull * G, cudaMemcpyHostToDevice, st));
  PGS_CUDA(cudaStreamSynchronize(st));                 // the host vectors die with this call
  const Geo g{reinterpret_cast<const uint64_t*>(ws + L.koff), reinterpret_cast<const uint32_t*>(ws + L.Pt),
              reinterpret_cast<const uint32_t*>(ws + L.R0), reinterpret_cast<const uint64_t*>(ws + L.mat),
              reinterpret_cast<const uint64_t*>(ws + L.seg), reinterpret_cast<const uint64_t*>(ws + L.st),
              reinterpret_cast<const uint64_t*>(ws + L.run_off), reinterpret_cast<const uint32_t*>(ws + L.run_inst),
              1u, G};
  uint64_t* lb = reinterpret_cast<uint64_t*>(ws + L.lb);
  uint64_t* cnt = reinterpret_cast<uint64_t*>(ws + L.cnt);
  K* t = reinterpret_cast<K*>(ws + L.t);
  const int f32 = o.dtype == PGS_F32;
  Ctx c;
  c.st = st;
  c.timer = o.timer;
  if (G > 1) {
    PGS_TRY(launch(c, PGS_KERNEL_INVESTIGATOR, 4, 16ull * G * (G - 1), [&] {
      klaunch(st, c.pdl, k_rank_unpack, grid_for((uint64_t)G * (G - 1), 256), 256, 0, counts_all, G, lb, cnt);
    }));
    PGS_TRY(launch(c, PGS_KERNEL_SPLITTERS, 3, 2ull * G * sizeof(K), [&] {
      klaunch(st, c.pdl, k_rank_splitters<K>, grid_for(G, 256), 256, 0, spl, G, t, f32);
    }));
  }
  PGS_TRY(launch(c, PGS_KERNEL_INVESTIGATOR, 4, 24ull * G, [&] {
    klaunch(st, c.pdl, k_cut_edges, grid_for(G, 256), 256, 0, g, cut_out, e_out);
  }));
  if (G == 1) return PGS_OK;
  return launch(c, PGS_KERNEL_INVESTIGATOR, 4, 24ull * G * (G + 1), [&] {
    klaunch(st, c.pdl, k_investigator<K>, G, 256, 0, lb, cnt, t, g, o.investigator, cut_out, e_out);
  });
}

// The shape of a merge of k sorted lists of n keys in all: one instance whose
// k segments form one bucket (the single-sort tables for P = k size the
// geometry; step 1 is not run).
inline Shape merge_shape(uint64_t n, uint32_t k, bool vals, const Options& o) {
  Shape sh;
  sh.n = n;
  sh.w = key_bytes(o.dtype);
  sh.vals = vals;
  sh.I = 1;
  sh.R = k;
  sh.Pmax = k;
  sh.Q = k;                                             // the k segments of the one bucket
  sh.MAT = 1;                                           // no cut matrices
  sh.maxlen = kTile;                                    // no run formation
  sh.s = 0;
  sh.S = 0;
  sh.four = use_four_way(sh.n, o);
  finish_shape(sh);
  sh.pre_rounds = 0;                                    // the rounds are planned one by one
  return sh;
}

// The key at every 64th position of src, in order form (the index a merge
// round's partition and four-way boundaries read).
template <typename K>
__global__ void k_build_index(const K* __restrict__ src, uint64_t n, K* kidx, int f32) {
  pdl_enter();
  const uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (e * kIdxStride >= n) return;
  kidx[e] = to_order<K>(src[e * kIdxStride], f32);
}

// Statistics of a merge: its size, the lists, passes, launches and the device
// error word (pgs_get_stats reads them).
static __global__ void k_merge_stats(DevStats* st, uint64_t n, uint32_t k, uint32_t passes, uint32_t launches,
                                     const uint32_t* err) {
  pdl_enter();
  st->n = n;
  st->P = k;
  st->s = 0;
  st->max_bucket = n;
  st->min_bucket = n;
  st->splitter_mode = 0;
  st->fallback = 0;
  st->error = *err;
  st->passes = passes;
  st->launches = launches;
  st->max_over_mean = 1.0f;
  st->learned_over_mean = 0.0f;
  st->reserved = 0;
}

// Step 6 on one rank: the stable merge of k sorted lists that lie one after
// another in kin (list j = [host_off[j], host_off[j+1])), earlier lists first
// on ties, with the Fig. 2 schedule: four-way passes while two tree levels
// remain (merge_ways 4), else pairwise ones.  Round i writes kout when the
// rounds left after it are even, else the workspace's alternate buffer, so the
// last round lands in kout and kin is only read.
template <typename K, bool V>
int run_merge_lists(const Shape& sh, const Options& o, const K* kin, const uint32_t* vin, K* kout, uint32_t* vout,
                    const uint64_t* host_off, uint32_t k, cudaStream_t st) {
  const uint64_t n = sh.n;
  int levels = k > 1 ? ceil_log2(k) : 0;
  int passes = 0;
  for (int l = levels; l > 0; ++passes) l -= (sh.four && l >= 2) ? 2 : 1;
  if (passes == 0) {                                    // one list: a copy
    if (kout != kin) PGS_CUDA(cudaMemcpyAsync(kout, kin, n * sizeof(K), cudaMemcpyDeviceToDevice, st));
    if (V && vout != vin) PGS_CUDA(cudaMemcpyAsync(vout, vin, n * 4ull, cudaMemcpyDeviceToDevice, st));
  }
  PGS_TRY((set_all_smem_attrs<K, V>()));
  Ctx c;
  c.st = st;
  c.timer = o.timer;
  c.variant = o.tile_variant;
  c.wait_ns = o.spin_limit;
  c.inject_timeout = o.fault_inject == PGS_FAULT_WAIT_TIMEOUT;
  c.pdl = n <= kPdlMaxKeys;
  Buffers b;
  carve(sh, o.workspace, &b);
  const int f32 = o.dtype == PGS_F32;
  const uint32_t mtile = (uint32_t)(kMergeShapes[c.variant].nt * kMergeShapes[c.variant].vt);
  PGS_CUDA(cudaMemsetAsync(b.err, 0, sizeof(uint32_t), st));
  if (passes > 0) {
    PGS_TRY(launch(c, PGS_KERNEL_OFFSETS, 0, 16ull * (k + 1), [&] {
      klaunch(st, c.pdl, k_tables_single, grid_for(k + 1, 256), 256, 0, b.koff, b.Pt, b.R0, b.mat, b.seg, b.st, b.run_off,
                                                            b.run_inst, n, k, 0);
    }));
    PGS_CUDA(cudaMemcpyAsync(b.off, host_off, (k + 1) * sizeof(uint64_t), cudaMemcpyHostToDevice, st));
    PGS_CUDA(cudaStreamSynchronize(st));               // host_off may be pageable memory of the caller
    K* alt = static_cast<K*>(b.alt_k);
    K* kidx = static_cast<K*>(b.kidx);
    const K* src = kin;
    const uint32_t* vsrc = vin;
    if (f32) {                                          // the rounds compare order-form keys
      K* conv = passes % 2 ? alt : kout;                // never a buffer the first round writes
      PGS_TRY(launch(c, PGS_KERNEL_SAMPLE, 6, 2 * n * sizeof(K), [&] {
        klaunch(st, c.pdl, k_to_order<K>, grid_for(n, 256), 256, 0, kin, conv, n, 1);
      }));
      src = conv;
    }
    PGS_TRY(launch(c, PGS_KERNEL_PARTITION, 6, 2 * ceil_div(n, kIdxStride) * sizeof(K), [&] {
      klaunch(st, c.pdl, k_build_index<K>, grid_for(ceil_div(n, kIdxStride), 256), 256, 0, src, n, kidx, 0);
    }));
    const Geo g = b.geo(sh);
    uint32_t step = 1;
    for (int i = 1; levels > 0; ++i) {
      const bool to_out = (passes - i) % 2 == 0;
      K* kd = to_out ? kout : alt;
      uint32_t* vd = V ? (to_out ? vout : b.alt_v) : nullptr;
      const bool last = i == passes;
      K* io = last ? nullptr : kidx;
      if (sh.four && levels >= 2) {
        PGS_TRY(launch(c, PGS_KERNEL_PAIRS, 6, 112ull * k, [&] {
          klaunch(st, c.pdl, k_quads4_buckets, grid_for(k, 256), 256, 0, b.quads, b.tcount4, b.pairs, b.tcount, g, b.off, 0, k,
                                                             step, merge4_q<K>(), mtile);
        }));
        PGS_TRY((merge4_round<K, V>(c, src, vsrc, kd, vd, k, n, b, last ? f32 : 0, 6, kidx, io,
                                    ceil_div(k, 4ull * step) + 1)));
        step *= 4;
        levels -= 2;
      } else {
        PGS_TRY((merge_round<K, V>(c, GenBucketLists{b.pairs, b.tcount, g, b.off, 0, step, mtile}, src, vsrc, kd,
                                   vd, k, n, b, last ? f32 : 0, 6, kidx, io, ceil_div(k, 2ull * step) + 1)));
        step *= 2;
        levels -= 1;
      }
      src = kd;
      vsrc = vd;
    }
  }
  if (!o.stats) return PGS_OK;
  const uint32_t launches = c.launches + 1;
  return launch(c, PGS_KERNEL_STATS, 0, 64, [&] {
    klaunch(st, c.pdl, k_merge_stats, 1, 1, 0, static_cast<DevStats*>(o.stats), n, k, (uint32_t)passes, launches, b.err);
  });
}

}  // namespace pgs
