/*
 * pgs.h - C ABI of the GB300 load-balanced sample sort (libpgs.so).
 *
 * The method is the six-step distributed sort of "A Load-Balanced Parallel and
 * Distributed Sorting Algorithm Implemented with PGX.D" (arXiv 1611.00463),
 * Section IV: local sort of every processor's data, regular sampling, splitter
 * selection by the Master, binary search of the splitters with the duplicate-
 * aware "investigator" (Section IV-B, Fig. 5), exchange of ranges at known
 * offsets (Section IV-C), and the balanced pairwise merge of Fig. 2
 * (Section IV-A).  The paper's p processors are P logical partitions ("runs")
 * of one array in device memory; the exchange is a copy inside HBM.
 *
 * Conventions shared by every entry point:
 *  - Every pointer argument is DEVICE memory owned by the caller, unless the
 *    comment says host.  The library never allocates or frees device memory;
 *    temporary storage is the caller's workspace (pgs_workspace_bytes).
 *  - Every call is asynchronous on `stream` (a cudaStream_t passed as void*,
 *    NULL = the legacy default stream) unless its comment says it synchronises.
 *  - Every call returns a pgs_status; none aborts, traps or exits.  Invalid
 *    arguments are rejected before anything is launched.
 *  - Keys are sorted ascending by their total order: unsigned integers by
 *    value, float32 by IEEE 754 totalOrder on the bit pattern
 *    (-NaN < -inf < ... < -0 < +0 < ... < +inf < +NaN).  Output keys keep the
 *    input bit patterns.  The sort is stable: equal keys keep input order, and
 *    the uint32 payload ("vals", the paper's previous-processor/index record,
 *    step 6) travels with its key.
 *  - Logical partitions: run r holds input positions
 *    [floor(r n / P), floor((r+1) n / P)).  P is clamped to max(1, min(P, n)).
 */
#ifndef PGS_H
#define PGS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum { PGS_U32 = 0, PGS_U64 = 1, PGS_F32 = 2 } pgs_dtype;

typedef enum {
  PGS_OK = 0,
  PGS_ERR_INVALID = -1,      /* bad argument (NULL pointer with n > 0, P = 0, bad enum, ...) */
  PGS_ERR_WORKSPACE = -2,    /* workspace NULL, misaligned (needs 256 B) or too small */
  PGS_ERR_CUDA = -3,         /* a CUDA runtime call or launch failed */
  PGS_ERR_TIMEOUT = -4,      /* a bounded device-side wait ran out */
  PGS_ERR_UNSUPPORTED = -5   /* valid request the library does not implement */
} pgs_status;

/* Investigator variants (Section IV-B).  With e_b the number of stable ranks
 * given to buckets 0..b-1, L_b = #keys < t_b and G_b = #keys == t_b:
 *  RANK  : e_b = clamp(floor(b n / P), L_b, L_b + G_b)   (default)
 *  EQUAL : a group of k equal splitters t_j..t_{j+k-1} splits the range of
 *          their value into k equal parts, e_{j+i} = L + floor(G (i+1) / k);
 *          a non-duplicated splitter is cut by plain binary search (upper bound)
 *  OFF   : plain upper bound e_b = L_b + G_b, the failure mode of Fig. 5(b).
 * These three divide a value's range by global stable rank, so the output is
 * the same stable sort; only the bucket sizes differ.
 *  LOCAL : the rule as the text words it: every run divides its own range of
 *          a duplicated value, cut[r][j+i] = lb[r][j] + floor(cnt[r][j] (i+1) / k)
 *          for a group of k equal splitters, upper bound otherwise; e_b is the
 *          sum of the runs' cuts.  The keys come out sorted, but equal keys are
 *          ordered by bucket, then run (not by input position: not stable). */
typedef enum {
  PGS_INVESTIGATOR_RANK = 0,
  PGS_INVESTIGATOR_EQUAL = 1,
  PGS_INVESTIGATOR_OFF = 2,
  PGS_INVESTIGATOR_LOCAL = 3
} pgs_investigator;

/* Step 5 (Section IV-C): SCATTER copies every run segment to its bucket before
 * the merge (one pass of its own); FUSED lets the first merge round of step 6
 * read each pair of segments where the sorted runs left them and write the
 * merged pair to its place in the bucket.  AUTO picks FUSED. */
typedef enum { PGS_EXCHANGE_AUTO = 0, PGS_EXCHANGE_SCATTER = 1, PGS_EXCHANGE_FUSED = 2 } pgs_exchange;

/* Splitter source.  SAMPLED: steps 2-3 of Section IV.  LEARNED: an MLP CDF
 * model trained on the same sample predicts bucket ids; the sampled splitters
 * judge it and take over when its imbalance exceeds 1 + eps.  For P > 64 no
 * model is trained (about 64 linear pieces cannot place more bucket
 * boundaries): the sampled cuts stand, stats report fallback = 1 and
 * learned_over_mean = NaN, and model_out receives an invalid all-zero model;
 * a caller-given cfg->model is still judged at any P. */
typedef enum { PGS_SPLITTERS_SAMPLED = 0, PGS_SPLITTERS_LEARNED = 1 } pgs_splitter_mode;

/* How pgs_sort_host copies its output back.  GROUPS (default): the host waits
 * once step 5 has fixed the bucket bounds, then each group of buckets is
 * copied back while the next group merges (shortest single call).  AT_END:
 * the call never waits; the whole output is copied back after step 6 (a longer
 * single call, but several calls in flight keep the GPU and both copy
 * directions busy).  Ignored by the device-buffer calls. */
typedef enum { PGS_COPY_BACK_AUTO = 0, PGS_COPY_BACK_AT_END = 1, PGS_COPY_BACK_GROUPS = 2 } pgs_copy_back;

/* Launch-sequence replay for pgs_sort / pgs_sort_copy and pgs_sort_batched /
 * pgs_sort_batched_copy.  AUTO: the second call with the same arguments and
 * options (pointers, sizes, every option; for a batch the plan, its workspace
 * and buffers) captures its launch sequence into a CUDA graph on a stream of
 * the library's own, and that call and later identical ones launch the graph
 * on `stream`: the same kernels on the same buffers, without the host's
 * per-launch work.  A call with a timer, on a stream that is itself being
 * captured, or from pgs_batch_tune always launches directly.  At most 16
 * graphs are kept per process (least recently used first out).  OFF: always
 * launch directly. */
typedef enum { PGS_GRAPH_CACHE_AUTO = 0, PGS_GRAPH_CACHE_OFF = 1 } pgs_graph_cache;

/* Kernels of the pipeline, as reported by the launch timer. */
typedef enum {
  PGS_KERNEL_BLOCK_SORT = 0,   /* step 1: shared-memory block sort of one tile */
  PGS_KERNEL_MERGE = 1,        /* steps 1, 3, 6: pairwise merge-path merge of one round */
  PGS_KERNEL_PARTITION = 2,    /* one round's plan: merge-path splits, a small round's tile jobs, four-way co-ranks */
  PGS_KERNEL_PAIRS = 3,        /* pair descriptors of one round */
  PGS_KERNEL_SCAN = 4,         /* device-wide exclusive scan */
  PGS_KERNEL_SAMPLE = 5,       /* step 2: regular samples */
  PGS_KERNEL_SPLITTERS = 6,    /* step 3: splitter pick (a sort's pick runs inside the cut search), learned model */
  PGS_KERNEL_CUT_SEARCH = 7,   /* steps 3-4: splitter pick, binary searches, fixed cuts */
  PGS_KERNEL_INVESTIGATOR = 8, /* step 4: investigator cuts */
  PGS_KERNEL_OFFSETS = 9,      /* step 5 set-up: segment sizes, receive offsets (and small sorts' bucket round plans) */
  PGS_KERNEL_SCATTER = 10,     /* step 5: the exchange */
  PGS_KERNEL_STATS = 11,       /* load statistics */
  PGS_KERNEL_MERGE4 = 12,      /* steps 1, 6: four-way merge of one pass (two tree levels) */
  PGS_KERNEL_COUNT = 13
} pgs_kernel;

/* One timed launch.  `bytes` are the algorithmic bytes the launch must move
 * (reads + writes of the data it is defined to touch), `ms` its duration
 * between CUDA events recorded on the call's stream around it. */
typedef struct pgs_launch_record {
  uint32_t kernel;            /* pgs_kernel */
  uint32_t step;              /* step of Section IV (1-6), 0 = bookkeeping */
  uint64_t bytes;
  float    ms;
  uint32_t reserved;
} pgs_launch_record;

/* Opaque launch timer (host object holding CUDA events; no device memory). */
typedef struct pgs_timer pgs_timer;

#define PGS_TILE_VARIANTS 4

/* Options.  A zeroed struct, or a NULL pointer, means all defaults. */
typedef struct pgs_config {
  int32_t  dtype;             /* pgs_dtype, default PGS_U32 */
  uint32_t samples_per_run;   /* s; 0 = the paper's budget floor(262144 / (P * key_bytes)) */
  float    eps;               /* target imbalance; 0 = 0.05 */
  int32_t  guaranteed;        /* 1: s = max(s, ceil(P / eps)).  With runs of equal length m = n / P every
                                 bucket is then below (1 + P/s) m + P <= (1 + eps) m + P, and below
                                 (1 + eps) m when s divides m (regular-sampling bound, any input) */
  int32_t  investigator;      /* pgs_investigator, default RANK */
  int32_t  exchange;          /* pgs_exchange, default AUTO */
  int32_t  splitter_mode;     /* pgs_splitter_mode, default SAMPLED */
  int32_t  tile_variant;      /* merge tile shape, 0..PGS_TILE_VARIANTS-1 (threads x outputs per thread:
                                 0 = 128 x 17 (default), 1 = 256 x 13, 2 = 128 x 9, 3 = 64 x 17);
                                 pgs_batch_tune picks one for a batch */
  void*    workspace;         /* device, 256-byte aligned, >= pgs_workspace_bytes(n, P, cfg) */
  uint64_t workspace_bytes;
  /* Optional device outputs, written when non-NULL: */
  uint64_t* bucket_bounds;    /* e[0..P] (P+1 entries, P effective): bucket b = output [e_b, e_{b+1}) */
  uint64_t* cuts;             /* cut[r][0..P], P x (P+1), row-major: run r sends its sorted
                                 positions [cut[r][b], cut[r][b+1]) to bucket b */
  void*     splitters;        /* t_1..t_{P-1}, P-1 keys of the key type (float keys as bits) */
  void*     stats;            /* a pgs_stats in device memory */
  uint64_t  spin_limit;       /* limit of every device-side wait (the merge kernels' waits for their bulk
                                 copies), in ns of %globaltimer; 0 = 2 s.  A wait that runs out sets bit 0
                                 of the device error word, the kernel lets its copies in flight land and
                                 returns, and pgs_get_stats reports PGS_ERR_TIMEOUT */
  pgs_timer* timer;           /* optional: record every launch's duration (host object) */
  /* LEARNED mode only (single sorts): */
  const float* model;         /* optional device model of PGS_MLP_WORDS words to use instead of
                                 training one; rejected (sampled cuts kept) if its signs do not make
                                 it monotone */
  float*    model_out;        /* optional device buffer of PGS_MLP_WORDS words: the model used */
  int32_t   merge_ways;       /* lists merged per pass over the data (Fig. 2 tree levels per pass):
                                 4 (two levels per pass), 2 (one level, pairwise rounds), or 0 (default):
                                 four-way from 2^23 keys (for a batch: keys of all instances), pairwise
                                 below, where the sort is bound by its launches.  Four-way tiles hold
                                 exactly their share of outputs: tile boundaries come from the key index
                                 the previous pass wrote */
  int32_t   copy_back;         /* pgs_copy_back, pgs_sort_host only; default AUTO */
  int32_t   graph_cache;       /* pgs_graph_cache, device and batched sorts; default AUTO */
  int32_t   fault_inject;      /* testing only, 0 = off.  PGS_FAULT_WAIT_TIMEOUT: the first tile of the
                                  call's first merge round announces its copies to its barrier but issues
                                  none (nothing is in flight), so its bounded wait runs out after
                                  spin_limit; the call's output is then incomplete */
} pgs_config;

/* pgs_config.fault_inject values. */
#define PGS_FAULT_WAIT_TIMEOUT 1

/* Load statistics of one sort (Table II reports the per-processor share). */
typedef struct pgs_stats {
  uint64_t n;                 /* keys sorted */
  uint32_t P;                 /* effective partitions */
  uint32_t samples_per_run;   /* s actually used */
  uint64_t max_bucket;        /* max_b (e_{b+1} - e_b) */
  uint64_t min_bucket;        /* min_b (e_{b+1} - e_b) */
  uint32_t splitter_mode;     /* mode that produced the buckets */
  uint32_t fallback;          /* LEARNED: 1 if the sampled splitters replaced the model's */
  uint32_t error;             /* device-side error word; 0 = none, bit 0 = a bounded wait expired,
                                 bit 1 = a merge tile did not fit its buffer (skipped) */
  uint32_t passes;            /* full passes over the data the sort made */
  uint32_t launches;          /* kernels the call launched */
  float    max_over_mean;     /* largest bucket / its instance's mean bucket n_i / P_i */
  float    learned_over_mean; /* LEARNED: the model's own largest bucket / mean, before the judge */
  uint32_t reserved;
} pgs_stats;

/* Bytes of device workspace pgs_sort / pgs_sort_copy need for n keys on P
 * partitions with these options (cfg may be NULL).  Returns 0 for an invalid
 * request.  Host-only; launches nothing. */
size_t pgs_workspace_bytes(uint64_t n, uint32_t P, const pgs_config* cfg);

/* Sort n keys (and their uint32 payload) in place, stably, ascending, with the
 * six steps of Section IV on P logical partitions.
 *   keys: n keys of cfg->dtype (device).  vals: n uint32 (device) or NULL for a
 *   keys-only sort.  P >= 1.  Asynchronous on stream. */
int pgs_sort(void* keys, uint32_t* vals, uint64_t n, uint32_t P, void* stream,
             const pgs_config* cfg);

/* Same as pgs_sort but out of place: reads keys_in/vals_in (left unchanged
 * unless they alias the outputs) and writes keys_out/vals_out.  vals_in and
 * vals_out are both NULL or both non-NULL. */
int pgs_sort_copy(const void* keys_in, const uint32_t* vals_in, void* keys_out,
                  uint32_t* vals_out, uint64_t n, uint32_t P, void* stream,
                  const pgs_config* cfg);

/* Bytes of device workspace pgs_sort_host needs: pgs_workspace_bytes plus the
 * device copies of input and output.  Returns 0 for an invalid request. */
size_t pgs_host_workspace_bytes(uint64_t n, uint32_t P, const pgs_config* cfg);

/* Sort host-resident keys (and payloads) out of place through the device: the
 * same sort as pgs_sort_copy, with the copies inside the call.
 *   keys_in/vals_in, keys_out/vals_out: host memory, pinned or pageable (a
 *   copy from or to pageable memory holds the host until it is done, so each
 *   group's copy is issued after the previous group's work is enqueued and
 *   the host waits while the GPU sorts); vals both NULL or both
 *   non-NULL; inputs and outputs must not overlap.  Device pointers are
 *   PGS_ERR_INVALID.  cfg->workspace (device, on the GPU that sorts) must hold
 *   pgs_host_workspace_bytes(n, P, cfg).
 *   cfg->copy_back = GROUPS: the input is copied in up to 8 groups of whole
 *   runs on a stream of the call's own, and step 1 of a group starts as soon
 *   as its copy has landed, while later groups are still copying; once step 5
 *   has fixed the bucket bounds the call reads them back (the host waits for
 *   steps 1-5 there), then runs the remaining merge rounds of step 6 in up to
 *   8 groups of buckets and copies each group's sorted keys back while the
 *   next group merges.  AT_END: the input in groups as with GROUPS, the whole
 *   output copied back after the last pass, and the call never waits (so does
 *   GROUPS for P = 1).  AUTO (the default): sorts of fewer than 2^25 keys copy
 *   their input in one piece and their output after the last pass and never
 *   wait (measured faster up to 2^24 keys: 11.2 against 8.2 Gkeys/s at 2^24
 *   u32 keys, two calls in flight), larger ones as GROUPS.  The rest is
 *   asynchronous on `stream` for pinned memory: synchronise it before reading
 *   the outputs.
 *   The paper has no counterpart (its data starts in each machine's memory);
 *   this is the host-to-host form of pgs_sort_copy. */
int pgs_sort_host(const void* keys_in, const uint32_t* vals_in, void* keys_out,
                  uint32_t* vals_out, uint64_t n, uint32_t P, void* stream,
                  const pgs_config* cfg);

/* pgs_sort without a workspace, for callers that cannot allocate device
 * memory (an allocator or memory-pool callback, a plug-in whose host owns all
 * device allocations, a path that must never wait on the driver's allocator).
 * The paper has no counterpart: this is a deployment variant of pgs_sort.
 *   Temporary storage is one file-scope device array of
 *   PGS_STATIC_SCRATCH_BYTES inside the library, present on every GPU that
 *   loads it until the process exits; the call allocates and frees nothing.
 *   Limits: n <= PGS_STATIC_MAX_KEYS and max(1, min(P, n)) <= PGS_STATIC_MAX_P,
 *   otherwise PGS_ERR_UNSUPPORTED before anything is launched.  Within those
 *   limits every option combination fits the array.  cfg->workspace must be
 *   NULL (PGS_ERR_INVALID otherwise); cfg->graph_cache has no effect (every
 *   launch is issued directly); every other option works as in pgs_sort.
 *   The first call on a device is its set-up: it looks up the array's device
 *   address with that device current, and the CUDA runtime may load the
 *   library's device code there (lazy loading), which can allocate device
 *   memory.  Make that first call outside any allocation-free context and
 *   before any stream capture.  The looked-up address is kept per device for
 *   the process's lifetime: after cudaDeviceReset the entry point must not be
 *   used again in that process.
 *   All calls share the array and it keeps the last call's contents: two calls
 *   whose work overlaps on the GPU race and corrupt each other's results;
 *   serialise them (one stream). */
#define PGS_STATIC_MAX_KEYS (1u << 16)
#define PGS_STATIC_MAX_P 64u
#define PGS_STATIC_SCRATCH_BYTES (8u << 20)
int pgs_sort_static(void* keys, uint32_t* vals, uint64_t n, uint32_t P, void* stream,
                    const pgs_config* cfg);

/* Batched sort: many independent instances in one launch sequence.  The
 * paper's library sorts several data sets simultaneously (end of Section
 * IV-C); here instance i is keys[offsets[i], offsets[i+1]) with its own P_i
 * logical partitions, and every step of Section IV runs for all instances at
 * once (one kernel per phase), so the whole batch is about as many launches
 * as one sort and can be captured in one CUDA graph.
 *   pgs_batch_create plans a batch on the host: offsets (HOST, num+1
 *   entries, non-decreasing, offsets[0] = 0), P (HOST, num entries, or NULL
 *   for the automatic rule pgs_batch_auto_partitions), cfg->dtype and
 *   with_vals fix the key type and whether a payload travels.  Each P_i is
 *   clamped to max(1, min(P_i, n_i)) and must stay <= 8192.
 *   pgs_batch_workspace_bytes: device workspace the batch needs.
 *   pgs_batch_upload copies the batch's tables into that workspace (256-byte
 *   aligned) and waits for the copy; call it once per workspace, outside any
 *   stream capture.
 *   pgs_sort_batched sorts every instance in place, stably, with the same
 *   options as pgs_sort (cfg->workspace must be the uploaded workspace; the
 *   optional outputs bucket_bounds, cuts and splitters are not written for a
 *   batch).  It only launches kernels on `stream`, so it may be captured.
 *   pgs_batch_destroy frees the host plan. */
typedef struct pgs_batch pgs_batch;
uint32_t pgs_batch_auto_partitions(uint64_t n);   /* clamp(2^floor(log2(n / 65536)), 1, 256) */
int pgs_batch_create(const uint64_t* offsets, uint32_t num, const uint32_t* P, int with_vals,
                     const pgs_config* cfg, pgs_batch** out);
size_t pgs_batch_workspace_bytes(const pgs_batch* batch);
int pgs_batch_upload(pgs_batch* batch, void* workspace, uint64_t workspace_bytes, void* stream);
int pgs_sort_batched(pgs_batch* batch, void* keys, uint32_t* vals, void* stream, const pgs_config* cfg);
/* Out-of-place form: reads keys_in/vals_in, writes keys_out/vals_out (the
 * inputs are left unchanged, so a captured graph can be replayed on them). */
int pgs_sort_batched_copy(pgs_batch* batch, const void* keys_in, const uint32_t* vals_in, void* keys_out,
                          uint32_t* vals_out, void* stream, const pgs_config* cfg);
/* Autotuner: times the whole batched sort once per merge tile shape on
 * pseudo-random keys written into the caller's scratch buffers (device, one
 * key and, for a batch with payload, one uint32 per key of the batch; their
 * contents are overwritten), keeps the fastest shape in the batch (used by
 * later calls whose cfg->tile_variant is 0) and returns it in *chosen (host,
 * may be NULL) with the times in ms_out (host, PGS_TILE_VARIANTS floats, may
 * be NULL).  Synchronises `stream`; call it outside any stream capture. */
int pgs_batch_tune(pgs_batch* batch, void* scratch_keys, uint32_t* scratch_vals, void* stream,
                   const pgs_config* cfg, uint32_t* chosen, float* ms_out);
int pgs_batch_destroy(pgs_batch* batch);

/* Step 3 of Section IV on a caller-given sample: sort m sample keys (device,
 * any order) stably and write the P-1 splitters t_b = sample at sorted index
 * floor(b m / P) - 1 to splitters_out (device, P-1 keys).  In LEARNED mode it
 * also trains the CDF model on the sorted sample and writes its
 * PGS_MLP_WORDS words to model_out (device, may be NULL).  Needs cfg->workspace of at least
 * pgs_fit_workspace_bytes(m, P, cfg). */
/* Learned-CDF model: 1 -> 32 -> 32 -> 1 ReLU, FP32.  Layout of its
 * PGS_MLP_WORDS 4-byte words: w1[32], b1[32], W2[32][32] (row = output unit),
 * b2[32], w3[32], b3 (the PGS_MLP_FLOATS weights), then the input
 * normalisation kmin (low word, high word), scale (float), and a validity flag
 * (1 = monotone).  Input x = f32(f64(max(key, kmin) - kmin)) * scale on the
 * key's total-order bits; bucket = min(P-1, floor(P * clamp(y, 0, 1))).
 * Units 0..15 must have w1 >= 0 and w3 >= 0, units 16..31 w1 <= 0 and
 * w3 <= 0, W2 >= 0 within each half (entries across halves are ignored), so
 * that the bucket id never decreases as the key grows. */
#define PGS_MLP_HIDDEN 32
#define PGS_MLP_FLOATS (1 * 32 + 32 + 32 * 32 + 32 + 32 * 1 + 1)
#define PGS_MLP_WORDS (PGS_MLP_FLOATS + 4)
size_t pgs_fit_workspace_bytes(uint64_t m, uint32_t P, const pgs_config* cfg);
int pgs_fit_splitters(const void* samples, uint64_t m, uint32_t P, void* stream,
                      const pgs_config* cfg, void* splitters_out, float* model_out);

/* ---------------------------------------------------------------------------
 * Sharded sort: one global array spread over G ranks (processes, one GPU
 * each), sorted by the six steps of Section IV with the ranks as the paper's
 * processors.  Rank r holds shard r; the global input is the shards in rank
 * order, so the result is the stable sort of that concatenation and rank b
 * ends with bucket b, the stable ranks [e_b, e_{b+1}).  The library runs each
 * rank's steps on its GPU; the caller moves data between the ranks with its
 * own collectives:
 *   1. pgs_sort_copy the shard (any P; the result is the sorted shard);
 *   2. pgs_rank_samples (s = pgs_samples_per_run(G, cfg)); all-gather the
 *      samples in rank order;
 *   3. pgs_fit_splitters(all samples, G) -> the G-1 splitters, identical on
 *      every rank (no broadcast needed);
 *   4. pgs_rank_counts; all-gather the counts in rank order;
 *      pgs_rank_cuts -> the cut matrix and bucket bounds, identical on every
 *      rank (step 4's investigator, Section IV-B);
 *   5. all-to-all: rank r sends its sorted positions [cut[r][b], cut[r][b+1])
 *      to rank b, which receives them in rank order (sizes known from the cut
 *      matrix on every rank: Section IV-C);
 *   6. pgs_merge_lists of the G received segments -> bucket b.
 * ------------------------------------------------------------------------- */

/* Regular samples per run (per rank) for P runs: the paper's budget
 * floor(262144 / (P * key_bytes)), or at least ceil(P / eps) in guaranteed
 * mode (Section IV-B); 0 for P = 1 or an invalid request.  Host-only. */
uint64_t pgs_samples_per_run(uint32_t P, const pgs_config* cfg);

/* Step 2 on one rank (Section IV): from the rank's sorted keys (device, n
 * keys of cfg->dtype) write sr = min(s, n) regular samples, the keys at
 * positions floor((i+1) n / sr) - 1, to samples_out (device, sr keys).
 * Asynchronous on stream. */
int pgs_rank_samples(const void* sorted, uint64_t n, uint32_t s, void* samples_out, void* stream,
                     const pgs_config* cfg);

/* Step 4's binary searches on one rank (Section IV-B): for each splitter t_b,
 * b = 1..G-1 (device, G-1 keys, as pgs_fit_splitters writes them), the number
 * of the rank's sorted keys (device, n keys) ordered before t_b and equal to
 * it.  counts_out (device, 2 (G-1) uint64): [lb_1..lb_{G-1}, cnt_1..cnt_{G-1}].
 * Nothing is written for G = 1.  Asynchronous on stream. */
int pgs_rank_counts(const void* sorted, uint64_t n, const void* splitters, uint32_t G, uint64_t* counts_out,
                    void* stream, const pgs_config* cfg);

/* Device workspace of pgs_rank_cuts for G ranks (0 for an invalid request). */
size_t pgs_rank_cuts_workspace_bytes(uint32_t G, const pgs_config* cfg);

/* Step 4's investigator over all ranks (Section IV-B, Fig. 5), the same on
 * every rank: counts_all (device, G rows of 2 (G-1) uint64 in rank order, each
 * as pgs_rank_counts writes it), shard_sizes (HOST, G uint64), the splitters
 * (device, G-1 keys).  Writes cut_out (device, G x (G+1) uint64, row r: rank
 * r sends its sorted positions [cut[r][b], cut[r][b+1]) to rank b) and
 * bounds_out (device, G+1 uint64: bucket b = global stable ranks [e_b,
 * e_{b+1})), with cfg->investigator's rule on global stable ranks (the target
 * floor(b N / G), N = sum of the shard sizes).  Needs cfg->workspace of
 * pgs_rank_cuts_workspace_bytes(G, cfg).  Synchronises stream (the shard
 * sizes are uploaded from the host). */
int pgs_rank_cuts(const uint64_t* counts_all, const uint64_t* shard_sizes, uint32_t G, const void* splitters,
                  uint64_t* cut_out, uint64_t* bounds_out, void* stream, const pgs_config* cfg);

/* Device workspace of pgs_merge_lists for n keys in k lists (0: invalid). */
size_t pgs_merge_workspace_bytes(uint64_t n, uint32_t k, const pgs_config* cfg);

/* Step 6 on one rank (Section IV-C: the receiver merges what it received with
 * the balanced merge of Fig. 2): the stable merge of k sorted lists that lie
 * one after another in keys_in (list j = [offsets[j], offsets[j+1]); offsets
 * HOST, k+1 uint64, offsets[0] = 0, non-decreasing), earlier lists first on
 * equal keys, into keys_out (and vals_in into vals_out; both NULL or both
 * set).  Inputs are only read; inputs and outputs must not overlap.  Four-way
 * passes while two tree levels remain (cfg->merge_ways), else pairwise.
 * Needs cfg->workspace of pgs_merge_workspace_bytes(n, k, cfg); cfg->stats
 * (optional) receives the passes, launches and device error word.
 * Synchronises stream once (the offsets are uploaded), then runs
 * asynchronously. */
int pgs_merge_lists(const void* keys_in, const uint32_t* vals_in, const uint64_t* offsets, uint32_t k,
                    void* keys_out, uint32_t* vals_out, void* stream, const pgs_config* cfg);

/* Bytes of device workspace pgs_search can use for n sorted keys (0: it uses
 * none at this size).  With that much cfg->workspace the search first bisects a
 * compact copy of every 64th key, which stays in L2, then one 64-key block of
 * the array (a plain bisection of a large array misses in L2 on most of its
 * lower levels). */
size_t pgs_search_workspace_bytes(uint64_t n, const pgs_config* cfg);

/* Binary search on sorted output (Section IV-C: the library lets its users
 * search the sorted data).
 *   keys: n keys of cfg->dtype (cfg may be NULL: u32) sorted by key order, e.g.
 *   a pgs_sort output (float32 by IEEE totalOrder of the bits); queries: m keys
 *   of the same type.  side 0 = lower bound (the number of keys ordered before
 *   the query), 1 = upper bound (ordered before or equal).  pos_out: m uint64.
 *   bucket_bounds (the sort's e[0..P]) and bucket_out (m uint32) are both NULL
 *   or both set: bucket_out[i] = the bucket b with e[b] <= pos < e[b+1], or P
 *   for pos = n.  cfg->workspace (optional, 256-byte aligned): scratch of
 *   pgs_search_workspace_bytes(n, cfg) bytes for the indexed search; without
 *   it (or smaller) the search bisects the array directly, same results.  All
 *   pointers device memory; asynchronous on stream; allocates nothing. */
int pgs_search(const void* keys, uint64_t n, const void* queries, uint64_t m, int side,
               const uint64_t* bucket_bounds, uint32_t P, uint64_t* pos_out, uint32_t* bucket_out,
               void* stream, const pgs_config* cfg);

/* Previous processor and index of sorted entries whose payload is their input
 * position (Section IV step 6 keeps this provenance): for v = vals[i] < n,
 * run_out[i] = r with floor(r n / P') <= v < floor((r+1) n / P'),
 * P' = max(1, min(P, n)), and index_out[i] = v - floor(r n / P'); v >= n gives
 * run P' and index v - n.  run_out or index_out may be NULL (not both).  All
 * pointers device memory; asynchronous on stream. */
int pgs_provenance(const uint32_t* vals, uint64_t m, uint64_t n, uint32_t P, uint32_t* run_out,
                   uint64_t* index_out, void* stream);

/* Copy a device pgs_stats to host memory; synchronises `stream` and returns
 * PGS_ERR_TIMEOUT if the device error word reports an expired wait, PGS_ERR_CUDA
 * if it reports any other device-side inconsistency. */
int pgs_get_stats(const void* stats_dev, pgs_stats* host_out, void* stream);

/* Launch timer.  pgs_timer_create makes a host object with room for
 * `capacity` launches (2 * capacity CUDA events on the current device); give
 * it to calls through pgs_config.timer and every launch they make is bracketed
 * by events on their stream, until the timer is full (later launches are
 * counted as dropped).  pgs_timer_read waits for the recorded events, writes
 * up to `max` records with their durations to host memory `out`, and stores
 * the number recorded in *count and the number dropped in *dropped (either
 * may be NULL).  pgs_timer_reset forgets all records.  A timer must not be
 * shared by calls that run concurrently. */
int pgs_timer_create(uint32_t capacity, pgs_timer** out);
int pgs_timer_destroy(pgs_timer* timer);
int pgs_timer_reset(pgs_timer* timer);
int pgs_timer_read(pgs_timer* timer, pgs_launch_record* out, uint32_t max, uint32_t* count,
                   uint32_t* dropped);

/* Name of a pgs_kernel value ("block_sort", "merge", ...; never NULL). */
const char* pgs_kernel_name(uint32_t kernel);

/* Static description of a status code (never NULL). */
const char* pgs_strerror(int status);

/* Library version, "major.minor.patch". */
const char* pgs_version(void);

/* Text of the last CUDA failure seen by this thread (the call and the CUDA
 * error string), or "" if none.  Host-only; the pointer stays valid for the
 * thread's lifetime and is overwritten by its next failure. */
const char* pgs_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* PGS_H */
