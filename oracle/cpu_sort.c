/*
 * cpu_sort.c - the oracle's definition of the result (a stable ascending sort
 * of keys by their total order, the uint32 payload travelling with its key;
 * Section IV: smaller keys end on processors with smaller IDs and every entry
 * keeps its previous processor and index) run on all host cores, to time a
 * CPU baseline beside the GPU.  Test infrastructure: nothing in the GPU
 * library uses it, and it shares no code with it.
 *
 * Method: the array is cut into T chunks, each thread sorts its chunk with a
 * bottom-up stable merge sort, then pairs of sorted lists are merged round by
 * round (earlier list first on equal keys); in every round each thread takes
 * an equal share of the output positions and finds where its share starts in
 * each pair by a merge-path bisection, so all threads work in every round.
 * Keys are handled as uint64 order keys (uint32 widened; float32 mapped to
 * IEEE 754 totalOrder and back).
 */
#define _POSIX_C_SOURCE 200809L
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
  uint64_t *ka, *kb;      /* keys: current and other buffer */
  uint32_t *va, *vb;      /* payloads */
  uint64_t n;
  int T;
  uint64_t width;         /* list length of the current round */
  pthread_barrier_t bar;
} Job;

typedef struct {
  Job* job;
  int t;
} Arg;

/* Merge a[0..na) and b[0..nb) into out (stable: a first on ties), only the
 * outputs [d0, d1). */
static uint64_t split_of(const uint64_t* a, uint64_t na, const uint64_t* b, uint64_t nb, uint64_t d) {
  uint64_t lo = d > nb ? d - nb : 0, hi = d < na ? d : na;
  while (lo < hi) {
    uint64_t mid = (lo + hi) / 2;
    if (a[mid] <= b[d - 1 - mid]) lo = mid + 1; else hi = mid;
  }
  return lo;
}

static void merge_range(const uint64_t* a, const uint32_t* av, uint64_t na, const uint64_t* b, const uint32_t* bv,
                        uint64_t nb, uint64_t d0, uint64_t d1, uint64_t* out, uint32_t* outv) {
  uint64_t i = split_of(a, na, b, nb, d0), j = d0 - i;
  for (uint64_t d = d0; d < d1; ++d) {
    if (j >= nb || (i < na && a[i] <= b[j])) {
      out[d] = a[i];
      if (outv) outv[d] = av[i];
      ++i;
    } else {
      out[d] = b[j];
      if (outv) outv[d] = bv[j];
      ++j;
    }
  }
}

/* Stable bottom-up merge sort of k[lo, hi) (with payloads), using tk/tv as the
 * other buffer; the result ends in k. */
static void sort_chunk(uint64_t* k, uint32_t* v, uint64_t* tk, uint32_t* tv, uint64_t lo, uint64_t hi) {
  const uint64_t run = 32;
  for (uint64_t s = lo; s < hi; s += run) {            /* insertion sort of short runs (stable) */
    uint64_t e = s + run < hi ? s + run : hi;
    for (uint64_t i = s + 1; i < e; ++i) {
      uint64_t key = k[i];
      uint32_t val = v ? v[i] : 0;
      uint64_t j = i;
      while (j > s && k[j - 1] > key) {
        k[j] = k[j - 1];
        if (v) v[j] = v[j - 1];
        --j;
      }
      k[j] = key;
      if (v) v[j] = val;
    }
  }
  uint64_t *src = k, *dst = tk;
  uint32_t *sv = v, *dv = tv;
  for (uint64_t w = run; w < hi - lo; w *= 2) {
    for (uint64_t s = lo; s < hi; s += 2 * w) {
      uint64_t m = s + w < hi ? s + w : hi, e = s + 2 * w < hi ? s + 2 * w : hi;
      merge_range(src + s, sv ? sv + s : NULL, m - s, src + m, sv ? sv + m : NULL, e - m, 0, e - s, dst + s,
                  dv ? dv + s : NULL);
    }
    uint64_t* tk2 = src; src = dst; dst = tk2;
    uint32_t* tv2 = sv; sv = dv; dv = tv2;
  }
  if (src != k) {
    memcpy(k + lo, src + lo, (hi - lo) * sizeof(uint64_t));
    if (v) memcpy(v + lo, sv + lo, (hi - lo) * sizeof(uint32_t));
  }
}

static void* worker(void* p) {
  Arg* a = (Arg*)p;
  Job* j = a->job;
  const uint64_t n = j->n;
  const int T = j->T;
  const uint64_t c0 = (uint64_t)a->t * n / T, c1 = (uint64_t)(a->t + 1) * n / T;
  sort_chunk(j->ka, j->va, j->kb, j->vb, c0, c1);
  pthread_barrier_wait(&j->bar);
  /* Lists are the T chunks, then pairs of them, ...: list i of round r spans
   * chunks [i 2^r, (i+1) 2^r). */
  for (uint64_t span = 1; span < (uint64_t)T; span *= 2) {
    const uint64_t d0 = c0, d1 = c1;                    /* this thread's output positions */
    for (uint64_t g = 0; g < (uint64_t)T; g += 2 * span) {
      const uint64_t lo = g * n / T;
      const uint64_t mid = (g + span < (uint64_t)T ? g + span : (uint64_t)T) * n / T;
      const uint64_t hi = (g + 2 * span < (uint64_t)T ? g + 2 * span : (uint64_t)T) * n / T;
      const uint64_t s = d0 > lo ? d0 : lo, e = d1 < hi ? d1 : hi;
      if (s >= e) continue;
      merge_range(j->ka + lo, j->va ? j->va + lo : NULL, mid - lo, j->ka + mid, j->va ? j->va + mid : NULL,
                  hi - mid, s - lo, e - lo, j->kb + lo, j->vb ? j->vb + lo : NULL);
    }
    pthread_barrier_wait(&j->bar);
    if (a->t == 0) {                                    /* swap buffers for the next round */
      uint64_t* tk = j->ka; j->ka = j->kb; j->kb = tk;
      uint32_t* tv = j->va; j->va = j->vb; j->vb = tv;
    }
    pthread_barrier_wait(&j->bar);
  }
  return NULL;
}

static uint64_t f32_to_order(uint32_t b) { return (b & 0x80000000u) ? (uint32_t)~b : (b | 0x80000000u); }
static uint32_t order_to_f32(uint64_t o) { return (o & 0x80000000u) ? (uint32_t)(o & 0x7FFFFFFFu) : ~(uint32_t)o; }

/* Sort n keys (key_bytes 4 or 8; is_f32 for float32 bit patterns) and their
 * payloads (vals may be NULL) in place on `threads` threads.  Returns 0, or -1
 * if memory could not be allocated or the arguments are invalid. */
int pgs_cpu_stable_sort(void* keys, uint32_t* vals, uint64_t n, int key_bytes, int is_f32, int threads) {
  if ((key_bytes != 4 && key_bytes != 8) || (is_f32 && key_bytes != 4) || threads < 1) return -1;
  if (n < 2) return 0;
  if ((uint64_t)threads > n) threads = (int)n;
  uint64_t* ka = (uint64_t*)malloc(n * sizeof(uint64_t));
  uint64_t* kb = (uint64_t*)malloc(n * sizeof(uint64_t));
  uint32_t* vb = vals ? (uint32_t*)malloc(n * sizeof(uint32_t)) : NULL;
  if (!ka || !kb || (vals && !vb)) {
    free(ka); free(kb); free(vb);
    return -1;
  }
  for (uint64_t i = 0; i < n; ++i) {
    if (key_bytes == 8) ka[i] = ((const uint64_t*)keys)[i];
    else ka[i] = is_f32 ? f32_to_order(((const uint32_t*)keys)[i]) : ((const uint32_t*)keys)[i];
  }
  Job job;
  job.ka = ka; job.kb = kb; job.va = vals; job.vb = vb; job.n = n; job.T = threads;
  pthread_barrier_init(&job.bar, NULL, (unsigned)threads);
  pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * threads);
  Arg* args = (Arg*)malloc(sizeof(Arg) * threads);
  for (int t = 0; t < threads; ++t) {
    args[t].job = &job;
    args[t].t = t;
    if (t) pthread_create(&th[t], NULL, worker, &args[t]);
  }
  worker(&args[0]);
  for (int t = 1; t < threads; ++t) pthread_join(th[t], NULL);
  pthread_barrier_destroy(&job.bar);
  for (uint64_t i = 0; i < n; ++i) {
    if (key_bytes == 8) ((uint64_t*)keys)[i] = job.ka[i];
    else ((uint32_t*)keys)[i] = is_f32 ? order_to_f32(job.ka[i]) : (uint32_t)job.ka[i];
  }
  if (vals && job.va != vals) memcpy(vals, job.va, n * sizeof(uint32_t));
  free(ka); free(kb); free(vb); free(th); free(args);
  return 0;
}
