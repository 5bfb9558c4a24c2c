/*
 * Oracle (test infrastructure only): a plain parallel-for over [0, n), used
 * by the threaded form of the timed CPU baseline.  With one thread (the
 * default) it is the serial loop.  The range is cut into chunks of a fixed
 * size that the threads claim one at a time; the body receives the chunk's
 * index for per-chunk accumulators.  Callers only use it for loops whose
 * iterations are independent (leaves of a reaction sub-step, rows of an
 * operator application) and combine per-chunk results in chunk order, so the
 * results do not depend on the thread count or the schedule.
 */
#include "oracle.h"
#include <pthread.h>
#include <stdlib.h>

static int g_threads = 1;

void orc_set_threads(int t) { g_threads = t < 1 ? 1 : (t > 1024 ? 1024 : t); }
int orc_get_threads(void) { return g_threads; }

typedef struct {
  orc_body body;
  void *ctx;
  int64_t n, chunk;
  int64_t next; /* next chunk index, claimed atomically */
} pf_args;

static void *pf_worker(void *p) {
  pf_args *a = (pf_args *)p;
  const int64_t nchunks = (a->n + a->chunk - 1) / a->chunk;
  for (;;) {
    const int64_t c = __atomic_fetch_add(&a->next, 1, __ATOMIC_RELAXED);
    if (c >= nchunks) break;
    const int64_t lo = c * a->chunk, hi = lo + a->chunk < a->n ? lo + a->chunk : a->n;
    a->body(a->ctx, lo, hi, (int)c);
  }
  return NULL;
}

void orc_parallel_for(int64_t n, int64_t chunk, orc_body body, void *ctx) {
  if (chunk < 1) chunk = 1;
  int t = g_threads;
  if (t <= 1 || n <= chunk) {
    for (int64_t lo = 0, c = 0; lo < n; lo += chunk, c++) body(ctx, lo, lo + chunk < n ? lo + chunk : n, (int)c);
    return;
  }
  pf_args a = {body, ctx, n, chunk, 0};
  pthread_t *th = malloc(sizeof(pthread_t) * t);
  for (int q = 1; q < t; q++) pthread_create(&th[q], NULL, pf_worker, &a);
  pf_worker(&a);
  for (int q = 1; q < t; q++) pthread_join(th[q], NULL);
  free(th);
}
