/*
 * _gen.c -- fast fills for the seeded synthetic inputs (same definitions as
 * synth/__init__.py): SplitMix64 stream element i of seed s is
 * mix(s + (i+1) * 0x9E3779B97F4A7C15); uniform = lo + (hi-lo) * (u >> 11) * 2^-53;
 * normal = std * sqrt(-2 ln u1) cos(2 pi u2) with u1 = ((r[2i] >> 11) + 1) * 2^-53,
 * u2 = (r[2i+1] >> 11) * 2^-53.  Each value is rounded f64 -> f32 (-> bf16,
 * round to nearest even) straight into the storage array.  Element ranges are
 * split over threads; the stream is counter-based, so the split does not
 * change any value.  Input generation only: no part of the DAG method.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <string.h>

static inline uint64_t sm64(uint64_t seed, uint64_t i) {
  uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

static inline uint16_t f32_to_bf16(float f) {
  uint32_t b;
  memcpy(&b, &f, 4);
  uint32_t lsb = (b >> 16) & 1u;
  return (uint16_t)((b + 0x7FFFu + lsb) >> 16);
}

typedef struct {
  int kind;        /* 0 uniform, 1 normal */
  uint64_t seed;
  double a, b;     /* uniform lo, hi; normal std */
  int bf16;
  void *out;
  int64_t i0, i1;
} job_t;

static void *run(void *arg) {
  job_t *j = (job_t *)arg;
  const double twopi = 6.283185307179586;
  for (int64_t i = j->i0; i < j->i1; ++i) {
    double x;
    if (j->kind == 0) {
      double u = (double)(sm64(j->seed, (uint64_t)i) >> 11) * 0x1p-53;
      x = j->a + (j->b - j->a) * u;
    } else {
      double u1 = ((double)(sm64(j->seed, 2 * (uint64_t)i) >> 11) + 1.0) * 0x1p-53;
      double u2 = (double)(sm64(j->seed, 2 * (uint64_t)i + 1) >> 11) * 0x1p-53;
      x = j->a * (sqrt(-2.0 * log(u1)) * cos(twopi * u2));
    }
    float f = (float)x;
    if (j->bf16) ((uint16_t *)j->out)[i] = f32_to_bf16(f);
    else ((float *)j->out)[i] = f;
  }
  return 0;
}

/* fill n values; returns 0 */
int synth_fill(int kind, uint64_t seed, double a, double b, int64_t n, int bf16, void *out, int threads) {
  if (threads < 1) threads = 1;
  if (threads > 64) threads = 64;
  if (n < 1 << 16) threads = 1;
  pthread_t tid[64];
  job_t jobs[64];
  for (int t = 0; t < threads; ++t) {
    jobs[t].kind = kind; jobs[t].seed = seed; jobs[t].a = a; jobs[t].b = b; jobs[t].bf16 = bf16;
    jobs[t].out = out; jobs[t].i0 = n * t / threads; jobs[t].i1 = n * (t + 1) / threads;
  }
  for (int t = 1; t < threads; ++t) pthread_create(&tid[t], 0, run, &jobs[t]);
  run(&jobs[0]);
  for (int t = 1; t < threads; ++t) pthread_join(tid[t], 0);
  return 0;
}
