/*
 * gen.c — seeded synthetic task-set generator (the paper's §7.1 generator).
 *
 * This file is the only code shared by the CUDA path and the CPU oracle's
 * tests: it draws the inputs (periods, deadlines, WCET parameters a and b,
 * types, utilisations) and holds none of the method's arithmetic (no WCET
 * evaluation, no conflict rule, no test).
 *
 * Randomness is counter-based: draw(seed, set, k) is a SplitMix64 hash
 * (Steele, Lea, Flood, "Fast splittable pseudorandom number generators",
 * OOPSLA 2014) of the three counters, so every set is independent of the
 * others and of the thread that generates it.  Floating point is used only
 * for log-uniform sampling, through the deterministic log/exp below (basic
 * IEEE operations only, built with -ffp-contract=off), so x86 and Arm hosts
 * produce identical batches.
 *
 * Utilisations: the paper uses UUniFast-Discard (§7.1), whose output is the
 * uniform distribution on the simplex sum_i u_i = U.  We sample that same
 * distribution exactly in integers: n-1 uniform cut points in [0, U_ppm],
 * sorted, whose spacings are the task utilisations.  "Discard" redraws a set
 * whose largest utilisation exceeds u_max_ppm.
 */
#include "gpa.h"

#include <pthread.h>
#include <stdlib.h>
#include <string.h>

static const uint64_t kGolden = 0x9E3779B97F4A7C15ULL;
static const double kLn2 = 0.69314718055994530942;

static uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

static uint64_t draw(uint64_t seed, uint64_t set, uint64_t k) {
  uint64_t s = mix64(seed + kGolden);
  s = mix64(s + (set + 1) * kGolden);
  return mix64(s + (k + 1) * kGolden);
}

/* uniform double in [0, 1) with 53 random bits */
static double u01(uint64_t z) { return (double)(z >> 11) * (1.0 / 9007199254740992.0); }

/* uniform integer in [lo, hi] */
static int64_t uint_range(uint64_t z, int64_t lo, int64_t hi) {
  uint64_t span = (uint64_t)(hi - lo) + 1u;
  return lo + (int64_t)(uint64_t)(((unsigned __int128)z * span) >> 64);
}

/* natural log for x > 0: exact binary scaling to [1, 2), then
 * ln(m) = 2 atanh((m - 1) / (m + 1)) by its odd power series. */
static double det_log(double x) {
  int e = 0;
  while (x >= 2.0) { x *= 0.5; e++; }
  while (x < 1.0) { x *= 2.0; e--; }
  double z = (x - 1.0) / (x + 1.0);
  double z2 = z * z, term = z, sum = 0.0;
  for (int k = 0; k < 40; k++) {
    sum += term / (double)(2 * k + 1);
    term *= z2;
  }
  return (double)e * kLn2 + 2.0 * sum;
}

/* exp(y): y = k ln2 + f with f in [0, ln2), exp(f) by its Taylor series,
 * then exact binary scaling by 2^k. */
static double det_exp(double y) {
  double kf = 0.0;
  while (y - kf * kLn2 >= kLn2) kf += 1.0;
  while (y - kf * kLn2 < 0.0) kf -= 1.0;
  double f = y - kf * kLn2;
  double term = 1.0, sum = 1.0;
  for (int i = 1; i < 30; i++) {
    term *= f / (double)i;
    sum += term;
  }
  int k = (int)kf;
  while (k > 0) { sum *= 2.0; k--; }
  while (k < 0) { sum *= 0.5; k++; }
  return sum;
}

/* log-uniform integer in [lo, hi] */
static int64_t loguniform_int(uint64_t z, int64_t lo, int64_t hi) {
  double a = det_log((double)lo), b = det_log((double)hi + 1.0);
  double v = det_exp(a + u01(z) * (b - a));
  int64_t t = (int64_t)v;
  if (t < lo) t = lo;
  if (t > hi) t = hi;
  return t;
}

static void sort_i64(int64_t* v, int n) {
  for (int i = 1; i < n; i++) {
    int64_t x = v[i];
    int j = i - 1;
    while (j >= 0 && v[j] > x) { v[j + 1] = v[j]; j--; }
    v[j + 1] = x;
  }
}

static void sort_f64(double* v, int n) {
  for (int i = 1; i < n; i++) {
    double x = v[i];
    int j = i - 1;
    while (j >= 0 && v[j] > x) { v[j + 1] = v[j]; j--; }
    v[j + 1] = x;
  }
}

/* draw-key layout of one attempt */
enum { KEY_N = 0, KEY_U = 1, KEY_TASK0 = 16, KEY_TASK_STRIDE = 8, KEY_CUT0 = 1100, KEY_ATTEMPT = 4096 };

static int64_t set_size(const gpa_gen_params* p, int64_t s) {
  uint64_t z = draw(p->seed, (uint64_t)s, KEY_N);
  if (p->n_dist == GPA_DIST_LOGUNIFORM && p->n_min >= 1) return loguniform_int(z, p->n_min, p->n_max);
  return uint_range(z, p->n_min, p->n_max);
}

static int64_t set_U(const gpa_gen_params* p, int64_t s) {
  if (p->U_steps > 0) {
    if (p->U_steps == 1) return p->U_lo_ppm;
    int64_t step = (p->U_hi_ppm - p->U_lo_ppm) / (p->U_steps - 1);
    return p->U_lo_ppm + (s % p->U_steps) * step;
  }
  return uint_range(draw(p->seed, (uint64_t)s, KEY_U), p->U_lo_ppm, p->U_hi_ppm);
}

typedef struct {
  const gpa_gen_params* p;
  gpa_gen_out* out;
  const int64_t* divisors;
  int ndiv;
  int64_t s0, s1;
} gen_job;

static void gen_set(const gpa_gen_params* p, gpa_gen_out* out, const int64_t* divisors, int ndiv, int64_t s) {
  const int64_t off = out->set_off[s];
  const int n = (int)(out->set_off[s + 1] - off);
  const int64_t U = set_U(p, s);
  int64_t cuts[GPA_NMAX + 1], u[GPA_NMAX];
  int tries = p->max_tries > 0 ? p->max_tries : 1;
  uint8_t flag = 0;
  for (int t = 0; t < tries; t++) {
    uint64_t base = (uint64_t)t * KEY_ATTEMPT;
    for (int k = 0; k + 1 < n; k++) cuts[k] = uint_range(draw(p->seed, (uint64_t)s, base + KEY_CUT0 + k), 0, U);
    sort_i64(cuts, n > 0 ? n - 1 : 0);
    int64_t prev = 0, umax = 0;
    for (int i = 0; i < n; i++) {
      int64_t c = (i + 1 < n) ? cuts[i] : U;
      u[i] = c - prev;
      prev = c;
      if (u[i] > umax) umax = u[i];
    }
    for (int i = 0; i < n; i++) {
      uint64_t kb = base + KEY_TASK0 + (uint64_t)KEY_TASK_STRIDE * (uint64_t)i;
      int64_t T;
      if (p->T_dist == GPA_DIST_LIST && ndiv > 0)
        T = divisors[uint_range(draw(p->seed, (uint64_t)s, kb + 0), 0, ndiv - 1)];
      else
        T = loguniform_int(draw(p->seed, (uint64_t)s, kb + 0), p->T_lo, p->T_hi);
      int64_t D = T * (int64_t)p->deadline_pm / 1000;
      if (D < 1) D = 1;
      int64_t alpha = uint_range(draw(p->seed, (uint64_t)s, kb + 1), p->alpha_lo_pm, p->alpha_hi_pm);
      int64_t mu;
      if (p->mu_dist == GPA_DIST_BETA25) {
        double x[6];
        for (int r = 0; r < 6; r++) x[r] = u01(draw(p->seed, (uint64_t)s, kb + 2 + r));
        sort_f64(x, 6);
        mu = (int64_t)(x[1] * 1000.0);  /* 2nd order statistic of 6 uniforms ~ Beta(2, 5) */
      } else {
        mu = (int64_t)(u01(draw(p->seed, (uint64_t)s, kb + 2)) * 1000.0);
      }
      if (mu > 999) mu = 999;
      uint8_t type = (mu >= p->prm_pm) ? GPA_MEMORY : GPA_COMPUTE;
      int64_t C1 = (u[i] * T + 500000) / 1000000;  /* round half up */
      if (C1 < 1) C1 = 1;
      int64_t A, B;
      if (p->mode == GPA_GEN_PAPER) {
        A = 1000 * C1;
        B = (type == GPA_MEMORY ? p->beta_m_pm : p->beta_c_pm) * C1;
      } else {
        A = C1 * (1000 - alpha);
        B = C1 * alpha;
      }
      out->T[off + i] = T;
      out->D[off + i] = D;
      out->A[off + i] = A;
      out->B[off + i] = B;
      out->u_ppm[off + i] = C1 * 1000000 / T;
      out->type[off + i] = type;
      if (out->C1) out->C1[off + i] = C1;
      if (out->alpha_pm) out->alpha_pm[off + i] = (int16_t)alpha;
      if (out->mu_pm) out->mu_pm[off + i] = (int16_t)mu;
    }
    if (p->u_max_ppm <= 0 || umax <= p->u_max_ppm) { flag = 0; break; }
    flag = 1;
  }
  if (out->flags) out->flags[s] = flag;
}

static void* gen_worker(void* arg) {
  gen_job* j = (gen_job*)arg;
  for (int64_t s = j->s0; s < j->s1; s++) gen_set(j->p, j->out, j->divisors, j->ndiv, s);
  return NULL;
}

int32_t gpa_gen_tasksets(const gpa_gen_params* p, gpa_gen_out* out, int64_t* ntasks) {
  if (!p || !ntasks) return GPA_ERR_ARG;
  if (p->nsets < 0 || p->n_min < 0 || p->n_max < p->n_min || p->n_max > GPA_NMAX) return GPA_ERR_RANGE;
  if (p->U_lo_ppm < 0 || p->U_hi_ppm < p->U_lo_ppm || p->U_hi_ppm > 1000000000LL) return GPA_ERR_RANGE;
  if (p->T_lo < 1 || p->T_hi < p->T_lo || p->T_hi > 2147483647LL) return GPA_ERR_RANGE;
  if (p->deadline_pm < 1 || p->deadline_pm > 1000) return GPA_ERR_RANGE;
  if (p->alpha_lo_pm < 0 || p->alpha_hi_pm < p->alpha_lo_pm || p->alpha_hi_pm > 1000) return GPA_ERR_RANGE;
  if (p->U_steps < 0) return GPA_ERR_RANGE;
  if (p->mode != GPA_GEN_ALPHA && p->mode != GPA_GEN_PAPER) return GPA_ERR_ARG;
  if (p->mode == GPA_GEN_PAPER && (p->beta_c_pm < 0 || p->beta_m_pm < 0 || p->beta_c_pm > 1000000 || p->beta_m_pm > 1000000))
    return GPA_ERR_RANGE;

  int64_t total = 0;
  for (int64_t s = 0; s < p->nsets; s++) total += set_size(p, s);
  *ntasks = total;
  if (!out) return GPA_OK;
  if (!out->set_off || (total > 0 && (!out->T || !out->D || !out->A || !out->B || !out->u_ppm || !out->type)))
    return GPA_ERR_ARG;

  out->set_off[0] = 0;
  for (int64_t s = 0; s < p->nsets; s++) out->set_off[s + 1] = out->set_off[s] + set_size(p, s);

  int64_t* divisors = NULL;
  int ndiv = 0;
  if (p->T_dist == GPA_DIST_LIST) {
    divisors = (int64_t*)malloc(sizeof(int64_t) * 4096);
    if (!divisors) return GPA_ERR_NOMEM;
    for (int64_t d = p->T_lo; d <= p->T_hi && ndiv < 4096; d++)
      if (p->T_hi % d == 0) divisors[ndiv++] = d;
    if (ndiv == 0) { free(divisors); return GPA_ERR_RANGE; }
  }

  int nth = p->nthreads > 0 ? p->nthreads : 1;
  if (nth > 256) nth = 256;
  if ((int64_t)nth > p->nsets) nth = p->nsets > 0 ? (int)p->nsets : 1;
  gen_job jobs[256];
  pthread_t th[256];
  for (int t = 0; t < nth; t++) {
    jobs[t].p = p;
    jobs[t].out = out;
    jobs[t].divisors = divisors;
    jobs[t].ndiv = ndiv;
    jobs[t].s0 = p->nsets * t / nth;
    jobs[t].s1 = p->nsets * (t + 1) / nth;
  }
  int started = 0;
  for (int t = 1; t < nth; t++) {
    if (pthread_create(&th[t], NULL, gen_worker, &jobs[t]) != 0) break;
    started = t;
  }
  gen_worker(&jobs[0]);
  for (int t = 1; t <= started; t++) pthread_join(th[t], NULL);
  for (int t = started + 1; t < nth; t++) gen_worker(&jobs[t]);  /* threads that failed to start */
  free(divisors);
  return GPA_OK;
}
