/*
 * oracle.c — plain, slow, obviously-correct CPU oracle for the contention-
 * aware partition/allocation schedulability path of Zahaf et al.,
 * "Contention-Aware GPU Partitioning and Task-to-Partition Allocation for
 * Real-Time Workloads" (arXiv 2105.10312).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the package's smoke check
 * and the CPU-baseline leg of the benchmark load this library.  It shares no
 * code, header, table or helper with the CUDA path; it takes its inputs as
 * plain arrays (the seeded generator feeds both sides).
 *
 * Every function below follows one passage of the paper and is written as
 * that passage's definition, with explicit loops over tasks and 128-bit
 * intermediates so that no overflow or rounding question arises:
 *
 *   wcet()          §3.3 two-curve model with the §7.1 scaling function
 *                   C = k (a/m + b): ceil(k (A + B m) / (10^6 m))
 *   in_conflict()   §4.2 conflict rule (another task of the same type in
 *                   the partition)
 *   rta()           §5.5 per-partition test; policy = deadline-monotonic
 *                   fixed priority, classic response-time iteration
 *   edf()           the second policy (EDF), processor-demand criterion
 *                   over the first synchronous busy period
 *   minm_linear()   Alg. 2 (merge): first size in [lo, hi] that passes
 *   minm_binary()   the binary-search variant the text of §5.2 mentions
 *   lemma1()        Lemma 1 (necessary utilisation test)
 *   allocate_one()  Alg. 1 with Lemma 2 (init), Lemma 3 (exit), Alg. 3
 *                   (select_partitions), Def. 2 (valid merge), Def. 3 (SMS
 *                   order), Def. 4 (BF order), forbidden list (§5.3, ACT/INA)
 *   one_gpu()       the 1G baseline of §7.2 (all tasks, one partition of M)
 *   search_rgs()    exhaustive optimum over set partitions (subset form)
 *   search_explicit() the same optimum by brute force over every split of M
 *                   into k parts and every task-to-part map
 *
 * Readings where the paper is silent (each also listed in the design notes):
 * DM priority order (D, then T, then index); response time -1 on a miss;
 * Lemma 1 with floor(10^6 C^n(1) / T) summed against 10^6 M; par_list in
 * decreasing sum of u_ppm (ties: lower lowest task index); forbidden list =
 * failing task pairs (ACT) plus failing exact partition pairs; Def. 4's U
 * read as the m-independent inflated workload W(S) = sum k_i(S) u_ppm_i;
 * ACT evaluated only when the loop of Alg. 1 will run (Pi > M after init);
 * partitions reported in order of their lowest task index.
 *
 * Pin status: allocate_one()'s trajectory (which merges Alg. 1-3 make, in
 * which order) is parity unpinned against the paper, which prints no worked
 * run: its tests check invariants every reading satisfies and a second
 * coding of the same readings, so a reading that differs from the authors'
 * intent would pass them.  Every other function above is pinned by values
 * the paper or the mathematics fix (worked example, closed forms,
 * schedule simulation, brute force, published bounds).
 */
#include <pthread.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

typedef __int128 i128;

#define ONMAX 256       /* tasks per set */
#define OSERVE_NMAX 128 /* tasks per serving tenant */

enum { O_OK = 0, O_ERR_ARG = -1, O_ERR_RANGE = -2, O_ERR_NOMEM = -3 };
enum { R_OK = 0, R_LEMMA1 = 1, R_LEMMA2 = 2, R_NO_MERGE = 3, R_TEST = 4, R_INVALID = 5 };
enum { P_SMS = 0, P_BF = 1, P_ONE_GPU = 2 };

typedef struct {
  int n;
  const int64_t *T, *D, *A, *B, *u;
  const uint8_t* type;
} oset;

enum { S_DM = 0, S_EDF = 1 };

typedef struct {
  int64_t M, g, kc, km;
  int64_t sched; /* per-partition policy: S_DM (the reading of §5.5) or S_EDF */
  const int32_t* sizes; /* admissible partition sizes, increasing; NULL: every multiple of g */
  int64_t nsizes;
} omodel;

/* Is m an admissible partition size of the model?  Without a size list,
 * every multiple of g in [g, M] is (§4.1 with the unit g); with one, only
 * its members are (partitions of whole GPCs / MIG slices, §2). */
static int admissible(const omodel* md, int64_t m) {
  if (m < md->g || m > md->M) return 0;
  if (md->nsizes == 0) return m % md->g == 0;
  for (int64_t k = 0; k < md->nsizes; k++)
    if (md->sizes[k] == m) return 1;
  return 0;
}

/* The smallest admissible size. */
static int64_t smallest_size(const omodel* md) {
  return md->nsizes == 0 ? md->g : md->sizes[0];
}

static oset view(int64_t s, const int64_t* set_off, const int64_t* T, const int64_t* D, const int64_t* A,
                 const int64_t* B, const int64_t* u, const uint8_t* type) {
  oset v;
  int64_t o = set_off[s];
  v.n = (int)(set_off[s + 1] - o);
  v.T = T + o;
  v.D = D + o;
  v.A = A + o;
  v.B = B + o;
  v.u = u ? u + o : NULL;
  v.type = type + o;
  return v;
}

/* ------------------------------------------------------------------ model */

/* §3.3 / §7.1: C(m) = k (a/m + b), integer per-mille form, one ceiling of the
 * exact rational. */
static int64_t wcet(int64_t A, int64_t B, int64_t k, int64_t m) {
  i128 num = (i128)k * ((i128)A + (i128)B * (i128)m);
  i128 den = (i128)1000000 * (i128)m;
  return (int64_t)((num + den - 1) / den);
}

/* §4.2: task i of partition `in` is in conflict iff at least one other task
 * of the same type is in the partition. */
static int in_conflict(const oset* s, const unsigned char* in, int i) {
  int same = 0;
  for (int j = 0; j < s->n; j++)
    if (in[j] && s->type[j] == s->type[i]) same++;
  return same >= 2;
}

/* §4.2 / §7.1: k = 1 without conflict, k_c or k_m (per mille) with one. */
static int64_t kfactor(const oset* s, const omodel* md, const unsigned char* in, int i) {
  if (!in_conflict(s, in, i)) return 1000;
  return s->type[i] == 1 ? md->km : md->kc;
}

/* deadline-monotonic priority: does task j have higher priority than i? */
static int higher_prio(const oset* s, int j, int i) {
  if (s->D[j] != s->D[i]) return s->D[j] < s->D[i];
  if (s->T[j] != s->T[i]) return s->T[j] < s->T[i];
  return j < i;
}

/* Inflated workload of a partition: W(S) = sum_{i in S} k_i(S) u_i. */
static int64_t workload(const oset* s, const omodel* md, const unsigned char* in) {
  int64_t w = 0;
  for (int i = 0; i < s->n; i++)
    if (in[i]) w += kfactor(s, md, in, i) * s->u[i];
  return w;
}

/* §5.5: the partition `in` of m SMs, run as one processor under DM fixed
 * priorities with interference folded into the WCETs.  R[i] receives the
 * least fixed point of R = C_i + sum_{hp} ceil(R/T_j) C_j when it is <= D_i,
 * else -1.  Returns 1 iff every task of the partition meets its deadline. */
static int rta(const oset* s, const omodel* md, const unsigned char* in, int64_t m, int64_t* R) {
  int64_t C[ONMAX];
  for (int i = 0; i < s->n; i++)
    if (in[i]) C[i] = wcet(s->A[i], s->B[i], kfactor(s, md, in, i), m);
  int all = 1;
  for (int i = 0; i < s->n; i++) {
    if (!in[i]) continue;
    i128 r = C[i];
    for (int j = 0; j < s->n; j++)
      if (in[j] && j != i && higher_prio(s, j, i)) r += C[j];
    int ok;
    for (;;) {
      if (r > s->D[i]) { ok = 0; break; }
      i128 next = C[i];
      for (int j = 0; j < s->n; j++)
        if (in[j] && j != i && higher_prio(s, j, i)) next += ((r + s->T[j] - 1) / s->T[j]) * (i128)C[j];
      if (next == r) { ok = 1; break; }
      r = next;
    }
    if (R) R[i] = ok ? (int64_t)r : -1;
    if (!ok) all = 0;
  }
  return all;
}

/* Set when an analysis was refused (see edf); read and cleared by
 * orc_take_refused after each call. */
static int g_refused;
static void refuse(void) { __atomic_store_n(&g_refused, 1, __ATOMIC_RELAXED); }
int orc_take_refused(void) { return __atomic_exchange_n(&g_refused, 0, __ATOMIC_RELAXED); }

/* ------------------------------------------------ exact utilisation bound
 *
 * Multi-limb unsigned integers (little-endian 32-bit limbs), just enough to
 * decide sum_i C_i / T_i <= 1 exactly: with T_i < 2^32 and at most ONMAX
 * tasks the common denominator prod_i T_i has at most 32 ONMAX bits. */
#define BIG_LIMBS (ONMAX + 4)
typedef struct {
  int n; /* limbs in use; the value is 0 when n == 0 */
  uint32_t d[BIG_LIMBS];
} bigu;

static void big_set(bigu* a, uint32_t v) {
  a->n = v ? 1 : 0;
  a->d[0] = v;
}

/* out = a * x */
static void big_mul(bigu* out, const bigu* a, uint32_t x) {
  uint64_t carry = 0;
  int i;
  for (i = 0; i < a->n; i++) {
    uint64_t v = (uint64_t)a->d[i] * x + carry;
    out->d[i] = (uint32_t)v;
    carry = v >> 32;
  }
  out->n = a->n;
  if (carry) out->d[out->n++] = (uint32_t)carry;
  while (out->n > 0 && out->d[out->n - 1] == 0) out->n--;
}

/* a += b */
static void big_add(bigu* a, const bigu* b) {
  uint64_t carry = 0;
  int n = a->n > b->n ? a->n : b->n;
  for (int i = 0; i < n; i++) {
    uint64_t v = carry + (i < a->n ? a->d[i] : 0) + (i < b->n ? b->d[i] : 0);
    a->d[i] = (uint32_t)v;
    carry = v >> 32;
  }
  a->n = n;
  if (carry) a->d[a->n++] = (uint32_t)carry;
}

static int big_cmp(const bigu* a, const bigu* b) {
  if (a->n != b->n) return a->n < b->n ? -1 : 1;
  for (int i = a->n - 1; i >= 0; i--)
    if (a->d[i] != b->d[i]) return a->d[i] < b->d[i] ? -1 : 1;
  return 0;
}

/* Sign of U - 1 for U = sum over the k tasks idx[] of C_i / T_i, exactly:
 * the running fraction p / q takes each task as p <- p T_i + C_i q,
 * q <- q T_i, and the end compares p with q. */
static int utilisation_vs_one(const oset* s, const int64_t* C, const int* idx, int k) {
  bigu p, q, t;
  big_set(&p, 0);
  big_set(&q, 1);
  for (int a = 0; a < k; a++) {
    const int i = idx[a];
    if (s->T[i] < 1 || s->T[i] > (int64_t)UINT32_MAX || C[i] < 0 || C[i] > (int64_t)UINT32_MAX) {
      fprintf(stderr, "oracle edf: a period or WCET beyond 2^32, refusing\n");
      refuse();
      return 1;
    }
    big_mul(&t, &q, (uint32_t)C[i]);
    big_mul(&p, &p, (uint32_t)s->T[i]);
    big_add(&p, &t);
    big_mul(&q, &q, (uint32_t)s->T[i]);
  }
  return big_cmp(&p, &q);
}

/* Second per-partition policy (the paper leaves the policy of §5.5 open):
 * preemptive EDF on the partition as one processor, synchronous periodic
 * release, constrained deadlines.  Written as the processor-demand criterion
 * (Baruah, Rosier & Howell, 1990): every deadline is met iff U <= 1 and
 *     dbf(t) = sum_{D_i <= t} (floor((t - D_i) / T_i) + 1) C_i  <=  t
 * at every absolute deadline t up to the end L of the first synchronous busy
 * period (George, Rivierre & Spuri, 1996), the least fixed point of
 * w = sum_i ceil(w / T_i) C_i from w = sum_i C_i, which exists iff U <= 1
 * (at U = 1 it is the first instant the processor idles, a multiple of the
 * hyperperiod).  Every step is exact: U is compared with 1 as a fraction of
 * multi-limb integers, and the deadlines are enumerated one by one.  A task
 * with C > D misses at t = D (so one task passes iff C <= D).  The oracle
 * refuses a partition whose busy period passes 2^100 or whose deadlines
 * below it need more than 2^34 demand terms (its analysis would not end in
 * reasonable time): it prints a message, sets the refusal flag that
 * orc_take_refused() reports (the Python wrapper raises on it) and returns 0. */
static int edf(const oset* s, const omodel* md, const unsigned char* in, int64_t m) {
  int64_t C[ONMAX];
  int idx[ONMAX], k = 0;
  for (int i = 0; i < s->n; i++)
    if (in[i]) {
      C[i] = wcet(s->A[i], s->B[i], kfactor(s, md, in, i), m);
      idx[k++] = i;
    }
  if (k == 0) return 1;
  for (int a = 0; a < k; a++)
    if (C[idx[a]] > s->D[idx[a]]) return 0;
  if (utilisation_vs_one(s, C, idx, k) > 0) return 0;
  const i128 Lmax = (i128)1 << 100;
  i128 L = 0;
  for (int a = 0; a < k; a++) L += C[idx[a]];
  for (;;) {
    i128 next = 0;
    for (int a = 0; a < k; a++) {
      int i = idx[a];
      next += ((L + s->T[i] - 1) / s->T[i]) * (i128)C[i];
    }
    if (next == L) break;
    L = next;
    if (L > Lmax) {
      fprintf(stderr, "oracle edf: busy period beyond 2^100, refusing\n");
      refuse();
      return 0;
    }
  }
  i128 checks = 0;
  for (int a = 0; a < k; a++) checks += (L / s->T[idx[a]] + 1) * k;
  if (checks > ((i128)1 << 34)) {
    fprintf(stderr, "oracle edf: more than 2^34 demand terms below the busy period, refusing\n");
    refuse();
    return 0;
  }
  for (int a = 0; a < k; a++) {
    int i = idx[a];
    for (i128 t = s->D[i]; t <= L; t += s->T[i]) {
      i128 dbf = 0;
      for (int b = 0; b < k; b++) {
        int j = idx[b];
        if (s->D[j] <= t) dbf += ((t - s->D[j]) / s->T[j] + 1) * (i128)C[j];
      }
      if (dbf > t) return 0;
    }
  }
  return 1;
}

/* The per-partition test of the model's policy (verdict only). */
static int test(const oset* s, const omodel* md, const unsigned char* in, int64_t m) {
  return md->sched == S_EDF ? edf(s, md, in, m) : rta(s, md, in, m, NULL);
}

/* Alg. 2: the first admissible size m in [lo, hi] at which the merged task
 * set passes the test; 0 when none does. */
static int64_t minm_linear(const oset* s, const omodel* md, const unsigned char* in, int64_t lo, int64_t hi) {
  for (int64_t m = lo; m <= hi; m++)
    if (admissible(md, m) && test(s, md, in, m)) return m;
  return 0;
}

/* §5.2: the same answer by binary search (valid because the test is
 * monotone in m under the no-timing-anomaly hypothesis of §4.1). */
static int64_t minm_binary(const oset* s, const omodel* md, const unsigned char* in, int64_t lo, int64_t hi) {
  int64_t cand[1025];
  int nc = 0;
  for (int64_t m = lo; m <= hi && m <= 1024; m++)
    if (admissible(md, m)) cand[nc++] = m;
  if (nc == 0 || !test(s, md, in, cand[nc - 1])) return 0;
  int a = 0, b = nc - 1;
  while (a < b) {
    int mid = a + (b - a) / 2;
    if (test(s, md, in, cand[mid])) b = mid;
    else a = mid + 1;
  }
  return cand[a];
}

static int64_t minm(const oset* s, const omodel* md, const unsigned char* in, int64_t lo, int64_t hi, int linear) {
  return linear ? minm_linear(s, md, in, lo, hi) : minm_binary(s, md, in, lo, hi);
}

/* Lemma 1: the set is unschedulable if sum_i C^n_i(1) / T_i > M. */
static int lemma1_rejects(const oset* s, const omodel* md) {
  i128 sum = 0;
  for (int i = 0; i < s->n; i++) sum += ((i128)wcet(s->A[i], s->B[i], 1000, 1) * 1000000) / s->T[i];
  return sum > (i128)1000000 * md->M;
}

/* -------------------------------------------------------------- heuristic */

typedef struct {
  unsigned char in[ONMAX];
  int64_t m;
} opart;

typedef struct {
  unsigned char a[ONMAX], b[ONMAX];
} opair;

typedef struct {
  uint8_t verdict, reason;
  int32_t n_parts, Pi, n_tests;
  int64_t W;
} ores;

static int lowest_task(const unsigned char* in, int n) {
  for (int i = 0; i < n; i++)
    if (in[i]) return i;
  return n;
}

static int64_t usum(const oset* s, const unsigned char* in) {
  int64_t t = 0;
  for (int i = 0; i < s->n; i++)
    if (in[i]) t += s->u[i];
  return t;
}

/* par_list order: decreasing utilisation, ties by lower lowest task index */
static int before_in_par_list(const oset* s, const opart* x, const opart* y) {
  int64_t ux = usum(s, x->in), uy = usum(s, y->in);
  if (ux != uy) return ux > uy;
  return lowest_task(x->in, s->n) < lowest_task(y->in, s->n);
}

static void sort_par_list(const oset* s, opart* list, int np) {
  for (int i = 1; i < np; i++) {
    opart x = list[i];
    int j = i - 1;
    while (j >= 0 && before_in_par_list(s, &x, &list[j])) { list[j + 1] = list[j]; j--; }
    list[j + 1] = x;
  }
}

static int same_tasks(const unsigned char* a, const unsigned char* b, int n) { return memcmp(a, b, (size_t)n) == 0; }

typedef struct {
  opair* v;
  int len, cap;
} pairlist;

static int pairlist_add(pairlist* pl, const unsigned char* a, const unsigned char* b) {
  if (pl->len == pl->cap) {
    int nc = pl->cap ? 2 * pl->cap : 64;
    opair* nv = (opair*)realloc(pl->v, sizeof(opair) * (size_t)nc);
    if (!nv) return 0;
    pl->v = nv;
    pl->cap = nc;
  }
  memcpy(pl->v[pl->len].a, a, ONMAX);
  memcpy(pl->v[pl->len].b, b, ONMAX);
  pl->len++;
  return 1;
}

/* §5.3 and Alg. 3: is the merge of P and Q forbidden? */
static int forbidden(const oset* s, const pairlist* pl, unsigned char act_pair[ONMAX][ONMAX], const opart* P,
                     const opart* Q) {
  for (int k = 0; k < pl->len; k++) {
    if (same_tasks(pl->v[k].a, P->in, s->n) && same_tasks(pl->v[k].b, Q->in, s->n)) return 1;
    if (same_tasks(pl->v[k].a, Q->in, s->n) && same_tasks(pl->v[k].b, P->in, s->n)) return 1;
  }
  for (int i = 0; i < s->n; i++)
    for (int j = 0; j < s->n; j++)
      if (P->in[i] && Q->in[j] && act_pair[i][j]) return 1;
  return 0;
}

static void union_of(const opart* P, const opart* Q, unsigned char* out, int n) {
  for (int i = 0; i < n; i++) out[i] = (unsigned char)(P->in[i] || Q->in[i]);
}

/* replace list[a] and list[b] by the merged partition (in, m) */
static int apply_merge(opart* list, int np, int a, int b, const unsigned char* in, int64_t m) {
  opart merged;
  memset(&merged, 0, sizeof merged);
  memcpy(merged.in, in, ONMAX);
  merged.m = m;
  opart keep[ONMAX];
  int k = 0;
  for (int i = 0; i < np; i++)
    if (i != a && i != b) keep[k++] = list[i];
  keep[k++] = merged;
  for (int i = 0; i < k; i++) list[i] = keep[i];
  return k;
}

static void write_partitions(const oset* s, const omodel* md, opart* list, int np, ores* r, uint8_t* part_of_task,
                             int16_t* size_of_part) {
  /* report partitions in increasing order of their lowest task index */
  opart sorted[ONMAX];
  for (int i = 0; i < np; i++) sorted[i] = list[i];
  for (int i = 1; i < np; i++) {
    opart x = sorted[i];
    int j = i - 1;
    while (j >= 0 && lowest_task(sorted[j].in, s->n) > lowest_task(x.in, s->n)) { sorted[j + 1] = sorted[j]; j--; }
    sorted[j + 1] = x;
  }
  int64_t Pi = 0, W = 0;
  for (int p = 0; p < np; p++) {
    Pi += sorted[p].m;
    W += workload(s, md, sorted[p].in);
    for (int i = 0; i < s->n; i++)
      if (sorted[p].in[i]) part_of_task[i] = (uint8_t)p;
    size_of_part[p] = (int16_t)sorted[p].m;
  }
  r->n_parts = np;
  r->Pi = (int32_t)Pi;
  r->W = W;
}

/* Alg. 1 (partition and allocate) for one task set. */
static int allocate_one(const oset* s, const omodel* md, int policy, int act, int linear, ores* r,
                        uint8_t* part_of_task, int16_t* size_of_part) {
  const int n = s->n;
  memset(r, 0, sizeof *r);
  for (int i = 0; i < n; i++) { part_of_task[i] = 255; size_of_part[i] = 0; }

  /* Lemma 1, applied before the heuristic starts */
  if (lemma1_rejects(s, md)) { r->reason = R_LEMMA1; return O_OK; }

  /* init_partitions: one partition per task at its Lemma 2 size */
  static __thread opart list[ONMAX];
  int np = n;
  int64_t Pi = 0;
  for (int i = 0; i < n; i++) {
    memset(&list[i], 0, sizeof(opart));
    list[i].in[i] = 1;
    list[i].m = minm_linear(s, md, list[i].in, md->g, md->M);
    if (list[i].m == 0) { r->reason = R_LEMMA2; return O_OK; }
    Pi += list[i].m;
  }

  static __thread unsigned char act_pair[ONMAX][ONMAX];
  memset(act_pair, 0, sizeof act_pair);
  pairlist pl = {NULL, 0, 0};
  int tests = 0;

  /* ACT: test every task pair, forbid those that cannot merge */
  if (act && Pi > md->M) {
    for (int i = 0; i < n; i++)
      for (int j = i + 1; j < n; j++) {
        opart a = list[i], b = list[j];
        unsigned char in[ONMAX];
        union_of(&a, &b, in, n);
        int64_t lo = a.m > b.m ? a.m : b.m;
        int64_t hi = a.m + b.m - 1;
        tests++;
        if (minm(s, md, in, lo, hi, linear) == 0) act_pair[i][j] = act_pair[j][i] = 1;
      }
  }

  int status = O_OK;
  while (Pi > md->M) {
    sort_par_list(s, list, np);
    /* Alg. 3: first partition (in par_list order) with a non-empty eligible list */
    int p1 = -1;
    int elig[ONMAX], ne = 0;
    for (int c = 0; c < np && p1 < 0; c++) {
      ne = 0;
      for (int e = 0; e < np; e++)
        if (e != c && !forbidden(s, &pl, act_pair, &list[c], &list[e])) elig[ne++] = e;
      if (ne > 0) p1 = c;
    }
    if (p1 < 0) { r->reason = R_NO_MERGE; break; }

    unsigned char in[ONMAX];
    if (policy == P_SMS) {
      /* Def. 3: every candidate merge is computed; the smallest merged size wins,
       * ties to the earlier par_list position */
      int best = -1;
      int64_t best_m = 0;
      for (int k = 0; k < ne; k++) {
        const opart* Q = &list[elig[k]];
        union_of(&list[p1], Q, in, n);
        int64_t lo = list[p1].m > Q->m ? list[p1].m : Q->m;
        int64_t hi = list[p1].m + Q->m - 1;
        int64_t m3 = minm(s, md, in, lo, hi, linear);
        tests++;
        if (m3 > 0 && (best < 0 || m3 < best_m)) { best = elig[k]; best_m = m3; }
      }
      if (best >= 0) {
        union_of(&list[p1], &list[best], in, n);
        Pi -= list[p1].m + list[best].m - best_m;
        np = apply_merge(list, np, p1, best, in, best_m);
      } else {
        for (int k = 0; k < ne; k++)
          if (!pairlist_add(&pl, list[p1].in, list[elig[k]].in)) { status = O_ERR_NOMEM; goto done; }
      }
    } else {
      /* Def. 4: eligible partitions sorted by the workload of the merge, ties
       * to the earlier par_list position; tried in that order */
      int64_t w[ONMAX];
      for (int k = 0; k < ne; k++) {
        union_of(&list[p1], &list[elig[k]], in, n);
        w[k] = workload(s, md, in);
      }
      for (int i = 1; i < ne; i++) {
        int xe = elig[i];
        int64_t xw = w[i];
        int j = i - 1;
        while (j >= 0 && w[j] > xw) { elig[j + 1] = elig[j]; w[j + 1] = w[j]; j--; }
        elig[j + 1] = xe;
        w[j + 1] = xw;
      }
      for (int k = 0; k < ne; k++) {
        const opart* Q = &list[elig[k]];
        union_of(&list[p1], Q, in, n);
        int64_t lo = list[p1].m > Q->m ? list[p1].m : Q->m;
        int64_t hi = list[p1].m + Q->m - 1;
        int64_t m3 = minm(s, md, in, lo, hi, linear);
        tests++;
        if (m3 > 0) {
          Pi -= list[p1].m + Q->m - m3;
          np = apply_merge(list, np, p1, elig[k], in, m3);
          break;
        }
        if (!pairlist_add(&pl, list[p1].in, Q->in)) { status = O_ERR_NOMEM; goto done; }
      }
    }
  }
  if (Pi <= md->M) { r->verdict = 1; r->reason = R_OK; }
  write_partitions(s, md, list, np, r, part_of_task, size_of_part);
done:
  r->n_tests = tests;
  free(pl.v);
  return status;
}

/* §7.2 1G baseline: the GPU as one non-partitioned resource. */
static void one_gpu(const oset* s, const omodel* md, ores* r, uint8_t* part_of_task, int16_t* size_of_part) {
  unsigned char in[ONMAX];
  memset(r, 0, sizeof *r);
  for (int i = 0; i < s->n; i++) { in[i] = 1; part_of_task[i] = 0; size_of_part[i] = 0; }
  r->n_tests = 1;
  if (s->n == 0) { r->verdict = 1; r->reason = R_OK; return; }
  int ok = test(s, md, in, md->M);
  r->verdict = (uint8_t)ok;
  r->reason = ok ? R_OK : R_TEST;
  r->n_parts = 1;
  r->Pi = (int32_t)md->M;
  r->W = workload(s, md, in);
  size_of_part[0] = (int16_t)md->M;
}

/* ------------------------------------------------------ exhaustive optimum */

typedef struct {
  int found;
  int64_t W;
  int64_t sum_minm;
  int nb;
  unsigned char rgs[ONMAX];
  int64_t minm_block[8];
} obest;

/* key order: W, then sum of block minimum sizes, then the RGS lexicographically */
static int key_less(int64_t W, int64_t sm, const unsigned char* rgs, const obest* b, int n) {
  if (!b->found) return 1;
  if (W != b->W) return W < b->W;
  if (sm != b->sum_minm) return sm < b->sum_minm;
  for (int i = 0; i < n; i++)
    if (rgs[i] != b->rgs[i]) return rgs[i] < b->rgs[i];
  return 0;
}

typedef struct {
  const oset* s;
  const omodel* md;
  int kmin, kmax;
  const int64_t* minm_sub;  /* [2^n] */
  const int64_t* W_sub;     /* [2^n] */
  unsigned char rgs[ONMAX];
  obest* best;
} rgs_walk;

static void rgs_leaf(rgs_walk* w) {
  const int n = w->s->n;
  int nb = 0;
  for (int i = 0; i < n; i++)
    if (w->rgs[i] + 1 > nb) nb = w->rgs[i] + 1;
  uint32_t mask[8] = {0};
  for (int i = 0; i < n; i++) mask[w->rgs[i]] |= 1u << i;
  int64_t sm = 0, W = 0;
  for (int b = 0; b < nb; b++) {
    if (w->minm_sub[mask[b]] == 0) return;
    sm += w->minm_sub[mask[b]];
    W += w->W_sub[mask[b]];
  }
  int64_t empty = w->kmin > nb ? (int64_t)(w->kmin - nb) : 0;
  if (sm + empty * smallest_size(w->md) > w->md->M) return;
  if (key_less(W, sm, w->rgs, w->best, n)) {
    w->best->found = 1;
    w->best->W = W;
    w->best->sum_minm = sm;
    w->best->nb = nb;
    memcpy(w->best->rgs, w->rgs, (size_t)n);
    for (int b = 0; b < 8; b++) w->best->minm_block[b] = b < nb ? w->minm_sub[mask[b]] : 0;
  }
}

/* every restricted-growth string a_0..a_{n-1} with a_0 = 0 and
 * a_i <= 1 + max(a_0..a_{i-1}), using at most kmax blocks */
static void rgs_rec(rgs_walk* w, int i, int used) {
  if (i == w->s->n) { rgs_leaf(w); return; }
  int top = used < w->kmax ? used : w->kmax - 1;
  for (int b = 0; b <= top; b++) {
    w->rgs[i] = (unsigned char)b;
    rgs_rec(w, i + 1, b + 1 > used ? b + 1 : used);
  }
}

static void mask_to_in(uint32_t mask, int n, unsigned char* in) {
  for (int i = 0; i < n; i++) in[i] = (unsigned char)((mask >> i) & 1u);
}

/* Optimum via subsets: the minimum size and workload of every non-empty
 * subset of tasks, then every set partition into at most kmax blocks. */
static int search_rgs(const oset* s, const omodel* md, int kmin, int kmax, obest* best) {
  const int n = s->n;
  memset(best, 0, sizeof *best);
  if (n == 0) {
    /* no tasks: the empty partition, realisable iff kmin parts fit */
    int64_t need = (int64_t)kmin * smallest_size(md);
    if (need <= md->M) { best->found = 1; best->nb = 0; }
    return O_OK;
  }
  size_t nsub = (size_t)1 << n;
  int64_t* minm_sub = (int64_t*)calloc(nsub, sizeof(int64_t));
  int64_t* W_sub = (int64_t*)calloc(nsub, sizeof(int64_t));
  if (!minm_sub || !W_sub) { free(minm_sub); free(W_sub); return O_ERR_NOMEM; }
  unsigned char in[ONMAX];
  for (size_t mask = 1; mask < nsub; mask++) {
    mask_to_in((uint32_t)mask, n, in);
    minm_sub[mask] = minm_linear(s, md, in, md->g, md->M);
    W_sub[mask] = workload(s, md, in);
  }
  rgs_walk w;
  memset(&w, 0, sizeof w);
  w.s = s;
  w.md = md;
  w.kmin = kmin;
  w.kmax = kmax;
  w.minm_sub = minm_sub;
  w.W_sub = W_sub;
  w.best = best;
  rgs_rec(&w, 1, 1); /* task 0 is always in block 0 */
  free(minm_sub);
  free(W_sub);
  return O_OK;
}

/* Optimum by brute force: every composition of M/g into k parts (k in
 * [kmin, kmax]; with a size list: every k admissible sizes of sum <= M)
 * times every map of tasks to parts; a candidate is feasible iff every
 * non-empty part passes the test at its size. */
typedef struct {
  const oset* s;
  const omodel* md;
  int kmin, kmax, k;
  int64_t parts[8];
  obest* best;
  int64_t candidates;
} explicit_walk;

static void explicit_candidates(explicit_walk* w) {
  const oset* s = w->s;
  const int n = s->n, k = w->k;
  int64_t nmaps = 1;
  for (int i = 0; i < n; i++) nmaps *= k;
  unsigned char map[ONMAX], in[ONMAX];
  for (int64_t code = 0; code < nmaps; code++) {
    int64_t c = code;
    for (int i = 0; i < n; i++) { map[i] = (unsigned char)(c % k); c /= k; }
    w->candidates++;
    int feasible = 1;
    for (int p = 0; p < k && feasible; p++) {
      int any = 0;
      for (int i = 0; i < n; i++) { in[i] = map[i] == p; any |= in[i]; }
      if (any && !test(s, w->md, in, w->parts[p])) feasible = 0;
    }
    if (!feasible) continue;
    /* induced set partition, blocks relabelled by first occurrence */
    int label[8];
    for (int p = 0; p < 8; p++) label[p] = -1;
    int nb = 0;
    unsigned char rgs[ONMAX];
    for (int i = 0; i < n; i++) {
      if (label[map[i]] < 0) label[map[i]] = nb++;
      rgs[i] = (unsigned char)label[map[i]];
    }
    int64_t W = 0, sm = 0, mb[8] = {0};
    for (int b = 0; b < nb; b++) {
      for (int i = 0; i < n; i++) in[i] = rgs[i] == b;
      W += workload(s, w->md, in);
      mb[b] = minm_linear(s, w->md, in, w->md->g, w->md->M);
      sm += mb[b];
    }
    if (key_less(W, sm, rgs, w->best, n)) {
      w->best->found = 1;
      w->best->W = W;
      w->best->sum_minm = sm;
      w->best->nb = nb;
      memcpy(w->best->rgs, rgs, (size_t)n);
      for (int b = 0; b < 8; b++) w->best->minm_block[b] = mb[b];
    }
  }
}

/* parts in SMs; `left` in units of g (exact sums) */
static void compositions(explicit_walk* w, int part, int64_t left) {
  if (part == w->k - 1) {
    w->parts[part] = left * w->md->g;
    explicit_candidates(w);
    return;
  }
  for (int64_t v = 1; v <= left - (w->k - 1 - part); v++) {
    w->parts[part] = v * w->md->g;
    compositions(w, part + 1, left - v);
  }
}

/* with a size list: every admissible size for each part, sum <= M (`left`
 * in SMs) */
static void admissible_splits(explicit_walk* w, int part, int64_t left) {
  const int64_t zmin = smallest_size(w->md);
  for (int64_t k = 0; k < w->md->nsizes; k++) {
    const int64_t v = w->md->sizes[k];
    if (v + (int64_t)(w->k - 1 - part) * zmin > left) break;
    w->parts[part] = v;
    if (part == w->k - 1) explicit_candidates(w);
    else admissible_splits(w, part + 1, left - v);
  }
}

static int64_t search_explicit(const oset* s, const omodel* md, int kmin, int kmax, obest* best) {
  memset(best, 0, sizeof *best);
  explicit_walk w;
  memset(&w, 0, sizeof w);
  w.s = s;
  w.md = md;
  w.kmin = kmin;
  w.kmax = kmax;
  w.best = best;
  int64_t Mu = md->M / md->g;
  for (int k = kmin; k <= kmax; k++) {
    if (k > Mu) break;
    w.k = k;
    if (md->nsizes == 0) compositions(&w, 0, Mu);
    else admissible_splits(&w, 0, md->M);
  }
  return w.candidates;
}

/* ------------------------------------------------------------ validation */

/* The library's input bounds.  Model: 1 <= g, g | M, 1 <= M <= 1024, an
 * increasing size list of multiples of g in [g, M], DM or EDF, factors in
 * [1000, 16000] per mille.  Task: 1 <= D <= T <= 2^31 - 1, A, B >= 0,
 * 1 <= A + B <= 2^36, 0 <= u_ppm < 2^32, type 0 or 1.  A set with a task
 * outside them is marked invalid; a model outside them fails the call. */
static int valid_model(const omodel* md) {
  if (md->g < 1 || md->M < 1 || md->M > 1024 || md->M % md->g != 0) return 0;
  if (md->sched != S_DM && md->sched != S_EDF) return 0;
  if (md->nsizes < 0 || md->nsizes > 1024 || (md->nsizes > 0 && !md->sizes)) return 0;
  for (int64_t k = 0; k < md->nsizes; k++) {
    const int64_t z = md->sizes[k];
    if (z < md->g || z > md->M || z % md->g != 0 || (k > 0 && z <= md->sizes[k - 1])) return 0;
  }
  if (md->kc < 1000 || md->kc > 16000 || md->km < 1000 || md->km > 16000) return 0;
  return 1;
}

static int valid_set(const oset* s) {
  if (s->n < 0 || s->n > ONMAX) return 0;
  for (int i = 0; i < s->n; i++) {
    if (s->D[i] < 1 || s->D[i] > s->T[i] || s->T[i] > 2147483647LL) return 0;
    if (s->A[i] < 0 || s->B[i] < 0 || s->A[i] + s->B[i] < 1 || s->A[i] + s->B[i] > ((int64_t)1 << 36)) return 0;
    if (s->u && (s->u[i] < 0 || s->u[i] >= ((int64_t)1 << 32))) return 0;
    if (s->type[i] > 1) return 0;
  }
  return 1;
}

/* ------------------------------------------------------- exported batch API */

typedef struct {
  const int64_t *set_off, *T, *D, *A, *B, *u;
  const uint8_t* type;
} obatch;

int orc_wcet(int64_t A, int64_t B, int64_t k, int64_t m, int64_t* out) {
  if (m < 1 || !out) return O_ERR_ARG;
  *out = wcet(A, B, k, m);
  return O_OK;
}

/* WCET tables, layout [set][m-index][task] (same as the library). */
int orc_wcet_tables(int64_t nsets, const int64_t* set_off, const int64_t* A, const int64_t* B, const uint8_t* type,
                    int64_t M, int64_t g, int64_t kc, int64_t km, int64_t* Cn, int64_t* Cc) {
  int64_t Mu = M / g;
  for (int64_t s = 0; s < nsets; s++) {
    int64_t o = set_off[s], n = set_off[s + 1] - o;
    for (int64_t mi = 0; mi < Mu; mi++)
      for (int64_t t = 0; t < n; t++) {
        int64_t m = g * (mi + 1);
        int64_t kx = type[o + t] == 1 ? km : kc;
        Cn[o * Mu + mi * n + t] = wcet(A[o + t], B[o + t], 1000, m);
        Cc[o * Mu + mi * n + t] = wcet(A[o + t], B[o + t], kx, m);
      }
  }
  return O_OK;
}

/* One partition: the per-task response times of the tasks selected by
 * in_mask (bytes) at m SMs.  Returns the verdict (0/1). */
int orc_rta(int n, const int64_t* T, const int64_t* D, const int64_t* A, const int64_t* B, const uint8_t* type,
            const uint8_t* in_mask, int64_t m, int64_t kc, int64_t km, int64_t* R) {
  oset s = {n, T, D, A, B, NULL, type};
  omodel md = {1024, 1, kc, km, S_DM, NULL, 0};
  unsigned char in[ONMAX];
  for (int i = 0; i < n; i++) in[i] = in_mask[i] ? 1 : 0;
  return rta(&s, &md, in, m, R);
}

/* One partition under EDF at m SMs: the verdict (0/1). */
int orc_edf(int n, const int64_t* T, const int64_t* D, const int64_t* A, const int64_t* B, const uint8_t* type,
            const uint8_t* in_mask, int64_t m, int64_t kc, int64_t km) {
  oset s = {n, T, D, A, B, NULL, type};
  omodel md = {1024, 1, kc, km, S_EDF, NULL, 0};
  unsigned char in[ONMAX];
  for (int i = 0; i < n; i++) in[i] = in_mask[i] ? 1 : 0;
  return edf(&s, &md, in, m);
}

int orc_minm(int n, const int64_t* T, const int64_t* D, const int64_t* A, const int64_t* B, const uint8_t* type,
             const uint8_t* in_mask, int64_t lo, int64_t hi, int64_t g, int64_t kc, int64_t km, int64_t sched,
             const int32_t* sizes, int64_t nsizes, int linear, int64_t* out) {
  oset s = {n, T, D, A, B, NULL, type};
  omodel md = {hi, g, kc, km, sched, sizes, nsizes};
  unsigned char in[ONMAX];
  for (int i = 0; i < n; i++) in[i] = in_mask[i] ? 1 : 0;
  *out = minm(&s, &md, in, lo, hi, linear);
  return O_OK;
}

int orc_workload(int n, const int64_t* u, const uint8_t* type, const uint8_t* in_mask, int64_t kc, int64_t km,
                 int64_t* out) {
  int64_t zeros[ONMAX] = {0};
  oset s = {n, zeros, zeros, zeros, zeros, u, type};
  omodel md = {1024, 1, kc, km, S_DM, NULL, 0};
  unsigned char in[ONMAX];
  for (int i = 0; i < n; i++) in[i] = in_mask[i] ? 1 : 0;
  *out = workload(&s, &md, in);
  return O_OK;
}

int orc_lemma1_rejects(int n, const int64_t* T, const int64_t* A, const int64_t* B, int64_t M) {
  oset s = {n, T, T, A, B, NULL, NULL};
  omodel md = {M, 1, 1000, 1000, S_DM, NULL, 0};
  return lemma1_rejects(&s, &md);
}

int orc_test_schedulable(int64_t nsets, const int64_t* set_off, const int64_t* T, const int64_t* D, const int64_t* A,
                         const int64_t* B, const uint8_t* type, int64_t M, int64_t g, int64_t kc, int64_t km,
                         int64_t sched, const int32_t* sizes, int64_t nsizes, int64_t ncands,
                         const int64_t* cand_set, const uint8_t* part_of_task, int64_t map_stride, int64_t kparts,
                         const int32_t* size_of_part, uint8_t* verdict, int64_t* R) {
  omodel md = {M, g, kc, km, sched, sizes, nsizes};
  if (!valid_model(&md) || kparts < 1 || kparts > 255) return O_ERR_RANGE;
  for (int64_t c = 0; c < ncands; c++) {
    int64_t si = cand_set[c];
    if (si < 0 || si >= nsets) return O_ERR_RANGE;
    oset s = view(si, set_off, T, D, A, B, NULL, type);
    if (!valid_set(&s) || s.n > map_stride) return O_ERR_RANGE;
    const uint8_t* map = part_of_task + c * map_stride;
    const int32_t* size = size_of_part + c * kparts;
    int64_t total = 0;
    for (int64_t p = 0; p < kparts; p++) {
      if (size[p] != 0 && !admissible(&md, size[p])) return O_ERR_RANGE;
      total += size[p];
    }
    for (int i = 0; i < s.n; i++)
      if (map[i] >= kparts) return O_ERR_RANGE;
    int ok = total <= M;
    int64_t Rt[ONMAX];
    for (int i = 0; i < s.n; i++) Rt[i] = -1;
    for (int64_t p = 0; p < kparts; p++) {
      unsigned char in[ONMAX];
      int any = 0;
      for (int i = 0; i < s.n; i++) { in[i] = map[i] == p; any |= in[i]; }
      if (!any) continue;
      if (size[p] == 0) { ok = 0; continue; }
      if (md.sched == S_EDF) {
        /* EDF gives no response times: 0 for the tasks of a passing part */
        int pass = edf(&s, &md, in, size[p]);
        for (int i = 0; i < s.n; i++)
          if (in[i]) Rt[i] = pass ? 0 : -1;
        if (!pass) ok = 0;
      } else if (!rta(&s, &md, in, size[p], Rt)) {
        ok = 0;
      }
    }
    verdict[c] = (uint8_t)ok;
    if (R)
      for (int i = 0; i < s.n; i++) R[c * map_stride + i] = Rt[i];
  }
  return O_OK;
}

typedef struct {
  obatch b;
  omodel md;
  int policy, act, linear;
  int64_t s0, s1;
  uint8_t *verdict, *reason, *part_of_task;
  int32_t *n_parts, *Pi, *n_tests;
  int64_t* W;
  int16_t* size_of_part;
  int status;
} alloc_job;

static void* alloc_worker(void* arg) {
  alloc_job* j = (alloc_job*)arg;
  for (int64_t si = j->s0; si < j->s1; si++) {
    oset s = view(si, j->b.set_off, j->b.T, j->b.D, j->b.A, j->b.B, j->b.u, j->b.type);
    int64_t o = j->b.set_off[si];
    ores r;
    memset(&r, 0, sizeof r);
    if (!valid_set(&s)) {
      r.reason = R_INVALID;
      for (int i = 0; i < s.n && i < ONMAX; i++) { j->part_of_task[o + i] = 255; j->size_of_part[o + i] = 0; }
    } else if (j->policy == P_ONE_GPU) {
      one_gpu(&s, &j->md, &r, j->part_of_task + o, j->size_of_part + o);
    } else {
      int st = allocate_one(&s, &j->md, j->policy, j->act, j->linear, &r, j->part_of_task + o, j->size_of_part + o);
      if (st != O_OK) j->status = st;
    }
    j->verdict[si] = r.verdict;
    j->reason[si] = r.reason;
    j->n_parts[si] = r.n_parts;
    j->Pi[si] = r.Pi;
    j->W[si] = r.W;
    if (j->n_tests) j->n_tests[si] = r.n_tests;
  }
  return NULL;
}

static int run_threads(void* (*fn)(void*), void* jobs, size_t job_size, int nth) {
  pthread_t th[256];
  int started = 0;
  for (int t = 1; t < nth; t++) {
    if (pthread_create(&th[t], NULL, fn, (char*)jobs + job_size * (size_t)t) != 0) break;
    started = t;
  }
  fn(jobs);
  for (int t = 1; t <= started; t++) pthread_join(th[t], NULL);
  for (int t = started + 1; t < nth; t++) fn((char*)jobs + job_size * (size_t)t);
  return O_OK;
}

int orc_allocate(int64_t nsets, const int64_t* set_off, const int64_t* T, const int64_t* D, const int64_t* A,
                 const int64_t* B, const int64_t* u, const uint8_t* type, int64_t M, int64_t g, int64_t kc,
                 int64_t km, int64_t sched, const int32_t* sizes, int64_t nsizes, int policy, int act, int linear,
                 uint8_t* verdict, uint8_t* reason, int32_t* n_parts, int32_t* Pi, int64_t* W, int32_t* n_tests,
                 uint8_t* part_of_task, int16_t* size_of_part, int nthreads) {
  omodel md = {M, g, kc, km, sched, sizes, nsizes};
  if (!valid_model(&md)) return O_ERR_RANGE;
  if (policy < P_SMS || policy > P_ONE_GPU) return O_ERR_ARG;
  int nth = nthreads < 1 ? 1 : (nthreads > 256 ? 256 : nthreads);
  if (nsets < nth) nth = nsets > 0 ? (int)nsets : 1;
  alloc_job* jobs = (alloc_job*)calloc((size_t)nth, sizeof(alloc_job));
  if (!jobs) return O_ERR_NOMEM;
  for (int t = 0; t < nth; t++) {
    alloc_job* j = &jobs[t];
    j->b = (obatch){set_off, T, D, A, B, u, type};
    j->md = md;
    j->policy = policy;
    j->act = act;
    j->linear = linear;
    j->s0 = nsets * t / nth;
    j->s1 = nsets * (t + 1) / nth;
    j->verdict = verdict;
    j->reason = reason;
    j->n_parts = n_parts;
    j->Pi = Pi;
    j->W = W;
    j->n_tests = n_tests;
    j->part_of_task = part_of_task;
    j->size_of_part = size_of_part;
  }
  run_threads(alloc_worker, jobs, sizeof(alloc_job), nth);
  int st = O_OK;
  for (int t = 0; t < nth; t++)
    if (jobs[t].status != O_OK) st = jobs[t].status;
  free(jobs);
  return st;
}

typedef struct {
  obatch b;
  omodel md;
  int kmin, kmax, explicit_form;
  int64_t s0, s1;
  uint8_t *feasible, *rgs;
  int64_t* W;
  int32_t *sum_minm, *n_blocks, *spare;
  int16_t* minm_block;
  int64_t candidates;
  int status;
} best_job;

static void* best_worker(void* arg) {
  best_job* j = (best_job*)arg;
  for (int64_t si = j->s0; si < j->s1; si++) {
    oset s = view(si, j->b.set_off, j->b.T, j->b.D, j->b.A, j->b.B, j->b.u, j->b.type);
    int64_t o = j->b.set_off[si];
    obest best;
    memset(&best, 0, sizeof best);
    if (!valid_set(&s) || s.n > 14) {
      j->status = O_ERR_RANGE;
    } else if (j->explicit_form) {
      j->candidates += search_explicit(&s, &j->md, j->kmin, j->kmax, &best);
    } else {
      int st = search_rgs(&s, &j->md, j->kmin, j->kmax, &best);
      if (st != O_OK) j->status = st;
    }
    j->feasible[si] = (uint8_t)best.found;
    j->W[si] = best.found ? best.W : 0;
    j->sum_minm[si] = best.found ? (int32_t)best.sum_minm : 0;
    j->n_blocks[si] = best.found ? best.nb : 0;
    int64_t empty = (best.found && j->kmin > best.nb) ? (int64_t)(j->kmin - best.nb) : 0;
    j->spare[si] = best.found ? (int32_t)(j->md.M - best.sum_minm - empty * smallest_size(&j->md)) : 0;
    for (int i = 0; i < s.n && i < ONMAX; i++) j->rgs[o + i] = best.found ? best.rgs[i] : 255;
    for (int b = 0; b < j->kmax; b++)
      j->minm_block[si * j->kmax + b] = (int16_t)((best.found && b < best.nb) ? best.minm_block[b] : 0);
  }
  return NULL;
}

static int search_batch(int explicit_form, int64_t nsets, const int64_t* set_off, const int64_t* T, const int64_t* D,
                        const int64_t* A, const int64_t* B, const int64_t* u, const uint8_t* type, int64_t M,
                        int64_t g, int64_t kc, int64_t km, int64_t sched, const int32_t* sizes, int64_t nsizes,
                        int kmin, int kmax, uint8_t* feasible, int64_t* W, int32_t* sum_minm, int32_t* n_blocks,
                        int32_t* spare, uint8_t* rgs, int16_t* minm_block, int nthreads, int64_t* candidates) {
  omodel md = {M, g, kc, km, sched, sizes, nsizes};
  if (!valid_model(&md)) return O_ERR_RANGE;
  if (kmin < 1 || kmax < kmin || kmax > 8) return O_ERR_RANGE;
  int nth = nthreads < 1 ? 1 : (nthreads > 256 ? 256 : nthreads);
  if (nsets < nth) nth = nsets > 0 ? (int)nsets : 1;
  best_job* jobs = (best_job*)calloc((size_t)nth, sizeof(best_job));
  if (!jobs) return O_ERR_NOMEM;
  for (int t = 0; t < nth; t++) {
    best_job* j = &jobs[t];
    j->b = (obatch){set_off, T, D, A, B, u, type};
    j->md = md;
    j->kmin = kmin;
    j->kmax = kmax;
    j->explicit_form = explicit_form;
    j->s0 = nsets * t / nth;
    j->s1 = nsets * (t + 1) / nth;
    j->feasible = feasible;
    j->W = W;
    j->sum_minm = sum_minm;
    j->n_blocks = n_blocks;
    j->spare = spare;
    j->rgs = rgs;
    j->minm_block = minm_block;
  }
  run_threads(best_worker, jobs, sizeof(best_job), nth);
  int st = O_OK;
  int64_t cand = 0;
  for (int t = 0; t < nth; t++) {
    if (jobs[t].status != O_OK) st = jobs[t].status;
    cand += jobs[t].candidates;
  }
  if (candidates) *candidates = cand;
  free(jobs);
  return st;
}

int orc_search_best(int64_t nsets, const int64_t* set_off, const int64_t* T, const int64_t* D, const int64_t* A,
                    const int64_t* B, const int64_t* u, const uint8_t* type, int64_t M, int64_t g, int64_t kc,
                    int64_t km, int64_t sched, const int32_t* sizes, int64_t nsizes, int kmin, int kmax,
                    uint8_t* feasible, int64_t* W, int32_t* sum_minm, int32_t* n_blocks, int32_t* spare, uint8_t* rgs,
                    int16_t* minm_block, int nthreads) {
  return search_batch(0, nsets, set_off, T, D, A, B, u, type, M, g, kc, km, sched, sizes, nsizes, kmin, kmax,
                      feasible, W, sum_minm, n_blocks, spare, rgs, minm_block, nthreads, NULL);
}

int orc_search_explicit(int64_t nsets, const int64_t* set_off, const int64_t* T, const int64_t* D, const int64_t* A,
                        const int64_t* B, const int64_t* u, const uint8_t* type, int64_t M, int64_t g, int64_t kc,
                        int64_t km, int64_t sched, const int32_t* sizes, int64_t nsizes, int kmin, int kmax,
                        uint8_t* feasible, int64_t* W, int32_t* sum_minm, int32_t* n_blocks, int32_t* spare,
                        uint8_t* rgs, int16_t* minm_block, int nthreads, int64_t* candidates) {
  return search_batch(1, nsets, set_off, T, D, A, B, u, type, M, g, kc, km, sched, sizes, nsizes, kmin, kmax,
                      feasible, W, sum_minm, n_blocks, spare, rgs, minm_block, nthreads, candidates);
}

/* ------------------------------------------------------- serving operations
 *
 * One tenant's state: n tasks and an allocation (partition of each task,
 * size of each partition, partitions numbered by their lowest task index)
 * that passes the test (Lemma 3).  These are the operations of the serving
 * loop, defined on top of Alg. 1-3: ADD tries, in order, to fit the new task
 * into an existing partition at its size (first fit by partition number),
 * to grow a partition into the spare SMs (Alg. 2 from its size + g up to
 * its size + spare), a new Lemma 2 partition in the spare SMs, and Alg. 1 on
 * all tasks; REMOVE drops a task and shrinks its partition to its minimum. */

enum { PATH_NONE = 0, PATH_FIT = 1, PATH_GROW = 2, PATH_NEW = 3, PATH_REALLOC = 4 };

static void summarise(const oset* s, const omodel* md, const uint8_t* part, const int16_t* size, int np,
                      int32_t* Pi, int64_t* W) {
  int64_t pi = 0, w = 0;
  unsigned char in[ONMAX];
  for (int p = 0; p < np; p++) {
    pi += size[p];
    for (int i = 0; i < s->n; i++) in[i] = part[i] == p;
    w += workload(s, md, in);
  }
  *Pi = (int32_t)pi;
  *W = w;
}

/* renumber partitions by their lowest task index */
static void canonical(int n, uint8_t* part, int16_t* size, int np) {
  int lowest[ONMAX], order[ONMAX], newid[ONMAX];
  for (int p = 0; p < np; p++) lowest[p] = n;
  for (int i = n - 1; i >= 0; i--) lowest[part[i]] = i;
  for (int p = 0; p < np; p++) order[p] = p;
  for (int a = 1; a < np; a++) {
    int x = order[a], b = a - 1;
    while (b >= 0 && lowest[order[b]] > lowest[x]) { order[b + 1] = order[b]; b--; }
    order[b + 1] = x;
  }
  int16_t sz[ONMAX];
  for (int r = 0; r < np; r++) { newid[order[r]] = r; sz[r] = size[order[r]]; }
  for (int r = 0; r < np; r++) size[r] = sz[r];
  for (int i = 0; i < n; i++) part[i] = (uint8_t)newid[part[i]];
}

int orc_serve_admit(int n, const int64_t* T, const int64_t* D, const int64_t* A, const int64_t* B, const int64_t* u,
                    const uint8_t* type, int64_t M, int64_t g, int64_t kc, int64_t km, int64_t sched,
                    const int32_t* sizes, int64_t nsizes, int policy, int act, uint8_t* verdict, uint8_t* reason,
                    uint8_t* part_out, int16_t* size_out, int32_t* n_parts, int32_t* Pi, int64_t* W) {
  oset s = {n, T, D, A, B, u, type};
  omodel md = {M, g, kc, km, sched, sizes, nsizes};
  if (n > OSERVE_NMAX || !valid_model(&md) || !valid_set(&s)) return O_ERR_RANGE;
  ores r;
  int st = allocate_one(&s, &md, policy, act, 1, &r, part_out, size_out);
  *verdict = r.verdict;
  *reason = r.reason;
  *n_parts = r.n_parts;
  *Pi = r.Pi;
  *W = r.W;
  return st;
}

/* tasks: n + 1 entries (the state's n tasks, then the new one) */
int orc_serve_add(int n, const int64_t* T, const int64_t* D, const int64_t* A, const int64_t* B, const int64_t* u,
                  const uint8_t* type, const uint8_t* part_in, const int16_t* size_in, int np_in, int64_t M,
                  int64_t g, int64_t kc, int64_t km, int64_t sched, const int32_t* sizes, int64_t nsizes, int policy,
                  int act, uint8_t* verdict, uint8_t* reason, uint8_t* path, uint8_t* part_out, int16_t* size_out,
                  int32_t* n_parts, int32_t* Pi, int64_t* W) {
  oset s = {n + 1, T, D, A, B, u, type};
  omodel md = {M, g, kc, km, sched, sizes, nsizes};
  if (n + 1 > OSERVE_NMAX || !valid_model(&md) || !valid_set(&s)) return O_ERR_RANGE;
  const int nw = n;  /* index of the new task */
  int np = np_in;
  for (int i = 0; i < n; i++) part_out[i] = part_in[i];
  for (int p = 0; p < np; p++) size_out[p] = size_in[p];
  int64_t pi = 0;
  for (int p = 0; p < np; p++) pi += size_in[p];
  const int64_t spare = M - pi;
  unsigned char in[ONMAX];
  *verdict = 0;
  *reason = R_OK;
  *path = PATH_NONE;
  /* fit into an existing partition at its size */
  for (int p = 0; p < np && *path == PATH_NONE; p++) {
    for (int i = 0; i <= n; i++) in[i] = (i == nw) || (i < n && part_in[i] == p);
    if (test(&s, &md, in, size_in[p])) { part_out[nw] = (uint8_t)p; *path = PATH_FIT; }
  }
  /* grow a partition into the spare SMs */
  for (int p = 0; p < np && *path == PATH_NONE && spare >= g; p++) {
    for (int i = 0; i <= n; i++) in[i] = (i == nw) || (i < n && part_in[i] == p);
    int64_t m = minm_linear(&s, &md, in, size_in[p] + 1, size_in[p] + spare);
    if (m) { part_out[nw] = (uint8_t)p; size_out[p] = (int16_t)m; *path = PATH_GROW; }
  }
  /* a new partition of the task's Lemma 2 size */
  if (*path == PATH_NONE) {
    for (int i = 0; i <= n; i++) in[i] = i == nw;
    int64_t z = minm_linear(&s, &md, in, g, M);
    if (z && z <= spare) { part_out[nw] = (uint8_t)np; size_out[np] = (int16_t)z; np++; *path = PATH_NEW; }
  }
  if (*path != PATH_NONE) {
    *verdict = 1;
    *n_parts = np;
    summarise(&s, &md, part_out, size_out, np, Pi, W);
    return O_OK;
  }
  /* Alg. 1 on every task */
  ores r;
  uint8_t pt[ONMAX];
  int16_t sz[ONMAX];
  int st = allocate_one(&s, &md, policy, act, 1, &r, pt, sz);
  if (st != O_OK) return st;
  *reason = r.reason;
  if (r.verdict) {
    *verdict = 1;
    *path = PATH_REALLOC;
    for (int i = 0; i <= n; i++) part_out[i] = pt[i];
    for (int p = 0; p <= n; p++) size_out[p] = sz[p];
    *n_parts = r.n_parts;
    *Pi = r.Pi;
    *W = r.W;
    return O_OK;
  }
  /* rejected: the state is unchanged (n tasks) */
  oset s0 = {n, T, D, A, B, u, type};
  *n_parts = np_in;
  summarise(&s0, &md, part_out, size_out, np_in, Pi, W);
  return O_OK;
}

/* tasks: the state's n tasks; removes task `index` */
int orc_serve_remove(int n, const int64_t* T, const int64_t* D, const int64_t* A, const int64_t* B,
                     const int64_t* u, const uint8_t* type, const uint8_t* part_in, const int16_t* size_in,
                     int np_in, int index, int64_t M, int64_t g, int64_t kc, int64_t km, int64_t sched,
                     const int32_t* sizes, int64_t nsizes, int64_t* T_out, int64_t* D_out, int64_t* A_out,
                     int64_t* B_out, int64_t* u_out, uint8_t* type_out, uint8_t* part_out, int16_t* size_out,
                     int32_t* n_parts, int32_t* Pi, int64_t* W) {
  omodel md = {M, g, kc, km, sched, sizes, nsizes};
  if (index < 0 || index >= n || !valid_model(&md)) return O_ERR_RANGE;
  int k = 0;
  for (int i = 0; i < n; i++) {
    if (i == index) continue;
    T_out[k] = T[i];
    D_out[k] = D[i];
    A_out[k] = A[i];
    B_out[k] = B[i];
    u_out[k] = u[i];
    type_out[k] = type[i];
    part_out[k] = part_in[i];
    k++;
  }
  const int n2 = n - 1;
  oset s = {n2, T_out, D_out, A_out, B_out, u_out, type_out};
  int np = np_in;
  for (int p = 0; p < np; p++) size_out[p] = size_in[p];
  const int pr = part_in[index];
  int still = 0;
  for (int i = 0; i < n2; i++) still |= part_out[i] == pr;
  if (!still) {
    /* the partition is gone: close the gap in the numbering */
    for (int i = 0; i < n2; i++)
      if (part_out[i] > pr) part_out[i]--;
    for (int p = pr; p + 1 < np; p++) size_out[p] = size_out[p + 1];
    np--;
  } else {
    unsigned char in[ONMAX];
    for (int i = 0; i < n2; i++) in[i] = part_out[i] == pr;
    size_out[pr] = (int16_t)minm_linear(&s, &md, in, g, size_in[pr]);
  }
  canonical(n2, part_out, size_out, np);
  *n_parts = np;
  summarise(&s, &md, part_out, size_out, np, Pi, W);
  return O_OK;
}
