/*
 * gpa.h — C ABI of libgpa: contention-aware GPU-partition schedulability
 * (Zahaf, Sañudo Olmedo, Singh, Capodieci, Faucou, "Contention-Aware GPU
 * Partitioning and Task-to-Partition Allocation for Real-Time Workloads",
 * arXiv 2105.10312).
 *
 * The library evaluates the paper's per-partition schedulability test over
 * candidate splits of M SMs into partitions and task-to-partition maps, for
 * large batches of task sets.  All time quantities are integer ticks; the
 * interference factors are integer per-mille rationals; every result is
 * exact (bit-identical to a plain CPU evaluation of the same definitions).
 *
 * Conventions (all entry points)
 *  - Return value: int32_t status, GPA_OK (0) or a negative GPA_ERR_*.
 *    No C++ exception crosses the ABI.  gpa_last_error() returns the message
 *    of the last failing call on this thread.
 *  - Ownership: the caller owns every array it passes (host or device).  The
 *    library owns only the gpa_ctx (its stream binding, autotune cache,
 *    cached CUDA graphs and device scratch) and the serving state.
 *  - Memory tag: structs carrying arrays have a `mem` field, GPA_HOST or
 *    GPA_DEVICE, that applies to every array of that struct.  Host inputs
 *    are copied into the context's device buffers and checked against the
 *    bounds there before any computation (GPA_ERR_RANGE naming the first
 *    offending set; nothing is computed and no output is written); the call
 *    is synchronous.  gpa_allocate instead checks host sets in the kernels
 *    that compute them and splits a large batch into slices whose copies
 *    and kernels overlap (GPA_OPT_HOST_SLICES): a rejected batch returns
 *    GPA_ERR_RANGE naming the first offending set, and its outputs are
 *    unspecified (GPA_OPT_HOST_SLICES = 1 restores check-before-compute).
 *    Page-locked host arrays are read and written by a staging kernel over
 *    the host link, pageable ones by cudaMemcpyAsync (GPA_OPT_HOST_COPY).  Device inputs are validated by
 *    the kernels: an invalid set gets reason GPA_REASON_INVALID, its other
 *    outputs are zero, and the context's sticky error word is set; the call
 *    itself is asynchronous on the context stream and gpa_ctx_sync() reports
 *    GPA_ERR_RANGE afterwards.  The task columns of a device batch must hold
 *    set_off[nsets] tasks; a set whose slice is not inside [0, set_off[nsets])
 *    is invalid and its per-task outputs are left untouched.
 *  - Streams are passed as void* (a cudaStream_t); NULL is the legacy stream.
 *
 * Task model (paper §4.2, §7.1)
 *  A task set is a slice [set_off[s], set_off[s+1]) of structure-of-arrays
 *  task columns.  Task i has period T_i, relative deadline D_i (D_i <= T_i),
 *  WCET parameters A_i, B_i, type (0 = compute-intensive, 1 = memory-
 *  intensive; Def. 1) and utilisation u_ppm_i (parts per million, used for
 *  ordering and for the inflated workload W).  Its WCET on a partition of
 *  m SMs with interference factor k (per mille) is the scaling function of
 *  §7.1, C = k (a/m + b), in integer form:
 *
 *      C_i^k(m) = ceil( k * (A_i + B_i * m) / (10^6 * m) )
 *
 *  with k = 1000 when the task is not in conflict (C^n of §3.3) and
 *  k = k_c_pm (compute) or k_m_pm (memory) when it is (C^c of §3.3).  A task
 *  is in conflict when at least one other task of its own type shares its
 *  partition (§4.2).
 *
 * Per-partition test (§5.5 leaves the policy open): a partition of m SMs is
 * one processor running its tasks under deadline-monotonic fixed priorities
 * (priority order: D ascending, then T ascending, then task index); each
 * task's response time is the least fixed point of
 *      R_i = C_i + sum_{j in hp(i)} ceil(R_i / T_j) * C_j
 * started from R_i^0 = C_i + sum_{hp(i)} C_j.  A task meets its deadline iff
 * that fixed point is <= D_i; otherwise its reported R is -1.
 * Second policy (GPA_SCHED_EDF, model->sched; not from the paper): preemptive
 * EDF on the partition, synchronous periodic release.  Exact processor-demand
 * test: U <= 1 (compared exactly) and dbf(t) = sum_{D_i <= t}
 * (floor((t - D_i) / T_i) + 1) C_i <= t at every absolute deadline up to the
 * first synchronous busy period (evaluated with QPA, Zhang & Burns 2009).
 * One task passes iff C <= D.  EDF gives no response times: R is 0 for the
 * tasks of a passing part.
 *
 * Undecided tests.  Every test is bounded: a DM fixed point stops after 2^20
 * steps per task, an EDF analysis after 2^20 busy-period or QPA steps, or
 * when its busy period would pass 2^62, or when U lies within n 2^-64 of 1
 * and the periods' least common multiple exceeds 2^62.  Such a test is
 * undecided, never reported as a miss: the set gets GPA_REASON_UNDECIDED
 * (gpa_allocate), the candidate verdict 2 (gpa_test_schedulable), the
 * optimum feasible = 2 (gpa_search_best), the serving request status
 * GPA_ERR_TIMEOUT; and gpa_ctx_sync returns GPA_ERR_TIMEOUT.  Near U = 1 an
 * EDF analysis takes about 1 / (1 - U) steps, so undecided tests are rare.
 *
 * Validation bounds (GPA_ERR_RANGE): 0 <= n <= 256 tasks per set (128 for
 * serving tenants and gpa_allocate_noalloc),
 * 1 <= D <= T <= 2^31 - 1, A >= 0, B >= 0, 1 <= A + B <= 2^36,
 * 0 <= u_ppm < 2^32, type in {0, 1}; model: 1 <= g, g | M, 1 <= M <= 1024,
 * 1000 <= k_c_pm, k_m_pm <= 16000.  These keep every WCET below 2^31 and
 * every intermediate product inside 64 bits.
 */
#ifndef GPA_H_
#define GPA_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GPA_ABI_VERSION 4
#define GPA_NMAX 256          /* tasks per set */
#define GPA_SERVE_NMAX 128    /* tasks per serving tenant and per set of gpa_allocate_noalloc */
#define GPA_MMAX 1024         /* SMs on the modelled GPU */
#define GPA_SEARCH_NMAX 14    /* tasks per set in gpa_search_best */
#define GPA_SEARCH_KMAX 8     /* partitions per candidate in gpa_search_best */

enum {
  GPA_OK = 0,
  GPA_ERR_ARG = -1,      /* NULL where an array is required, bad enum, bad size */
  GPA_ERR_RANGE = -2,    /* input outside the validation bounds above */
  GPA_ERR_NOMEM = -3,    /* device or host allocation failed */
  GPA_ERR_CUDA = -4,     /* a CUDA runtime call failed */
  GPA_ERR_TIMEOUT = -5,  /* a bounded wait expired */
  GPA_ERR_BUSY = -6,     /* serving: the host queue is full */
  GPA_ERR_NOTFOUND = -7  /* serving: unknown request id / tenant */
};

enum { GPA_HOST = 0, GPA_DEVICE = 1 };

/* Task types (Def. 1). */
enum { GPA_COMPUTE = 0, GPA_MEMORY = 1 };

/* Per-set outcome of gpa_allocate. */
enum {
  GPA_REASON_OK = 0,        /* schedulable allocation found (Lemma 3) */
  GPA_REASON_LEMMA1 = 1,    /* rejected by the necessary utilisation test (Lemma 1) */
  GPA_REASON_LEMMA2 = 2,    /* a task meets its deadline on no size <= M (Lemma 2) */
  GPA_REASON_NO_MERGE = 3,  /* Alg. 3 found no eligible merge while Pi > M */
  GPA_REASON_TEST = 4,      /* 1G baseline: the single partition fails the test */
  GPA_REASON_INVALID = 5,   /* device-side validation rejected the set */
  GPA_REASON_UNDECIDED = 6  /* a per-partition test hit its step limit: the verdict is unknown (0 is
                               written); the set's other outputs are unspecified */
};

/* Allocation policies (§7.2). */
enum {
  GPA_POLICY_SMS = 0,       /* order >> of Def. 3: smallest merged size first */
  GPA_POLICY_BF = 1,        /* order > of Def. 4: smallest merged workload first */
  GPA_POLICY_ONE_GPU = 2    /* 1G baseline: all tasks in one partition of M SMs */
};

/* Per-partition scheduling policies (gpa_model.sched). */
enum {
  GPA_SCHED_DM = 0,   /* deadline-monotonic fixed priority, response-time analysis (§5.5 reading) */
  GPA_SCHED_EDF = 1   /* preemptive EDF, processor-demand test */
};

/* ---------------------------------------------------------------- context */

typedef struct gpa_ctx gpa_ctx;

/* Create a context bound to CUDA device `device` and stream `stream`
 * (cudaStream_t, may be NULL).  *out receives the context.
 * Errors: GPA_ERR_ARG (out NULL, bad device), GPA_ERR_CUDA. */
int32_t gpa_ctx_create(int32_t device, void* stream, gpa_ctx** out);
/* Destroy a context; frees its scratch, graphs and serving state. NULL is a no-op. */
int32_t gpa_ctx_destroy(gpa_ctx* ctx);
/* Rebind the context to another stream of the same device. */
int32_t gpa_ctx_set_stream(gpa_ctx* ctx, void* stream);
/* Wait for the context stream; return GPA_ERR_TIMEOUT if any kernel since
 * the last call left a test undecided (see "Undecided tests" above), else
 * GPA_ERR_RANGE if one flagged an invalid device-resident set (and clear
 * both flags), GPA_ERR_CUDA on an asynchronous CUDA error, else GPA_OK. */
int32_t gpa_ctx_sync(gpa_ctx* ctx);
/* Copy the last error message of this thread into buf (NUL-terminated). */
int32_t gpa_last_error(char* buf, int32_t len);
/* Number of GPU kernel launches the context has issued since creation. */
int32_t gpa_ctx_launch_count(gpa_ctx* ctx, int64_t* out);

/* Context options (gpa_ctx_set_option).  None changes any result. */
enum {
  GPA_OPT_AUTOTUNE = 1,       /* 1: on the first gpa_allocate call of each batch signature, time the
                                 launch shapes of the kernels the call runs (the fast kernel's loads,
                                 warps and sets per ticket; the merge kernel's warps per CTA, warps
                                 per set, CTAs per SM and top-size round; the 1G deferred-set
                                 kernel's warps per CTA) and keep the fastest for that signature
                                 (default 0) */
  GPA_OPT_GRAPH = 2,          /* 1: capture gpa_allocate's launches in a CUDA graph per argument set and
                                 replay it (default 0); not allowed while the stream is being captured */
  GPA_OPT_FAST_WARPS = 3,     /* force warps per CTA of the fast allocate kernel: 1, 2, 4 or 8 (the staged
                                 form adds a copy warp) (0 = tuned/default) */
  GPA_OPT_FAST_CHUNK = 4,     /* force task sets per work-queue ticket (0 = tuned/default) */
  GPA_OPT_FAST_BLOCKS = 5,    /* force CTAs of the persistent grid (0 = tuned/default) */
  GPA_OPT_PER_SET_LAUNCH = 6, /* 1: the plain form, one launch sequence per task set (comparison only) */
  GPA_OPT_PROFILE = 7,        /* 1: record CUDA events around each kernel of every call (also inside
                                 captured graphs) so that gpa_ctx_last_timing can report them */
  GPA_OPT_FAST_STAGES = 8,    /* force how the fast allocate kernel reads the task columns: 1 = direct
                                 loads; 2..5 = through that many shared-memory stages filled by bulk
                                 copies, used only when every task column starts on a 16-byte
                                 boundary (direct loads otherwise) (0 = tuned/default) */
  GPA_OPT_HOST_SLICES = 9,    /* gpa_allocate on host buffers: 0 = sets checked by the computing
                                 kernels, batches of more than 48 MB of task columns split into
                                 max(2, ceil(MB / 64)) slices (at most 16) whose copies in, kernels and
                                 copies out overlap; 1 = the whole batch checked before any computation (a
                                 rejected batch leaves the outputs untouched); n in 2..64 = as 0 but
                                 every batch split into n slices (fewer when it has fewer sets)
                                 (default 0) */
  GPA_OPT_HOST_COPY = 10,     /* how host buffers move: 0 = arrays that are page-locked (cudaHostAlloc,
                                 cudaHostRegister) are read and written by one staging kernel per
                                 direction and slice, over the host link, with up to 16 CTAs per array;
                                 other arrays by cudaMemcpyAsync; 1 = cudaMemcpyAsync for every array;
                                 n in 2..256 = the staging kernel with n CTAs per array (default 0) */
  GPA_OPT_MERGE_WARPS = 11,   /* force warps per CTA of the merge kernel (Alg. 1 for the sets the fast
                                 kernel could not decide): 1..8, a multiple of GPA_OPT_MERGE_GROUP; lowered
                                 to the largest such multiple whose shared memory fits one SM
                                 (0 = tuned/default) */
  GPA_OPT_MERGE_GROUP = 12,   /* force warps per task set in the merge kernel: 1, 2, 4 or 8; a set's
                                 candidate merges are spread over its warps (0 = tuned/default) */
  GPA_OPT_MERGE_BLOCKS = 13,  /* force CTAs of the persistent merge grid (0 = tuned/default) */
  GPA_OPT_TEST_WARPS = 14,    /* force warps per CTA of the 1G deferred-set kernel (the sets the 1G
                                 pre-pass does not decide in closed form: one test of all tasks at M
                                 per set, one warp per set): 1..8 (0 = tuned/default) */
  GPA_OPT_MERGE_TOPFIRST = 15 /* force whether the merge kernel's SMS steps first test every candidate
                                 merge with several sizes in its range at its top size (a failure there
                                 rules it out at every size): 1 = off, 2 = on (0 = tuned/default) */
};
int32_t gpa_ctx_set_option(gpa_ctx* ctx, int32_t option, int64_t value);

/* Device time (ms) of each kernel of the last call made with GPA_OPT_PROFILE
 * on, in launch order (gpa_allocate: the fast kernel, then the merge kernel;
 * every other entry point: its one kernel).  Waits for that call's work.
 * ms[0 .. *count) are written, at most n of them. */
int32_t gpa_ctx_last_timing(gpa_ctx* ctx, float* ms, int32_t n, int32_t* count);

/* Interference terms evaluated by the kernels of the context's last
 * gpa_allocate, gpa_test_schedulable, gpa_search_best or gpa_search_explicit
 * call on device buffers (one launch sequence; a call on host buffers may
 * run several, and the count then covers its last slice).  A term is one
 * ceil(R / T_j) C_j of a response-time iteration (§5.5, DM), or one task's
 * demand in a busy-period or QPA step (EDF).  Waits for the context stream. */
int32_t gpa_ctx_last_terms(gpa_ctx* ctx, int64_t* terms);

/* --------------------------------------------------------------- task sets */

typedef struct {
  int64_t nsets;
  int32_t mem;              /* GPA_HOST or GPA_DEVICE for every array below */
  int32_t n_max;            /* upper bound on tasks per set (<= GPA_NMAX) */
  const int64_t* set_off;   /* [nsets + 1], set_off[0] = 0, non-decreasing */
  const int64_t* T;         /* [ntasks] period */
  const int64_t* D;         /* [ntasks] relative deadline */
  const int64_t* A;         /* [ntasks] WCET parameter a (per-mille scaled) */
  const int64_t* B;         /* [ntasks] WCET parameter b (per-mille scaled) */
  const int64_t* u_ppm;     /* [ntasks] utilisation, parts per million */
  const uint8_t* type;      /* [ntasks] GPA_COMPUTE / GPA_MEMORY */
} gpa_tasksets;

typedef struct {
  int32_t M;       /* SMs of the modelled GPU (§4.1) */
  int32_t g;       /* partition granularity in SMs (1 = SM, 2 = TPC); sizes are multiples of g */
  int32_t k_c_pm;  /* conflict factor of compute-intensive tasks, per mille (§7.1: 1200) */
  int32_t k_m_pm;  /* conflict factor of memory-intensive tasks, per mille (§7.1: 2300) */
  int32_t sched;   /* per-partition policy: GPA_SCHED_DM or GPA_SCHED_EDF */
  int32_t nsizes;  /* 0: every multiple of g in [g, M] is a partition size; else the length of `sizes` */
  const int32_t* sizes; /* host array, strictly increasing multiples of g in [g, M]: the only admissible
                           partition sizes (whole GPCs or MIG slices, §2).  Used by gpa_allocate
                           (Lemma 2 sizes round up to the next listed size; a merge is sized over the
                           listed sizes below the sum of the two), gpa_test_schedulable (a non-empty
                           part's size must be listed) and gpa_search_best (blocks take listed sizes; an
                           empty part counts the smallest).  1G uses M; serving takes its list in
                           gpa_serve_cfg; gpa_allocate_noalloc takes none (GPA_ERR_ARG). */
} gpa_model;

/* Host-side validation of a task batch and model against the bounds above
 * (host arrays only; no GPU needed).  *bad_set receives the first invalid
 * set index or -1.  Returns GPA_OK or GPA_ERR_RANGE / GPA_ERR_ARG. */
int32_t gpa_validate(const gpa_tasksets* sets, const gpa_model* model, int64_t* bad_set);

/* --------------------------------------------------------------- generator */

enum { GPA_DIST_UNIFORM = 0, GPA_DIST_LOGUNIFORM = 1, GPA_DIST_LIST = 2, GPA_DIST_BETA25 = 3 };
enum { GPA_GEN_ALPHA = 0, GPA_GEN_PAPER = 1 };

typedef struct {
  uint64_t seed;
  int64_t nsets;
  int32_t n_min, n_max;        /* tasks per set */
  int32_t n_dist;              /* UNIFORM or LOGUNIFORM over [n_min, n_max] */
  int32_t U_steps;             /* 0: U ~ U[U_lo, U_hi]; > 0: U = U_lo + (s mod U_steps) * (U_hi - U_lo) / (U_steps - 1) */
  int64_t U_lo_ppm, U_hi_ppm;  /* total utilisation per set, ppm */
  int64_t T_lo, T_hi;          /* period range, ticks */
  int32_t T_dist;              /* LOGUNIFORM over [T_lo, T_hi], or LIST = divisors of T_hi in [T_lo, T_hi] */
  int32_t deadline_pm;         /* D = max(1, floor(T * deadline_pm / 1000)) */
  int32_t alpha_lo_pm, alpha_hi_pm; /* ALPHA mode: serial fraction alpha ~ U{lo..hi} per mille */
  int32_t mu_dist;             /* memory intensity: UNIFORM or BETA25 (Beta(2,5)), per mille */
  int32_t prm_pm;              /* type = MEMORY iff mu_pm >= prm_pm */
  int32_t mode;                /* GPA_GEN_ALPHA: A = C1 (1000 - alpha), B = C1 alpha
                                  GPA_GEN_PAPER:    A = 1000 C1, B = beta C1 (beta by type) */
  int32_t beta_c_pm, beta_m_pm;/* PAPER mode serial parts (§7.1: 20 and 100 per mille) */
  int64_t u_max_ppm;           /* discard and redraw a set whose largest task utilisation exceeds this (0 = never) */
  int32_t max_tries;           /* redraw limit per set (the last draw is kept, flagged) */
  int32_t nthreads;            /* host threads (<= 0: 1) */
} gpa_gen_params;

typedef struct {
  int64_t* set_off;    /* [nsets + 1] */
  int64_t* T;          /* [ntasks] */
  int64_t* D;
  int64_t* A;
  int64_t* B;
  int64_t* u_ppm;      /* floor(10^6 C1 / T) after rounding C1 */
  uint8_t* type;
  int64_t* C1;         /* baseline single-SM execution time (ticks) */
  int16_t* alpha_pm;
  int16_t* mu_pm;
  uint8_t* flags;      /* [nsets] bit 0: discard limit reached */
} gpa_gen_out;

/* Seeded, counter-based synthetic task-set generator (§7.1; utilisations are
 * drawn uniformly on the simplex sum u_i = U).  Host memory only.
 * Call with out == NULL to get the total task count in *ntasks; then call
 * again with every array of *out allocated to that size. */
int32_t gpa_gen_tasksets(const gpa_gen_params* params, gpa_gen_out* out, int64_t* ntasks);

/* ------------------------------------------------------------- WCET tables */

/* a2: Cn and Cc tables, layout [set][m-index][task]: for set s with n_s tasks
 * at offset o_s, the entry of task t at size m = g (mi + 1), mi < M/g, is at
 * o_s * (M/g) + mi * n_s + t.  Cn uses k = 1000; Cc uses k_c_pm or k_m_pm by
 * type (§3.3, §7.1).  Both arrays hold ntasks * (M/g) int64 and live in the
 * memory named by sets->mem. */
int32_t gpa_build_wcet_tables(gpa_ctx* ctx, const gpa_tasksets* sets, const gpa_model* model,
                              int64_t* Cn, int64_t* Cc);

/* ---------------------------------------------------- partition enumeration */

/* Number of compositions of Mu = M/g units into k parts, summed over
 * k in [kmin, kmax] (candidate SM splits, §4.1). */
int32_t gpa_enumerate_partitions(int32_t Mu, int32_t kmin, int32_t kmax, uint64_t* count);
/* The composition of Mu into k positive parts of rank `rank` in
 * lexicographic order of (parts[0], ..., parts[k-1]). */
int32_t gpa_unrank_composition(int32_t Mu, int32_t k, uint64_t rank, int32_t* parts);
/* Number of set partitions of n tasks into at most kmax blocks. */
int32_t gpa_count_rgs(int32_t n, int32_t kmax, uint64_t* count);
/* The restricted-growth string of rank `rank` (lexicographic order) among
 * set partitions of n tasks into at most kmax blocks. */
int32_t gpa_unrank_rgs(int32_t n, int32_t kmax, uint64_t rank, uint8_t* rgs);

/* ------------------------------------------------------- explicit candidates */

typedef struct {
  int64_t ncands;
  int32_t mem;
  int32_t map_stride;       /* bytes per candidate in part_of_task (>= tasks of its set) */
  int32_t kparts;           /* parts per candidate = entries per candidate in size_of_part */
  int32_t pad_;
  const int64_t* set;       /* [ncands] task-set index */
  const uint8_t* part_of_task; /* [ncands * map_stride] part of each task (< kparts) */
  const int32_t* size_of_part; /* [ncands * kparts] SMs of each part: 0 or a multiple of g in [g, M] */
} gpa_candidates;

/* a4 over a flat batch: candidate c is schedulable iff sum of its part sizes
 * <= M and every non-empty part meets the per-partition test at its size (a
 * non-empty part of size 0 fails).  verdict[c] in {0,1}, or 2 when a part's
 * test was undecided and no other part fails; R (nullable) gets
 * each task's response time at R[c * map_stride + t], -1 for a miss (under
 * EDF: 0 for the tasks of a passing part, -1 otherwise).
 * Arrays live in cands->mem (which must equal sets->mem). */
int32_t gpa_test_schedulable(gpa_ctx* ctx, const gpa_tasksets* sets, const gpa_model* model,
                             const gpa_candidates* cands, uint8_t* verdict, int64_t* R);

/* ------------------------------------------------------------- heuristic */

typedef struct {
  int32_t policy;       /* GPA_POLICY_SMS / BF / ONE_GPU */
  int32_t act;          /* 1: fill the forbidden list with failing task pairs first (ACT); 0: INA */
  int32_t linear_merge; /* 1: Alg. 2 linear scan; 0: binary search (same result) */
  int32_t pad_;
} gpa_params;

typedef struct {
  int32_t mem;
  int32_t pad_;
  uint8_t* verdict;       /* [nsets] 1 iff a schedulable allocation was found */
  uint8_t* reason;        /* [nsets] GPA_REASON_* */
  int32_t* n_parts;       /* [nsets] partitions in the final list */
  int32_t* Pi;            /* [nsets] sum of partition sizes (SMs) */
  int64_t* W;             /* [nsets] inflated workload sum_P sum_{i in P} k_i(P) u_ppm_i */
  int32_t* n_tests;       /* [nsets] merge candidates evaluated (nullable) */
  uint8_t* part_of_task;  /* [ntasks] partition of each task, 255 when none */
  int16_t* size_of_part;  /* [ntasks] size of partition p of set s at set_off[s] + p (p < n_parts), else 0 */
} gpa_alloc_result;

/* a7/a9: the paper's partition-and-allocate heuristic (Alg. 1-3 with
 * Lemmas 1-3, SMS/BF x ACT/INA) or the 1G baseline, for every set of the
 * batch.  Partitions are numbered by their lowest task index.  result->mem
 * must equal sets->mem. */
int32_t gpa_allocate(gpa_ctx* ctx, const gpa_tasksets* sets, const gpa_model* model,
                     const gpa_params* params, gpa_alloc_result* result);

/* Most policies per gpa_allocate_multi call. */
#define GPA_MULTI_MAX_POLICIES 8

/* gpa_allocate under several policies in one call.  The paper's evaluation
 * (§7) decides every task set of a sweep under each allocation policy it
 * compares (SMS, BF, the 1G baseline, with ACT or INA); this call does that
 * for one batch.  results[i] receives exactly what
 * gpa_allocate(ctx, sets, model, &params[i], &results[i]) would write, for
 * every i < npolicies (1 to GPA_MULTI_MAX_POLICIES, else GPA_ERR_RANGE).
 *  - Host arrays: the batch crosses the host link once for all the
 *    policies.  Each slice of sets is copied in once, decided under every
 *    policy in order, and its results of every policy are copied out while
 *    the next slice is decided.  The call returns when every result is in
 *    the caller's arrays.
 *  - Device arrays: the same work as npolicies gpa_allocate calls in order on
 *    the context stream (asynchronous, as gpa_allocate).
 *  - Every results[i] must have mem == sets->mem and arrays of its own (no
 *    two results may share an array); the argument checks of gpa_allocate
 *    apply to each params[i] and results[i], and an argument that fails
 *    them is reported before any copy or launch.
 *  - Status: the first error, as gpa_allocate reports it; an undecided or
 *    invalid set under any of the policies gives GPA_ERR_TIMEOUT or
 *    GPA_ERR_RANGE, and each result's reason[] marks its own sets.  Host
 *    sets out of bounds are handled as by gpa_allocate (GPA_ERR_RANGE naming
 *    the first; the outputs unspecified when the batch was split into
 *    slices, untouched otherwise). */
int32_t gpa_allocate_multi(gpa_ctx* ctx, const gpa_tasksets* sets, const gpa_model* model,
                           const gpa_params* params, int32_t npolicies, gpa_alloc_result* results);

/* Task sets per call of gpa_allocate_noalloc. */
#define GPA_NOALLOC_MAX_SETS 262144

/* gpa_allocate for callers that cannot allocate device memory (the paper has
 * no counterpart: this is a deployment variant).  Some callers may not call
 * cudaMalloc: a host application or plug-in whose device memory belongs to
 * someone else's pool or a fixed budget, or a real-time process that must not
 * allocate once it runs.  This call takes no context and allocates nothing
 * (no cudaMalloc, cudaFree or allocating library routine); its scratch -- the
 * work-queue counters, the error word, a queue of up to GPA_NOALLOC_MAX_SETS
 * deferred sets and the reciprocal table, about 2 MB -- is a static device
 * array of the library.  A device holds those 2 MB until the process exits
 * from the moment the library's device code is loaded on it: at the first
 * call of this entry point on that device under CUDA's default lazy module
 * loading, and as soon as the process creates a CUDA context on it under
 * eager loading (CUDA_MODULE_LOADING=EAGER), whether or not it ever calls
 * this entry point.
 *  - Same computation and outputs as gpa_allocate with GPA_POLICY_SMS or
 *    GPA_POLICY_BF (GPA_ERR_ARG otherwise), either per-partition policy;
 *    device arrays only (both `mem` fields GPA_DEVICE); work is enqueued on
 *    `stream` (a cudaStream_t), which must belong to the current device
 *    (GPA_ERR_ARG otherwise).
 *  - More than GPA_NOALLOC_MAX_SETS sets: GPA_ERR_RANGE, nothing launched.
 *  - The first call on a device (the current device) sets that device up
 *    synchronously (uploads the reciprocal table, looks up the scratch
 *    address); make it before any stream capture.
 *  - Every call shares the one scratch array, which keeps the previous
 *    call's contents; each call clears the counters it needs zeroed.  Calls
 *    whose GPU work overlaps (other streams, other threads) race on it: the
 *    caller must serialise them.
 *  - Problems found on the device are marked per set as gpa_allocate marks
 *    them (GPA_REASON_INVALID, GPA_REASON_UNDECIDED) and recorded in the
 *    scratch's error word; the call itself returns before they are known.
 *    gpa_allocate_noalloc_status reports and clears that word. */
int32_t gpa_allocate_noalloc(void* stream, const gpa_tasksets* sets, const gpa_model* model,
                             const gpa_params* params, gpa_alloc_result* result);
/* The error word of gpa_allocate_noalloc on the current device: waits for
 * `stream` (which must belong to the current device), then returns
 * GPA_ERR_TIMEOUT if a set of the calls since the last status was left
 * undecided, else GPA_ERR_RANGE if one failed validation, else GPA_OK, and
 * clears the word.  Allocates nothing. */
int32_t gpa_allocate_noalloc_status(void* stream);

/* ------------------------------------------------------ exhaustive optimum */

typedef struct {
  int32_t mem;
  int32_t pad_;
  uint8_t* feasible;      /* [nsets] 1 feasible, 0 not, 2 undecided (a test hit its step limit) */
  int64_t* W;             /* [nsets] inflated workload of the optimum */
  int32_t* sum_minm;      /* [nsets] sum over blocks of the block's minimum size */
  int32_t* n_blocks;      /* [nsets] */
  int32_t* spare;         /* [nsets] M - sum_minm - max(0, kmin - n_blocks) * g */
  uint8_t* rgs;           /* [ntasks] block of each task (restricted growth string) */
  int16_t* minm_block;    /* [nsets * kmax] minimum size of each block, 0 past n_blocks */
} gpa_best_result;

/* a6/a8: exact optimum over every split of M into k in [kmin, kmax]
 * partitions (multiples of g) and every task-to-partition map, for sets of
 * at most GPA_SEARCH_NMAX tasks.  Key (lexicographic, minimised): W, then
 * sum_minm, then the restricted-growth string of the induced set partition.
 * A set partition with b blocks is realisable iff b <= kmax, every block
 * has a minimum size, and sum_minm + max(0, kmin - b) g <= M. */
int32_t gpa_search_best(gpa_ctx* ctx, const gpa_tasksets* sets, const gpa_model* model,
                        int32_t kmin, int32_t kmax, gpa_best_result* result);

/* a6/a8 on the explicit candidates, enumerated on the device: for each set,
 * every composition of Mu = M / g into k in [kmin, min(kmax, Mu)] positive
 * parts (part b gets parts[b] * g SMs) times every map of its n tasks to the
 * k parts (problem statement of §5: an SM split and a task-to-partition
 * allocation).  Candidate ranks run over k, then the composition in
 * lexicographic order of its parts, then the map code c, which sends task i
 * (in set order) to part (c / k^i) mod k.  A candidate is feasible iff
 * every non-empty part passes the model's test at its size; the result is
 * the optimum of gpa_search_best (the same key and fields; identical
 * values), here found over the explicit space.
 *  - cand_verdict (nullable; memory of sets->mem): [nsets * cand_stride]
 *    bytes, candidate r of set s at s * cand_stride + r: 1 feasible,
 *    0 not, 2 undecided (a test of one of its parts' task sets hit its step
 *    limit); entries past a set's
 *    own count are 255.  cand_stride = the count for n_max tasks, returned
 *    in *ncand (nullable) by every call, also when cand_verdict is NULL.
 *  - Limits: n_max <= GPA_SEARCH_NMAX, 1 <= kmin <= kmax <= GPA_SEARCH_KMAX,
 *    at most GPA_EXPLICIT_MAX candidates per set (GPA_ERR_RANGE);
 *    admissible size lists are not supported (GPA_ERR_ARG). */
#define GPA_EXPLICIT_MAX (1ll << 26)
int32_t gpa_search_explicit(gpa_ctx* ctx, const gpa_tasksets* sets, const gpa_model* model, int32_t kmin,
                            int32_t kmax, gpa_best_result* result, uint8_t* cand_verdict, int64_t* ncand);

/* ----------------------------------------------------------------- serving */

/* Admission control as a service: tenants (task sets of up to
 * GPA_SERVE_NMAX tasks) and their current allocation live in device memory; requests are
 * queued, packed into micro-batches (at most one request per tenant per
 * batch, each tenant's requests in submission order) and run one warp per
 * request on one of several streams, so a batch starts while earlier ones are
 * still on the GPU.  A tenant's state is always an allocation that passes
 * (Lemma 3).  Every request's result depends only on its tenant's earlier
 * requests, never on what else shares its batch.
 *
 * Operations:
 *  GPA_SERVE_ADMIT  create tenant `tenant` from n tasks: Alg. 1 (the
 *                   configured policy); admitted iff it succeeds.  Waits in
 *                   the queue while no tenant slot is free and the device
 *                   has no memory left to add slots (cudaMemGetInfo).
 *  GPA_SERVE_ADD    append one task (index n): first partition (in order of
 *                   lowest task index) that still passes at its size with the
 *                   task; else the first that passes after growing into the
 *                   spare SMs (Alg. 2 search from its size + g up to its size
 *                   + spare); else a new partition of the task's Lemma 2 size
 *                   if it fits in the spare SMs; else Alg. 1 on all tasks.  If
 *                   all fail the task is rejected and the state is unchanged.
 *  GPA_SERVE_REMOVE remove task `index` (later tasks shift down by one); its
 *                   partition shrinks to its new minimum size (or disappears).
 *  GPA_SERVE_EVICT  delete the tenant and free its slot. */
enum { GPA_SERVE_ADMIT = 0, GPA_SERVE_ADD = 1, GPA_SERVE_REMOVE = 2, GPA_SERVE_EVICT = 3 };
/* How an ADD was placed. */
enum { GPA_PATH_NONE = 0, GPA_PATH_FIT = 1, GPA_PATH_GROW = 2, GPA_PATH_NEW = 3, GPA_PATH_REALLOC = 4 };

typedef struct {
  int32_t M, g, k_c_pm, k_m_pm;  /* the GPU model of every tenant */
  int32_t policy;                /* GPA_POLICY_SMS or GPA_POLICY_BF for ADMIT and ADD's re-allocation */
  int32_t act;
  int32_t max_batch;             /* requests per micro-batch (<= 4096) */
  int32_t nstreams;              /* concurrent micro-batches (1..8) */
  int32_t queue_cap;             /* pending requests before GPA_ERR_BUSY */
  int32_t slots_per_chunk;       /* tenant slots added per device allocation */
  int64_t max_tenants;           /* upper bound on live tenants */
  int64_t reserve_bytes;         /* device memory left free when adding slots */
  int32_t sched;                 /* per-partition policy: GPA_SCHED_DM or GPA_SCHED_EDF */
  int32_t nsizes;                /* admissible partition sizes as in gpa_model (0: every multiple of g) */
  const int32_t* sizes;          /* host array, copied by gpa_serve_start */
} gpa_serve_cfg;

typedef struct {
  int32_t op;                    /* GPA_SERVE_* */
  int32_t n;                     /* ADMIT: tasks; ADD: 1 */
  int64_t tenant;                /* caller's tenant id (>= 0) */
  int32_t index;                 /* REMOVE: task index */
  int32_t pad_;
  const int64_t* T;              /* ADMIT/ADD host arrays of n tasks, copied at submit */
  const int64_t* D;
  const int64_t* A;
  const int64_t* B;
  const int64_t* u_ppm;
  const uint8_t* type;
} gpa_request;

typedef struct {
  uint64_t req_id;
  int32_t status;                /* GPA_OK, or the request's error (GPA_ERR_RANGE / ARG / NOTFOUND), or
                                    GPA_ERR_TIMEOUT when a test of the request was undecided (the tenant's
                                    state is still an allocation whose every partition passes) */
  uint8_t verdict;               /* ADMIT/ADD: 1 if accepted; REMOVE/EVICT: 1 */
  uint8_t reason;                /* GPA_REASON_* of the Alg. 1 run (ADMIT, ADD re-allocation) */
  uint8_t path;                  /* GPA_PATH_* (ADD) */
  uint8_t pad_;
  int32_t n_tasks, n_parts, Pi;  /* the tenant's state after the request */
  int64_t W;
  uint8_t part_of_task[GPA_SERVE_NMAX];
  int16_t size_of_part[GPA_SERVE_NMAX];
  double latency_us;             /* submit to completion, host clock */
} gpa_response;

/* Start the server on the context's device (one server per context). */
int32_t gpa_serve_start(gpa_ctx* ctx, const gpa_serve_cfg* cfg);
/* Queue a request; *req_id identifies it.  GPA_ERR_BUSY only when the host
 * queue is full; malformed requests are answered with an error status. */
int32_t gpa_serve_submit(gpa_ctx* ctx, const gpa_request* req, uint64_t* req_id);
/* Wait up to timeout_us (0: do not wait) for request req_id and move its
 * response into *out.  GPA_ERR_TIMEOUT if not done in time (ask again later),
 * GPA_ERR_NOTFOUND for an unknown or already collected id.  Never blocks
 * beyond timeout_us. */
int32_t gpa_serve_poll(gpa_ctx* ctx, uint64_t req_id, gpa_response* out, int64_t timeout_us);
/* Finish the queued requests, stop the server and free its device state. */
int32_t gpa_serve_stop(gpa_ctx* ctx);
/* Counters: requests completed, micro-batches launched, largest batch,
 * batches that overlapped another on the GPU, tenant slots allocated. */
int32_t gpa_serve_stats(gpa_ctx* ctx, int64_t* completed, int64_t* batches, int64_t* max_batch,
                        int64_t* overlapped, int64_t* slots);

/* ---------------------------------------------- measured WCET curves (§3)
 *
 * The execution time C(m) of a kernel on m SMs, measured as §3 describes for
 * Fig. 1: a blocker kernel takes sm_count - m SMs (one CTA per SM, each
 * holding the whole 227 KB of opt-in shared memory so that no other CTA fits
 * beside it) for a fixed time window, and the kernel under test, launched on
 * another stream, runs on the m SMs left.  With `interfere` set the blocker
 * streams a 1 GB buffer from HBM meanwhile, the memory-intensive co-runner
 * of §3.3, so that C_interfered(m) / C(m) estimates the interference factor
 * k of the kernel's type.  Every CTA records its SM (%smid): a measurement
 * counts only if the two kernels ran on disjoint SMs, the kernel under test
 * on exactly m of them, and it finished inside the blocker's window; a
 * repetition that fails this is retried (at most 3 times per repetition).
 * No kernel waits on another: the blocker's window is a %globaltimer bound.
 *
 * Kernels under test, written from the published definitions of those §3
 * used (vector add, transpose, hotspot-like stencil) plus an FMA loop:
 * GPA_PROBE_VADD (n floats), GPA_PROBE_TRANSPOSE (n x n floats through 32 x
 * 32 tiles), GPA_PROBE_STENCIL (one 5-point sweep of an n x n grid),
 * GPA_PROBE_COMPUTE (64 dependent FMAs per each of n floats). */
enum { GPA_PROBE_VADD = 0, GPA_PROBE_TRANSPOSE = 1, GPA_PROBE_STENCIL = 2, GPA_PROBE_COMPUTE = 3 };

typedef struct {
  int32_t kernel;     /* GPA_PROBE_* */
  int32_t interfere;  /* 0: the blocked SMs idle; 1: they stream HBM */
  int64_t n;          /* problem size: elements (VADD, COMPUTE) or matrix side (TRANSPOSE, STENCIL) */
  int32_t reps;       /* timed repetitions per m (the median is reported), 1..100 */
  int32_t ctas;       /* CTAs of the kernel under test (0: 4 per SM of the whole GPU) */
} gpa_probe_cfg;

/* For each m[i] (1 <= m[i] <= the device's SM count): ms[i] = median device
 * time (CUDA events on the kernel's stream) of the kernel under test on
 * m[i] SMs, sms_used[i] = the SMs it ran on (m[i]), or ms[i] = -1 and
 * sms_used[i] = -1 when no repetition passed the placement check.  Device
 * buffers (3 arrays of the problem, 1 GB with `interfere`) are allocated
 * and freed by the call; it is synchronous and uses its own two streams.
 * Errors: GPA_ERR_ARG (NULL, bad kernel or counts), GPA_ERR_RANGE (n, m or
 * reps out of range: n in [1, 2^28] elements, side in [32, 16384]),
 * GPA_ERR_NOMEM, GPA_ERR_CUDA. */
int32_t gpa_measure_wcet(gpa_ctx* ctx, const gpa_probe_cfg* cfg, const int32_t* m, int32_t nm, double* ms,
                         int32_t* sms_used);

/* Least-squares fit of C(m) = a / m + b (§3.3's model without interference;
 * in the task model of this header, with times in microseconds, A = 1000 a
 * and B = 1000 b) to n points (m[i], ms[i]); points with ms[i] < 0 are
 * skipped.  Errors: GPA_ERR_ARG (NULL, fewer than two usable points or all
 * at one m). */
int32_t gpa_fit_wcet(const int32_t* m, const double* ms, int32_t n, double* a, double* b);

/* The kernel under test of gpa_measure_wcet run once, on the whole device,
 * on the caller's data, so that what it computes can be checked: `a` (and
 * `b` for GPA_PROBE_VADD; may be NULL otherwise) are host arrays of n
 * floats (VADD, COMPUTE) or n x n floats, row-major (TRANSPOSE, STENCIL);
 * `out` (host, same size) receives c = a + b (VADD), the transpose of a
 * (TRANSPOSE), one sweep c = a + 0.1 (left + right + up + down - 4 a) with
 * edge cells reusing their own value for a missing neighbour (STENCIL), or
 * y_64 with y_0 = 1, y_{k+1} = y_k a + 0.5 (COMPUTE, fused multiply-adds).
 * ctas = 0: 4 per SM.  Synchronous; allocates and frees its device buffers.
 * Errors as gpa_measure_wcet. */
int32_t gpa_probe_run(gpa_ctx* ctx, int32_t kernel, int64_t n, int32_t ctas, const float* a, const float* b,
                      float* out);

/* -------------------------------------- integer throughput of the device
 *
 * The ceiling against which the tests' throughput is reported: the rate at
 * which every SM of the context's device evaluates interference terms
 * ceil(R / T_j) C_j of the response-time iteration (§5.5) with the same
 * arithmetic the test kernels use (the period's reciprocal from shared
 * memory, a 32 x 32 -> 64-bit multiply and shift, a 64-bit product with C_j,
 * the D + 1 cap and a 64-bit sum), four independent iterations per thread,
 * all warps busy; and, for context, the rate of dependent-free 32-bit
 * integer multiply-adds.  Each is the best of five timed launches (CUDA
 * events on the context stream) of about 2-5 ms.  Synchronous; allocates
 * and frees a small device buffer. */
typedef struct {
  double terms_per_s;  /* interference terms per second, whole device */
  double imad_per_s;   /* 32-bit integer multiply-adds per second, whole device */
  double term_ms;      /* device time of the best term launch */
  int64_t terms;       /* terms evaluated by one term launch */
} gpa_alu_peak;
int32_t gpa_measure_alu_peak(gpa_ctx* ctx, gpa_alu_peak* out);

#ifdef __cplusplus
}
#endif

#endif /* GPA_H_ */
