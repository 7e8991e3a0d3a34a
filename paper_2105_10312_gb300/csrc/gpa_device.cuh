// gpa_device.cuh — device building blocks shared by the libgpa kernels.
//
//  * exact integer division by invariant divisors (Granlund & Montgomery,
//    "Division by invariant integers using multiplication", PLDI 1994,
//    Theorem 4.2), used for ceil(R / T_j) in the response-time iteration and
//    for the WCET's division by 10^6 m;
//  * staging of one task set from the caller's int64 structure-of-arrays
//    into shared memory in deadline-monotonic order;
//  * the WCET of §3.3/§7.1, C = ceil(k (A + B m) / (10^6 m)), with
//    the conflict rule of §4.2;
//  * the warp-cooperative per-partition response-time test of §5.5
//    and the minimum-size search of Alg. 2.
#pragma once

#include <cstdint>

#include "gpa.h"
#include "gpa_ns.h"

GPA_NS_BEGIN

constexpr unsigned kFull = 0xffffffffu;
constexpr int kNmax = GPA_KNMAX;
constexpr int kWords = kNmax / 32;        // 32-bit words of a task mask
constexpr int kIterCap = 1 << 20;         // response-time iterations per task before GPA_ERR_TIMEOUT

// error bits of the context's sticky error word
constexpr unsigned kErrRange = 1u;        // a set failed device-side validation
constexpr unsigned kErrIter = 2u;         // a per-partition test hit its step limit: undecided
constexpr unsigned kErrWait = 4u;         // a pipeline barrier wait hit its time limit

// floor(x / d) for 0 <= x < 2^60 and d = 10^6 m (m <= GPA_MMAX):
// magic = ceil(2^(60+l) / d) with l = ceil(log2 d), then
// floor(x / d) = floor(x * magic / 2^(60+l)) = umulhi64(x, magic) >> (l - 4).
struct MagicDiv {
  unsigned long long magic;
  unsigned int shift;  // l - 4
  unsigned int pad;
};

__device__ __forceinline__ unsigned long long div_by_1e6m(unsigned long long x, const MagicDiv& md) {
  return __umul64hi(x, md.magic) >> md.shift;
}

// 32-bit divisor T (1 <= T < 2^31), dividend n < 2^31:
// magic = ceil(2^(31+l) / T) < 2^32 with l = ceil(log2 T), shift = l;
// floor(n / T) = floor(n magic / 2^(31+l)) = floor(2n magic / 2^(32+l)): the
// high word of the 32 x 32-bit product (2n) magic, shifted right by l.
__device__ __forceinline__ void magic_for_period(unsigned int T, unsigned int* magic, unsigned int* shift) {
  unsigned int l = (T <= 1u) ? 0u : 32u - __clz(T - 1u);
  unsigned long long num = (1ull << (31 + l)) + T - 1;
  *magic = (unsigned int)(num / T);
  *shift = l;
}

// floor(n / T) from n2 = 2n (n < 2^31) and T's reciprocal.
__device__ __forceinline__ unsigned int floor_div_T2(unsigned int n2, unsigned int magic, unsigned int shift) {
  return __umulhi(n2, magic) >> shift;
}

// ceil(R / T) for 1 <= R <= 2^31 as floor((R - 1) / T) + 1.
__device__ __forceinline__ unsigned int ceil_div_T(unsigned int R, unsigned int magic, unsigned int shift) {
  return floor_div_T2(2u * (R - 1u), magic, shift) + 1u;
}

// WCET at m SMs with factor k per mille: ceil(k (A + B m) / (10^6 m)).
__device__ __forceinline__ unsigned int wcet(unsigned long long A, unsigned long long B, unsigned int k, unsigned int m,
                                             const MagicDiv& md) {
  unsigned long long x = (unsigned long long)k * (A + B * m);
  return (unsigned int)(div_by_1e6m(x - 1ull, md) + 1ull);
}

// Validation bounds of gpa.h for one task: 1 <= D <= T <= 2^31 - 1,
// A, B >= 0, 1 <= A + B <= 2^36, 0 <= u < 2^32, type in {0, 1}.  Written
// with unsigned ranges (a negative value wraps to a huge one), so each bound
// is one 64-bit compare.
__device__ __forceinline__ bool task_valid(long long T, long long D, long long A, long long B, long long u,
                                           unsigned int type) {
  const unsigned long long uT = (unsigned long long)T, uD = (unsigned long long)D;
  const unsigned long long uA = (unsigned long long)A, uB = (unsigned long long)B;
  return (uT >> 31) == 0ull && uD - 1ull < uT && uA <= (1ull << 36) && uB <= (1ull << 36) &&
         uA + uB - 1ull < (1ull << 36) && ((unsigned long long)u >> 32) == 0ull && type <= 1u;
}

// The admissible partition sizes of a model: every multiple of g in [g, M]
// (list == nullptr), or a listed increasing subset of them (whole GPCs or
// MIG slices, §2).  rank[m], m in [0, M + 1], counts the listed sizes < m.
struct Sizes {
  unsigned int M, g;
  const unsigned short* list;
  const unsigned short* rank;
  int n;
  // number of admissible sizes below m (m <= M + 1); unit 1 needs no division
  __device__ __forceinline__ int below(unsigned int m) const {
    if (!list) return m == 0u ? 0 : (int)(g == 1u ? m - 1u : (m - 1u) / g);
    return rank[m];
  }
  __device__ __forceinline__ int count() const { return list ? n : (int)(g == 1u ? M : M / g); }
  __device__ __forceinline__ unsigned int at(int k) const { return list ? (unsigned int)list[k] : (unsigned int)(k + 1) * g; }
  // smallest admissible size >= m (1 <= m), 0 if none
  __device__ __forceinline__ unsigned int next(unsigned int m) const {
    if (m > M) return 0u;
    const int k = below(m);
    return k < count() ? at(k) : 0u;
  }
  __device__ __forceinline__ bool admissible(unsigned int m) const {
    return m >= 1u && m <= M && below(m + 1u) - below(m) == 1 && (list || m % g == 0u);
  }
};

// Lemma 2 in closed form: the smallest admissible size m with C^n(m) <= D,
// i.e. 1000 (A + B m) <= 10^6 D m  <=>  A <= m (1000 D - B).  Returns 0 when
// no admissible size qualifies.
__device__ __forceinline__ unsigned int lemma2_size(unsigned long long A, unsigned long long B, unsigned long long D,
                                                    const Sizes& z) {
  long long den = (long long)(1000ull * D) - (long long)B;
  if (den < 0) return 0u;
  unsigned long long m1;
  if (A == 0ull) m1 = 1ull;
  else if (den == 0) return 0u;
  else m1 = (A + (unsigned long long)den - 1ull) / (unsigned long long)den;
  if (m1 < 1ull) m1 = 1ull;
  return m1 <= z.M ? z.next((unsigned int)m1) : 0u;
}

// The same size without 64-bit division: if A <= M (1000 D - B), the
// quotient q = ceil(A / den) is at most M <= 1024, so a float estimate is
// within one of it and two exact integer checks settle it.  m_one is the
// smallest admissible size.
__device__ __forceinline__ unsigned int lemma2_size_fast(unsigned long long A, unsigned long long B,
                                                         unsigned long long D, const Sizes& z, unsigned int m_one) {
  const unsigned int M = z.M;
  const long long den = (long long)(1000ull * D) - (long long)B;
  if (den < 0) return 0u;
  if (A == 0ull) return m_one;
  if (den == 0) return 0u;
  const unsigned long long ud = (unsigned long long)den;
  if (A <= ud) return m_one;  // one SM already meets the deadline (the common case)
  if (A > ud * M) return 0u;
  unsigned int q = (unsigned int)__fdividef((float)A, (float)ud);
  q = min(max(q, 1u), M);
  if ((unsigned long long)q * ud < A) q++;                        // estimate too small by one
  if ((unsigned long long)q * ud < A) q++;
  if (q > 1u && (unsigned long long)(q - 1u) * ud >= A) q--;      // estimate too large by one
  if (q > 1u && (unsigned long long)(q - 1u) * ud >= A) q--;
  if (!z.list) {
    const unsigned int mg = (z.g == 1u) ? q : (q + z.g - 1u) / z.g * z.g;
    return mg <= M ? mg : 0u;
  }
  return z.next(q);
}

// One task set staged in shared memory, rows in deadline-monotonic order
// (D ascending, then T, then original index).
struct SetSmem {
  unsigned long long key[kNmax];  // staging: deadline-monotonic sort key (D, T) of each original task
  unsigned int T[kNmax];
  unsigned int D[kNmax];
  unsigned int mT[kNmax];    // Granlund-Montgomery magic of T
  unsigned char shT[kNmax];  // its shift
  unsigned char orig[kNmax]; // original index of the row's task
  unsigned long long A[kNmax];
  unsigned long long B[kNmax];
  unsigned int u[kNmax];
  float rT[kNmax];               // 1 / T (float, correctly rounded)
  unsigned int memmask[kWords];  // rows holding memory-intensive tasks
  int n;
};

// Per-warp scratch of the response-time test: the partition's tasks,
// compacted in priority order.
struct RtaScratch {
  uint2 cm[kNmax];  // .x: the task's WCET at the tested size, .y: the reciprocal of its period
  unsigned int T[kNmax];
  unsigned int D[kNmax];
  unsigned char sh[kNmax];
  unsigned char pos[kNmax];
  unsigned int Rcur[kNmax];  // verdict-only test: each task's latest iterate (saturated at 2^32 - 1)
  float Uex[kNmax];          // float sum of C_j / T_j over the tasks before each (when every C <= D)
  unsigned long long Cin[kNmax];  // sum of the WCETs up to and including each task (when every C <= D)
  unsigned char need[kNmax];      // verdict-only test: the tasks the utilisation bound leaves undecided
  // interference terms evaluated by this warp's tests: ceil(R / T_j) C_j of
  // the response-time iteration, or one task's demand of an EDF step
  unsigned long long terms;
};

// Adds the lanes' term counts (each below 2^32) to a per-warp counter.
__device__ __forceinline__ void warp_add_terms(unsigned long long& total, unsigned int nt) {
  const unsigned int lo = __reduce_add_sync(0xffffffffu, nt & 0xFFFFu), hi = __reduce_add_sync(0xffffffffu, nt >> 16);
  if ((threadIdx.x & 31) == 0) total += ((unsigned long long)hi << 16) + lo;
}

// Stage set [o, o + n) into st (warp-cooperative).  Returns false (on all
// lanes) if any task violates the validation bounds.
__device__ __forceinline__ bool stage_set(SetSmem& st, long long o, int n, const long long* __restrict__ T,
                                          const long long* __restrict__ D, const long long* __restrict__ A,
                                          const long long* __restrict__ B, const long long* __restrict__ u,
                                          const unsigned char* __restrict__ type) {
  const int lane = threadIdx.x & 31;
  long long Tv[kWords], Dv[kWords];
  unsigned int ty[kWords];
  bool ok = true;
  // first pass: load and validate; keep (D, T) for ranking
  for (int c = 0; c < kWords; c++) {
    int t = c * 32 + lane;
    Tv[c] = 0;
    Dv[c] = 0;
    ty[c] = 0;
    if (t < n) {
      long long Tt = __ldg(T + o + t), Dt = __ldg(D + o + t), At = __ldg(A + o + t), Bt = __ldg(B + o + t);
      long long ut = u ? __ldg(u + o + t) : 0;
      unsigned int yt = __ldg(type + o + t);
      ok = ok && task_valid(Tt, Dt, At, Bt, ut, yt);
      Tv[c] = Tt;
      Dv[c] = Dt;
      ty[c] = yt;
      // temporary: stash original-order values in the A/B/u rows of the
      // original index; they are permuted below
      st.A[t] = (unsigned long long)At;
      st.B[t] = (unsigned long long)Bt;
      st.u[t] = (unsigned int)ut;
      st.key[t] = ((unsigned long long)Dt << 31) | (unsigned long long)Tt;
    }
  }
  ok = __all_sync(kFull, ok);
  if (!ok) return false;
  __syncwarp();
  // DM rank of each task by counting: smaller (D, T), or the same and a
  // lower index
  int rank[kWords];
  for (int c = 0; c < kWords; c++) {
    int t = c * 32 + lane;
    int r = 0;
    if (t < n) {
      const unsigned long long key = ((unsigned long long)Dv[c] << 31) | (unsigned long long)Tv[c];
      for (int j = 0; j < t; j++) r += st.key[j] <= key;
      for (int j = t + 1; j < n; j++) r += st.key[j] < key;
    }
    rank[c] = r;
  }
  // gather original-order values into registers, then scatter by rank
  unsigned long long Av[kWords], Bv[kWords];
  unsigned int uv[kWords];
  for (int c = 0; c < kWords; c++) {
    int t = c * 32 + lane;
    if (t < n) {
      Av[c] = st.A[t];
      Bv[c] = st.B[t];
      uv[c] = st.u[t];
    }
  }
  __syncwarp();
  for (int w = 0; w < kWords; w++) st.memmask[w] = 0u;  // lanes write the same value
  __syncwarp();
  for (int c = 0; c < kWords; c++) {
    int t = c * 32 + lane;
    if (t < n) {
      int r = rank[c];
      st.T[r] = (unsigned int)Tv[c];
      st.rT[r] = __frcp_rn((float)Tv[c]);
      st.D[r] = (unsigned int)Dv[c];
      unsigned int mg, sh;
      magic_for_period((unsigned int)Tv[c], &mg, &sh);
      st.mT[r] = mg;
      st.shT[r] = (unsigned char)sh;
      st.orig[r] = (unsigned char)t;
      st.A[r] = Av[c];
      st.B[r] = Bv[c];
      st.u[r] = uv[c];
    }
  }
  // memory mask by rank
  for (int c = 0; c < kWords; c++) {
    int t = c * 32 + lane;
    bool mem = (t < n) && ty[c] == 1u;
    int r = rank[c];
    // each lane sets its bit with an atomic on shared memory
    if (mem) atomicOr(&st.memmask[r >> 5], 1u << (r & 31));
  }
  if (lane == 0) st.n = n;
  __syncwarp();
  return true;
}

__device__ __forceinline__ int mask_popc(const unsigned int* S) {
  int c = 0;
#pragma unroll
  for (int w = 0; w < kWords; w++) c += __popc(S[w]);
  return c;
}

// Inflated workload W(S) = sum_{i in S} k_i(S) u_i from the per-type sums.
__device__ __forceinline__ unsigned long long workload_from_sums(unsigned long long Uc, unsigned long long Um, int nc,
                                                                 int nm, unsigned int kc, unsigned int km) {
  return (unsigned long long)(nc >= 2 ? kc : 1000u) * Uc + (unsigned long long)(nm >= 2 ? km : 1000u) * Um;
}

// §5.5 per-partition test, warp-cooperative: the tasks of S (rows of st, a
// mask in priority order) on one processor of m SMs.  Lane l owns the l-th,
// (l+32)-th, ... task of S; its fixed point reads the higher-priority tasks
// from the compacted scratch (broadcast shared-memory reads).
// If R_row != nullptr, R_row[row] receives the response time or -1.
// With early_exit the test stops at the first deadline miss (verdict only).
// Returns the verdict on every lane.  *err |= kErrIter if the iteration cap
// was reached (the verdict is then 0).
// Compacts S's rows (priority order) into sc with their WCETs at m SMs
// (conflict factors of §4.2); returns the number of tasks (every lane).
__device__ __forceinline__ int compact_partition(const SetSmem& st, const unsigned int* S, unsigned int m,
                                                 unsigned int kc, unsigned int km, const MagicDiv& md,
                                                 RtaScratch& sc) {
  const int lane = threadIdx.x & 31;
  int nm = 0, ns = 0;
#pragma unroll
  for (int w = 0; w < kWords; w++) {
    nm += __popc(S[w] & st.memmask[w]);
    ns += __popc(S[w]);
  }
  const unsigned int kmem = nm >= 2 ? km : 1000u;
  const unsigned int kcmp = (ns - nm) >= 2 ? kc : 1000u;
  int base = 0;
  for (int w = 0; w < kWords && w * 32 < st.n; w++) {
    unsigned int word = S[w];
    if (word) {
      int row = w * 32 + lane;
      if ((word >> lane) & 1u) {
        int idx = base + __popc(word & ((1u << lane) - 1u));
        bool mem = (st.memmask[w] >> lane) & 1u;
        sc.cm[idx] = make_uint2(wcet(st.A[row], st.B[row], mem ? kmem : kcmp, m, md), st.mT[row]);
        sc.T[idx] = st.T[row];
        sc.sh[idx] = st.shT[row];
        sc.D[idx] = st.D[row];
        sc.pos[idx] = (unsigned char)row;
      }
      base += __popc(word);
    }
  }
  __syncwarp();
  return base;
}

// A lower bound of task i's least fixed point from the utilisation U_hp of
// the tasks before it (Sjodin & Hansson, 1998): R = C_i + sum ceil(R / T_j)
// C_j >= C_i + R U_hp, so R >= C_i / (1 - U_hp), and there is no fixed
// point when U_hp >= 1.  uhp is a float sum of the C_j / T_j (each at most
// 1, at most 255 of them, each quotient from __fdividef: within 2 ulp) within
// 2^-15 of U_hp; the bound uses uhp - 2^-14 and rounds down with a 2^-20
// margin (its own quotient within 2 ulp too), so it never exceeds the fixed
// point.
// Returns 2^32 (above every deadline) when U_hp >= 1 is proven.
__device__ __forceinline__ unsigned long long util_start(unsigned int Ci, float uhp) {
  const float u = uhp - 0x1p-14f;
  if (u <= 0.0f) return Ci;
  if (u >= 1.0f) return 1ull << 32;
  const float b = __fdividef((float)Ci, 1.0f - u) * (1.0f - 0x1p-20f);
  if (!(b < 4294967296.0f)) return 1ull << 32;
  const unsigned long long lb = (unsigned long long)b;
  return lb > Ci ? lb : (unsigned long long)Ci;
}

// An upper bound of task i's least fixed point, the counterpart of util_start.
// With f(t) = C_i + sum_{j<i} ceil(t / T_j) C_j and ceil(t / T_j) C_j <=
// t U_j + C_j, the value X = (C_i + sum_{j<i} C_j) / (1 - U_hp) satisfies
// f(X) <= X U_hp + C_i + sum_{j<i} C_j = X.  f is non-decreasing, so every
// iterate started at or below the least fixed point stays at or below X, and
// R_i <= X: X <= D_i proves that task i meets its deadline without iterating.
// uhp is within 2^-15 of U_hp (see util_start) and chp is the exact sum of
// the C_j.  X <= D_i is tested as (C_i + sum C_j) <= D_i (1 - U_hp), with
// U_hp + 2^-14 for U_hp and the left side raised by 2^-17, which covers the
// five roundings of the two sides (conversions, 1 - u, products; each at most
// 2^-24 relative), so a true result is never wrong.
__device__ __forceinline__ bool util_pass(unsigned int Ci, unsigned long long chp, float uhp, unsigned int Di) {
  const float u = uhp + 0x1p-14f;
  return u < 1.0f && (float)(chp + Ci) * (1.0f + 0x1p-17f) <= (float)Di * (1.0f - u);
}

// A float sum of the terms C_i / T_i (each at most 1, each within 2 ulp) of
// at most 256 tasks is within 2^-15 of U when U <= 1, so a sum above 1 + 2^-13 proves U > 1,
// and with it a miss under any policy on one processor.
constexpr float kUtilFail = 1.0f + 0x1p-13f;

// One step of task i's response-time iteration: next = C_i + sum_{j<i}
// ceil(R / T_j) C_j over the compacted tasks (uncapped when every C_j <= D_j,
// see warp_rta).  Uncapped, ceil(R / T_j) = floor((R - 1) / T_j) + 1 and the
// +1 terms add up to C_0 + ... + C_{i-1}: next = Cin[i] + sum floor(...) C_j.
__device__ __forceinline__ unsigned long long rta_step(const RtaScratch& sc, int i, unsigned long long R,
                                                      unsigned int Ci, unsigned int Di, bool c_le_d) {
  const unsigned int Rc = (unsigned int)R;
  unsigned long long next;
  if (c_le_d) {
    next = sc.Cin[i];
    const unsigned int R2 = 2u * (Rc - 1u);
    for (int j = 0; j < i; j++) {
      const uint2 v = sc.cm[j];  // one 8-byte broadcast load: C_j and T_j's reciprocal
      next += (unsigned long long)floor_div_T2(R2, v.y, sc.sh[j]) * v.x;
    }
  } else {
    next = Ci;
    // terms capped at D_i + 1: a capped term already puts the sum above D_i
    const unsigned long long cap = (unsigned long long)Di + 1ull;
    for (int j = 0; j < i; j++) {
      const uint2 v = sc.cm[j];
      const unsigned long long t = (unsigned long long)ceil_div_T(Rc, v.y, sc.sh[j]) * v.x;
      next += t < cap ? t : cap;
    }
  }
  return next;
}

// Verdict-only response-time test of the q tasks listed in sc.need (indices
// of compacted tasks in priority order: those util_pass could not settle),
// lanes taking tasks in list order as they finish: lane l starts with the
// l-th, and a lane whose task reached its fixed point takes the next
// unassigned one, so no lane idles while another iterates.  Task i starts at
// the larger of util_start and a bound from the last task q assigned before
// it: R_i >= R_q + C_{q+1} + ... + C_i (each task's least fixed point is at
// least the previous one's plus its own WCET), with R_q replaced by q's
// latest iterate, which is at most R_q.  The first tasks start at
// C_0 + ... + C_i.  Returns false at the first step in which some task
// passed its deadline (or hit the step limit: *eb |= kErrIter).  Every
// C_j <= D_j, so the sums need no cap (see warp_rta).
__device__ __forceinline__ bool rta_verdict(RtaScratch& sc, int q, unsigned int* eb, unsigned int& nt) {
  const int lane = threadIdx.x & 31;
  const unsigned int lt = (1u << lane) - 1u;
  int i = lane < q ? sc.need[lane] : -1;
  unsigned int Ci = i >= 0 ? sc.cm[i].x : 0u, Di = i >= 0 ? sc.D[i] : 0u;
  unsigned long long R = 0ull;
  if (i >= 0) {
    const unsigned long long lb = util_start(Ci, sc.Uex[i]);
    R = lb > sc.Cin[i] ? lb : sc.Cin[i];
  }
  int next = q < 32 ? q : 32;  // the first list position not yet assigned
  int iter = 0;
  bool probe = true;  // the task's first step evaluates f(D_i) (see rta_verdict_seq)
  for (;;) {
    bool miss = false, conv = i < 0;
    if (i >= 0) {
      if (R > Di) {
        miss = true;
      } else if (probe) {
        probe = false;
        conv = rta_step(sc, i, Di, Ci, Di, true) <= Di;
        nt += (unsigned int)i;
      } else {
        const unsigned long long nx = rta_step(sc, i, R, Ci, Di, true);
        nt += (unsigned int)i;
        if (nx == R) {
          conv = true;
        } else {
          R = nx;
          if (++iter > kIterCap) {
            *eb |= kErrIter;
            miss = true;
          }
        }
      }
      sc.Rcur[i] = R > 0xffffffffull ? 0xffffffffu : (unsigned int)R;
    }
    if (__any_sync(kFull, miss)) return false;
    const unsigned int freem = __ballot_sync(kFull, conv);
    if (next >= q) {
      if (freem == kFull) return true;
      if (conv) i = -1;
      continue;  // nothing left to assign
    }
    if (freem == 0u) continue;  // no lane is free
    __syncwarp();
    // free lanes take list positions next, next + 1, ... in lane order
    const int idx = next + __popc(freem & lt);
    const int prev = sc.need[next - 1];  // the last task assigned so far
    if (conv && idx < q) {
      i = sc.need[idx];
      Ci = sc.cm[i].x;
      Di = sc.D[i];
      R = (unsigned long long)sc.Rcur[prev] + (sc.Cin[i] - sc.Cin[prev]);
      const unsigned long long lb = util_start(Ci, sc.Uex[i]);
      R = lb > R ? lb : R;
      iter = 0;
      probe = true;
    } else if (conv) {
      i = -1;
    }
    next = min(q, next + __popc(freem));
    __syncwarp();
  }
}

// Lists of at most this many undecided tasks are tested one task at a time
// by the whole warp (rta_verdict_seq), longer ones a task per lane.
constexpr int kSeqTasksMax = 16;

// Verdict-only response-time test of the q tasks listed in sc.need, one task
// at a time by the whole warp: in a step of task i, lane l evaluates the
// terms of tasks l, l + 32, ... below i, and the warp adds them.  Task i
// starts at the larger of util_start and R_p + C_{p+1} + ... + C_i, p being
// the listed task before it and R_p its least fixed point (the first at
// C_0 + ... + C_i).  Returns false as soon as a task passes its deadline (or
// hits the step limit: *eb |= kErrIter).  Every C_j <= D_j, so the sums need
// no cap (see warp_rta); a lane's terms each stay below 2^32, at most
// kNmax / 32 of them, so the halves of its sum below 2^16 and above add up
// without overflow in 32-bit warp reductions.
__device__ __forceinline__ bool rta_verdict_seq(const RtaScratch& sc, int q, unsigned int* eb, unsigned int& nt) {
  const int lane = threadIdx.x & 31;
  unsigned long long Rp = 0ull, Cp = 0ull;
  for (int k = 0; k < q; k++) {
    const int i = sc.need[k];
    const unsigned int Ci = sc.cm[i].x, Di = sc.D[i];
    unsigned long long R = Rp + (sc.Cin[i] - Cp);
    const unsigned long long lb = util_start(Ci, sc.Uex[i]);
    R = lb > R ? lb : R;
    int iter = 0;
    const unsigned long long Cin = sc.Cin[i];
    if (R > Di) return false;
    // R_i is the least t with f(t) <= t (f: the step's function, which is
    // non-decreasing), so f(D_i) <= D_i proves R_i <= D_i: one evaluation at
    // D_i first; R (at most R_i) then serves the next listed task's start
    bool probe = true;
    for (;;) {
      if (R > Di) return false;
      // next = C_0 + ... + C_i + sum_{j<i} floor((t - 1) / T_j) C_j (see
      // rta_step) at t = D_i for the probe, else at t = R
      const unsigned int R2 = 2u * ((probe ? Di : (unsigned int)R) - 1u);
      unsigned long long part = 0ull;
      for (int j = lane; j < i; j += 32) {
        const uint2 v = sc.cm[j];
        part += (unsigned long long)floor_div_T2(R2, v.y, sc.sh[j]) * v.x;
      }
      const unsigned int lo = __reduce_add_sync(kFull, (unsigned int)(part & 0xFFFFull));
      const unsigned int hi = __reduce_add_sync(kFull, (unsigned int)(part >> 16));
      const unsigned long long next = Cin + ((unsigned long long)hi << 16) + lo;
      if (lane == 0) nt += (unsigned int)i;
      if (probe) {
        probe = false;
        if (next <= Di) break;
        continue;
      }
      if (next == R) break;
      R = next;
      if (++iter > kIterCap) {
        *eb |= kErrIter;
        return false;
      }
    }
    Rp = R;
    Cp = sc.Cin[i];
  }
  return true;
}

static __device__ __noinline__ bool warp_rta(const SetSmem& st, const unsigned int* S, unsigned int m, unsigned int kc,
                                      unsigned int km, const MagicDiv* __restrict__ mdiv, RtaScratch& sc,
                                      long long* R_row, bool early_exit, unsigned int* err) {
  const int lane = threadIdx.x & 31;
  const int s = compact_partition(st, S, m, kc, km, mdiv[m], sc);
  // Every C_j <= D_j (<= T_j) bounds each term ceil(R / T_j) C_j by R + T_j
  // < 2^32 while R <= D < 2^31, so the sums need no cap; a task with
  // C > D misses.  For a verdict alone, such a task or U > 1 decides it at
  // once.
  bool c_le_d = true;
  float uf = 0.0f;
  for (int i = lane; i < s; i += 32) {
    const unsigned int C = sc.cm[i].x;
    c_le_d = c_le_d && C <= sc.D[i];
    uf += __fdividef((float)C, (float)sc.T[i]);
  }
  c_le_d = __all_sync(kFull, c_le_d);
  if (early_exit) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) uf += __shfl_xor_sync(kFull, uf, o);
    if (!c_le_d || uf > kUtilFail) return false;
  }
  bool all_ok = true;
  unsigned int errbits = 0u, nt = 0u;
  const bool verdict_only = early_exit && !R_row;
  int q = 0;  // verdict only: tasks util_pass leaves undecided
  if (c_le_d) {
    // exclusive prefix sums of C_j / T_j and inclusive ones of C_j, chunk by
    // chunk; for a verdict, the list of tasks util_pass does not settle
    float carry = 0.0f;
    unsigned long long ccarry = 0ull;
    const unsigned int lt = (1u << lane) - 1u;
    for (int c0 = 0; c0 < s; c0 += 32) {
      const int i = c0 + lane;
      const unsigned int C = i < s ? sc.cm[i].x : 0u;
      float u = i < s ? __fdividef((float)C, (float)sc.T[i]) : 0.0f;
      float incl = u;
      unsigned long long cin = C;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const float v = __shfl_up_sync(kFull, incl, o);
        const unsigned long long w = __shfl_up_sync(kFull, cin, o);
        if (lane >= o) {
          incl += v;
          cin += w;
        }
      }
      const float uex = carry + (incl - u);
      cin += ccarry;
      if (i < s) {
        sc.Uex[i] = uex;
        sc.Cin[i] = cin;
      }
      if (verdict_only) {
        const bool nd = i < s && !util_pass(C, cin - C, uex, sc.D[i]);
        const unsigned int b = __ballot_sync(kFull, nd);
        if (nd) sc.need[q + __popc(b & lt)] = (unsigned char)i;
        q += __popc(b);
      }
      carry += __shfl_sync(kFull, incl, 31);
      ccarry = __shfl_sync(kFull, cin, 31);
    }
    __syncwarp();
  }
  if (verdict_only) {
    all_ok = q == 0 || (q <= kSeqTasksMax ? rta_verdict_seq(sc, q, &errbits, nt) : rta_verdict(sc, q, &errbits, nt));
    errbits = __reduce_or_sync(kFull, errbits);
    if (errbits && lane == 0) atomicOr(err, errbits);
    warp_add_terms(sc.terms, nt);
    __syncwarp();
    return all_ok;
  }
  // Start values: the least fixed points grow along the priority order by at
  // least each task's own WCET (R_i >= R_{i-1} + C_i), so task i starts at
  // R_last + C_{c0} + ... + C_i, R_last being where the previous chunk's last
  // task stopped (its fixed point, or an iterate below it); every start is
  // at most the fixed point, so the iteration reaches the same one.
  unsigned long long Rlast = 0ull;
  for (int c0 = 0; c0 < s; c0 += 32) {
    const int i = c0 + lane;
    const bool active = i < s;
    unsigned int Ci = 0, Di = 0;
    if (active) {
      Ci = sc.cm[i].x;
      Di = sc.D[i];
    }
    unsigned long long pre = Ci;  // inclusive prefix sum of the chunk's WCETs
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long v = __shfl_up_sync(kFull, pre, o);
      if (lane >= o) pre += v;
    }
    unsigned long long R = active ? Rlast + pre : 0ull;
    if (c_le_d && active) {
      const unsigned long long lb = util_start(Ci, sc.Uex[i]);
      R = lb > R ? lb : R;
    }
    bool done = !active, ok = true;
    int iter = 0;
    while (__any_sync(kFull, !done)) {
      if (!done) {
        if (R > Di) {
          ok = false;
          done = true;
        } else {
          const unsigned long long next = rta_step(sc, i, R, Ci, Di, c_le_d);
          nt += (unsigned int)i;
          if (next == R) done = true;
          else R = next;
          if (++iter > kIterCap) {
            ok = false;
            done = true;
            errbits |= kErrIter;
          }
        }
      }
      if (early_exit && __any_sync(kFull, !ok)) break;
    }
    if (R_row && active) R_row[sc.pos[i]] = ok ? (long long)R : -1LL;
    all_ok = __all_sync(kFull, ok) && all_ok;
    if (early_exit && !all_ok) break;
    Rlast = __shfl_sync(kFull, R, min(31, s - 1 - c0));
  }
  errbits = __reduce_or_sync(kFull, errbits);
  if (errbits && lane == 0) atomicOr(err, errbits);
  warp_add_terms(sc.terms, nt);
  __syncwarp();
  return all_ok;
}

// ------------------------------------------------------------------ EDF
//
// Second per-partition policy (the paper leaves §5.5's policy open):
// preemptive EDF on the partition as one processor, synchronous periodic
// release, constrained deadlines.  Exact processor-demand criterion: every
// deadline is met iff U <= 1 and dbf(t) <= t at every absolute deadline up to
// L, with dbf(t) = sum_{D_i <= t} (floor((t - D_i)/T_i) + 1) C_i (Baruah,
// Rosier & Howell, 1990).  Evaluated by QPA (Zhang & Burns, 2009): start from
// the largest absolute deadline t < L and repeat
//     h = dbf(t);  h > t: miss;  h <= d_min: schedulable;
//     t = h if h < t, else the largest absolute deadline below t,
// where L = min(L_a, L_b): L_a = max(D_max, sum (T_i - D_i) U_i / (1 - U))
// (bounded from above in floating point with a margin, when U < 1) and L_b
// the synchronous busy period (least fixed point of sum ceil(w/T_i) C_i).
// U is compared with 1 exactly: a float sum first (it is within 2^-14 of U),
// then, near 1, integer terms floor(2^64 C_i / T_i) (U 2^64 lies in
// [sum, sum + number of inexact terms)), then, if that still straddles 1,
// the exact fraction over the periods' least common multiple when it stays
// below 2^62.  One task passes iff C <= D; a task with C > D misses at t = D.
// When an analysis cannot finish -- U within n 2^-64 of 1 with periods whose
// least common multiple exceeds 2^62, a busy period beyond 2^62, or more than
// kIterCap busy-period or QPA steps -- the test is undecided: it sets
// kErrIter in *err and returns false, and the caller reports the set as
// undecided (never as a miss).
// Values stay below 2^63: C <= D <= T bounds each demand term by t + C.

constexpr unsigned long long kEdfLmax = 1ull << 62;  // also "no L_a bound"
constexpr unsigned long long kEdfLcmMax = 1ull << 62;

// Float screen: uf = sum of float C_i / T_i is within 2^-14 of U for n <= 256
// (each term within 3 ulp, the sums within n ulp: at most 2^-16 of U for
// U <= 2).  uf above kEdfFail proves U > 1, below kEdfPass proves
// 1 - U >= 1 - uf - 2^-14.
constexpr float kEdfPass = 1.0f - 0x1p-13f;
constexpr float kEdfFail = 1.0f + 0x1p-13f;
// Density: sum C_i / D_i <= 1 makes a constrained-deadline set EDF-feasible
// (dbf(t) <= sum C_i (t / D_i) <= t); the float sum is within 2^-14 of the
// exact one, so dens <= 1 - 2^-14 proves it.
constexpr float kEdfDensity = 1.0f - 0x1p-14f;

// 128-bit unsigned (hi, lo) accumulation.
struct U128 {
  unsigned long long hi, lo;
};
__device__ __forceinline__ void add128(U128& a, unsigned long long bhi, unsigned long long blo) {
  const unsigned long long lo = a.lo + blo;
  a.hi += bhi + (lo < a.lo ? 1ull : 0ull);
  a.lo = lo;
}

// Adds floor(2^64 C / T) to q and counts an inexact term in nz (C <= T < 2^31):
// long division in base 2^32, q1 = floor(C 2^32 / T) <= 2^32, then the next
// 32 bits from the remainder.
__device__ __forceinline__ void edf_uterm64(unsigned int C, unsigned int T, U128& q, unsigned int& nz) {
  const unsigned long long n1 = (unsigned long long)C << 32;
  const unsigned long long q1 = n1 / T, r1 = n1 - q1 * T;
  const unsigned long long n2 = r1 << 32;
  const unsigned long long q2 = n2 / T, r2 = n2 - q2 * T;
  add128(q, q1 >> 32, (q1 << 32) + q2);
  nz += r2 != 0ull ? 1u : 0u;
}

// Sign of U - 1 from q = sum floor(2^64 C_i / T_i) and nz inexact terms:
// -1, 0 or 1, or 2 when U 2^64 in [q, q + nz) straddles 2^64.  With -1,
// *gap gets a lower bound of 1 - U (possibly 0).
__device__ __forceinline__ int edf_classify64(const U128& q, unsigned int nz, double* gap) {
  if (q.hi > 1ull || (q.hi == 1ull && q.lo != 0ull)) return 1;
  if (q.hi == 1ull) return nz == 0u ? 0 : 1;
  // q < 2^64: the gap 2^64 - q, as an integer
  const unsigned long long g = 0ull - q.lo;  // 2^64 - lo (lo > 0 since every C >= 1)
  if (nz == 0u) {
    *gap = (double)g * 0x1p-64 * (1.0 - 0x1p-50);
    return -1;
  }
  if (q.lo == 0ull || g >= nz) {
    *gap = q.lo == 0ull ? 1.0 - 0x1p-50 : (double)(g - nz) * 0x1p-64 * (1.0 - 0x1p-50);
    return -1;
  }
  return 2;
}

__device__ __forceinline__ unsigned long long gcd64(unsigned long long a, unsigned long long b) {
  while (b) {
    const unsigned long long r = a % b;
    a = b;
    b = r;
  }
  return a;
}

// Sign of U - 1 over the k tasks get(a, C, T) yields, exactly, by the
// periods' least common multiple H: U - 1 = (sum C_i H / T_i - H) / H.
// Returns 2 when H exceeds 2^62.
template <class Get>
__device__ int edf_lcm_classify(int k, Get get) {
  unsigned long long H = 1ull;
  for (int a = 0; a < k; a++) {
    unsigned int C, T;
    get(a, C, T);
    const unsigned long long f = T / gcd64(H, T);
    if (H > kEdfLcmMax / f) return 2;
    H *= f;
  }
  U128 N{0ull, 0ull};
  for (int a = 0; a < k; a++) {
    unsigned int C, T;
    get(a, C, T);
    const unsigned long long term = (H / T) * C;  // <= H since C <= T
    add128(N, 0ull, term);
  }
  if (N.hi != 0ull || N.lo > H) return 1;
  return N.lo == H ? 0 : -1;
}

// L_a from a numerator bound num >= sum (T_i - D_i) U_i and gap <= 1 - U:
// num / gap rounded up with margins, at least D_max; kEdfLmax when that
// reaches 2^62 or gap is 0 (no usable bound).
__device__ __forceinline__ unsigned long long edf_la(double num, double gap, unsigned int dmax) {
  if (!(gap > 0.0)) return kEdfLmax;
  const double la = num * (1.0 + 0x1p-20) / gap * (1.0 + 0x1p-30) + 2.0;
  if (!(la < (double)kEdfLmax)) return kEdfLmax;
  const unsigned long long up = (unsigned long long)la;
  return up > dmax ? up : (unsigned long long)dmax;
}

__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long w = __shfl_xor_sync(kFull, v, o);
    v = w > v ? w : v;
  }
  return v;
}

__device__ __forceinline__ double warp_sum_f64(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

__device__ __forceinline__ unsigned long long warp_sum_u64_edf(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

__device__ __forceinline__ U128 warp_sum_u128(U128 v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long hi = __shfl_xor_sync(kFull, v.hi, o), lo = __shfl_xor_sync(kFull, v.lo, o);
    add128(v, hi, lo);
  }
  return v;
}

// floor(x / T) and ceil(x / T) for 64-bit x: the period's reciprocal while
// x stays below 2^31 (the common case), a 64-bit division above.
__device__ __forceinline__ unsigned long long floor_div_T64(unsigned long long x, unsigned int T, unsigned int mg,
                                                            unsigned int sh) {
  return x < 0x7fffffffull ? (unsigned long long)(ceil_div_T((unsigned int)x + 1u, mg, sh) - 1u) : x / T;
}

__device__ __forceinline__ unsigned long long ceil_div_T64(unsigned long long x, unsigned int T, unsigned int mg,
                                                           unsigned int sh) {
  if (x == 0ull) return 0ull;
  return x < 0x80000000ull ? (unsigned long long)ceil_div_T((unsigned int)x, mg, sh) : (x + T - 1ull) / T;
}

// The largest absolute deadline k T + D (k >= 0) strictly below t, or 0.
__device__ __forceinline__ unsigned long long edf_deadline_below(unsigned long long t, unsigned int T, unsigned int D,
                                                                 unsigned int mg, unsigned int sh) {
  if (t <= D) return 0ull;
  return floor_div_T64(t - 1ull - D, T, mg, sh) * T + D;
}

// Warp-cooperative EDF test of S at m SMs; lane l holds the compacted tasks
// l, l + 32, ...  Returns the verdict on every lane; an undecided test sets
// kErrIter in *err and returns false.
static __device__ __noinline__ bool warp_edf(const SetSmem& st, const unsigned int* S, unsigned int m, unsigned int kc,
                                      unsigned int km, const MagicDiv* __restrict__ mdiv, RtaScratch& sc,
                                      unsigned int* err) {
  const int lane = threadIdx.x & 31;
  const int s = compact_partition(st, S, m, kc, km, mdiv[m], sc);
  if (s == 0) return true;
  if (s == 1) return sc.cm[0].x <= sc.D[0];
  bool late = false;
  unsigned long long csum = 0;
  float uf = 0.0f;
  double numf = 0.0;
  unsigned int dmin = 0xffffffffu, dmax = 0u;
  float dens = 0.0f;
  for (int i = lane; i < s; i += 32) {
    const unsigned int C = sc.cm[i].x, T = sc.T[i], D = sc.D[i];
    late = late || C > D;
    const float r = (float)C / (float)T;
    uf += r;
    dens += (float)C / (float)D;
    numf += (double)(T - D) * (double)r;
    csum += C;
    dmin = min(dmin, D);
    dmax = max(dmax, D);
  }
  if (__any_sync(kFull, late)) return false;
  uf = (float)warp_sum_f64((double)uf);  // the butterfly leaves the same sum on every lane
  dens = (float)warp_sum_f64((double)dens);
  csum = warp_sum_u64_edf(csum);
  dmin = __reduce_min_sync(kFull, dmin);
  dmax = __reduce_max_sync(kFull, dmax);
  if (uf > kEdfFail) return false;
  if (dens <= kEdfDensity) return true;  // density <= 1 suffices
  unsigned long long La;
  if (uf < kEdfPass) {
    La = edf_la(warp_sum_f64(numf), 1.0 - ((double)uf + 0x1p-14), dmax);
  } else {
    U128 q{0ull, 0ull};
    unsigned int nz = 0u;
    double num = 0.0;
    for (int i = lane; i < s; i += 32) {
      const unsigned long long hi0 = q.hi, lo0 = q.lo;
      edf_uterm64(sc.cm[i].x, sc.T[i], q, nz);
      // this term's value (q after - q before) times (T - D) / 2^64
      const unsigned long long dlo = q.lo - lo0, dhi = q.hi - hi0 - (q.lo < lo0 ? 1ull : 0ull);
      num += (double)(sc.T[i] - sc.D[i]) * ((double)dhi + (double)dlo * 0x1p-64);
    }
    q = warp_sum_u128(q);
    nz = __reduce_add_sync(kFull, nz);
    num = warp_sum_f64(num);
    double gap = 0.0;
    int cmp = edf_classify64(q, nz, &gap);
    if (cmp == 2) {
      cmp = edf_lcm_classify(s, [&](int a, unsigned int& C, unsigned int& T) {
        C = sc.cm[a].x;
        T = sc.T[a];
      });
      gap = 0.0;  // exact sign only: no L_a bound
    }
    if (cmp == 2) {
      if (lane == 0) atomicOr(err, kErrIter);
      return false;
    }
    if (cmp > 0) return false;
    La = cmp < 0 ? edf_la(num, gap, dmax) : kEdfLmax;
  }
  // synchronous busy period, stopped at La
  unsigned long long L = csum;
  int iter = 0;
  for (;;) {
    unsigned long long part = 0;
    if (lane == 0) sc.terms += (unsigned int)s;
    for (int i = lane; i < s; i += 32) part += ceil_div_T64(L, sc.T[i], sc.cm[i].y, sc.sh[i]) * sc.cm[i].x;
    const unsigned long long next = warp_sum_u64_edf(part);
    if (next == L) break;
    if (next >= La) {
      if (La == kEdfLmax) {  // no bound below 2^62: undecided
        if (lane == 0) atomicOr(err, kErrIter);
        return false;
      }
      L = La;
      break;
    }
    L = next;
    if (++iter > kIterCap) {
      if (lane == 0) atomicOr(err, kErrIter);
      return false;
    }
  }
  // QPA
  unsigned long long t = 0;
  for (int i = lane; i < s; i += 32) {
    const unsigned long long d = edf_deadline_below(L, sc.T[i], sc.D[i], sc.cm[i].y, sc.sh[i]);
    t = d > t ? d : t;
  }
  t = warp_max_u64(t);
  iter = 0;
  while (t > 0ull) {
    unsigned long long part = 0;
    if (lane == 0) sc.terms += (unsigned int)s;
    for (int i = lane; i < s; i += 32) {
      const unsigned int D = sc.D[i];
      if (D <= t) part += (floor_div_T64(t - D, sc.T[i], sc.cm[i].y, sc.sh[i]) + 1ull) * sc.cm[i].x;
    }
    const unsigned long long h = warp_sum_u64_edf(part);
    if (h > t) return false;
    if (h <= dmin) return true;
    if (h < t) {
      t = h;
    } else {
      unsigned long long d = 0;
      for (int i = lane; i < s; i += 32) {
        const unsigned long long e = edf_deadline_below(t, sc.T[i], sc.D[i], sc.cm[i].y, sc.sh[i]);
        d = e > d ? e : d;
      }
      t = warp_max_u64(d);
    }
    if (++iter > kIterCap) {
      if (lane == 0) atomicOr(err, kErrIter);
      return false;
    }
  }
  return true;
}

// The same EDF test by one thread over k tasks; get(a, C, T, D, mg, sh)
// yields the a-th with its period's reciprocal.  An undecided test sets
// kErrIter in *errbits and returns false.  nterms counts the demand terms
// evaluated (k per busy-period or QPA step).
template <class Get>
__device__ bool serial_edf(int k, Get get, unsigned int* errbits, unsigned int& nterms) {
  unsigned int C, T, D, mg, sh;
  if (k == 0) return true;
  if (k == 1) {
    get(0, C, T, D, mg, sh);
    return C <= D;
  }
  unsigned long long csum = 0;
  float uf = 0.0f;
  double numf = 0.0;
  unsigned int dmin = 0xffffffffu, dmax = 0u;
  float dens = 0.0f;
  for (int a = 0; a < k; a++) {
    get(a, C, T, D, mg, sh);
    if (C > D) return false;
    const float r = (float)C / (float)T;
    uf += r;
    dens += (float)C / (float)D;
    numf += (double)(T - D) * (double)r;
    csum += C;
    dmin = min(dmin, D);
    dmax = max(dmax, D);
  }
  if (uf > kEdfFail) return false;
  if (dens <= kEdfDensity) return true;  // density <= 1 suffices
  unsigned long long La;
  if (uf < kEdfPass) {
    La = edf_la(numf, 1.0 - ((double)uf + 0x1p-14), dmax);
  } else {
    U128 q{0ull, 0ull};
    unsigned int nz = 0u;
    double num = 0.0;
    for (int a = 0; a < k; a++) {
      get(a, C, T, D, mg, sh);
      const unsigned long long hi0 = q.hi, lo0 = q.lo;
      edf_uterm64(C, T, q, nz);
      const unsigned long long dlo = q.lo - lo0, dhi = q.hi - hi0 - (q.lo < lo0 ? 1ull : 0ull);
      num += (double)(T - D) * ((double)dhi + (double)dlo * 0x1p-64);
    }
    double gap = 0.0;
    int cmp = edf_classify64(q, nz, &gap);
    if (cmp == 2) {
      cmp = edf_lcm_classify(k, [&](int a, unsigned int& Ca, unsigned int& Ta) {
        unsigned int Da, mga, sha;
        get(a, Ca, Ta, Da, mga, sha);
      });
      gap = 0.0;
    }
    if (cmp == 2) {
      *errbits |= kErrIter;
      return false;
    }
    if (cmp > 0) return false;
    La = cmp < 0 ? edf_la(num, gap, dmax) : kEdfLmax;
  }
  unsigned long long L = csum;
  int iter = 0;
  for (;;) {
    unsigned long long next = 0;
    nterms += (unsigned int)k;
    for (int a = 0; a < k; a++) {
      get(a, C, T, D, mg, sh);
      next += ceil_div_T64(L, T, mg, sh) * C;
    }
    if (next == L) break;
    if (next >= La) {
      if (La == kEdfLmax) {
        *errbits |= kErrIter;
        return false;
      }
      L = La;
      break;
    }
    L = next;
    if (++iter > kIterCap) {
      *errbits |= kErrIter;
      return false;
    }
  }
  unsigned long long t = 0;
  for (int a = 0; a < k; a++) {
    get(a, C, T, D, mg, sh);
    const unsigned long long d = edf_deadline_below(L, T, D, mg, sh);
    t = d > t ? d : t;
  }
  iter = 0;
  while (t > 0ull) {
    unsigned long long h = 0;
    nterms += (unsigned int)k;
    for (int a = 0; a < k; a++) {
      get(a, C, T, D, mg, sh);
      if (D <= t) h += (floor_div_T64(t - D, T, mg, sh) + 1ull) * C;
    }
    if (h > t) return false;
    if (h <= dmin) return true;
    if (h < t) {
      t = h;
    } else {
      unsigned long long d = 0;
      for (int a = 0; a < k; a++) {
        get(a, C, T, D, mg, sh);
        const unsigned long long e = edf_deadline_below(t, T, D, mg, sh);
        d = e > d ? e : d;
      }
      t = d;
    }
    if (++iter > kIterCap) {
      *errbits |= kErrIter;
      return false;
    }
  }
  return true;
}

// The per-partition test of the model's policy.  Under EDF the test gives
// no response times: R_row receives 0 for S's tasks when S passes, else -1.
__device__ __forceinline__ bool warp_test(const SetSmem& st, const unsigned int* S, unsigned int m, unsigned int kc,
                                          unsigned int km, int sched, const MagicDiv* __restrict__ mdiv,
                                          RtaScratch& sc, long long* R_row, bool early_exit, unsigned int* err) {
  if (sched != GPA_SCHED_EDF) return warp_rta(st, S, m, kc, km, mdiv, sc, R_row, early_exit, err);
  const bool ok = warp_edf(st, S, m, kc, km, mdiv, sc, err);
  if (R_row) {
    const int lane = threadIdx.x & 31;
    for (int w = 0; w < kWords; w++)
      if ((S[w] >> lane) & 1u) R_row[w * 32 + lane] = ok ? 0ll : -1ll;
  }
  __syncwarp();
  return ok;
}

// Alg. 2: smallest admissible size in [lo, hi] at which S passes; 0 if none.
// The binary form (§5.2) returns the same size because the test is monotone
// in m (no timing anomalies, §4.1).
__device__ __forceinline__ unsigned int warp_minm(const SetSmem& st, const unsigned int* S, unsigned int lo,
                                                  unsigned int hi, const Sizes& z, bool linear, unsigned int kc,
                                                  unsigned int km, int sched, const MagicDiv* __restrict__ mdiv,
                                                  RtaScratch& sc, unsigned int* err) {
  if (lo > hi) return 0u;
  hi = min(hi, z.M);
  int a = z.below(lo);
  const int e = z.below(hi + 1u);  // admissible sizes in [lo, hi]: indices a .. e - 1
  if (a >= e) return 0u;
  if (linear) {
    for (int k = a; k < e; k++)
      if (warp_test(st, S, z.at(k), kc, km, sched, mdiv, sc, nullptr, true, err)) return z.at(k);
    return 0u;
  }
  int b = e - 1;
  if (!warp_test(st, S, z.at(b), kc, km, sched, mdiv, sc, nullptr, true, err)) return 0u;
  while (a < b) {
    const int mid = a + (b - a) / 2;
    if (warp_test(st, S, z.at(mid), kc, km, sched, mdiv, sc, nullptr, true, err)) b = mid;
    else a = mid + 1;
  }
  return z.at(a);
}

// Warp-wide sums.
__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

__device__ __forceinline__ int warp_sum_i32(int v) { return __reduce_add_sync(kFull, (unsigned int)v); }

GPA_NS_END
