// k_search.cu — exact optimum over every SM split and task-to-partition map
// (the exhaustive yardstick for the heuristic of §5).
//
// The explicit space is every composition of M/g into k in [kmin, kmax]
// parts times every map of the n tasks to the k parts.  Because the test is
// monotone in m (§4.1) and in the task set, that space reduces exactly to
// set partitions of the tasks: a set partition with b blocks is realisable
// iff b <= kmax, every block has a minimum size minm(block) <= M, and
// sum minm + max(0, kmin - b) g <= M (empty parts still take g SMs).  So one
// CTA per task set
//   phase A: computes minm(S) and the inflated workload W(S) of every
//            non-empty subset S (one thread per subset, serial test);
//   phase B: enumerates restricted-growth strings (RGS) with at most kmax
//            blocks depth first.  A job is an RGS prefix (jobs in
//            lexicographic order, spread over the threads); a thread extends
//            it label by label with the block masks, sum minm and W updated
//            in place.  A branch is cut when a block becomes infeasible, sum
//            minm exceeds M, or W plus the singleton W of the tasks still to
//            place exceeds the CTA's best W so far: all three only grow as
//            tasks are added (a task adds at least its singleton W), so no
//            cut branch holds the optimum.  Leaves are compared by the key
//            (W, sum minm, RGS) and a CTA-wide shuffle argmin finishes.
#include <cuda_runtime.h>

#include "gpa_device.cuh"
#include "gpa_internal.h"

namespace gpa {

namespace {

constexpr int kSN = GPA_SEARCH_NMAX;  // tasks per set
constexpr int kSK = GPA_SEARCH_KMAX;  // blocks per set partition
constexpr int kSThreads = 256;
constexpr int kSuffix = 4;            // RGS positions enumerated below a job's prefix
constexpr int kTableMax = 2048;       // WCET table entries per curve (sizes x kSN)

struct SearchHead {
  unsigned int T[kSN], D[kSN], mT[kSN], sh[kSN];
  unsigned long long A[kSN], B[kSN];
  unsigned int u[kSN];
  unsigned int memmask;        // rows of memory tasks
  unsigned int rowbit[kSN];    // original task -> bit of its DM row
  unsigned int singleton[kSN]; // Lemma 2 size of each row
  unsigned long long cnt[kSN + 1][kSK + 2];  // prefix-completion counts (positions i..L-1)
  unsigned long long bestK1[kSThreads / 32];
  unsigned long long bestK2[kSThreads / 32];
  unsigned long long gbestW;   // best W found by any thread of the CTA (for cutting)
  unsigned long long restW[kSN + 1];  // sum of the singleton W of tasks i..n-1 (phase B's bound)
  unsigned int err;            // error bits of the set (kErrIter: a test hit its step limit)
  int n;
  long long set;
};

// Per-thread working storage in shared memory, laid out [field][thread] so
// that a warp's accesses to one field hit 32 different banks.
struct SearchThreads {
  unsigned int C[kSN][kSThreads];           // WCETs of the current test (phase A)
  unsigned short msk[kSK][kSThreads];       // block masks (phase B)
  unsigned char lab[kSN][kSThreads];        // labels of the current path
  unsigned char used[kSN + 1][kSThreads];   // blocks open before each position
  unsigned int terr[kSThreads];             // error bits of the current candidate (explicit search)
};

// WCETs of one set at every size, when they fit in shared memory:
// tn[mi * kSN + row] = C^n, tc[...] = C^c at m = g (mi + 1).
struct WcetTables {
  const unsigned int* tn;
  const unsigned int* tc;
};

// Serial per-partition test (one thread): rows of S in priority order at m.
// A fixed point that needs more than kIterCap steps leaves the test
// undecided: kErrIter goes to *errp and the test returns false.
__device__ bool serial_rta(const SearchHead& h, SearchThreads& w, unsigned int S, unsigned int m, unsigned int g,
                           unsigned int kc, unsigned int km, const MagicDiv& md, const WcetTables& tb,
                           unsigned int* errp, unsigned int& nt) {
  const int tid = threadIdx.x;
  const int nm = __popc(S & h.memmask), ns = __popc(S);
  const bool cm = nm >= 2, cc = (ns - nm) >= 2;
  const unsigned int kmem = cm ? km : 1000u, kcmp = cc ? kc : 1000u;
  const int mi = (int)(m / g) - 1;
  // Tasks are visited in priority order, and every one before task i met its
  // deadline (the test stops at the first miss), so R_i >= R_prev + C_i and
  // R_i >= C_i / (1 - U_hp) (util_start): the iteration starts at the larger
  // instead of at the sum of the WCETs (same least fixed point, fewer steps).
  unsigned long long Rprev = 0, chp = 0;
  float ua = 0.0f;  // sum of C_j / T_j over the tasks before i (each at most 1: they met their deadlines)
  for (unsigned int rest = S; rest; rest &= rest - 1u) {
    const int i = __ffs(rest) - 1;
    const bool mem = (h.memmask >> i) & 1u;
    unsigned int Ci;
    if (tb.tn) Ci = ((mem ? cm : cc) ? tb.tc : tb.tn)[mi * kSN + i];
    else Ci = wcet(h.A[i], h.B[i], mem ? kmem : kcmp, m, md);
    w.C[i][tid] = Ci;
    unsigned long long R = Rprev + Ci;
    const unsigned long long lb = util_start(Ci, ua);
    R = lb > R ? lb : R;
    const unsigned int Di = h.D[i];
    // a task the utilisation bound settles keeps its start value, at most
    // its least fixed point, as the next task's lower bound
    bool settled = util_pass(Ci, chp, ua, Di);
    ua += __fdividef((float)Ci, (float)h.T[i]);
    chp += Ci;
    const unsigned int hp = S & ((1u << i) - 1u);
    if (!settled && R <= Di) {
      // R_i is the least t with f(t) <= t (f: the iteration's non-decreasing
      // function), so f(D_i) <= D_i settles the task too
      unsigned long long fd = chp;
      nt += (unsigned int)__popc(hp);
      const unsigned int D2 = 2u * (Di - 1u);
      for (unsigned int r2 = hp; r2; r2 &= r2 - 1u) {
        const int j = __ffs(r2) - 1;
        fd += (unsigned long long)floor_div_T2(D2, h.mT[j], h.sh[j]) * w.C[j][tid];
      }
      settled = fd <= Di;
    }
    int iter = 0;
    for (; !settled;) {
      if (R > Di) return false;
      // every earlier task met its deadline (C_j <= D_j <= T_j): each term
      // stays below R + T_j < 2^32 and the sum cannot overflow
      // ceil(R / T_j) = floor((R - 1) / T_j) + 1: C_i and the +1 terms add up to
      // chp, which already holds C_i here
      unsigned long long next = chp;
      nt += (unsigned int)__popc(hp);
      const unsigned int R2 = 2u * ((unsigned int)R - 1u);
      for (unsigned int r2 = hp; r2; r2 &= r2 - 1u) {
        const int j = __ffs(r2) - 1;
        next += (unsigned long long)floor_div_T2(R2, h.mT[j], h.sh[j]) * w.C[j][tid];
      }
      if (next == R) break;
      R = next;
      if (++iter > kIterCap) {
        atomicOr(errp, kErrIter);
        return false;
      }
    }
    Rprev = R;
  }
  return true;
}

// The model's per-partition test, serially: DM as above, or EDF (the
// tasks' WCETs into w.C, then the processor-demand test).
__device__ bool serial_test(const SearchHead& h, SearchThreads& w, unsigned int S, unsigned int m, unsigned int g,
                            unsigned int kc, unsigned int km, int sched, const MagicDiv& md, const WcetTables& tb,
                            unsigned int* errp, unsigned int& nt) {
  if (sched != GPA_SCHED_EDF) return serial_rta(h, w, S, m, g, kc, km, md, tb, errp, nt);
  const int tid = threadIdx.x;
  const int nm = __popc(S & h.memmask), ns = __popc(S);
  const bool cm = nm >= 2, cc = (ns - nm) >= 2;
  const unsigned int kmem = cm ? km : 1000u, kcmp = cc ? kc : 1000u;
  const int mi = (int)(m / g) - 1;
  for (unsigned int rest = S; rest; rest &= rest - 1u) {
    const int i = __ffs(rest) - 1;
    const bool mem = (h.memmask >> i) & 1u;
    w.C[i][tid] = tb.tn ? ((mem ? cm : cc) ? tb.tc : tb.tn)[mi * kSN + i]
                        : wcet(h.A[i], h.B[i], mem ? kmem : kcmp, m, md);
  }
  unsigned int eb = 0u;
  const bool ok = serial_edf(
      ns,
      [&](int a, unsigned int& C, unsigned int& T, unsigned int& D, unsigned int& mg, unsigned int& sh) {
        const int i = (int)__fns(S, 0u, a + 1);
        C = w.C[i][tid];
        T = h.T[i];
        D = h.D[i];
        mg = h.mT[i];
        sh = h.sh[i];
      },
      &eb, nt);
  if (eb) atomicOr(errp, eb);
  return ok;
}

__device__ __forceinline__ Sizes sizes_of(const DevModel& md) {
  return Sizes{(unsigned int)md.M, (unsigned int)md.g, md.zlist, md.zrank, md.nz};
}

// Smallest admissible size in [lo, M] at which S passes (0 if none), for a
// lo known not to exceed the answer (the largest Lemma 2 size of S's tasks):
// a binary search over the admissible sizes from lo with one past the last
// standing for "no size passes" (valid because the test is monotone in m,
// §4.1).
__device__ unsigned int serial_minm(const SearchHead& h, SearchThreads& w, unsigned int S, unsigned int lo,
                                    const DevModel& md, const Sizes& z, const MagicDiv* __restrict__ mdiv,
                                    const WcetTables& tb, unsigned int* errp, unsigned int& nt) {
  const int e = z.count();
  int a = z.below(lo), b = e;
  while (a < b) {
    const int mid = a + (b - a) / 2;
    const unsigned int m = z.at(mid);
    if (serial_test(h, w, S, m, (unsigned)md.g, md.kc, md.km, md.sched, mdiv[m], tb, errp, nt)) b = mid;
    else a = mid + 1;
  }
  return a < e ? z.at(a) : 0u;
}

__device__ __forceinline__ bool key_less(unsigned long long a1, unsigned long long a2, unsigned long long b1,
                                         unsigned long long b2) {
  return a1 < b1 || (a1 == b1 && a2 < b2);
}

// Shared-memory layout of the search kernels: the head, the per-thread
// arrays, then minm and W of every subset and the WCET tables.
struct SearchSmem {
  SearchHead* h;
  SearchThreads* w;
  unsigned long long* Wsub;
  unsigned short* msub;
  unsigned int* tabn;
  unsigned int* tabc;
};

__device__ __forceinline__ SearchSmem search_smem(unsigned char* raw, int nsub_max, int tab_cap) {
  SearchSmem m;
  m.h = reinterpret_cast<SearchHead*>(raw);
  m.w = reinterpret_cast<SearchThreads*>(raw + sizeof(SearchHead));
  m.Wsub = reinterpret_cast<unsigned long long*>(raw + sizeof(SearchHead) + sizeof(SearchThreads));
  m.msub = reinterpret_cast<unsigned short*>(m.Wsub + nsub_max);
  m.tabn = reinterpret_cast<unsigned int*>(m.msub + nsub_max + (nsub_max & 1));
  m.tabc = m.tabn + tab_cap;
  return m;
}

// Stages set [o, o + n) by warp 0: validation, deadline-monotonic rows,
// Lemma 2 sizes; h.n = n, or -1 when the set is invalid (bad: its slice or
// size is out of range).  With L > 0 also the RGS prefix-completion counts
// for prefixes of length L.
__device__ void stage_search_set(SearchHead& h, const DevSets& S, long long o, int n, bool bad, int kmax, int L,
                                 const Sizes& z) {
  const int lane = threadIdx.x & 31;
  bool ok = !bad;
  long long Tt = 0, Dt = 0, At = 0, Bt = 0, ut = 0;
  unsigned int yt = 0;
  if (ok && lane < n) {
    Tt = S.T[o + lane];
    Dt = S.D[o + lane];
    At = S.A[o + lane];
    Bt = S.B[o + lane];
    ut = S.u[o + lane];
    yt = S.type[o + lane];
    ok = task_valid(Tt, Dt, At, Bt, ut, yt);
  }
  ok = __all_sync(kFull, ok);
  // deadline-monotonic rank by all-pairs compare through shuffles
  int r = 0;
  const unsigned long long key = ((unsigned long long)Dt << 31) | (unsigned long long)Tt;
  for (int j = 0; j < kSN; j++) {
    const unsigned long long kj = __shfl_sync(kFull, key, j);
    if (ok && lane < n && j < n) r += (kj < key) || (kj == key && j < lane);
  }
  if (ok && lane < n) {
    h.T[r] = (unsigned int)Tt;
    h.D[r] = (unsigned int)Dt;
    unsigned int mg, sh;
    magic_for_period((unsigned int)Tt, &mg, &sh);
    h.mT[r] = mg;
    h.sh[r] = sh;
    h.A[r] = (unsigned long long)At;
    h.B[r] = (unsigned long long)Bt;
    h.u[r] = (unsigned int)ut;
    h.rowbit[lane] = 1u << r;
    h.singleton[r] = lemma2_size((unsigned long long)At, (unsigned long long)Bt, (unsigned long long)Dt, z);
  }
  const unsigned int mem = __ballot_sync(kFull, ok && lane < n && yt == 1u);
  unsigned int mm = 0u;
  for (int j = 0; j < kSN; j++) {
    const int rj = __shfl_sync(kFull, r, j);
    if ((mem >> j) & 1u) mm |= 1u << rj;
  }
  if (lane == 0) {
    h.memmask = mm;
    h.n = ok ? n : -1;
    h.gbestW = ~0ull;
    h.err = 0u;
  }
  // prefix-completion counts: cnt[i][j] = ways to label positions i..L-1
  // with j blocks already open and at most kmax blocks in total
  if (lane == 0 && ok && L > 0) {
    for (int j = 0; j <= kmax + 1; j++) h.cnt[L][j] = 1ull;
    for (int i = L - 1; i >= 0; i--)
      for (int j = 0; j <= kmax; j++) {
        unsigned long long c = (unsigned long long)j * h.cnt[i + 1][j];
        if (j < kmax) c += h.cnt[i + 1][j + 1];
        h.cnt[i][j] = c;
      }
  }
}

// Result of a set that failed validation (h.n < 0).
__device__ void write_search_invalid(long long s, long long o, long long nl, int kmax, const BestOut& out,
                                     unsigned int* err) {
  const int tid = threadIdx.x;
  if (tid == 0) {
    out.feasible[s] = 0;
    out.W[s] = 0;
    out.sum_minm[s] = 0;
    out.n_blocks[s] = 0;
    out.spare[s] = 0;
    atomicOr(err, kErrRange);
  }
  for (int b = tid; b < kmax; b += kSThreads) out.minm_block[s * kmax + b] = 0;
  for (long long t = tid; t < nl && nl > 0; t += kSThreads) out.rgs[o + t] = 255;
}

// Result of an empty set: feasible iff kmin empty parts fit.
__device__ void write_search_empty(long long s, int kmin, int kmax, const DevModel& md, unsigned int zmin,
                                   const Sizes& z, const BestOut& out) {
  const int tid = threadIdx.x;
  if (tid == 0) {
    const bool f = z.count() > 0 && (long long)kmin * zmin <= md.M;
    out.feasible[s] = f ? 1 : 0;
    out.W[s] = 0;
    out.sum_minm[s] = 0;
    out.n_blocks[s] = 0;
    out.spare[s] = f ? md.M - kmin * (int)zmin : 0;
  }
  for (int b = tid; b < kmax; b += kSThreads) out.minm_block[s * kmax + b] = 0;
}

// Phase A: minm(S) and W(S) of every non-empty subset S of the n rows (one
// thread per subset); the WCET tables first when they fit.  Counts the
// interference terms of its tests into nt.  With flag_undecided, a subset
// whose size search hit a test's step limit gets kMsubUndecided in msub.
constexpr unsigned short kMsubUndecided = 0x8000;
__device__ WcetTables subset_table(SearchHead& h, SearchThreads& w, const SearchSmem& sm, int n, int tab_cap,
                                   const DevModel& md, const Sizes& z, const MagicDiv* __restrict__ mdiv,
                                   unsigned int& nt, bool flag_undecided = false) {
  const int tid = threadIdx.x;
  const unsigned int nsub = 1u << n;
  const int Mu = md.M / md.g;
  WcetTables tb{nullptr, nullptr};
  if (Mu * kSN <= tab_cap) {
    for (int e = tid; e < Mu * n; e += kSThreads) {
      const int mi = e / n, row = e % n;
      const unsigned int m = (unsigned)md.g * (unsigned)(mi + 1);
      const bool mem = (h.memmask >> row) & 1u;
      sm.tabn[mi * kSN + row] = wcet(h.A[row], h.B[row], 1000u, m, mdiv[m]);
      sm.tabc[mi * kSN + row] = wcet(h.A[row], h.B[row], mem ? (unsigned)md.km : (unsigned)md.kc, m, mdiv[m]);
    }
    tb = WcetTables{sm.tabn, sm.tabc};
  }
  __syncthreads();
  for (unsigned int S2 = tid; S2 < nsub; S2 += kSThreads) {
    if (S2 == 0u) {
      sm.msub[0] = 0;
      sm.Wsub[0] = 0;
      continue;
    }
    // lower bound: the largest Lemma 2 size of its tasks (0: some task alone is infeasible)
    unsigned int lo = 0u;
    bool dead = false;
    for (unsigned int r = S2; r; r &= r - 1u) {
      const unsigned int zs = h.singleton[__ffs(r) - 1];
      dead = dead || zs == 0u;
      lo = max(lo, zs);
    }
    if (!flag_undecided) {
      sm.msub[S2] = (unsigned short)(dead ? 0u
                                          : (__popc(S2) == 1 ? lo
                                                             : serial_minm(h, w, S2, lo, md, z, mdiv, tb, &h.err, nt)));
    } else {
      w.terr[tid] = 0u;
      const unsigned int mm =
          dead ? 0u : (__popc(S2) == 1 ? lo : serial_minm(h, w, S2, lo, md, z, mdiv, tb, &w.terr[tid], nt));
      const unsigned int te = w.terr[tid];
      if (te) atomicOr(&h.err, te);
      sm.msub[S2] = (unsigned short)(mm | ((te & kErrIter) ? kMsubUndecided : 0u));
    }
    const int nmS = __popc(S2 & h.memmask), ncS = __popc(S2) - nmS;
    unsigned long long Uc = 0, Um = 0;
    for (unsigned int r = S2; r; r &= r - 1u) {
      const int i = __ffs(r) - 1;
      ((h.memmask >> i) & 1u ? Um : Uc) += h.u[i];
    }
    sm.Wsub[S2] = workload_from_sums(Uc, Um, ncS, nmS, md.kc, md.km);
  }
  __syncthreads();
  return tb;
}

// CTA argmin of the threads' keys (k1 = W << 11 | sum minm, k2 = packed RGS,
// 3 bits per task with task 0 most significant), then the set's result.
__device__ void write_search_best(SearchHead& h, const SearchSmem& sm, unsigned long long best1,
                                  unsigned long long best2, long long s, long long o, int n, int kmin, int kmax,
                                  const DevModel& md, unsigned int zmin, const BestOut& out, unsigned int* err) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const unsigned long long kNoKey = ~0ull;
  for (int off = 16; off > 0; off >>= 1) {
    const unsigned long long o1 = __shfl_xor_sync(kFull, best1, off);
    const unsigned long long o2 = __shfl_xor_sync(kFull, best2, off);
    if (key_less(o1, o2, best1, best2)) {
      best1 = o1;
      best2 = o2;
    }
  }
  if (lane == 0) {
    h.bestK1[warp] = best1;
    h.bestK2[warp] = best2;
  }
  __syncthreads();
  if (warp == 0) {
    best1 = lane < kSThreads / 32 ? h.bestK1[lane] : kNoKey;
    best2 = lane < kSThreads / 32 ? h.bestK2[lane] : kNoKey;
    for (int off = 16; off > 0; off >>= 1) {
      const unsigned long long o1 = __shfl_xor_sync(kFull, best1, off);
      const unsigned long long o2 = __shfl_xor_sync(kFull, best2, off);
      if (key_less(o1, o2, best1, best2)) {
        best1 = o1;
        best2 = o2;
      }
    }
    const bool found = best1 != kNoKey;
    // decode the winning RGS (3 bits per task, task 0 most significant)
    int ai = 0;
    if (lane < n) ai = found ? (int)((best2 >> (3 * (n - 1 - lane))) & 7ull) : 255;
    if (lane < n) out.rgs[o + lane] = (unsigned char)ai;
    int nb = 0;
    unsigned int bm[kSK];
    for (int b = 0; b < kSK; b++) bm[b] = 0u;
    if (found) {
      for (int i = 0; i < n; i++) {
        const int ab = (int)((best2 >> (3 * (n - 1 - i))) & 7ull);
        bm[ab] |= h.rowbit[i];
        nb = max(nb, ab + 1);
      }
    }
    if (lane < kmax) {
      short zb = 0;
      for (int b = 0; b < kSK; b++)
        if (b == lane && b < nb) zb = (short)sm.msub[bm[b]];
      out.minm_block[s * kmax + lane] = zb;
    }
    if (lane == 0) {
      const unsigned int smm = found ? (unsigned int)(best1 & 2047ull) : 0u;
      const int empty = (found && kmin > nb) ? kmin - nb : 0;
      // a minimum size computed from an undecided test may be wrong: the
      // optimum is then undecided (feasible = 2)
      const unsigned int e = *(volatile unsigned int*)&h.err;
      out.feasible[s] = e & kErrIter ? 2 : found ? 1 : 0;
      if (e) atomicOr(err, e);
      out.W[s] = found ? (long long)(best1 >> 11) : 0;
      out.sum_minm[s] = (int)smm;
      out.n_blocks[s] = found ? nb : 0;
      out.spare[s] = found ? md.M - (int)smm - empty * (int)zmin : 0;
    }
  }
}

// Adds the CTA's interference-term counts to *terms (every thread calls it).
__device__ __forceinline__ void flush_search_terms(unsigned long long t, unsigned long long* terms) {
  t = warp_sum_u64(t);
  if ((threadIdx.x & 31) == 0 && t) atomicAdd(terms, t);
}

__global__ void __launch_bounds__(kSThreads) search_sets(DevSets S, DevModel md, int kmin, int kmax, BestOut out,
                                                         unsigned int* err, const MagicDiv* __restrict__ mdiv,
                                                         unsigned long long* ticket, int nsub_max, int tab_cap) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const SearchSmem smm = search_smem(smem_raw, nsub_max, tab_cap);
  SearchHead& h = *smm.h;
  SearchThreads& w = *smm.w;
  const unsigned long long* Wsub = smm.Wsub;
  const unsigned short* msub = smm.msub;
  const int tid = threadIdx.x, warp = tid >> 5;
  const unsigned long long kNoKey = ~0ull;
  const Sizes z = sizes_of(md);
  const unsigned int zmin = z.count() > 0 ? z.at(0) : (unsigned)md.M + 1u;  // an empty part's size
  unsigned long long terms = 0;

  for (;;) {
    __syncthreads();
    if (tid == 0) h.set = (long long)atomicAdd(ticket, 1ull);
    __syncthreads();
    const long long s = h.set;
    if (s >= S.nsets) break;
    const long long o = S.set_off[s];
    const long long nl = S.set_off[s + 1] - o;
    // ---- stage (warp 0): validate, DM order, Lemma 2 sizes
    const bool bad = nl < 0 || nl > kSN || (1ll << (nl < 0 ? 0 : nl)) > nsub_max || o < 0 ||
                     o > S.set_off[S.nsets] - nl;
    const int n = bad ? 0 : (int)nl;
    const int L = n > kSuffix ? n - kSuffix : (n > 0 ? 1 : 0);  // job prefix length
    if (warp == 0) stage_search_set(h, S, o, n, bad, kmax, L, z);
    __syncthreads();
    if (h.n < 0) {
      write_search_invalid(s, o, nl, kmax, out, err);
      continue;
    }
    if (n == 0) {
      write_search_empty(s, kmin, kmax, md, zmin, z, out);
      continue;
    }
    // ---- phase A: minm and W of every non-empty subset of rows
    unsigned int nt = 0;
    subset_table(h, w, smm, n, tab_cap, md, z, mdiv, nt);
    terms += nt;
    // Adding a task to a block adds at least its own W alone (1000 u, its
    // factor at least 1000 per mille) and never lowers the others' factors,
    // so a prefix's W plus the singleton W of the tasks still to place is a
    // lower bound of every completion's W.
    if (tid == 0) {
      h.restW[n] = 0ull;
      for (int i = n - 1; i >= 0; i--) h.restW[i] = h.restW[i + 1] + Wsub[h.rowbit[i]];
    }
    __syncthreads();
    // ---- phase B: depth-first over RGS, jobs = prefixes of length L
    const unsigned long long njobs = h.cnt[1][1];
    const unsigned int M = (unsigned)md.M;
    unsigned long long best1 = kNoKey, best2 = kNoKey;  // (W << 11 | sum minm, packed RGS)
    for (unsigned long long job = tid; job < njobs; job += kSThreads) {
#pragma unroll
      for (int b = 0; b < kSK; b++) w.msk[b][tid] = 0;
      unsigned long long Wp = 0;
      unsigned int Sp = 0;
      bool dead = false;
      // unrank the prefix; task 0 is in block 0
      unsigned long long rank = job;
      int used = 0;
      for (int i = 0; i < L; i++) {
        int b = 0;
        if (i > 0) {
          const int top = used < kmax ? used : kmax - 1;
          for (b = 0; b <= top; b++) {
            const int nu = b + 1 > used ? b + 1 : used;
            const unsigned long long c = h.cnt[i + 1][nu];
            if (rank < c) break;
            rank -= c;
          }
        }
        w.lab[i][tid] = (unsigned char)b;
        w.used[i][tid] = (unsigned char)used;
        used = b + 1 > used ? b + 1 : used;
        const unsigned int old = w.msk[b][tid], nw = old | h.rowbit[i];
        w.msk[b][tid] = (unsigned short)nw;
        Wp += Wsub[nw] - Wsub[old];
        Sp += (unsigned)msub[nw] - (unsigned)msub[old];
        dead = dead || msub[nw] == 0;
      }
      w.used[L][tid] = (unsigned char)used;
      if (dead || Sp > M || Wp + h.restW[L] > *(volatile unsigned long long*)&h.gbestW) continue;
      // depth-first over positions L..n-1; lab = 255 means "not placed yet"
      int i = L;
      if (i == n) {
        // the whole RGS is the prefix
        const int nb = used;
        const int empty = kmin > nb ? kmin - nb : 0;
        if ((long long)Sp + (long long)empty * zmin <= md.M) {
          unsigned long long packed = 0;
          for (int k = 0; k < n; k++) packed = (packed << 3) | w.lab[k][tid];
          const unsigned long long k1 = (Wp << 11) | Sp;
          if (key_less(k1, packed, best1, best2)) {
            best1 = k1;
            best2 = packed;
            atomicMin(&h.gbestW, Wp);
          }
        }
        continue;
      }
      w.lab[i][tid] = 255;
      while (i >= L) {
        unsigned int lb = w.lab[i][tid];
        const unsigned int bit = h.rowbit[i];
        if (lb != 255u) {  // take task i out of its current block
          const unsigned int old = w.msk[lb][tid], nw = old & ~bit;
          w.msk[lb][tid] = (unsigned short)nw;
          Wp -= Wsub[old] - Wsub[nw];
          Sp -= (unsigned)msub[old] - (unsigned)msub[nw];
        }
        lb = lb == 255u ? 0u : lb + 1u;
        const unsigned int u_i = w.used[i][tid];
        const unsigned int top = u_i < (unsigned)kmax ? u_i : (unsigned)kmax - 1u;
        if (lb > top) {  // labels exhausted: back up
          w.lab[i][tid] = 255;
          i--;
          continue;
        }
        w.lab[i][tid] = (unsigned char)lb;
        const unsigned int old = w.msk[lb][tid], nw = old | bit;
        w.msk[lb][tid] = (unsigned short)nw;
        Wp += Wsub[nw] - Wsub[old];
        Sp += (unsigned)msub[nw] - (unsigned)msub[old];
        if (msub[nw] == 0 || Sp > M || Wp + h.restW[i + 1] > *(volatile unsigned long long*)&h.gbestW) continue;
        const unsigned int u_next = lb + 1u > u_i ? lb + 1u : u_i;
        if (i + 1 == n) {
          const int empty = kmin > (int)u_next ? kmin - (int)u_next : 0;
          if ((long long)Sp + (long long)empty * zmin <= md.M) {
            const unsigned long long k1 = (Wp << 11) | Sp;
            if (k1 <= best1) {
              unsigned long long packed = 0;
              for (int k = 0; k < n; k++) packed = (packed << 3) | w.lab[k][tid];
              if (key_less(k1, packed, best1, best2)) {
                best1 = k1;
                best2 = packed;
                atomicMin(&h.gbestW, Wp);
              }
            }
          }
          continue;
        }
        w.used[i + 1][tid] = (unsigned char)u_next;
        i++;
        w.lab[i][tid] = 255;
      }
    }
    // ---- CTA argmin of (k1, k2) and the set's result
    write_search_best(h, smm, best1, best2, s, o, n, kmin, kmax, md, zmin, out, err);
  }
  flush_search_terms(terms, ticket + 1);  // the context's term counter follows the ticket
}

// C(a, b) for small b (exact while the result and a C(a, b - 1) fit in 64 bits).
__device__ __forceinline__ unsigned long long binom_small(int a, int b) {
  if (b < 0 || a < b) return 0ull;
  unsigned long long r = 1ull;
  for (int i = 1; i <= b; i++) r = r * (unsigned long long)(a - b + i) / (unsigned long long)i;
  return r;
}

// The explicit candidate space of one set: for k = kmin .. kmax (k <= Mu),
// C(Mu - 1, k - 1) compositions of Mu = M / g into k positive parts, in
// lexicographic order of the parts, times k^n maps of the tasks to the
// parts (map code c: task i goes to part (c / k^i) mod k).  Candidate ranks
// run over k, then the composition, then the map code.
struct ExplicitPlan {
  int kmin, kmax, Mu;
  unsigned long long comps[kSK + 1];  // compositions into k parts
};

// Candidate `rank` of a set of n tasks: its part count k, its parts (in
// units of g) and its map code.  A set has at most GPA_EXPLICIT_MAX (2^26)
// candidates, so ranks, codes and every k^n with compositions fit in 32 bits.
__device__ __forceinline__ void unrank_candidate(const ExplicitPlan& pl, int n, unsigned int rank, int* k_out,
                                                 int* parts, unsigned int* code) {
  int k = pl.kmin;
  unsigned int nmaps = 1u;
  for (; k <= pl.kmax; k++) {
    if (pl.comps[k] == 0ull) continue;
    nmaps = 1u;
    for (int i = 0; i < n; i++) nmaps *= (unsigned int)k;
    const unsigned int c = (unsigned int)pl.comps[k] * nmaps;
    if (rank < c) break;
    rank -= c;
  }
  *k_out = k;
  unsigned int comp = rank / nmaps;
  *code = rank - comp * nmaps;
  // lexicographic unrank: parts[i] = p leaves C(left - p - 1, rest - 1)
  // completions of the remaining parts
  int left = pl.Mu;
  for (int i = 0; i < k; i++) {
    const int rest = k - i - 1;
    if (rest == 0) {
      parts[i] = left;
      break;
    }
    for (int pv = 1; pv <= left - rest; pv++) {
      const unsigned long long c = binom_small(left - pv - 1, rest - 1);
      if (comp < c) {
        parts[i] = pv;
        left -= pv;
        break;
      }
      comp -= (unsigned int)c;
    }
  }
}

// a6 / a8 on the explicit space: every candidate (composition x map) is
// tested part by part (each non-empty part at its size, §5.5's test), and
// the feasible ones are ranked by the key of the optimum (W, sum of the
// blocks' minimum sizes, RGS of the induced set partition); minm and W of
// the blocks come from the subset table of phase A.  cverdict (nullable)
// receives every candidate's verdict: 1 feasible, 0 not, 2 undecided.
__global__ void __launch_bounds__(kSThreads) search_explicit(DevSets S, DevModel md, ExplicitPlan pl, BestOut out,
                                                             unsigned char* cverdict, long long cstride,
                                                             unsigned int* err, const MagicDiv* __restrict__ mdiv,
                                                             unsigned long long* ticket, int nsub_max, int tab_cap) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const SearchSmem smm = search_smem(smem_raw, nsub_max, tab_cap);
  SearchHead& h = *smm.h;
  SearchThreads& w = *smm.w;
  const int tid = threadIdx.x, warp = tid >> 5;
  const unsigned long long kNoKey = ~0ull;
  const Sizes z = sizes_of(md);
  const unsigned int zmin = (unsigned)md.g;
  unsigned long long terms = 0;

  for (;;) {
    __syncthreads();
    if (tid == 0) h.set = (long long)atomicAdd(ticket, 1ull);
    __syncthreads();
    const long long s = h.set;
    if (s >= S.nsets) break;
    const long long o = S.set_off[s];
    const long long nl = S.set_off[s + 1] - o;
    const bool bad = nl < 0 || nl > kSN || (1ll << (nl < 0 ? 0 : nl)) > nsub_max || o < 0 ||
                     o > S.set_off[S.nsets] - nl;
    const int n = bad ? 0 : (int)nl;
    if (warp == 0) stage_search_set(h, S, o, n, bad, pl.kmax, 0, z);
    __syncthreads();
    if (h.n < 0) {
      write_search_invalid(s, o, nl, pl.kmax, out, err);
      if (cverdict)
        for (long long c = tid; c < cstride; c += kSThreads) cverdict[s * cstride + c] = 255;
      continue;
    }
    unsigned int nt = 0;
    if (n > 0) subset_table(h, w, smm, n, tab_cap, md, z, mdiv, nt, true);
    terms += nt;
    nt = 0;
    // this set's candidate count
    unsigned long long ncand = 0;
    for (int k = pl.kmin; k <= pl.kmax; k++) {
      unsigned long long nm = 1ull;
      for (int i = 0; i < n; i++) nm *= (unsigned long long)k;
      ncand += pl.comps[k] * nm;
    }
    unsigned long long best1 = kNoKey, best2 = kNoKey;
    for (unsigned long long r = tid; r < ncand; r += kSThreads) {
      int k, parts[kSK];
      unsigned int code;
      unrank_candidate(pl, n, (unsigned int)r, &k, parts, &code);
      // the parts' task masks (rows)
      unsigned int pm[kSK];
      for (int b = 0; b < kSK; b++) pm[b] = 0u;
      unsigned int c = code;
      for (int i = 0; i < n; i++) {
        const unsigned int q = c / (unsigned int)k;
        pm[c - q * (unsigned int)k] |= h.rowbit[i];
        c = q;
      }
      // A part passes at its size m iff its task set's minimum passing size
      // is at most m: the test is monotone in m (§4.1), and every size is
      // admissible here (no size lists).  A part whose size search hit a
      // test's step limit leaves the candidate (and the optimum) undecided.
      bool feasible = true, undecided = false;
      for (int b = 0; b < k; b++) {
        if (!pm[b]) continue;
        const unsigned int m = (unsigned)parts[b] * (unsigned)md.g;
        const unsigned int ms = smm.msub[pm[b]];
        if (ms & kMsubUndecided) undecided = true;
        else feasible = feasible && ms != 0u && ms <= m;
      }
      if (cverdict) cverdict[s * cstride + (long long)r] = undecided ? 2 : feasible ? 1 : 0;
      if (undecided || !feasible) continue;
      // induced set partition: blocks relabelled by first occurrence (task order)
      int label[kSK];
      for (int b = 0; b < kSK; b++) label[b] = -1;
      int nb = 0;
      unsigned long long packed = 0, W = 0;
      unsigned int summ = 0;
      c = code;
      for (int i = 0; i < n; i++) {
        const unsigned int q = c / (unsigned int)k;
        const int part = (int)(c - q * (unsigned int)k);
        c = q;
        if (label[part] < 0) {
          label[part] = nb++;
          W += smm.Wsub[pm[part]];
          summ += smm.msub[pm[part]];
        }
        packed = (packed << 3) | (unsigned long long)label[part];
      }
      const unsigned long long k1 = (W << 11) | summ;
      if (key_less(k1, packed, best1, best2)) {
        best1 = k1;
        best2 = packed;
      }
    }
    if (cverdict)
      for (long long cc = (long long)ncand + tid; cc < cstride; cc += kSThreads) cverdict[s * cstride + cc] = 255;
    if (n == 0) {
      // the empty set: the all-empty candidate of kmin parts, when it exists
      write_search_empty(s, pl.kmin, pl.kmax, md, zmin, z, out);
      continue;
    }
    write_search_best(h, smm, best1, best2, s, o, n, pl.kmin, pl.kmax, md, zmin, out, err);
  }
  flush_search_terms(terms, ticket + 1);
}

size_t search_smem_bytes(int nsub_max, int tab_cap) {
  return sizeof(SearchHead) + sizeof(SearchThreads) +
         (size_t)nsub_max * (sizeof(unsigned long long) + sizeof(unsigned short)) + 4 +
         2 * (size_t)tab_cap * sizeof(unsigned int);
}

}  // namespace

cudaError_t search_kernels_init() {
  cudaError_t e = cudaFuncSetAttribute(search_sets, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)search_smem_bytes(1 << kSN, kTableMax));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(search_explicit, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)search_smem_bytes(1 << kSN, kTableMax));
}

cudaError_t launch_search_best(const DevSets& s, const DevModel& md, int kmin, int kmax, const BestOut& out,
                               const AllocQueue& q, const MagicDivHost* mdiv, int sm_count, cudaStream_t st,
                               long long* launches, Prof* prof) {
  int nmax = s.n_max < 0 ? 0 : (s.n_max > kSN ? kSN : s.n_max);
  const int nsub_max = 1 << nmax;
  const int Mu = md.M / md.g;
  const int tab_cap = Mu * kSN <= kTableMax ? Mu * kSN : 0;  // WCET tables only when they are small
  const size_t smem = search_smem_bytes(nsub_max, tab_cap);
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, search_sets, kSThreads, smem);
  if (per_sm < 1) per_sm = 1;
  long long blocks = (long long)sm_count * per_sm;
  if (blocks > s.nsets) blocks = s.nsets > 0 ? s.nsets : 1;
  unsigned long long* ticket = q.counters + 3;  // followed by the interference-term counter
  unsigned int* err = q.err;
  cudaError_t e = cudaMemsetAsync(ticket, 0, 2 * sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  prof_mark(prof, st);
  search_sets<<<(int)blocks, kSThreads, smem, st>>>(s, md, kmin, kmax, out, err,
                                                     reinterpret_cast<const MagicDiv*>(mdiv), ticket, nsub_max, tab_cap);
  e = cudaGetLastError();
  prof_mark(prof, st);
  *launches += 1;
  return e;
}

cudaError_t launch_search_explicit(const DevSets& s, const DevModel& md, int kmin, int kmax, const BestOut& out,
                                   unsigned char* cverdict, long long cstride, const AllocQueue& q,
                                   const MagicDivHost* mdiv, int sm_count, cudaStream_t st, long long* launches,
                                   Prof* prof) {
  int nmax = s.n_max < 0 ? 0 : (s.n_max > kSN ? kSN : s.n_max);
  const int nsub_max = 1 << nmax;
  const int Mu = md.M / md.g;
  const int tab_cap = Mu * kSN <= kTableMax ? Mu * kSN : 0;
  ExplicitPlan pl{};
  pl.kmin = kmin;
  pl.kmax = kmax;  // part counts above Mu have no composition (comps = 0)
  pl.Mu = Mu;
  for (int k = 1; k <= kSK; k++) {
    // C(Mu - 1, k - 1): the host has checked that the whole space is small
    unsigned long long r = 1ull;
    for (int i = 1; i <= k - 1; i++) r = r * (unsigned long long)(Mu - 1 - (k - 1) + i) / (unsigned long long)i;
    pl.comps[k] = k <= Mu ? r : 0ull;
  }
  const size_t smem = search_smem_bytes(nsub_max, tab_cap);
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, search_explicit, kSThreads, smem);
  if (per_sm < 1) per_sm = 1;
  long long blocks = (long long)sm_count * per_sm;
  if (blocks > s.nsets) blocks = s.nsets > 0 ? s.nsets : 1;
  unsigned long long* ticket = q.counters + 3;  // followed by the interference-term counter
  cudaError_t e = cudaMemsetAsync(ticket, 0, 2 * sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  prof_mark(prof, st);
  search_explicit<<<(int)blocks, kSThreads, smem, st>>>(s, md, pl, out, cverdict, cstride, q.err,
                                                         reinterpret_cast<const MagicDiv*>(mdiv), ticket, nsub_max,
                                                         tab_cap);
  e = cudaGetLastError();
  prof_mark(prof, st);
  *launches += 1;
  return e;
}

}  // namespace gpa
