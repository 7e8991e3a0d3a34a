// alloc_dev.cuh — device pieces of the heuristic shared by the batch
// allocate kernels (k_alloc.cu) and the serving kernel (k_serve.cu): the
// per-set result writers and Alg. 1 for one task set in shared memory
// (Lemma 1, Lemma 2, ACT, and the merge loop with Alg. 3, Alg. 2 and the
// SMS / BF orders of Def. 3 / Def. 4).
#pragma once

#include "gpa_device.cuh"
#include "gpa_internal.h"

GPA_NS_BEGIN

namespace {

// A set's task slice [o, o + n) lies inside the task columns, whose length
// is set_off[nsets].
__device__ __forceinline__ bool slice_inside(long long o, long long n, long long ntasks) {
  return o >= 0 && n >= 0 && o <= ntasks - n;
}

__device__ __forceinline__ void write_invalid(long long s, long long o, long long n, const AllocOut& out,
                                              unsigned int* err) {
  const int lane = threadIdx.x & 31;
  if (lane == 0) {
    out.verdict[s] = 0;
    out.reason[s] = GPA_REASON_INVALID;
    out.n_parts[s] = 0;
    out.Pi[s] = 0;
    out.W[s] = 0;
    if (out.n_tests) out.n_tests[s] = 0;
    atomicOr(err, kErrRange);
  }
  for (long long t = lane; t < n; t += 32) {
    out.part_of_task[o + t] = 255;
    out.size_of_part[o + t] = 0;
  }
}

__device__ __forceinline__ void write_empty(long long s, long long o, int n, unsigned char reason, const AllocOut& out,
                                            int tests) {
  const int lane = threadIdx.x & 31;
  if (lane == 0) {
    out.verdict[s] = 0;
    out.reason[s] = reason;
    out.n_parts[s] = 0;
    out.Pi[s] = 0;
    out.W[s] = 0;
    if (out.n_tests) out.n_tests[s] = tests;
  }
  for (int t = lane; t < n; t += 32) {
    out.part_of_task[o + t] = 255;
    out.size_of_part[o + t] = 0;
  }
}


// After a set's run with its own error word e: a per-partition test that hit
// its step limit (kErrIter) leaves the set undecided (verdict 0, reason
// GPA_REASON_UNDECIDED; its other outputs are those of the run, unspecified);
// the bits go to the sticky error word too.
__device__ __forceinline__ void finish_set_errors(long long s, unsigned int e, const AllocOut& out,
                                                  unsigned int* gerr) {
  if ((threadIdx.x & 31) == 0 && e) {
    if (e & kErrIter) {
      out.verdict[s] = 0;
      out.reason[s] = GPA_REASON_UNDECIDED;
    }
    atomicOr(gerr, e);
  }
  __syncwarp();
}

// ------------------------------------------------------------ merge kernel
//
// Alg. 1 for one task set is run by a group of warps: the whole CTA, or one
// warp of it.  The group stages the set, then repeats Alg. 3's selection
// and the candidate merges of Def. 3 / Def. 4 until Π <= M or no partition
// has an eligible partner.  The candidate tests of a step are spread over
// the group: a merged set of at most kLaneMax tasks is tested by one thread
// (serially), a larger one by one warp (warp_test).
//
// Two facts keep the work per step small without changing any result:
//  * the test is monotone in m (§4.1: C(m) never grows with m), so a merge
//    passes somewhere in its range iff it passes at the range's top size,
//    and the smallest passing size is found by testing sizes upwards;
//  * a step whose candidates all fail changes neither the utilisations nor
//    the lowest task indices, so par_list keeps its order, and forbidding
//    pairs only removes eligibility: the next Alg. 3 scan resumes after the
//    position of the partition that just failed.
// SMS (Def. 3: the smallest merged size, ties to the earlier par_list
// position) is evaluated size level by size level (optionally after a round
// that tests every thread-tested candidate with more than one size in its
// range at its top size; a failure there rules it out): at level L every candidate whose range holds
// the L-th admissible size and that failed below it is tested at that size,
// in position order, and the first pass at the lowest level is the chosen
// merge; no later candidate of that level, and no higher level, is tested.  BF (Def. 4) tests each candidate, in its order,
// at its top size; the first that passes is merged at its smallest passing
// size and every earlier one is forbidden.  The number of candidate merges
// counted in n_tests is the algorithm's (every candidate of an SMS step,
// BF's candidates up to the first success).

constexpr int kLaneMax = 16;      // merged sets of up to this many tasks are tested by one thread
constexpr int kGrpWarpsMax = 8;   // warps of a group
constexpr int kWinMax = 256;      // jobs per window of first_pass

// One thread's serial test of a candidate merge: WCETs and rows of the
// merged set's tasks in priority order, [position][lane] (conflict-free
// banks), and the thread's count of interference terms.
struct LaneScratch {
  uint2 cm[kLaneMax][32];             // .x: WCET, .y: reciprocal of the period
  unsigned char sh[kLaneMax][32];     // shift of that reciprocal
  unsigned char row[kLaneMax][32];
  unsigned long long terms[32];
};

// Per-warp test scratch.
struct WarpScratch {
  RtaScratch sc;
  LaneScratch ls;
};

struct MergeSmem {
  SetSmem st;
  RtaScratch sc;                     // test scratch of the group's warp 0
  LaneScratch ls;
  unsigned int mask[kNmax][kWords];  // tasks (rows) of each partition slot
  unsigned int actm[kNmax][kWords];  // rows forbidden to the slot by ACT pairs
  unsigned int forb[kNmax][kWords];  // slots whose exact pair with this slot failed
  unsigned int act[kNmax][kWords];   // ACT pair matrix over rows
  unsigned long long Uc[kNmax];      // utilisation of the slot's compute tasks
  unsigned long long Um[kNmax];      // utilisation of the slot's memory tasks
  unsigned long long wkey[kNmax];    // BF: workload of each candidate merge
  unsigned short m[kNmax];           // slot size (SMs)
  unsigned short ka[kNmax];          // candidate: index of its lowest admissible size
  unsigned short kb[kNmax];          // candidate: index of its top admissible size
  unsigned short kx[kNmax];          // candidate: upper end of a binary search
  unsigned char nc[kNmax], nm[kNmax];
  unsigned char lowest[kNmax];       // lowest original task index in the slot
  unsigned char alive[kNmax];
  unsigned char order[kNmax];        // par_list: slots in order
  unsigned char cand[kNmax];         // candidate partners of p1 (SMS: par_list order; BF: its order)
  unsigned char big[kNmax];          // candidate's merged set exceeds kLaneMax tasks
  unsigned char live[kNmax];         // candidate's range holds an admissible size
  unsigned char jk[kNmax];           // jobs: candidate of each
  unsigned char pass[kNmax];         // jobs: result of each (binary search rounds)
  unsigned char wl[kWinMax];         // warp-tested jobs of a window (offsets in the window)
  unsigned char slot_of[kNmax];      // slot of each row
  unsigned char rank[kNmax];         // output numbering of each slot
  int redi[kGrpWarpsMax];            // group reductions
  unsigned long long redl[kGrpWarpsMax];
  int ctl[8];                        // values broadcast to the group
  long long ticket;                  // set popped from the queue
  unsigned int err;                  // error bits of the set being processed
};

// A group of nwarps consecutive warps (nthreads threads); sync() is its
// barrier: __syncwarp for one warp, named barrier `bar` for several.
struct Grp {
  int nthreads, tid, nwarps, warp, lane, bar;
  __device__ __forceinline__ void sync() const {
    if (nwarps == 1) __syncwarp();
    else asm volatile("bar.sync %0, %1;" ::"r"(bar), "r"(nthreads) : "memory");
  }
};

// The calling warp as a group of one.
__device__ __forceinline__ Grp warp_group() {
  Grp g;
  g.nthreads = 32;
  g.tid = g.lane = (int)(threadIdx.x & 31);
  g.nwarps = 1;
  g.warp = 0;
  g.bar = 0;
  return g;
}

__device__ __forceinline__ RtaScratch& grp_sc(MergeSmem& sm, WarpScratch* extra, const Grp& g) {
  return g.warp == 0 ? sm.sc : extra[g.warp - 1].sc;
}
__device__ __forceinline__ LaneScratch& grp_ls(MergeSmem& sm, WarpScratch* extra, const Grp& g) {
  return g.warp == 0 ? sm.ls : extra[g.warp - 1].ls;
}

// Group-wide reductions (every thread gets the result; they end with the
// group's barrier, so values written before them are visible after).
__device__ __forceinline__ int grp_min_int(const Grp& g, MergeSmem& sm, int v) {
  v = __reduce_min_sync(kFull, v);
  if (g.nwarps == 1) {
    __syncwarp();
    return v;
  }
  if (g.lane == 0) sm.redi[g.warp] = v;
  g.sync();
  int r = sm.redi[0];
  for (int w = 1; w < g.nwarps; w++) r = min(r, sm.redi[w]);
  g.sync();
  return r;
}
__device__ __forceinline__ int grp_max_int(const Grp& g, MergeSmem& sm, int v) {
  return -grp_min_int(g, sm, -v);
}
__device__ __forceinline__ int grp_sum_int(const Grp& g, MergeSmem& sm, int v) {
  v = warp_sum_i32(v);
  if (g.nwarps == 1) {
    __syncwarp();
    return v;
  }
  if (g.lane == 0) sm.redi[g.warp] = v;
  g.sync();
  int r = 0;
  for (int w = 0; w < g.nwarps; w++) r += sm.redi[w];
  g.sync();
  return r;
}
__device__ __forceinline__ unsigned long long grp_sum_u64(const Grp& g, MergeSmem& sm, unsigned long long v) {
  v = warp_sum_u64(v);
  if (g.nwarps == 1) {
    __syncwarp();
    return v;
  }
  if (g.lane == 0) sm.redl[g.warp] = v;
  g.sync();
  unsigned long long r = 0;
  for (int w = 0; w < g.nwarps; w++) r += sm.redl[w];
  g.sync();
  return r;
}

// §5.5 per-partition test of a merged set S (at most kLaneMax tasks) by one
// thread, serially.  First the tasks' WCETs in priority order, with a
// float utilisation sum: a task with C > D, or a sum above 1 + 2^-13
// (U > 1, see kUtilFail), fails the set before any iteration.  Then tasks
// are visited in priority order and each earlier task met its deadline: a
// task the response-time upper bound settles (util_pass) needs no
// iteration; the others start at the larger of R_prev + C_i and the
// utilisation bound (util_start), both at most the least fixed point.
__device__ bool lane_rta(const SetSmem& st, const unsigned int* S, unsigned int m, unsigned int kc, unsigned int km,
                         const MagicDiv& md, LaneScratch& ls, int lane, unsigned int* err) {
  int nm = 0, ns = 0;
#pragma unroll
  for (int w = 0; w < kWords; w++) {
    nm += __popc(S[w] & st.memmask[w]);
    ns += __popc(S[w]);
  }
  const unsigned int kmem = nm >= 2 ? km : 1000u, kcmp = (ns - nm) >= 2 ? kc : 1000u;
  int n = 0;
  float uf = 0.0f;
  bool c_le_d = true;
  for (int w = 0; w < kWords; w++) {
    for (unsigned int bits = S[w]; bits; bits &= bits - 1u) {
      const int row = w * 32 + __ffs(bits) - 1;
      const bool mem = (st.memmask[w] >> (row & 31)) & 1u;
      const unsigned int Ci = wcet(st.A[row], st.B[row], mem ? kmem : kcmp, m, md);
      ls.cm[n][lane] = make_uint2(Ci, st.mT[row]);
      ls.sh[n][lane] = st.shT[row];
      ls.row[n][lane] = (unsigned char)row;
      c_le_d = c_le_d && Ci <= st.D[row];
      uf += (float)Ci * st.rT[row];
      n++;
    }
  }
  if (!c_le_d || uf > kUtilFail) return false;
  unsigned long long Rprev = 0, chp = 0;
  unsigned int nt = 0;
  float ua = 0.0f;  // sum of C_q / T_q over the tasks before pos
  bool ok = true;
  for (int pos = 0; pos < n && ok; pos++) {
    const uint2 self = ls.cm[pos][lane];
    const int row = ls.row[pos][lane];
    const unsigned int Ci = self.x, Di = st.D[row];
    // a task the utilisation bound settles keeps its start value, at most
    // its least fixed point, as the next task's lower bound
    // (unlike the warp and serial tests, no evaluation of f(D_i) first:
    // merge candidates fail often, and on the paper setting it cost 6 %)
    const bool settled = util_pass(Ci, chp, ua, Di);
    unsigned long long R = Rprev + Ci;
    if (!settled) {
      const unsigned long long lb = util_start(Ci, ua);
      R = lb > R ? lb : R;
    }
    ua += (float)Ci * st.rT[row];  // C_i / T_i within 2^-22 (two roundings)
    chp += Ci;
    int iter = 0;
    for (; !settled;) {
      if (R > Di) {
        ok = false;
        break;
      }
      // every earlier task met its deadline, so C_q <= D_q <= T_q and each
      // term stays below R + T_q < 2^32: the sum cannot overflow
      // ceil(R / T_q) = floor((R - 1) / T_q) + 1: C_i and the +1 terms add up to
      // chp, which already holds C_i here
      unsigned long long next = chp;
      nt += (unsigned int)pos;
      const unsigned int R2 = 2u * ((unsigned int)R - 1u);
      for (int q = 0; q < pos; q++) {
        const uint2 v = ls.cm[q][lane];
        next += (unsigned long long)floor_div_T2(R2, v.y, ls.sh[q][lane]) * v.x;
      }
      if (next == R) break;
      R = next;
      if (++iter > kIterCap) {
        atomicOr(err, kErrIter);
        ok = false;
        break;
      }
    }
    Rprev = R;
  }
  ls.terms[lane] += nt;
  return ok;
}

// The EDF test of S (at most kLaneMax tasks) by one thread.
__device__ bool lane_edf(const SetSmem& st, const unsigned int* S, unsigned int m, unsigned int kc, unsigned int km,
                         const MagicDiv& md, LaneScratch& ls, int lane, unsigned int* err) {
  int nm = 0, ns = 0;
#pragma unroll
  for (int w = 0; w < kWords; w++) {
    nm += __popc(S[w] & st.memmask[w]);
    ns += __popc(S[w]);
  }
  const unsigned int kmem = nm >= 2 ? km : 1000u, kcmp = (ns - nm) >= 2 ? kc : 1000u;
  int pos = 0;
  for (int w = 0; w < kWords; w++) {
    for (unsigned int bits = S[w]; bits; bits &= bits - 1u) {
      const int row = w * 32 + __ffs(bits) - 1;
      const bool mem = (st.memmask[w] >> (row & 31)) & 1u;
      ls.cm[pos][lane] = make_uint2(wcet(st.A[row], st.B[row], mem ? kmem : kcmp, m, md), st.mT[row]);
      ls.row[pos][lane] = (unsigned char)row;
      pos++;
    }
  }
  unsigned int eb = 0u, nt = 0u;
  const bool ok = serial_edf(
      pos,
      [&](int a, unsigned int& C, unsigned int& T, unsigned int& D, unsigned int& mg, unsigned int& sh) {
        const int r = ls.row[a][lane];
        C = ls.cm[a][lane].x;
        T = st.T[r];
        D = st.D[r];
        mg = st.mT[r];
        sh = st.shT[r];
      },
      &eb, nt);
  if (eb) atomicOr(err, eb);
  ls.terms[lane] += nt;
  return ok;
}

__device__ __forceinline__ bool lane_test(const SetSmem& st, const unsigned int* S, unsigned int m, unsigned int kc,
                                          unsigned int km, int sched, const MagicDiv& md, LaneScratch& ls, int lane,
                                          unsigned int* err) {
  return sched == GPA_SCHED_EDF ? lane_edf(st, S, m, kc, km, md, ls, lane, err)
                                : lane_rta(st, S, m, kc, km, md, ls, lane, err);
}

// The admissible sizes of the model.
__device__ __forceinline__ Sizes sizes_of(const DevModel& md) {
  return Sizes{(unsigned int)md.M, (unsigned int)md.g, md.zlist, md.zrank, md.nz};
}

// What a candidate test needs besides the set and the merge.
struct TestCtx {
  Sizes z;
  unsigned int kc, km;
  int sched;
  const MagicDiv* mdiv;
  unsigned int* err;
};

// Candidate k (the merge of slot p1 with cand[k]) at the L-th admissible
// size: by the calling thread, or by the calling warp.
__device__ __forceinline__ bool cand_lane(MergeSmem& sm, LaneScratch& ls, int p1, int k, int L, const TestCtx& tc,
                                          int lane) {
  const int e = sm.cand[k];
  unsigned int U[kWords];
#pragma unroll
  for (int w = 0; w < kWords; w++) U[w] = sm.mask[p1][w] | sm.mask[e][w];
  const unsigned int m = tc.z.at(L);
  return lane_test(sm.st, U, m, tc.kc, tc.km, tc.sched, tc.mdiv[m], ls, lane, tc.err);
}
__device__ __forceinline__ bool cand_warp(MergeSmem& sm, RtaScratch& sc, int p1, int k, int L, const TestCtx& tc) {
  const int e = sm.cand[k];
  unsigned int U[kWords];
#pragma unroll
  for (int w = 0; w < kWords; w++) U[w] = sm.mask[p1][w] | sm.mask[e][w];
  return warp_test(sm.st, U, tc.z.at(L), tc.kc, tc.km, tc.sched, tc.mdiv, sc, nullptr, true, tc.err);
}

// The first passing job (nj when none) of jobs 0 .. nj - 1, job(j, k, L)
// giving candidate k at size index L.  Jobs go in windows of up to
// min(nthreads, kWinMax): a window's thread-tested jobs run at once, one per
// thread; then its warp-tested jobs that precede the window's first thread
// pass run in order, one per warp, until a round holds a pass.  No job after
// the first pass of a window is needed, and no later window is opened.
template <class Job>
__device__ int first_pass(const Grp& g, MergeSmem& sm, RtaScratch& sc, LaneScratch& ls, int p1, int nj, Job job,
                          const TestCtx& tc) {
  const int span = min(g.nthreads, kWinMax);
  for (int c0 = 0; c0 < nj; c0 += span) {
    const int c1 = min(nj, c0 + span);
    const int j = c0 + g.tid;
    int f = c1;
    if (g.tid < span && j < c1) {
      int k, L;
      job(j, k, L);
      if (!sm.big[k] && cand_lane(sm, ls, p1, k, L, tc, g.lane)) f = j;
    }
    f = grp_min_int(g, sm, f);
    // the warp-tested jobs of [c0, f), in order
    if (g.warp == 0) {
      int cnt = 0;
      for (int b0 = c0; b0 < f; b0 += 32) {
        const int jj = b0 + g.lane;
        bool w = false;
        if (jj < f) {
          int k, L;
          job(jj, k, L);
          w = sm.big[k] != 0;
        }
        const unsigned int bm = __ballot_sync(kFull, w);
        if (w) sm.wl[cnt + __popc(bm & ((1u << g.lane) - 1u))] = (unsigned char)(jj - c0);
        cnt += __popc(bm);
      }
      if (g.lane == 0) sm.ctl[4] = cnt;
    }
    g.sync();
    const int nw = sm.ctl[4];
    int win = f;
    for (int r0 = 0; r0 < nw; r0 += g.nwarps) {
      const int q = r0 + g.warp;
      int hit = c1;
      if (q < nw) {
        const int jj = c0 + sm.wl[q];
        int k, L;
        job(jj, k, L);
        if (cand_warp(sm, sc, p1, k, L, tc)) hit = jj;
      }
      hit = grp_min_int(g, sm, hit);
      if (hit < c1) {
        win = hit;
        break;
      }
    }
    if (win < c1) return win;
  }
  return nj;
}

// Every job's result into sm.pass[j] (no early exit).
template <class Job>
__device__ void eval_all(const Grp& g, MergeSmem& sm, RtaScratch& sc, LaneScratch& ls, int p1, int nj, Job job,
                         const TestCtx& tc) {
  for (int j = g.tid; j < nj; j += g.nthreads) {
    int k, L;
    job(j, k, L);
    if (!sm.big[k]) sm.pass[j] = cand_lane(sm, ls, p1, k, L, tc, g.lane) ? 1 : 0;
  }
  for (int j = g.warp; j < nj; j += g.nwarps) {
    int k, L;
    job(j, k, L);
    if (sm.big[k]) {
      const bool ok = cand_warp(sm, sc, p1, k, L, tc);
      if (g.lane == 0) sm.pass[j] = ok ? 1 : 0;
    }
  }
  g.sync();
}

// Compacts, in order, the candidates k < ne with pred(k) into sm.jk (warp 0);
// returns their number to the whole group.
template <class Pred>
__device__ int compact_jobs(const Grp& g, MergeSmem& sm, int ne, Pred pred) {
  if (g.warp == 0) {
    int cnt = 0;
    for (int b0 = 0; b0 < ne; b0 += 32) {
      const int k = b0 + g.lane;
      const bool in = k < ne && pred(k);
      const unsigned int bm = __ballot_sync(kFull, in);
      if (in) sm.jk[cnt + __popc(bm & ((1u << g.lane) - 1u))] = (unsigned char)k;
      cnt += __popc(bm);
    }
    if (g.lane == 0) sm.ctl[3] = cnt;
  }
  g.sync();
  const int nj = sm.ctl[3];
  g.sync();
  return nj;
}

__device__ __forceinline__ bool mask_meets(const unsigned int* a, const unsigned int* b) {
  unsigned int x = 0;
#pragma unroll
  for (int w = 0; w < kWords; w++) x |= a[w] & b[w];
  return x != 0u;
}

// par_list key of slot x: larger first; utilisation, then the lower lowest
// task index (unique among live slots, their task sets being disjoint).
__device__ __forceinline__ unsigned long long par_key(const MergeSmem& sm, int x) {
  return ((sm.Uc[x] + sm.Um[x]) << 8) | (unsigned long long)(255u - sm.lowest[x]);
}

// par_list order (decreasing utilisation, ties to the lower lowest index),
// by counting larger keys.
__device__ int sort_par_list(const Grp& g, MergeSmem& sm, int nslots) {
  int alive_count = 0;
  for (int x = g.tid; x < nslots; x += g.nthreads) alive_count += sm.alive[x];
  alive_count = grp_sum_int(g, sm, alive_count);
  for (int x = g.tid; x < nslots; x += g.nthreads) sm.wkey[x] = sm.alive[x] ? par_key(sm, x) : 0ull;
  g.sync();
  for (int x = g.tid; x < nslots; x += g.nthreads) {
    if (!sm.alive[x]) continue;
    const unsigned long long kx = sm.wkey[x];
    int r = 0;
#pragma unroll 4
    for (int y = 0; y < nslots; y++) r += sm.wkey[y] > kx;  // dead slots have key 0
    sm.order[r] = (unsigned char)x;
  }
  g.sync();
  return alive_count;
}

// Eligibility of every slot for a merge with slot c (Alg. 3: partners in a
// forbidden pair are excluded), by one warp; act: some ACT pair is forbidden.
__device__ __forceinline__ void eligible_of(const MergeSmem& sm, int c, int nslots, bool act, unsigned int* elig) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int w = 0; w < kWords; w++) {
    const int e = w * 32 + lane;
    bool ok = e < nslots && w * 32 < nslots && sm.alive[e] && e != c && !((sm.forb[c][w] >> lane) & 1u) &&
              !(act && mask_meets(sm.mask[e], sm.actm[c]));
    elig[w] = __ballot_sync(kFull, ok);
  }
}

__device__ void apply_merge(const Grp& g, MergeSmem& sm, int a, int b, unsigned int m3, int nslots) {
  g.sync();
  if (g.tid < kWords) {
    sm.mask[a][g.tid] |= sm.mask[b][g.tid];
    sm.actm[a][g.tid] |= sm.actm[b][g.tid];
    sm.forb[a][g.tid] = 0u;
    sm.forb[b][g.tid] = 0u;
  }
  if (g.tid == 0) {
    sm.m[a] = (unsigned short)m3;
    sm.Uc[a] += sm.Uc[b];
    sm.Um[a] += sm.Um[b];
    sm.nc[a] = (unsigned char)(sm.nc[a] + sm.nc[b]);
    sm.nm[a] = (unsigned char)(sm.nm[a] + sm.nm[b]);
    sm.lowest[a] = min(sm.lowest[a], sm.lowest[b]);
    sm.alive[b] = 0;
  }
  g.sync();
  // the merged slot holds a task set never seen before: clear its column
  for (int x = g.tid; x < nslots; x += g.nthreads) {
    sm.forb[x][a >> 5] &= ~(1u << (a & 31));
    sm.forb[x][b >> 5] &= ~(1u << (b & 31));
    if (sm.slot_of[x] == b) sm.slot_of[x] = (unsigned char)a;
  }
  g.sync();
}

// par_list after slot b was merged into slot a (positions pa, pb in the old
// order): the others keep their order, b leaves and a moves to its new rank,
// the number of the others with a larger key.  Returns the new length.
__device__ int reorder_after_merge(const Grp& g, MergeSmem& sm, int a, int b, int nal) {
  const unsigned long long ka = par_key(sm, a);
  int pa = -1, pb = -1, ra = 0;
  for (int p = g.tid; p < nal; p += g.nthreads) {
    const int x = sm.order[p];
    if (x == a) pa = p;
    else if (x == b) pb = p;
    else ra += par_key(sm, x) > ka;
  }
  pa = grp_max_int(g, sm, pa);
  pb = grp_max_int(g, sm, pb);
  ra = grp_sum_int(g, sm, ra);
  for (int p = g.tid; p < nal; p += g.nthreads) {
    const int x = sm.order[p];
    if (x == a || x == b) continue;
    int q = p - (pa < p) - (pb < p);
    q += q >= ra;
    sm.jk[q] = (unsigned char)x;
  }
  if (g.tid == 0) sm.jk[ra] = (unsigned char)a;
  g.sync();
  for (int p = g.tid; p < nal - 1; p += g.nthreads) sm.order[p] = sm.jk[p];
  g.sync();
  return nal - 1;
}

// Forbids the pairs (p1, cand[k]) for k < kend.
__device__ void forbid_cands(const Grp& g, MergeSmem& sm, int p1, int kend) {
  for (int k = g.tid; k < kend; k += g.nthreads) {
    const int e = sm.cand[k];
    atomicOr(&sm.forb[p1][e >> 5], 1u << (e & 31));
    atomicOr(&sm.forb[e][p1 >> 5], 1u << (p1 & 31));
  }
  g.sync();
}

// Size ranges of the candidates (indices of admissible sizes in
// [max(m1, m2), min(m1 + m2 - g, M)], ka > kb when there is none) and which
// are tested by a warp.  Returns the lowest and highest live index.
// Candidate k (slot e): its range, whether a warp tests it, whether it is
// live; lo_i / hi_i take in its range.
__device__ __forceinline__ void cand_range_of(MergeSmem& sm, int p1, int k, int e, const Sizes& z, int& lo_i,
                                              int& hi_i) {
  const unsigned int lo = max(sm.m[p1], sm.m[e]);
  const unsigned int hi = min((unsigned int)sm.m[p1] + sm.m[e] - 1u, z.M);
  const int a = z.below(lo), b = lo <= hi ? z.below(hi + 1u) - 1 : a - 1;
  sm.ka[k] = (unsigned short)a;
  sm.kb[k] = (unsigned short)(b < 0 ? 0 : b);
  // tasks of the merged set (the two slots' task sets are disjoint)
  const int cnt = sm.nc[p1] + sm.nm[p1] + sm.nc[e] + sm.nm[e];
  sm.big[k] = cnt > kLaneMax ? 1 : 0;
  sm.live[k] = b >= a ? 1 : 0;
  if (b >= a) {
    lo_i = min(lo_i, a);
    hi_i = max(hi_i, b);
  }
}

__device__ void cand_ranges(const Grp& g, MergeSmem& sm, int p1, int ne, const Sizes& z, int* lmin, int* lmax) {
  int lo_i = 1 << 30, hi_i = -1;
  for (int k = g.tid; k < ne; k += g.nthreads) cand_range_of(sm, p1, k, sm.cand[k], z, lo_i, hi_i);
  *lmin = grp_min_int(g, sm, lo_i);
  *lmax = grp_max_int(g, sm, hi_i);
}

// Alg. 1 for the set staged in sm.st (n tasks), by group g.  extra holds the
// test scratch of the group's warps after its first; top_first selects the
// SMS top-size round (same results either way).
__device__ void merge_set(const Grp& g, MergeSmem& sm, WarpScratch* extra, long long s, long long o, int n,
                          const DevModel& md, const gpa_params& p, const AllocOut& out, const MagicDiv* mdiv,
                          unsigned int* err, bool top_first) {
  const int tid = g.tid;
  RtaScratch& sc = grp_sc(sm, extra, g);
  LaneScratch& ls = grp_ls(sm, extra, g);
  const unsigned kc = (unsigned)md.kc, km = (unsigned)md.km, M = (unsigned)md.M;
  const int sched = md.sched;
  const Sizes z = sizes_of(md);
  const bool linear = p.linear_merge != 0;
  const TestCtx tc{z, kc, km, sched, mdiv, err};

  // Lemma 1: sum_i floor(10^6 C^n_i(1) / T_i) > 10^6 M rejects the set.
  unsigned long long l1 = 0;
  for (int r = tid; r < n; r += g.nthreads) {
    unsigned long long c1 = (sm.st.A[r] + sm.st.B[r] + 999ull) / 1000ull;  // C^n(1)
    l1 += c1 * 1000000ull / sm.st.T[r];
  }
  l1 = grp_sum_u64(g, sm, l1);
  if (l1 > 1000000ull * M) {
    if (g.warp == 0) write_empty(s, o, n, GPA_REASON_LEMMA1, out, 0);
    g.sync();
    return;
  }
  // init_partitions (Lemma 2): slot r = row r
  int none = 0, pi = 0;
  for (int r = tid; r < kNmax; r += g.nthreads) {
    unsigned int mr = 0;
    if (r < n) {
      mr = lemma2_size(sm.st.A[r], sm.st.B[r], sm.st.D[r], z);
      none += mr == 0u;
      pi += (int)mr;
      const bool mem = (sm.st.memmask[r >> 5] >> (r & 31)) & 1u;
      sm.m[r] = (unsigned short)mr;
      sm.Uc[r] = mem ? 0ull : sm.st.u[r];
      sm.Um[r] = mem ? sm.st.u[r] : 0ull;
      sm.nc[r] = mem ? 0 : 1;
      sm.nm[r] = mem ? 1 : 0;
      sm.lowest[r] = sm.st.orig[r];
      sm.alive[r] = 1;
      sm.slot_of[r] = (unsigned char)r;
    } else {
      sm.alive[r] = 0;
    }
#pragma unroll
    for (int w = 0; w < kWords; w++) {
      sm.mask[r][w] = (r < n && (r >> 5) == w) ? (1u << (r & 31)) : 0u;
      sm.actm[r][w] = 0u;
      sm.forb[r][w] = 0u;
      sm.act[r][w] = 0u;
    }
  }
  none = grp_sum_int(g, sm, none);
  pi = grp_sum_int(g, sm, pi);
  if (none) {
    if (g.warp == 0) write_empty(s, o, n, GPA_REASON_LEMMA2, out, 0);
    g.sync();
    return;
  }
  int tests = 0;
  bool act_any = false;  // some ACT pair is forbidden
  // ACT: every task pair is tried as a merge of two singletons; pairs that
  // fail are forbidden for the rest of the run (§5.3).  A pair merges iff
  // it passes at the top admissible size of its range.
  if (p.act && pi > (int)M) {
    for (int q = tid; q < n * n; q += g.nthreads) {
      const int a = q / n, b = q - a * n;
      if (a >= b) continue;
      unsigned int S2[kWords];
#pragma unroll
      for (int w = 0; w < kWords; w++) S2[w] = 0u;
      S2[a >> 5] |= 1u << (a & 31);
      S2[b >> 5] |= 1u << (b & 31);
      const unsigned int lo = max(sm.m[a], sm.m[b]), hi = min((unsigned int)sm.m[a] + sm.m[b] - 1u, M);
      const int ia = z.below(lo), ib = lo <= hi ? z.below(hi + 1u) - 1 : ia - 1;
      bool ok = false;
      if (ib >= ia) {
        const unsigned int mt = z.at(ib);
        ok = lane_test(sm.st, S2, mt, kc, km, sched, mdiv[mt], ls, g.lane, err);
      }
      if (!ok) {
        atomicOr(&sm.act[a][b >> 5], 1u << (b & 31));
        atomicOr(&sm.act[b][a >> 5], 1u << (a & 31));
      }
    }
    tests += n * (n - 1) / 2;
    g.sync();
    int any = 0;
    for (int r = tid; r < n; r += g.nthreads)
#pragma unroll
      for (int w = 0; w < kWords; w++) {
        sm.actm[r][w] = sm.act[r][w];
        any |= sm.act[r][w] != 0u;
      }
    act_any = grp_sum_int(g, sm, any) != 0;
  }

  bool stuck = false;
  int nal = pi > (int)M ? sort_par_list(g, sm, n) : 0, r0 = 0;
  while (pi > (int)M) {
    // Alg. 3 (warp 0): the first partition in par_list order, from r0, with
    // an eligible partner; its eligible partners in par_list order
    if (g.warp == 0) {
      int p1 = -1, rp = nal, ne = 0;
      unsigned int elig[kWords];
      for (int r = r0; r < nal; r++) {
        const int c = sm.order[r];
        eligible_of(sm, c, n, act_any, elig);
        unsigned int any = 0u;
#pragma unroll
        for (int w = 0; w < kWords; w++) any |= elig[w];
        if (any) {
          p1 = c;
          rp = r;
          break;
        }
      }
      // SMS keeps the candidates in par_list order, so their size ranges are
      // set here as they are listed (BF sorts them first: cand_ranges)
      const bool sms = p.policy == GPA_POLICY_SMS;
      int lo_i = 1 << 30, hi_i = -1;
      if (p1 >= 0) {
        for (int b0 = 0; b0 < nal; b0 += 32) {
          const int r = b0 + g.lane;
          const int e = r < nal ? sm.order[r] : 0;
          const bool in = r < nal && ((elig[e >> 5] >> (e & 31)) & 1u);
          const unsigned int bm = __ballot_sync(kFull, in);
          if (in) {
            const int k = ne + __popc(bm & ((1u << g.lane) - 1u));
            sm.cand[k] = (unsigned char)e;
            if (sms) cand_range_of(sm, p1, k, e, z, lo_i, hi_i);
          }
          ne += __popc(bm);
        }
      }
      lo_i = __reduce_min_sync(kFull, lo_i);
      hi_i = __reduce_max_sync(kFull, hi_i);
      if (g.lane == 0) {
        sm.ctl[0] = p1;
        sm.ctl[1] = rp;
        sm.ctl[2] = ne;
        sm.ctl[3] = lo_i;
        sm.ctl[4] = hi_i;
      }
    }
    g.sync();
    const int p1 = sm.ctl[0], rp = sm.ctl[1], ne = sm.ctl[2], lmin_sel = sm.ctl[3], lmax_sel = sm.ctl[4];
    g.sync();
    if (p1 < 0) {
      stuck = true;
      break;
    }
    int win = -1;            // chosen candidate
    unsigned int wm = 0u;    // its merged size
    if (p.policy == GPA_POLICY_SMS) {
      // Def. 3: compute every candidate merge; smallest size wins, ties to
      // the earlier par_list position (ranges set by the selection above)
      int lmin = lmin_sel, lmax = lmax_sel;
      if (linear) {
        // with top_first, a candidate tested by one thread with more than
        // one size in its range is first tested at its top size: failing
        // there, it fails at every size (§4.1) and leaves the scan, so a step
        // whose merges all fail takes one round.  (A top-size test costs more
        // than one at the range's bottom, so this pays where failing steps
        // with short ranges dominate -- the 50-task paper setting -- and not
        // on 200-task sets; the launch shape carries the choice, which the
        // autotuner times.)
        const int nt = !top_first ? 0 : compact_jobs(g, sm, ne, [&](int k) {
          return sm.live[k] && !sm.big[k] && sm.ka[k] < sm.kb[k];
        });
        if (nt > 0) {
          eval_all(
              g, sm, sc, ls, p1, nt,
              [&](int jj, int& k, int& Li) {
                k = sm.jk[jj];
                Li = sm.kb[k];
              },
              tc);
          int lo_i = 1 << 30, hi_i = -1;
          for (int jj = tid; jj < nt; jj += g.nthreads)
            if (!sm.pass[jj]) sm.live[sm.jk[jj]] = 0;
          g.sync();
          for (int k = tid; k < ne; k += g.nthreads)
            if (sm.live[k]) {
              lo_i = min(lo_i, (int)sm.ka[k]);
              hi_i = max(hi_i, (int)sm.kb[k]);
            }
          lmin = grp_min_int(g, sm, lo_i);
          lmax = grp_max_int(g, sm, hi_i);
        }
        for (int L = lmin; L <= lmax && win < 0; L++) {
          const int nj = compact_jobs(g, sm, ne, [&](int k) { return sm.live[k] && sm.ka[k] <= L && L <= sm.kb[k]; });
          if (nj == 0) continue;
          const int j = first_pass(
              g, sm, sc, ls, p1, nj,
              [&](int jj, int& k, int& Li) {
                k = sm.jk[jj];
                Li = L;
              },
              tc);
          if (j < nj) {
            win = sm.jk[j];
            wm = z.at(L);
          }
        }
      } else {
        // §5.2's binary search, for every candidate at once: kx is one past
        // the highest size still possible (kb + 1: none)
        for (int k = tid; k < ne; k += g.nthreads) sm.kx[k] = (unsigned short)(sm.kb[k] + 1);
        g.sync();
        for (;;) {
          const int nj = compact_jobs(g, sm, ne, [&](int k) { return sm.live[k] && sm.ka[k] < sm.kx[k]; });
          if (nj == 0) break;
          auto mid = [&](int jj, int& k, int& Li) {
            k = sm.jk[jj];
            Li = (sm.ka[k] + sm.kx[k]) / 2;
          };
          eval_all(g, sm, sc, ls, p1, nj, mid, tc);
          for (int jj = tid; jj < nj; jj += g.nthreads) {
            const int k = sm.jk[jj];
            const int Li = (sm.ka[k] + sm.kx[k]) / 2;
            if (sm.pass[jj]) sm.kx[k] = (unsigned short)Li;
            else sm.ka[k] = (unsigned short)(Li + 1);
          }
          g.sync();
        }
        // the smallest size, then the earliest position
        int key = 1 << 30;
        for (int k = tid; k < ne; k += g.nthreads)
          if (sm.live[k] && sm.ka[k] <= sm.kb[k]) key = min(key, ((int)sm.ka[k] << 8) | k);
        key = grp_min_int(g, sm, key);
        if (key < (1 << 30)) {
          win = key & 255;
          wm = z.at(key >> 8);
        }
      }
      tests += ne;
      if (win >= 0) {
        const int best = sm.cand[win];
        pi -= (int)sm.m[p1] + (int)sm.m[best] - (int)wm;
        apply_merge(g, sm, p1, best, wm, n);
        nal = reorder_after_merge(g, sm, p1, best, nal);
        r0 = 0;
      } else {
        forbid_cands(g, sm, p1, ne);
        r0 = rp + 1;
      }
    } else {
      // Def. 4: eligible partners sorted by the workload of the merge, ties
      // to the earlier par_list position; tried in that order
      for (int k = tid; k < ne; k += g.nthreads) {
        const int e = sm.cand[k];
        sm.wkey[k] = workload_from_sums(sm.Uc[p1] + sm.Uc[e], sm.Um[p1] + sm.Um[e], sm.nc[p1] + sm.nc[e],
                                        sm.nm[p1] + sm.nm[e], kc, km);
      }
      g.sync();
      unsigned char sorted_e[kWords];
      int sorted_r[kWords];
#pragma unroll
      for (int c = 0; c < kWords; c++) {
        const int x = c * g.nthreads + tid;
        sorted_r[c] = -1;
        if (x < ne) {
          int rr = 0;
          for (int y = 0; y < ne; y++) rr += (sm.wkey[y] < sm.wkey[x]) || (sm.wkey[y] == sm.wkey[x] && y < x);
          sorted_r[c] = rr;
          sorted_e[c] = sm.cand[x];
        }
      }
      g.sync();
#pragma unroll
      for (int c = 0; c < kWords; c++)
        if (sorted_r[c] >= 0) sm.cand[sorted_r[c]] = sorted_e[c];
      g.sync();
      int lmin, lmax;
      cand_ranges(g, sm, p1, ne, z, &lmin, &lmax);
      // the first candidate, in order, that passes at its top size
      const int nj = compact_jobs(g, sm, ne, [&](int k) { return sm.live[k] != 0; });
      const int j = first_pass(
          g, sm, sc, ls, p1, nj,
          [&](int jj, int& k, int& Li) {
            k = sm.jk[jj];
            Li = sm.kb[k];
          },
          tc);
      const int kw = j < nj ? (int)sm.jk[j] : ne;
      forbid_cands(g, sm, p1, kw);
      if (kw < ne) {
        tests += kw + 1;
        // its smallest passing size: sizes ka .. kb - 1 upwards (kb passes)
        const int a = sm.ka[kw], b = sm.kb[kw];
        const int jj = first_pass(
            g, sm, sc, ls, p1, b - a,
            [&](int q, int& k, int& Li) {
              k = kw;
              Li = a + q;
            },
            tc);
        win = kw;
        wm = z.at(a + jj);
        const int best = sm.cand[win];
        pi -= (int)sm.m[p1] + (int)sm.m[best] - (int)wm;
        apply_merge(g, sm, p1, best, wm, n);
        nal = reorder_after_merge(g, sm, p1, best, nal);
        r0 = 0;
      } else {
        tests += ne;
        r0 = rp + 1;
      }
    }
  }
  // report: partitions numbered by their lowest task index
  int nal2 = 0;
  unsigned long long W = 0;
  for (int x = tid; x < n; x += g.nthreads) {
    if (!sm.alive[x]) continue;
    nal2++;
    W += workload_from_sums(sm.Uc[x], sm.Um[x], sm.nc[x], sm.nm[x], kc, km);
    int r = 0;
    for (int y = 0; y < n; y++) r += sm.alive[y] && sm.lowest[y] < sm.lowest[x];
    sm.rank[x] = (unsigned char)r;
  }
  nal2 = grp_sum_int(g, sm, nal2);
  W = grp_sum_u64(g, sm, W);
  for (int r = tid; r < n; r += g.nthreads) out.size_of_part[o + r] = 0;
  g.sync();
  for (int x = tid; x < n; x += g.nthreads)
    if (sm.alive[x]) out.size_of_part[o + sm.rank[x]] = (short)sm.m[x];
  for (int r = tid; r < n; r += g.nthreads) out.part_of_task[o + sm.st.orig[r]] = sm.rank[sm.slot_of[r]];
  if (tid == 0) {
    const bool ok = !stuck && pi <= (int)M;
    out.verdict[s] = ok ? 1 : 0;
    out.reason[s] = ok ? GPA_REASON_OK : GPA_REASON_NO_MERGE;
    out.n_parts[s] = nal2;
    out.Pi[s] = pi;
    out.W[s] = (long long)W;
    if (out.n_tests) out.n_tests[s] = tests;
  }
  g.sync();
}

// Adds the group warp's interference-term counts (its thread counters and
// its warp counter) to *total, and clears them.  The whole warp calls it.
__device__ __forceinline__ void flush_terms(RtaScratch& sc, LaneScratch& ls, unsigned long long* total) {
  const int lane = threadIdx.x & 31;
  __syncwarp();
  unsigned long long t = warp_sum_u64(ls.terms[lane]) + sc.terms;
  __syncwarp();
  ls.terms[lane] = 0ull;
  if (lane == 0) sc.terms = 0ull;
  if (lane == 0 && t && total) atomicAdd(total, t);
  __syncwarp();
}

}  // namespace

GPA_NS_END
