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

constexpr int kLaneMax = 16;  // merged sets of up to this many tasks are tested by one lane

// One lane's serial test of a candidate merge: WCETs and rows of the merged
// set's tasks in priority order, [position][lane] (conflict-free banks).
struct LaneScratch {
  unsigned int C[kLaneMax][32];
  unsigned char row[kLaneMax][32];
  unsigned short res[kNmax];  // size found per candidate; 0 none; kLaneNone: not tried by a lane
};
constexpr unsigned short kLaneNone = 0xFFFFu;

struct MergeSmem {
  SetSmem st;
  RtaScratch sc;
  LaneScratch ls;
  unsigned int mask[kNmax][kWords];  // tasks (rows) of each partition slot
  unsigned int actm[kNmax][kWords];  // rows forbidden to the slot by ACT pairs
  unsigned int forb[kNmax][kWords];  // slots whose exact pair with this slot failed
  unsigned int act[kNmax][kWords];   // ACT pair matrix over rows
  unsigned long long Uc[kNmax];      // utilisation of the slot's compute tasks
  unsigned long long Um[kNmax];      // utilisation of the slot's memory tasks
  unsigned long long wkey[kNmax];    // BF: workload of each candidate merge
  unsigned short m[kNmax];           // slot size (SMs)
  unsigned char nc[kNmax], nm[kNmax];
  unsigned char lowest[kNmax];       // lowest original task index in the slot
  unsigned char alive[kNmax];
  unsigned char order[kNmax];        // par_list: slots in order
  unsigned char cand[kNmax];         // BF: eligible slots sorted by (W, position)
  unsigned char slot_of[kNmax];      // slot of each row
  unsigned char rank[kNmax];         // output numbering of each slot
  unsigned int err;                  // error bits of the set being processed
};


// §5.5 per-partition test of a merged set S (at most kLaneMax tasks) by one
// lane, serially.  Tasks are visited in priority order and each earlier task
// met its deadline, so R_i >= R_prev + C_i starts the iteration (same least
// fixed point as starting from the sum of the WCETs).
__device__ bool lane_rta(const SetSmem& st, const unsigned int* S, unsigned int m, unsigned int kc, unsigned int km,
                         const MagicDiv& md, LaneScratch& ls, int lane, unsigned int* err) {
  int nm = 0, ns = 0;
#pragma unroll
  for (int w = 0; w < kWords; w++) {
    nm += __popc(S[w] & st.memmask[w]);
    ns += __popc(S[w]);
  }
  const unsigned int kmem = nm >= 2 ? km : 1000u, kcmp = (ns - nm) >= 2 ? kc : 1000u;
  unsigned long long Rprev = 0;
  int pos = 0;
  for (int w = 0; w < kWords; w++) {
    for (unsigned int bits = S[w]; bits; bits &= bits - 1u) {
      const int row = w * 32 + __ffs(bits) - 1;
      const bool mem = (st.memmask[w] >> (row & 31)) & 1u;
      const unsigned int Ci = wcet(st.A[row], st.B[row], mem ? kmem : kcmp, m, md);
      ls.C[pos][lane] = Ci;
      ls.row[pos][lane] = (unsigned char)row;
      unsigned long long R = Rprev + Ci;
      const unsigned int Di = st.D[row];
      const unsigned long long cap = (unsigned long long)Di + 1ull;
      int iter = 0;
      for (;;) {
        if (R > Di) return false;
        unsigned long long next = Ci;
        for (int q = 0; q < pos; q++) {
          const int rq = ls.row[q][lane];
          const unsigned long long t = (unsigned long long)ceil_div_T((unsigned int)R, st.mT[rq], st.shT[rq]) *
                                       ls.C[q][lane];
          next += t < cap ? t : cap;
        }
        if (next == R) break;
        R = next;
        if (++iter > kIterCap) {
          atomicOr(err, kErrIter);
          return false;
        }
      }
      Rprev = R;
      pos++;
    }
  }
  return true;
}

// The EDF test of S (at most kLaneMax tasks) by one lane.
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
      ls.C[pos][lane] = wcet(st.A[row], st.B[row], mem ? kmem : kcmp, m, md);
      ls.row[pos][lane] = (unsigned char)row;
      pos++;
    }
  }
  unsigned int eb = 0u;
  const bool ok = serial_edf(
      pos,
      [&](int a, unsigned int& C, unsigned int& T, unsigned int& D, unsigned int& mg, unsigned int& sh) {
        const int r = ls.row[a][lane];
        C = ls.C[a][lane];
        T = st.T[r];
        D = st.D[r];
        mg = st.mT[r];
        sh = st.shT[r];
      },
      &eb);
  if (eb) atomicOr(err, eb);
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

// Alg. 2 by one lane: the first admissible size in [lo, hi] that passes.  A
// range of up to three sizes is scanned; a longer one is bisected (§5.2),
// which finds the same size because the test is monotone in m.
__device__ unsigned int lane_minm(const SetSmem& st, const unsigned int* S, unsigned int lo, unsigned int hi,
                                  const Sizes& z, unsigned int kc, unsigned int km, int sched,
                                  const MagicDiv* __restrict__ mdiv, LaneScratch& ls, int lane, unsigned int* err) {
  if (lo > hi) return 0u;
  hi = min(hi, z.M);
  int a = z.below(lo);
  const int e = z.below(hi + 1u);  // indices of the admissible sizes in [lo, hi]: a .. e - 1
  if (e - a <= 3) {
    for (int k = a; k < e; k++) {
      const unsigned int m = z.at(k);
      if (lane_test(st, S, m, kc, km, sched, mdiv[m], ls, lane, err)) return m;
    }
    return 0u;
  }
  int b = e;  // e stands for "no size passes"
  while (a < b) {
    const int mid = a + (b - a) / 2;
    const unsigned int m = z.at(mid);
    if (lane_test(st, S, m, kc, km, sched, mdiv[m], ls, lane, err)) b = mid;
    else a = mid + 1;
  }
  return a < e ? z.at(a) : 0u;
}

// Sizes of the candidate merges of slot p1 with cand[c0 .. c1) into ls.res:
// one lane per candidate when the merged set is small, then the warp for
// the others.  Warp-uniform arguments.
__device__ void size_candidates(MergeSmem& sm, int p1, int c0, int c1, const Sizes& z, bool linear, unsigned int kc,
                                unsigned int km, int sched, const MagicDiv* __restrict__ mdiv, unsigned int* err) {
  const int lane = threadIdx.x & 31;
  for (int b = c0; b < c1; b += 32) {
    const int k = b + lane;
    if (k < c1) {
      const int e = sm.cand[k];
      unsigned int U[kWords];
      int cnt = 0;
#pragma unroll
      for (int w = 0; w < kWords; w++) {
        U[w] = sm.mask[p1][w] | sm.mask[e][w];
        cnt += __popc(U[w]);
      }
      // merged sizes: admissible, from the larger of the two up to below their sum
      const unsigned int lo = max(sm.m[p1], sm.m[e]), hi = sm.m[p1] + sm.m[e] - 1u;
      sm.ls.res[k] = cnt <= kLaneMax ? (unsigned short)lane_minm(sm.st, U, lo, hi, z, kc, km, sched, mdiv, sm.ls, lane, err)
                                     : kLaneNone;
    }
  }
  __syncwarp();
  for (int k = c0; k < c1; k++) {
    if (sm.ls.res[k] != kLaneNone) continue;
    const int e = sm.cand[k];
    unsigned int U[kWords];
#pragma unroll
    for (int w = 0; w < kWords; w++) U[w] = sm.mask[p1][w] | sm.mask[e][w];
    const unsigned int lo = max(sm.m[p1], sm.m[e]), hi = sm.m[p1] + sm.m[e] - 1u;
    const unsigned int m3 = warp_minm(sm.st, U, lo, hi, z, linear, kc, km, sched, mdiv, sm.sc, err);
    __syncwarp();
    if (lane == 0) sm.ls.res[k] = (unsigned short)m3;
    __syncwarp();
  }
}

__device__ __forceinline__ bool mask_meets(const unsigned int* a, const unsigned int* b) {
  unsigned int x = 0;
#pragma unroll
  for (int w = 0; w < kWords; w++) x |= a[w] & b[w];
  return x != 0u;
}

// par_list order (decreasing utilisation, ties to the lower lowest index).
__device__ int sort_par_list(MergeSmem& sm, int nslots) {
  const int lane = threadIdx.x & 31;
  int alive_count = 0;
  for (int x = lane; x < nslots; x += 32) alive_count += sm.alive[x];
  alive_count = warp_sum_i32(alive_count);
  for (int x = lane; x < nslots; x += 32) {
    if (!sm.alive[x]) continue;
    unsigned long long ux = sm.Uc[x] + sm.Um[x];
    int r = 0;
    for (int y = 0; y < nslots; y++) {
      if (!sm.alive[y] || y == x) continue;
      unsigned long long uy = sm.Uc[y] + sm.Um[y];
      r += (uy > ux) || (uy == ux && sm.lowest[y] < sm.lowest[x]);
    }
    sm.order[r] = (unsigned char)x;
  }
  __syncwarp();
  return alive_count;
}

// Eligibility of every slot for a merge with slot c (Alg. 3: partners in a forbidden pair are excluded).
__device__ __forceinline__ void eligible_of(const MergeSmem& sm, int c, int nslots, unsigned int* elig) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int w = 0; w < kWords; w++) {
    const int e = w * 32 + lane;
    bool ok = e < nslots && sm.alive[e] && e != c && !((sm.forb[c][w] >> lane) & 1u) &&
              !mask_meets(sm.mask[e], sm.actm[c]);
    elig[w] = __ballot_sync(kFull, ok);
  }
}

__device__ void apply_merge(MergeSmem& sm, int a, int b, unsigned int m3, int nslots) {
  const int lane = threadIdx.x & 31;
  __syncwarp();
  if (lane < kWords) {
    sm.mask[a][lane] |= sm.mask[b][lane];
    sm.actm[a][lane] |= sm.actm[b][lane];
    sm.forb[a][lane] = 0u;
    sm.forb[b][lane] = 0u;
  }
  if (lane == 0) {
    sm.m[a] = (unsigned short)m3;
    sm.Uc[a] += sm.Uc[b];
    sm.Um[a] += sm.Um[b];
    sm.nc[a] = (unsigned char)(sm.nc[a] + sm.nc[b]);
    sm.nm[a] = (unsigned char)(sm.nm[a] + sm.nm[b]);
    sm.lowest[a] = min(sm.lowest[a], sm.lowest[b]);
    sm.alive[b] = 0;
  }
  __syncwarp();
  // the merged slot holds a task set never seen before: clear its column
  for (int x = lane; x < nslots; x += 32) {
    sm.forb[x][a >> 5] &= ~(1u << (a & 31));
    sm.forb[x][b >> 5] &= ~(1u << (b & 31));
    if (sm.slot_of[x] == b) sm.slot_of[x] = (unsigned char)a;
  }
  __syncwarp();
}

__device__ void merge_set(MergeSmem& sm, long long s, long long o, int n, const DevModel& md, const gpa_params& p,
                          const AllocOut& out, const MagicDiv* mdiv, unsigned int* err) {
  const int lane = threadIdx.x & 31;
  const unsigned kc = (unsigned)md.kc, km = (unsigned)md.km, M = (unsigned)md.M;
  const int sched = md.sched;
  const Sizes z = sizes_of(md);
  const bool linear = p.linear_merge != 0;

  // Lemma 1: sum_i floor(10^6 C^n_i(1) / T_i) > 10^6 M rejects the set.
  unsigned long long l1 = 0;
  for (int r = lane; r < n; r += 32) {
    unsigned long long c1 = (sm.st.A[r] + sm.st.B[r] + 999ull) / 1000ull;  // C^n(1)
    l1 += c1 * 1000000ull / sm.st.T[r];
  }
  l1 = warp_sum_u64(l1);
  if (l1 > 1000000ull * M) {
    write_empty(s, o, n, GPA_REASON_LEMMA1, out, 0);
    return;
  }
  // init_partitions (Lemma 2): slot r = row r
  bool none = false;
  int pi = 0;
  for (int r = lane; r < kNmax; r += 32) {
    unsigned int mr = 0;
    if (r < n) {
      mr = lemma2_size(sm.st.A[r], sm.st.B[r], sm.st.D[r], z);
      none = none || mr == 0u;
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
  none = __any_sync(kFull, none);
  pi = warp_sum_i32(pi);
  __syncwarp();
  if (none) {
    write_empty(s, o, n, GPA_REASON_LEMMA2, out, 0);
    return;
  }
  int tests = 0;
  // ACT: every task pair is tried as a merge of two singletons; pairs that
  // fail are forbidden for the rest of the run (§5.3).
  if (p.act && pi > (int)M) {
    // one lane per pair (a, b), b > a
    for (int a = 0; a < n; a++)
      for (int b0 = a + 1; b0 < n; b0 += 32) {
        const int b = b0 + lane;
        if (b < n) {
          unsigned int S2[kWords];
#pragma unroll
          for (int w = 0; w < kWords; w++) S2[w] = 0u;
          S2[a >> 5] |= 1u << (a & 31);
          S2[b >> 5] |= 1u << (b & 31);
          const unsigned int lo = max(sm.m[a], sm.m[b]), hi = sm.m[a] + sm.m[b] - 1u;
          if (lane_minm(sm.st, S2, lo, hi, z, kc, km, sched, mdiv, sm.ls, lane, err) == 0u) {
            atomicOr(&sm.act[a][b >> 5], 1u << (b & 31));
            atomicOr(&sm.act[b][a >> 5], 1u << (a & 31));
          }
        }
      }
    tests += n * (n - 1) / 2;
    __syncwarp();
    for (int r = lane; r < n; r += 32)
#pragma unroll
      for (int w = 0; w < kWords; w++) sm.actm[r][w] = sm.act[r][w];
    __syncwarp();
  }

  bool stuck = false;
  while (pi > (int)M) {
    const int nal = sort_par_list(sm, n);
    // Alg. 3: the first partition in par_list order with an eligible partner
    int p1 = -1;
    unsigned int elig[kWords];
    for (int r = 0; r < nal; r++) {
      const int c = sm.order[r];
      eligible_of(sm, c, n, elig);
      unsigned int any = 0u;
#pragma unroll
      for (int w = 0; w < kWords; w++) any |= elig[w];
      if (any) {
        p1 = c;
        break;
      }
    }
    if (p1 < 0) {
      stuck = true;
      break;
    }
    if (p.policy == GPA_POLICY_SMS) {
      // Def. 3: compute every candidate merge; smallest size wins, ties to
      // the earlier par_list position.
      int ne = 0;
      for (int r = 0; r < nal; r++) {
        const int e = sm.order[r];
        if (!((elig[e >> 5] >> (e & 31)) & 1u)) continue;
        if (lane == 0) sm.cand[ne] = (unsigned char)e;
        ne++;
      }
      __syncwarp();
      size_candidates(sm, p1, 0, ne, z, linear, kc, km, sched, mdiv, err);
      tests += ne;
      // smallest size, then earliest position: key = size << 8 | position
      unsigned int keyv = 0xFFFFFFFFu;
      for (int k = lane; k < ne; k += 32) {
        const unsigned int m3 = sm.ls.res[k];
        if (m3 != 0u) keyv = min(keyv, (m3 << 8) | (unsigned int)k);
      }
      keyv = __reduce_min_sync(kFull, keyv);
      const int best = keyv == 0xFFFFFFFFu ? -1 : (int)sm.cand[keyv & 0xFFu];
      const unsigned int best_m = keyv >> 8;
      if (best >= 0) {
        pi -= (int)sm.m[p1] + (int)sm.m[best] - (int)best_m;
        apply_merge(sm, p1, best, best_m, n);
      } else {
        __syncwarp();
        for (int e = lane; e < n; e += 32)
          if ((elig[e >> 5] >> (e & 31)) & 1u) {
            atomicOr(&sm.forb[p1][e >> 5], 1u << (e & 31));
            atomicOr(&sm.forb[e][p1 >> 5], 1u << (p1 & 31));
          }
        __syncwarp();
      }
    } else {
      // Def. 4: eligible partners sorted by the workload of the merge, ties
      // to the earlier par_list position; tried in that order.
      int ne = 0;
      for (int r = 0; r < nal; r++) {
        const int e = sm.order[r];
        if (!((elig[e >> 5] >> (e & 31)) & 1u)) continue;
        if (lane == 0) {
          sm.cand[ne] = (unsigned char)e;
          sm.wkey[ne] = workload_from_sums(sm.Uc[p1] + sm.Uc[e], sm.Um[p1] + sm.Um[e], sm.nc[p1] + sm.nc[e],
                                           sm.nm[p1] + sm.nm[e], kc, km);
        }
        ne++;
      }
      __syncwarp();
      unsigned char sorted_e[kWords];
      int sorted_r[kWords];
      for (int c = 0; c < kWords; c++) {
        const int x = c * 32 + lane;
        sorted_r[c] = -1;
        if (x < ne) {
          int rr = 0;
          for (int y = 0; y < ne; y++) rr += (sm.wkey[y] < sm.wkey[x]) || (sm.wkey[y] == sm.wkey[x] && y < x);
          sorted_r[c] = rr;
          sorted_e[c] = sm.cand[x];
        }
      }
      __syncwarp();
      for (int c = 0; c < kWords; c++)
        if (sorted_r[c] >= 0) sm.cand[sorted_r[c]] = sorted_e[c];
      __syncwarp();
      // tried in that order: chunks of 32 are sized together, the first
      // success (in order) is applied, every earlier failure is forbidden
      for (int c0 = 0; c0 < ne; c0 += 32) {
        const int c1 = min(ne, c0 + 32);
        size_candidates(sm, p1, c0, c1, z, linear, kc, km, sched, mdiv, err);
        const int k = c0 + lane;
        const unsigned int okb = __ballot_sync(kFull, k < c1 && sm.ls.res[k] != 0u);
        const int first = okb ? c0 + __ffs(okb) - 1 : c1;
        if (k < first) {
          const int e = sm.cand[k];
          atomicOr(&sm.forb[p1][e >> 5], 1u << (e & 31));
          atomicOr(&sm.forb[e][p1 >> 5], 1u << (p1 & 31));
        }
        __syncwarp();
        if (okb) {
          tests += first - c0 + 1;
          const int e = sm.cand[first];
          const unsigned int m3 = sm.ls.res[first];
          pi -= (int)sm.m[p1] + (int)sm.m[e] - (int)m3;
          apply_merge(sm, p1, e, m3, n);
          break;
        }
        tests += c1 - c0;
      }
    }
  }
  // report: partitions numbered by their lowest task index
  int nal = 0;
  unsigned long long W = 0;
  for (int x = lane; x < n; x += 32) {
    if (!sm.alive[x]) continue;
    nal++;
    W += workload_from_sums(sm.Uc[x], sm.Um[x], sm.nc[x], sm.nm[x], kc, km);
    int r = 0;
    for (int y = 0; y < n; y++) r += sm.alive[y] && sm.lowest[y] < sm.lowest[x];
    sm.rank[x] = (unsigned char)r;
  }
  nal = warp_sum_i32(nal);
  W = warp_sum_u64(W);
  __syncwarp();
  for (int r = lane; r < n; r += 32) out.size_of_part[o + r] = 0;
  __syncwarp();
  for (int x = lane; x < n; x += 32)
    if (sm.alive[x]) out.size_of_part[o + sm.rank[x]] = (short)sm.m[x];
  for (int r = lane; r < n; r += 32) out.part_of_task[o + sm.st.orig[r]] = sm.rank[sm.slot_of[r]];
  if (lane == 0) {
    const bool ok = !stuck && pi <= (int)M;
    out.verdict[s] = ok ? 1 : 0;
    out.reason[s] = ok ? GPA_REASON_OK : GPA_REASON_NO_MERGE;
    out.n_parts[s] = nal;
    out.Pi[s] = pi;
    out.W[s] = (long long)W;
    if (out.n_tests) out.n_tests[s] = tests;
  }
}


}  // namespace

GPA_NS_END
