// k_alloc.cu — the partition-and-allocate heuristic (Alg. 1-3), the 1G
// baseline, and the persistent work queue that batches them.
//
// Two persistent kernels run back to back on the context stream:
//  * alloc_fast: a warp streams a few consecutive task sets at a time,
//    registers only.  It validates each set, sizes every singleton partition
//    by Lemma 2 in closed form and sums Pi.  When Pi <= M the heuristic ends at its first exit
//    test (Lemma 3) with the singleton partitions, so the set is decided
//    here (Lemma 1 cannot reject then: m C^n(m) >= C^n(1) and C^n(m) <= T
//    give sum C^n(1)/T <= Pi).  Otherwise the set index is appended to a
//    device queue.
//  * alloc_merge: one warp per deferred set, state in shared memory.  It
//    runs Lemma 1, Lemma 2, the optional ACT pass, and the merge loop of
//    Alg. 1 with Alg. 3's selection, Alg. 2's size search and the SMS (Def. 3)
//    or BF (Def. 4) order, exactly as the CPU reading does.
#include <cuda_runtime.h>

#include "gpa_device.cuh"
#include "gpa_internal.h"

namespace gpa {

namespace {

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

// ------------------------------------------------------------- fast kernel
//
// Each warp takes K consecutive task sets at a time (grid-stride over chunks
// of K sets); their tasks are one contiguous range, which the lanes stream in
// coalesced 32-task slices, U slices (6 columns each) in flight together.
// Every task gets its Lemma 2 size in registers; a lane finds the set of its
// task with K-1 compares against the chunk's offsets and adds its values to
// per-set partial sums held in registers; K full-warp reductions finish the
// chunk.  Sets whose singleton partitions already fit (Pi <= M) are decided
// here; the others are appended to the merge kernel's queue, which rewrites
// their per-task outputs.

template <int K, int U>
__global__ void __launch_bounds__(256) alloc_fast(DevSets S, DevModel md, AllocOut out, AllocQueue q) {
  const int lane = threadIdx.x & 31;
  const long long warp0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  const unsigned M = (unsigned)md.M, g = (unsigned)md.g;
  // the offsets of the next chunk are loaded one iteration ahead
  long long offv_next = 0;
  {
    const long long b0 = warp0 * K;
    if (b0 < S.nsets && lane <= (int)min((long long)K, S.nsets - b0)) offv_next = __ldg(S.set_off + b0 + lane);
  }
  for (long long base = warp0 * K; base < S.nsets; base += nwarps * K) {
    const int ns = (int)min((long long)K, S.nsets - base);
    const long long offv = offv_next;
    {
      const long long bn = base + nwarps * K;
      if (bn < S.nsets && lane <= (int)min((long long)K, S.nsets - bn)) offv_next = __ldg(S.set_off + bn + lane);
    }
    long long o[K + 1];
#pragma unroll
    for (int k = 0; k <= K; k++) o[k] = __shfl_sync(kFull, offv, k <= ns ? k : ns);
    bool bad = false;
#pragma unroll
    for (int k = 0; k < K; k++) {
      const long long n = o[k + 1] - o[k];
      bad = bad || n < 0 || n > S.n_max || n > kNmax;
    }
    if (bad) {
      // a malformed size: the merge kernel validates these sets one by one
      if (lane < ns) {
        const unsigned long long idx = atomicAdd(q.counters + 1, 1ull);
        q.slow_sets[idx] = base + lane;
      }
      continue;
    }
    const long long o0 = o[0];
    const int nt = (int)(o[K] - o0);
    unsigned int pi[K], lo[K], hi[K], fl[K];
#pragma unroll
    for (int k = 0; k < K; k++) pi[k] = lo[k] = hi[k] = fl[k] = 0u;
    for (int c0 = 0; c0 < nt; c0 += 32 * U) {
      long long Tt[U], Dt[U], At[U], Bt[U], ut[U];
      unsigned int yt[U];
#pragma unroll
      for (int uu = 0; uu < U; uu++) {
        const int i = c0 + uu * 32 + lane;
        if (i < nt) {
          const long long t = o0 + i;
          Tt[uu] = __ldg(S.T + t);
          Dt[uu] = __ldg(S.D + t);
          At[uu] = __ldg(S.A + t);
          Bt[uu] = __ldg(S.B + t);
          ut[uu] = __ldg(S.u + t);
          yt[uu] = __ldg(S.type + t);
        }
      }
#pragma unroll
      for (int uu = 0; uu < U; uu++) {
        const int i = c0 + uu * 32 + lane;
        if (i < nt) {
          const long long t = o0 + i;
          int ks = 0;
#pragma unroll
          for (int k = 1; k < K; k++) ks += (t >= o[k]) ? 1 : 0;
          unsigned int mm = 0u, f = 0u, ulo = 0u, uhi = 0u;
          if (!task_valid(Tt[uu], Dt[uu], At[uu], Bt[uu], ut[uu], yt[uu])) {
            f = 1u;
          } else {
            mm = lemma2_size_fast((unsigned long long)At[uu], (unsigned long long)Bt[uu],
                                  (unsigned long long)Dt[uu], M, g);
            f = mm == 0u ? 2u : 0u;
            ulo = (unsigned int)ut[uu] & 0xffffu;
            uhi = (unsigned int)((unsigned long long)ut[uu] >> 16);
          }
          long long ok_ = o0;
#pragma unroll
          for (int k = 0; k < K; k++) {
            const bool mine = ks == k;
            pi[k] += mine ? mm : 0u;
            lo[k] += mine ? ulo : 0u;
            hi[k] += mine ? uhi : 0u;
            fl[k] |= mine ? f : 0u;
            ok_ = mine ? o[k] : ok_;
          }
          out.part_of_task[t] = (unsigned char)(t - ok_);
          out.size_of_part[t] = (short)mm;
        }
      }
    }
#pragma unroll
    for (int k = 0; k < K; k++) {
      const unsigned int pk = __reduce_add_sync(kFull, pi[k]);
      const unsigned int lk = __reduce_add_sync(kFull, lo[k]);
      const unsigned int hk = __reduce_add_sync(kFull, hi[k]);
      const unsigned int fk = __reduce_or_sync(kFull, fl[k]);
      if (lane == k && k < ns) {
        const long long s = base + k;
        if (fk != 0u || pk > M) {
          const unsigned long long idx = atomicAdd(q.counters + 1, 1ull);
          q.slow_sets[idx] = s;
        } else {
          // Lemma 3 holds for the singleton partitions (numbered by their task)
          out.verdict[s] = 1;
          out.reason[s] = GPA_REASON_OK;
          out.n_parts[s] = (int)(o[k + 1] - o[k]);
          out.Pi[s] = (int)pk;
          out.W[s] = (long long)(1000ull * (((unsigned long long)hk << 16) + lk));
          if (out.n_tests) out.n_tests[s] = 0;
        }
      }
    }
  }
}

// ------------------------------------------------------------ merge kernel

struct MergeSmem {
  SetSmem st;
  RtaScratch sc;
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
};

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
  const unsigned kc = (unsigned)md.kc, km = (unsigned)md.km, g = (unsigned)md.g, M = (unsigned)md.M;
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
      mr = lemma2_size(sm.st.A[r], sm.st.B[r], sm.st.D[r], M, g);
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
    for (int a = 0; a < n; a++)
      for (int b = a + 1; b < n; b++) {
        unsigned int S2[kWords];
#pragma unroll
        for (int w = 0; w < kWords; w++) S2[w] = 0u;
        S2[a >> 5] |= 1u << (a & 31);
        S2[b >> 5] |= 1u << (b & 31);
        unsigned int lo = max(sm.m[a], sm.m[b]), hi = sm.m[a] + sm.m[b] - g;
        unsigned int m3 = warp_minm(sm.st, S2, lo, hi, g, linear, kc, km, mdiv, sm.sc, err);
        tests++;
        if (m3 == 0u && lane == 0) {
          sm.act[a][b >> 5] |= 1u << (b & 31);
          sm.act[b][a >> 5] |= 1u << (a & 31);
        }
      }
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
    unsigned int U[kWords];
    if (p.policy == GPA_POLICY_SMS) {
      // Def. 3: compute every candidate merge; smallest size wins, ties to
      // the earlier par_list position.
      int best = -1;
      unsigned int best_m = 0u;
      for (int r = 0; r < nal; r++) {
        const int e = sm.order[r];
        if (!((elig[e >> 5] >> (e & 31)) & 1u)) continue;
#pragma unroll
        for (int w = 0; w < kWords; w++) U[w] = sm.mask[p1][w] | sm.mask[e][w];
        unsigned int lo = max(sm.m[p1], sm.m[e]), hi = sm.m[p1] + sm.m[e] - g;
        unsigned int m3 = warp_minm(sm.st, U, lo, hi, g, linear, kc, km, mdiv, sm.sc, err);
        tests++;
        if (m3 != 0u && (best < 0 || m3 < best_m)) {
          best = e;
          best_m = m3;
        }
      }
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
      for (int k = 0; k < ne; k++) {
        const int e = sm.cand[k];
#pragma unroll
        for (int w = 0; w < kWords; w++) U[w] = sm.mask[p1][w] | sm.mask[e][w];
        unsigned int lo = max(sm.m[p1], sm.m[e]), hi = sm.m[p1] + sm.m[e] - g;
        unsigned int m3 = warp_minm(sm.st, U, lo, hi, g, linear, kc, km, mdiv, sm.sc, err);
        tests++;
        if (m3 != 0u) {
          pi -= (int)sm.m[p1] + (int)sm.m[e] - (int)m3;
          apply_merge(sm, p1, e, m3, n);
          break;
        }
        if (lane == 0) {
          sm.forb[p1][e >> 5] |= 1u << (e & 31);
          sm.forb[e][p1 >> 5] |= 1u << (p1 & 31);
        }
        __syncwarp();
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

__global__ void __launch_bounds__(128) alloc_merge(DevSets S, DevModel md, gpa_params p, AllocOut out, AllocQueue q,
                                                   const MagicDiv* __restrict__ mdiv) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  MergeSmem& sm = reinterpret_cast<MergeSmem*>(smem_raw)[warp];
  const unsigned long long nslow = *(volatile unsigned long long*)(q.counters + 1);
  for (;;) {
    unsigned long long i = 0;
    if (lane == 0) i = atomicAdd(q.counters + 2, 1ull);
    i = __shfl_sync(kFull, i, 0);
    if (i >= nslow) break;
    const long long s = q.slow_sets[i];
    const long long o = S.set_off[s];
    const long long nl = S.set_off[s + 1] - o;
    if (nl < 0 || nl > S.n_max || nl > kNmax) {
      write_invalid(s, o, nl < 0 ? 0 : nl, out, q.err);
      continue;
    }
    const int n = (int)nl;
    if (!stage_set(sm.st, o, n, S.T, S.D, S.A, S.B, S.u, S.type)) {
      write_invalid(s, o, n, out, q.err);
      continue;
    }
    merge_set(sm, s, o, n, md, p, out, mdiv, q.err);
    __syncwarp();
  }
}

// --------------------------------------------------------------- 1G kernel

struct OneGpuSmem {
  SetSmem st;
  RtaScratch sc;
};

__global__ void __launch_bounds__(256) one_gpu(DevSets S, DevModel md, AllocOut out, unsigned int* err,
                                               const MagicDiv* __restrict__ mdiv, unsigned long long* ticket) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  OneGpuSmem& sm = reinterpret_cast<OneGpuSmem*>(smem_raw)[warp];
  for (;;) {
    unsigned long long s = 0;
    if (lane == 0) s = atomicAdd(ticket, 1ull);
    s = __shfl_sync(kFull, s, 0);
    if ((long long)s >= S.nsets) break;
    const long long o = S.set_off[s];
    const long long n = S.set_off[s + 1] - o;
    if (n < 0 || n > S.n_max || n > kNmax) {
      write_invalid((long long)s, o, n < 0 ? 0 : n, out, err);
      continue;
    }
    if (!stage_set(sm.st, o, (int)n, S.T, S.D, S.A, S.B, S.u, S.type)) {
      write_invalid((long long)s, o, n, out, err);
      continue;
    }
    unsigned int all[kWords];
#pragma unroll
    for (int w = 0; w < kWords; w++) {
      int lo = w * 32;
      all[w] = n >= lo + 32 ? kFull : (n > lo ? ((1u << (n - lo)) - 1u) : 0u);
    }
    bool ok = n == 0 ? true : warp_rta(sm.st, all, (unsigned)md.M, md.kc, md.km, mdiv, sm.sc, nullptr, true, err);
    unsigned long long Uc = 0, Um = 0;
    int nm = 0;
    for (int r = lane; r < n; r += 32) {
      const bool mem = (sm.st.memmask[r >> 5] >> (r & 31)) & 1u;
      (mem ? Um : Uc) += sm.st.u[r];
      nm += mem;
    }
    Uc = warp_sum_u64(Uc);
    Um = warp_sum_u64(Um);
    nm = warp_sum_i32(nm);
    for (long long t = lane; t < n; t += 32) {
      out.part_of_task[o + t] = 0;
      out.size_of_part[o + t] = (t == 0) ? (short)md.M : (short)0;
    }
    if (lane == 0) {
      out.verdict[s] = ok ? 1 : 0;
      out.reason[s] = ok ? GPA_REASON_OK : GPA_REASON_TEST;
      out.n_parts[s] = n > 0 ? 1 : 0;
      out.Pi[s] = n > 0 ? md.M : 0;
      out.W[s] = (long long)workload_from_sums(Uc, Um, (int)n - nm, nm, md.kc, md.km);
      if (out.n_tests) out.n_tests[s] = 1;
    }
    __syncwarp();
  }
}

}  // namespace

size_t slow_smem_bytes(int warps_per_block) { return sizeof(MergeSmem) * (size_t)warps_per_block; }
size_t one_gpu_smem_bytes(int warps_per_block) { return sizeof(OneGpuSmem) * (size_t)warps_per_block; }

cudaError_t launch_allocate(const DevSets& s, const DevModel& md, const gpa_params& p, const AllocOut& out,
                            const AllocQueue& q, const MagicDivHost* mdiv, const LaunchShape& fast,
                            const LaunchShape& slow, cudaStream_t st, long long* launches, Prof* prof) {
  cudaError_t e = cudaMemsetAsync(q.counters, 0, 4 * sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  prof_mark(prof, st);
  const int threads = fast.warps_per_block * 32;
  // grid: the requested CTAs, or (0) as many as fit on every SM at once
  auto grid = [&](const void* fn) {
    if (fast.blocks > 0) return fast.blocks;
    int per_sm = 0, dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, 0);
    return (per_sm > 0 ? per_sm : 1) * (sms > 0 ? sms : 1);
  };
  if (fast.chunk >= 8) {
    alloc_fast<8, 2><<<grid((const void*)alloc_fast<8, 2>), threads, 0, st>>>(s, md, out, q);
  } else if (fast.chunk >= 4) {
    alloc_fast<4, 3><<<grid((const void*)alloc_fast<4, 3>), threads, 0, st>>>(s, md, out, q);
  } else if (fast.chunk == 3) {
    alloc_fast<2, 3><<<grid((const void*)alloc_fast<2, 3>), threads, 0, st>>>(s, md, out, q);
  } else if (fast.chunk >= 2) {
    alloc_fast<2, 2><<<grid((const void*)alloc_fast<2, 2>), threads, 0, st>>>(s, md, out, q);
  } else {
    alloc_fast<1, 1><<<grid((const void*)alloc_fast<1, 1>), threads, 0, st>>>(s, md, out, q);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  prof_mark(prof, st);
  const size_t smem = slow_smem_bytes(slow.warps_per_block);
  alloc_merge<<<slow.blocks, slow.warps_per_block * 32, smem, st>>>(s, md, p, out, q,
                                                                     reinterpret_cast<const MagicDiv*>(mdiv));
  e = cudaGetLastError();
  prof_mark(prof, st);
  *launches += 2;
  return e;
}

cudaError_t launch_one_gpu(const DevSets& s, const DevModel& md, const AllocOut& out, const AllocQueue& q,
                           const MagicDivHost* mdiv, const LaunchShape& shape, cudaStream_t st, long long* launches,
                           Prof* prof) {
  unsigned long long* ticket = q.counters + 3;
  unsigned int* err = q.err;
  cudaError_t e = cudaMemsetAsync(ticket, 0, sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  prof_mark(prof, st);
  one_gpu<<<shape.blocks, shape.warps_per_block * 32, one_gpu_smem_bytes(shape.warps_per_block), st>>>(
      s, md, out, err, reinterpret_cast<const MagicDiv*>(mdiv), ticket);
  e = cudaGetLastError();
  prof_mark(prof, st);
  *launches += 1;
  return e;
}

// Record the next timing event of a profiled call (no-op when prof is null).
void prof_mark(Prof* p, cudaStream_t st) {
  if (!p || p->used >= 4) return;
  cudaEventRecordWithFlags(p->ev[p->used], st, p->capture ? cudaEventRecordExternal : cudaEventRecordDefault);
  p->used++;
}

// Opt in to the dynamic shared memory the kernels need (once per process).
cudaError_t alloc_kernels_init() {
  cudaError_t e = cudaFuncSetAttribute(alloc_merge, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)slow_smem_bytes(4));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(one_gpu, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)one_gpu_smem_bytes(8));
}

}  // namespace gpa
