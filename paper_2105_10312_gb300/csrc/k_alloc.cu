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

#include "alloc_dev.cuh"
#include "bulk_pipe.cuh"
#include "gpa_device.cuh"
#include "gpa_internal.h"

GPA_NS_BEGIN

namespace {

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

// Per-task step of the fast kernel for one task already loaded: validity
// (the same conditions as task_valid, grouped so that the common checks are
// a few 32-bit operations), the Lemma 2 size and the split utilisation.
// For a valid task A + B <= 2^36 and 1000 D < 2^41, and A <= 1000 D - B, the
// one-SM case, is A + B <= 1000 D, which also covers A = 0.
__device__ __forceinline__ void fast_task(long long T, long long D, long long A, long long B, long long u,
                                          unsigned int y, const Sizes& z, unsigned int m_one,
                                          unsigned int* mm, unsigned int* f, unsigned int* ulo, unsigned int* uhi) {
  const unsigned long long uT = (unsigned long long)T, uD = (unsigned long long)D;
  const unsigned long long uA = (unsigned long long)A, uB = (unsigned long long)B, uu = (unsigned long long)u;
  const unsigned long long high = ((uT | uD) >> 31) | (uu >> 32) | ((uA | uB) >> 37);
  const unsigned long long sAB = uA + uB;
  const unsigned int D32 = (unsigned int)uD;
  const bool valid = high == 0ull && D32 - 1u < (unsigned int)uT && sAB - 1ull < (1ull << 36) && y <= 1u;
  const unsigned long long w = 1000ull * D32;
  unsigned int m = m_one;
  if (sAB > w) m = uB >= w ? 0u : lemma2_size_fast(uA, uB, uD, z, m_one);
  *mm = valid ? m : 0u;
  *f = valid ? (m == 0u ? 2u : 0u) : 1u;
  *ulo = valid ? ((unsigned int)uu & 0xffffu) : 0u;
  *uhi = valid ? ((unsigned int)uu >> 16) : 0u;
}

constexpr unsigned kBadShift = 20;  // pi sums carry Pi + (invalid or unsizable tasks << kBadShift)

// Adds one task's values to the partial sums of its set (ks of the chunk's
// K) and returns the chunk-relative index of that set's first task.
template <int K>
__device__ __forceinline__ int accumulate(int ks, unsigned int mm, unsigned int f, unsigned int ulo, unsigned int uhi,
                                          const int (&orel)[K + 1], unsigned int (&pi)[K], unsigned int (&lo)[K],
                                          unsigned int (&hi)[K]) {
  const unsigned int v = mm + ((f != 0u ? 1u : 0u) << kBadShift);
  int first = 0;
#pragma unroll
  for (int k = 0; k < K; k++) {
    const bool mine = ks == k;
    pi[k] += mine ? v : 0u;
    lo[k] += mine ? ulo : 0u;
    hi[k] += mine ? uhi : 0u;
    first = mine ? orel[k] : first;
  }
  return first;
}

// Warp-wide totals of a chunk's K sets, gathered so that lane k holds set
// k's; lanes k < ns then write their set's result when its singleton
// partitions fit (Lemma 3: Pi <= M), or queue it for the merge kernel.
template <int K>
__device__ __forceinline__ void finish_chunk(const unsigned int (&pi)[K], const unsigned int (&lo)[K],
                                             const unsigned int (&hi)[K], const int (&orel)[K + 1], long long base,
                                             int ns, unsigned int M, int lane, const AllocOut& out,
                                             const AllocQueue& q) {
  unsigned int pk = 0u, lk = 0u, hk = 0u;
  int nk = 0;
#pragma unroll
  for (int k = 0; k < K; k++) {
    const unsigned int tp = __reduce_add_sync(kFull, pi[k]);
    const unsigned int tl = __reduce_add_sync(kFull, lo[k]);
    const unsigned int th = __reduce_add_sync(kFull, hi[k]);
    if (lane == k) {
      pk = tp;
      lk = tl;
      hk = th;
      nk = orel[k + 1] - orel[k];
    }
  }
  if (lane < ns) {
    const long long s = base + lane;
    const unsigned int Pi = pk & ((1u << kBadShift) - 1u);
    if ((pk >> kBadShift) != 0u || Pi > M) {
      const unsigned long long idx = atomicAdd(q.counters + 1, 1ull);
      q.slow_sets[idx] = s;
    } else {
      out.verdict[s] = 1;
      out.reason[s] = GPA_REASON_OK;
      out.n_parts[s] = nk;
      out.Pi[s] = (int)Pi;
      out.W[s] = (long long)(1000ull * (((unsigned long long)hk << 16) + lk));
      if (out.n_tests) out.n_tests[s] = 0;
    }
  }
}

template <int K, int U>
__global__ void __launch_bounds__(256) alloc_fast(DevSets S, DevModel md, AllocOut out, AllocQueue q) {
  asm volatile("griddepcontrol.launch_dependents;");  // the merge grid may be scheduled as CTAs drain
  const int lane = threadIdx.x & 31;
  const long long warp0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  const unsigned M = (unsigned)md.M;
  const Sizes z = sizes_of(md);
  const unsigned m_one = z.next(1u);  // the smallest admissible size
  const long long ntasks = __ldg(S.set_off + S.nsets);
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
    bool bad = o[0] < 0 || o[K] > ntasks;
#pragma unroll
    for (int k = 0; k < K; k++) {
      const long long n = o[k + 1] - o[k];
      bad = bad || n < 0 || n > S.n_max || n > kNmax;
    }
    if (bad) {
      if (lane < ns) {
        const unsigned long long idx = atomicAdd(q.counters + 1, 1ull);
        q.slow_sets[idx] = base + lane;
      }
      continue;
    }
    const long long o0 = o[0];
    int orel[K + 1];
#pragma unroll
    for (int k = 0; k <= K; k++) orel[k] = (int)(o[k] - o0);
    const int nt = orel[K];
    const long long* Tc = S.T + o0;
    const long long* Dc = S.D + o0;
    const long long* Ac = S.A + o0;
    const long long* Bc = S.B + o0;
    const long long* uc = S.u + o0;
    const unsigned char* yc = S.type + o0;
    unsigned char* pot = out.part_of_task + o0;
    short* sop = out.size_of_part + o0;
    unsigned int pi[K], lo[K], hi[K];
#pragma unroll
    for (int k = 0; k < K; k++) pi[k] = lo[k] = hi[k] = 0u;
    for (int c0 = 0; c0 < nt; c0 += 32 * U) {
      long long Tt[U], Dt[U], At[U], Bt[U], ut[U];
      unsigned int yt[U];
#pragma unroll
      for (int uu = 0; uu < U; uu++) {
        const int i = c0 + uu * 32 + lane;
        if (i < nt) {
          Tt[uu] = __ldg(Tc + i);
          Dt[uu] = __ldg(Dc + i);
          At[uu] = __ldg(Ac + i);
          Bt[uu] = __ldg(Bc + i);
          ut[uu] = __ldg(uc + i);
          yt[uu] = __ldg(yc + i);
        }
      }
#pragma unroll
      for (int uu = 0; uu < U; uu++) {
        const int i = c0 + uu * 32 + lane;
        if (i < nt) {
          int ks = 0;
#pragma unroll
          for (int k = 1; k < K; k++) ks += i >= orel[k] ? 1 : 0;
          unsigned int mm, f, ulo, uhi;
          fast_task(Tt[uu], Dt[uu], At[uu], Bt[uu], ut[uu], yt[uu], z, m_one, &mm, &f, &ulo, &uhi);
          const int first = accumulate<K>(ks, mm, f, ulo, uhi, orel, pi, lo, hi);
          pot[i] = (unsigned char)(i - first);
          sop[i] = (short)mm;
        }
      }
    }
    finish_chunk<K>(pi, lo, hi, orel, base, ns, M, lane, out, q);
  }
}

// ------------------------------------------------- staged fast kernel
//
// The same per-task and per-set work with the task columns brought into
// shared memory by bulk copies (the TMA engine), so that the HBM reads of
// later tiles overlap the arithmetic on the current one.  A tile is
// `tile_sets` consecutive sets (tile_sets * n_max <= kStageCap); CTAs take
// tiles grid-stride.  One producer warp per CTA loads a tile's set offsets,
// checks them (sizes in [0, n_max], inside the task columns), writes them into
// a free stage and issues six bulk copies: the five 8-byte columns from the
// even task at or below the tile's first task, the type column from the
// multiple of 16 at or below it.  A copy never reads past the last task: the
// unaligned end of the columns (at most one task, 15 type bytes) is copied by
// the producer's lanes with plain loads.  A tile with a malformed offset is
// not copied; its sets go to the merge kernel, which validates each one.  The
// other warps each take chunks of K sets of the tile as alloc_fast does.  The
// stages cycle through `full` (data landed) and `empty` (every compute warp
// done with it) barriers.

constexpr int kStageCap = 1024;      // task slots per stage
constexpr int kTileSetsMax = 64;     // sets per tile
constexpr int kStagesMax = 5;
constexpr unsigned long long kWaitLimitNs = 1000000000ull;  // a pipeline wait gives up after 1 s

struct alignas(16) FastStage {
  long long col[5][kStageCap + 2];   // T, D, A, B, u_ppm from task e8 on
  unsigned char ty[kStageCap + 16];  // type from task e1 on
  long long off[kTileSetsMax + 2];   // the tile's set offsets
  long long e8, e1;
  int bad;
  int pad[3];
};
constexpr size_t kStageHeader = 128;  // the barriers: full[kStagesMax], empty[kStagesMax]
static_assert(2 * kStagesMax * sizeof(unsigned long long) <= kStageHeader, "barrier header too small");
static_assert(sizeof(FastStage) % 16 == 0, "stages must keep 16-byte alignment");

template <int K>
__global__ void __launch_bounds__(288, 2) alloc_fast_staged(DevSets S, DevModel md, AllocOut out, AllocQueue q,
                                                            int tile_sets, int nstages) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  unsigned long long* full = reinterpret_cast<unsigned long long*>(smem_raw);
  unsigned long long* empty = full + kStagesMax;
  FastStage* stages = reinterpret_cast<FastStage*>(smem_raw + kStageHeader);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ncw = (int)(blockDim.x >> 5) - 1;  // compute warps; the last warp is the producer
  const long long ntiles = (S.nsets + tile_sets - 1) / tile_sets;
  asm volatile("griddepcontrol.launch_dependents;");
  if (threadIdx.x == 0) {
    for (int st = 0; st < nstages; st++) {
      mbar_init(&full[st], 1u);
      mbar_init(&empty[st], (unsigned)ncw);
    }
    mbar_init_fence();
  }
  __syncthreads();

  if (warp == ncw) {
    // ---------------------------------------------------------- producer
    const long long ntasks = __ldg(S.set_off + S.nsets);
    int it = 0;
    bool ok = true;
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x, it++) {
      const int st = it % nstages;
      const long long s0 = tile * tile_sets;
      const int nst = (int)min((long long)tile_sets, S.nsets - s0);
      long long ov[3];
      bool sizes_ok = true;
#pragma unroll
      for (int r = 0; r < 3; r++) {
        const int j = r * 32 + lane;
        ov[r] = j <= nst ? __ldg(S.set_off + s0 + j) : 0ll;
        if (j < nst) {
          const long long n = __ldg(S.set_off + s0 + j + 1) - ov[r];
          sizes_ok = sizes_ok && n >= 0 && n <= S.n_max && n <= kNmax;
        }
      }
      sizes_ok = __all_sync(kFull, sizes_ok);
      const long long o_first = __shfl_sync(kFull, ov[0], 0);
      const int last_r = nst >> 5;
      const long long o_last = __shfl_sync(kFull, last_r == 0 ? ov[0] : (last_r == 1 ? ov[1] : ov[2]), nst & 31);
      if (it >= nstages && !mbar_wait(&empty[st], (unsigned)((it / nstages) - 1) & 1u, kWaitLimitNs)) {
        ok = false;
        break;
      }
      FastStage& sg = stages[st];
#pragma unroll
      for (int r = 0; r < 3; r++) {
        const int j = r * 32 + lane;
        if (j <= nst) sg.off[j] = ov[r];
      }
      const bool bad = !sizes_ok || o_first < 0 || o_last < o_first || o_last > ntasks ||
                       o_last - o_first > kStageCap;
      const long long e8 = o_first & ~1ll, e1 = o_first & ~15ll;
      unsigned b8 = 0u, b1 = 0u;
      if (!bad) {
        const long long want8 = ((o_last - e8 + 1) & ~1ll) * 8, have8 = ((ntasks - e8) & ~1ll) * 8;
        const long long want1 = (o_last - e1 + 15) & ~15ll, have1 = (ntasks - e1) & ~15ll;
        b8 = (unsigned)min(want8, have8);
        b1 = (unsigned)min(want1, have1);
        // the unaligned end of the columns, by plain loads
        const long long t8 = e8 + b8 / 8;
        if (lane == 0 && t8 < o_last) {
          const int r = (int)(t8 - e8);
          sg.col[0][r] = __ldg(S.T + t8);
          sg.col[1][r] = __ldg(S.D + t8);
          sg.col[2][r] = __ldg(S.A + t8);
          sg.col[3][r] = __ldg(S.B + t8);
          sg.col[4][r] = __ldg(S.u + t8);
        }
        const long long t1 = e1 + b1 + lane;
        if (t1 < o_last) sg.ty[b1 + lane] = __ldg(S.type + t1);
      }
      if (lane == 0) {
        sg.e8 = e8;
        sg.e1 = e1;
        sg.bad = bad ? 1 : 0;
      }
      __threadfence_block();
      __syncwarp();
      if (lane == 0) {
        // order this warp's plain shared-memory writes before the copies
        // that may later overwrite the same bytes
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive_expect_tx(&full[st], 5u * b8 + b1);
        if (b8) {
          bulk_copy_g2s(sg.col[0], S.T + e8, b8, &full[st]);
          bulk_copy_g2s(sg.col[1], S.D + e8, b8, &full[st]);
          bulk_copy_g2s(sg.col[2], S.A + e8, b8, &full[st]);
          bulk_copy_g2s(sg.col[3], S.B + e8, b8, &full[st]);
          bulk_copy_g2s(sg.col[4], S.u + e8, b8, &full[st]);
        }
        if (b1) bulk_copy_g2s(sg.ty, S.type + e1, b1, &full[st]);
      }
    }
    if (!ok) {
      if (lane == 0) atomicOr(q.err, kErrWait);
      // let the copies already issued land before the CTA can exit
      const int issued = it < nstages ? it : nstages;
      for (int k = 1; k <= issued; k++) {
        const int j = it - k;
        (void)mbar_wait(&full[j % nstages], (unsigned)(j / nstages) & 1u, kWaitLimitNs);
      }
    }
    return;
  }

  // ------------------------------------------------------------- compute
  const unsigned M = (unsigned)md.M;
  const Sizes z = sizes_of(md);
  const unsigned m_one = z.next(1u);  // the smallest admissible size
  int it = 0;
  for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x, it++) {
    const int st = it % nstages;
    if (!mbar_wait(&full[st], (unsigned)(it / nstages) & 1u, kWaitLimitNs)) {
      if (lane == 0) atomicOr(q.err, kErrWait);
      return;
    }
    const FastStage& sg = stages[st];
    const long long s0 = tile * tile_sets;
    const int nst = (int)min((long long)tile_sets, S.nsets - s0);
    const int nchunks = (nst + K - 1) / K;
    const bool tile_bad = sg.bad != 0;
    const long long e8 = sg.e8, e1 = sg.e1;
    for (int c = warp; c < nchunks; c += ncw) {
      const long long base = s0 + (long long)c * K;
      const int ns = min(K, nst - c * K);
      if (tile_bad) {
        if (lane < ns) {
          const unsigned long long idx = atomicAdd(q.counters + 1, 1ull);
          q.slow_sets[idx] = base + lane;
        }
        continue;
      }
      // the producer checked every size of the tile: the chunk is well formed
      int orel[K + 1];
      const long long o0 = sg.off[c * K];
#pragma unroll
      for (int k = 0; k <= K; k++) orel[k] = (int)(sg.off[c * K + (k <= ns ? k : ns)] - o0);
      const int nt = orel[K];
      const int r8 = (int)(o0 - e8), r1 = (int)(o0 - e1);
      unsigned char* pot = out.part_of_task + o0;
      short* sop = out.size_of_part + o0;
      unsigned int pi[K], lo[K], hi[K];
#pragma unroll
      for (int k = 0; k < K; k++) pi[k] = lo[k] = hi[k] = 0u;
      for (int i = lane; i < nt; i += 32) {
        int ks = 0;
#pragma unroll
        for (int k = 1; k < K; k++) ks += i >= orel[k] ? 1 : 0;
        unsigned int mm, f, ulo, uhi;
        fast_task(sg.col[0][r8 + i], sg.col[1][r8 + i], sg.col[2][r8 + i], sg.col[3][r8 + i], sg.col[4][r8 + i],
                  sg.ty[r1 + i], z, m_one, &mm, &f, &ulo, &uhi);
        const int first = accumulate<K>(ks, mm, f, ulo, uhi, orel, pi, lo, hi);
        pot[i] = (unsigned char)(i - first);
        sop[i] = (short)mm;
      }
      finish_chunk<K>(pi, lo, hi, orel, base, ns, M, lane, out, q);
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[st]);
  }
}

// Bytes of one merge group (the set state plus the test scratch of each of
// its warps after the first).
__host__ __device__ constexpr size_t merge_group_bytes(int gw) {
  return (sizeof(MergeSmem) + (size_t)(gw - 1) * sizeof(WarpScratch) + 127) / 128 * 128;
}

// The merge kernel: CTAs of warps_per_block warps in groups of gw warps;
// each group pops deferred sets from the queue and runs Alg. 1 on them
// (top_first: the SMS top-size round of merge_set).
__global__ void __launch_bounds__(256, GPA_MERGE_MINB) alloc_merge(DevSets S, DevModel md, gpa_params p, AllocOut out, AllocQueue q,
                                                   const MagicDiv* __restrict__ mdiv, int gw, int top_first) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int gi = warp / gw;
  Grp g;
  g.nthreads = gw * 32;
  g.nwarps = gw;
  g.warp = warp - gi * gw;
  g.tid = (int)threadIdx.x - gi * gw * 32;
  g.lane = lane;
  g.bar = 1 + gi;
  unsigned char* base = smem_raw + (size_t)gi * merge_group_bytes(gw);
  MergeSmem& sm = *reinterpret_cast<MergeSmem*>(base);
  WarpScratch* extra = reinterpret_cast<WarpScratch*>(base + sizeof(MergeSmem));
  RtaScratch& sc = grp_sc(sm, extra, g);
  LaneScratch& ls = grp_ls(sm, extra, g);
  ls.terms[lane] = 0ull;
  if (lane == 0) sc.terms = 0ull;
  asm volatile("griddepcontrol.wait;" ::: "memory");  // the fast grid has finished and its writes are visible
  const unsigned long long nslow = *(volatile unsigned long long*)(q.counters + 1);
  if (nslow == 0ull) return;  // the fast kernel decided every set
  const long long ntasks = S.set_off[S.nsets];
  for (;;) {
    if (g.tid == 0) sm.ticket = (long long)atomicAdd(q.counters + 2, 1ull);
    g.sync();
    const unsigned long long i = (unsigned long long)sm.ticket;
    g.sync();
    if (i >= nslow) break;
    const long long s = q.slow_sets[i];
    const long long o = S.set_off[s];
    const long long nl = S.set_off[s + 1] - o;
    if (nl < 0 || nl > S.n_max || nl > kNmax || !slice_inside(o, nl, ntasks)) {
      if (g.warp == 0) write_invalid(s, o, slice_inside(o, nl, ntasks) ? nl : 0, out, q.err);
      continue;
    }
    const int n = (int)nl;
    if (g.warp == 0) {
      const bool ok = stage_set(sm.st, o, n, S.T, S.D, S.A, S.B, S.u, S.type);
      if (lane == 0) {
        sm.ctl[5] = ok ? 1 : 0;
        sm.err = 0u;
      }
    }
    g.sync();
    if (!sm.ctl[5]) {
      if (g.warp == 0) write_invalid(s, o, n, out, q.err);
      g.sync();
      continue;
    }
    merge_set(g, sm, extra, s, o, n, md, p, out, mdiv, &sm.err, top_first != 0);
    if (g.warp == 0) finish_set_errors(s, sm.err, out, q.err);
    g.sync();
  }
  flush_terms(sc, ls, q.counters + 4);
}

// --------------------------------------------------------------- 1G kernel

struct OneGpuSmem {
  SetSmem st;
  RtaScratch sc;
  unsigned int err;  // error bits of the set being tested
};

// Per-warp scratch of the 1G pre-pass: the set's columns in original order
// and, per task, D, C, C / T and a raised 1 / T (the last three as float
// bits).
struct PreSmem {
  unsigned long long A[kNmax], B[kNmax];
  unsigned int T[kNmax], D[kNmax];
  uint4 rec[kNmax];
};
// the dynamic shared memory opted in by alloc_kernels_init (227 KB per CTA at most)
static_assert(merge_group_bytes(1) <= 232448, "merge kernel: one group must fit 227 KB");
static_assert(8 * sizeof(OneGpuSmem) <= 232448, "1G kernel: eight warps must fit 227 KB");
static_assert(8 * sizeof(PreSmem) <= 232448, "1G pre-pass kernel: eight warps must fit 227 KB");

// Outcomes of the 1G pre-pass.
enum { kPreOpen = 0, kPrePass = 1, kPreMiss = 2, kPreInvalid = 3 };

// 1G pre-pass over set [o, o + n) (warp-cooperative, original task order):
// decides most sets without the deadline-monotonic staging of stage_set.
// It validates the tasks (kPreInvalid), computes every WCET at m = M with
// the conflict factors of the whole set, and returns kPreMiss when a task has
// C > D or U > 1 (either rules out every policy on one processor), kPrePass
// when the hyperbolic bound holds or every task passes one evaluation of the
// iteration at its deadline or its response-time upper bound (see
// util_pass), else kPreOpen.  The bound takes as higher-priority tasks every
// other task whose deadline is at most its own: a superset of its
// deadline-monotonic predecessors, which only raises the bound.  A set that
// passes under DM passes under EDF too (EDF meets every deadline that any
// policy meets on one processor).  Uc, Um: the per-type sums of u; nm: the
// memory-intensive tasks (every lane).
//
// The sums are float: for task t, a = sum of C_j and b = sum of C_j / T_j
// over the tasks with D_j <= D_t, t included; b then drops t's own term.
// Each of at most 256 non-negative terms is within 2^-22 of its value
// (relative: the conversion of C_j rounds once, the quotients C_j / T_j come
// from __fdividef, at most 2 ulp) and each partial sum is rounded once
// (2^-24), so a (the bound's numerator C_t + sum C_hp) is within 2^-16 of its
// true value (relative), and b within 2^-15 of U_hp (b and t's term add up
// to at most U <= 1 + 2^-13).
// The bound is tested as a <= D_t (1 - U_hp), with U_hp + 2^-14 for U_hp
// and a raised by 2^-13, which also covers the test's roundings and that of
// D_t, so a pass is never wrong.
__device__ __forceinline__ int one_gpu_prepass(PreSmem& st, long long o, int n, const DevSets& S,
                                               const DevModel& md, const MagicDiv& mdM, unsigned long long& Uc,
                                               unsigned long long& Um, int& nm) {
  uint4* __restrict__ rec = st.rec;
  const int lane = threadIdx.x & 31;
  const int nch = (n + 31) >> 5;  // chunks of 32 tasks
  bool ok = true;
  unsigned int mm[kWords];
  unsigned long long uc = 0ull, um = 0ull;
#pragma unroll
  for (int c = 0; c < kWords; c++) {
    mm[c] = 0u;
    if (c >= nch) continue;
    const int t = c * 32 + lane;
    bool mem = false;
    if (t < n) {
      const long long T = __ldg(S.T + o + t), D = __ldg(S.D + o + t), A = __ldg(S.A + o + t),
                      B = __ldg(S.B + o + t);
      const long long u = S.u ? __ldg(S.u + o + t) : 0;
      const unsigned int y = __ldg(S.type + o + t);
      ok = ok && task_valid(T, D, A, B, u, y);
      st.T[t] = (unsigned int)T;
      st.D[t] = (unsigned int)D;
      st.A[t] = (unsigned long long)A;
      st.B[t] = (unsigned long long)B;
      mem = y == 1u;
      (mem ? um : uc) += (unsigned long long)(unsigned int)u;
    }
    mm[c] = __ballot_sync(kFull, mem);
  }
  if (!__all_sync(kFull, ok)) return kPreInvalid;
  // a lane's sum of at most kNmax / 32 values below 2^32: its halves below
  // and above 2^16 add up in 32-bit warp reductions
  Uc = ((unsigned long long)__reduce_add_sync(kFull, (unsigned int)(uc >> 16)) << 16) +
       __reduce_add_sync(kFull, (unsigned int)(uc & 0xFFFFull));
  Um = ((unsigned long long)__reduce_add_sync(kFull, (unsigned int)(um >> 16)) << 16) +
       __reduce_add_sync(kFull, (unsigned int)(um & 0xFFFFull));
  nm = 0;
#pragma unroll
  for (int c = 0; c < kWords; c++) nm += __popc(mm[c]);
  const unsigned int kmem = nm >= 2 ? (unsigned int)md.km : 1000u;
  const unsigned int kcmp = (n - nm) >= 2 ? (unsigned int)md.kc : 1000u;
  bool c_le_d = true;
  float uf = 0.0f, hyp = 1.0f;
#pragma unroll
  for (int c = 0; c < kWords; c++) {
    const int t = c * 32 + lane;
    if (c < nch && t < n) {
      const unsigned int T = st.T[t], D = st.D[t];
      const unsigned int C = wcet(st.A[t], st.B[t], ((mm[c] >> lane) & 1u) ? kmem : kcmp, (unsigned int)md.M, mdM);
      const float f = __fdividef((float)C, (float)T);
      c_le_d = c_le_d && C <= D;
      uf += f;
      hyp *= 1.0f + __fdividef((float)C, (float)D);
      // .w: 1 / T raised by 2^-19 (above 1 / T despite the quotient's 2 ulp)
      rec[t] = make_uint4(D, __float_as_uint((float)C), __float_as_uint(f),
                          __float_as_uint(__fdividef(1.0f, (float)T) * (1.0f + 0x1p-19f)));
    }
  }
  if (!__all_sync(kFull, c_le_d)) return kPreMiss;
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) {
    uf += __shfl_xor_sync(kFull, uf, d);
    hyp *= __shfl_xor_sync(kFull, hyp, d);
  }
  if (uf > kUtilFail) return kPreMiss;
  // The hyperbolic bound (Bini, Buttazzo & Buttazzo, 2003): implicit-deadline
  // tasks with prod (1 + C_i / T_i) <= 2 meet every deadline under
  // rate-monotonic priorities.  Here the periods are taken as D_i: each term
  // ceil(t / T_j) C_j of the response-time iteration is at most
  // ceil(t / D_j) C_j, so every response time is at most that of the set
  // with periods D_i, where deadline-monotonic order is rate-monotonic order.
  // Each of the at most 256 factors 1 + C_i / D_i is within 2^-22 of its
  // value (the quotient from __fdividef, at most 2 ulp, and one rounding)
  // and each product is rounded once (2^-24), so the float product is
  // within 2^-14 of the true one (relative): at most 2 (1 - 2^-13) proves
  // the true one <= 2.
  if (hyp <= 2.0f * (1.0f - 0x1p-13f)) return kPrePass;
  __syncwarp();
  // chunk by chunk; the first chunk with a task that neither test passes
  // leaves the set open, and the later chunks are not examined
  for (int c = 0; c < nch; c++) {
    const int t = c * 32 + lane;
    const uint4 own = t < n ? rec[t] : make_uint4(0u, 0u, 0u, 0u);
    // One evaluation at the deadline.  The response time is the least t with
    // f(t) <= t, f(t) = C_t + sum_{hp} ceil(t / T_j) C_j, so f(D_t) <= D_t
    // proves D_t met.  The sum runs over every task with D_j <= D_t (a
    // superset of t's deadline-monotonic predecessors; t itself, with a
    // ceiling of at least 1, stands for C_t), and each ceiling comes from
    // D_t times 1 / T_j raised by 2^-19, which is above D_t / T_j: every term
    // is at least the exact one.  The float sum of at most 256 terms is
    // within 2^-16 of its value (relative), and the test's 2^-13 margin
    // covers that and the rounding of D_t.
    const float Dt = (float)own.x;
    float cs = 0.0f;
#pragma unroll 4
    for (int j = 0; j < n; j++) {
      const uint4 r = rec[j];
      if (r.x <= own.x) cs = fmaf(ceilf(Dt * __uint_as_float(r.w)), __uint_as_float(r.y), cs);
    }
    bool ok = t >= n || cs * (1.0f + 0x1p-13f) <= Dt;
    // Tasks it leaves open: the response-time upper bound over the same
    // tasks (see util_pass and the error analysis above).
    if (__any_sync(kFull, !ok)) {
      float a = 0.0f, b = 0.0f;
#pragma unroll 4
      for (int j = 0; j < n; j++) {
        const uint4 r = rec[j];
        if (r.x <= own.x) {
          a += __uint_as_float(r.y);
          b += __uint_as_float(r.z);
        }
      }
      if (!ok) {
        // a already holds C_t + sum C_j, the bound's numerator
        const float u = (b - __uint_as_float(own.z)) + 0x1p-14f;
        ok = u < 1.0f && a * (1.0f + 0x1p-13f) <= Dt * (1.0f - u);
      }
    }
    if (!__all_sync(kFull, ok)) return kPreOpen;
  }
  return kPrePass;
}

// 1G, first kernel: one warp per set, grid-stride.  The pre-pass decides a
// set (outputs written here), or the set goes to the deferred queue: the
// ones it leaves open, and the malformed ones, which the second kernel
// validates.  The second kernel may be scheduled as this grid drains.
__global__ void __launch_bounds__(256) one_gpu_fast(DevSets S, DevModel md, AllocOut out, AllocQueue q,
                                                    const MagicDiv* __restrict__ mdiv) {
  asm volatile("griddepcontrol.launch_dependents;");
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  PreSmem& ps = reinterpret_cast<PreSmem*>(smem_raw)[warp];
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  const long long ntasks = __ldg(S.set_off + S.nsets);
  const MagicDiv mdM = mdiv[md.M];
  long long s = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  // lanes 0 and 1 hold the offsets of the warp's next set
  long long offv = (s < S.nsets && lane < 2) ? __ldg(S.set_off + s + lane) : 0;
  for (; s < S.nsets; s += nw) {
    const long long o = __shfl_sync(kFull, offv, 0), n = __shfl_sync(kFull, offv, 1) - o;
    if (s + nw < S.nsets && lane < 2) offv = __ldg(S.set_off + s + nw + lane);
    int pre = kPreInvalid, nm = 0;
    unsigned long long Uc = 0, Um = 0;
    if (n >= 0 && n <= S.n_max && n <= kNmax && slice_inside(o, n, ntasks))
      pre = one_gpu_prepass(ps, o, (int)n, S, md, mdM, Uc, Um, nm);
    if (pre == kPreOpen || pre == kPreInvalid) {
      if (lane == 0) q.slow_sets[atomicAdd(q.counters + 1, 1ull)] = s;
      __syncwarp();
      continue;
    }
    const bool ok = pre == kPrePass;
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

// 1G, second kernel: the deferred sets, one warp per set from a ticket
// queue: validation, deadline-monotonic staging and the per-partition test
// of all tasks at m = M.
__global__ void __launch_bounds__(256, GPA_ONEGPU_MINB) one_gpu(DevSets S, DevModel md, AllocOut out, AllocQueue q,
                                                                const MagicDiv* __restrict__ mdiv) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  OneGpuSmem& sm = reinterpret_cast<OneGpuSmem*>(smem_raw)[warp];
  if (lane == 0) sm.sc.terms = 0ull;
  asm volatile("griddepcontrol.wait;" ::: "memory");  // the first grid has finished and its writes are visible
  const unsigned long long nslow = *(volatile unsigned long long*)(q.counters + 1);
  const long long ntasks = S.set_off[S.nsets];
  // lane 0 fetches the next ticket when a set starts and its queue entry once
  // the set is staged, so neither round trip delays the next set
  unsigned long long tnext = 0ull;
  long long snext = 0;
  if (lane == 0) {
    tnext = atomicAdd(q.counters + 2, 1ull);
    if (tnext < nslow) snext = q.slow_sets[tnext];
  }
  for (;;) {
    const unsigned long long i = __shfl_sync(kFull, tnext, 0);
    if (i >= nslow) break;
    const long long s = __shfl_sync(kFull, snext, 0);
    if (lane == 0) tnext = atomicAdd(q.counters + 2, 1ull);
    const long long o = S.set_off[s];
    const long long n = S.set_off[s + 1] - o;
    const bool inside = n >= 0 && n <= S.n_max && n <= kNmax && slice_inside(o, n, ntasks);
    const bool staged = inside && stage_set(sm.st, o, (int)n, S.T, S.D, S.A, S.B, S.u, S.type);
    if (lane == 0 && tnext < nslow) snext = q.slow_sets[tnext];
    if (!staged) {
      write_invalid(s, o, slice_inside(o, n, ntasks) ? n : 0, out, q.err);
      continue;
    }
    unsigned int all[kWords];
#pragma unroll
    for (int w = 0; w < kWords; w++) {
      int lo = w * 32;
      all[w] = n >= lo + 32 ? kFull : (n > lo ? ((1u << (n - lo)) - 1u) : 0u);
    }
    if (lane == 0) sm.err = 0u;
    __syncwarp();
    const bool ok = n == 0 ? true
                           : warp_test(sm.st, all, (unsigned)md.M, md.kc, md.km, md.sched, mdiv, sm.sc, nullptr,
                                       true, &sm.err);
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
    finish_set_errors(s, sm.err, out, q.err);
  }
  __syncwarp();
  if (lane == 0 && sm.sc.terms) atomicAdd(q.counters + 4, sm.sc.terms);
}

}  // namespace

size_t staged_smem_bytes(int stages) { return kStageHeader + sizeof(FastStage) * (size_t)stages; }
size_t slow_smem_bytes(int warps_per_block, int gw) {
  return merge_group_bytes(gw) * (size_t)(warps_per_block / (gw > 0 ? gw : 1));
}
size_t one_gpu_smem_bytes(int warps_per_block) { return sizeof(OneGpuSmem) * (size_t)warps_per_block; }

int merge_ctas_per_sm(int wpb, int gw) {
  if (gw < 1 || gw > kGrpWarpsMax || wpb < gw || wpb > 8 || wpb % gw) return 0;
  const size_t smem = slow_smem_bytes(wpb, gw);
  if (smem > 232448) return 0;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, alloc_merge, wpb * 32, smem) != cudaSuccess) return 0;
  return per_sm;
}

int one_gpu_ctas_per_sm(int wpb) {
  if (wpb < 1 || wpb > 8) return 0;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, one_gpu, wpb * 32, one_gpu_smem_bytes(wpb)) != cudaSuccess)
    return 0;
  return per_sm;
}

cudaError_t launch_allocate(const DevSets& s, const DevModel& md, const gpa_params& p, const AllocOut& out,
                            const AllocQueue& q, const MagicDivHost* mdiv, const LaunchShape& fast,
                            const LaunchShape& slow, cudaStream_t st, long long* launches, Prof* prof) {
  // tickets, deferred count and the interference-term counter start at zero
  cudaError_t e = cudaMemsetAsync(q.counters, 0, 5 * sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  prof_mark(prof, st);
  const int threads = min(fast.warps_per_block, 8) * 32;  // the direct kernel takes up to 8 warps
  // grid: the requested CTAs, or (0) as many as fit on every SM at once
  auto grid = [&](const void* fn) {
    if (fast.blocks > 0) return fast.blocks;
    int per_sm = 0, dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, 0);
    return (per_sm > 0 ? per_sm : 1) * (sms > 0 ? sms : 1);
  };
  // the staged kernel copies 16-byte aligned ranges: every column must start
  // on a 16-byte boundary
  const unsigned long long align = (unsigned long long)(size_t)s.T | (unsigned long long)(size_t)s.D |
                                   (unsigned long long)(size_t)s.A | (unsigned long long)(size_t)s.B |
                                   (unsigned long long)(size_t)s.u | (unsigned long long)(size_t)s.type;
  const int chunk = fast.chunk;
  if (fast.stages >= 2 && fast.stages <= kStagesMax && (align & 15ull) == 0 && s.nsets > 0) {
    const int nmax = s.n_max > 0 ? s.n_max : 1;
    const int tile_sets = min(kTileSetsMax, kStageCap / nmax);
    const long long ntiles = (s.nsets + tile_sets - 1) / tile_sets;
    const int cw = min(fast.warps_per_block, 8);  // compute warps (the kernel takes at most 9 warps)
    const int sthreads = (cw + 1) * 32;
    const size_t smem = staged_smem_bytes(fast.stages);
    auto sgrid = [&](const void* fn) -> int {
      long long b = fast.blocks;
      if (b <= 0) {
        int per_sm = 0, dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, sthreads, smem);
        b = (long long)(per_sm > 0 ? per_sm : 1) * (sms > 0 ? sms : 1);
      }
      return (int)min(b, ntiles);
    };
    if (chunk >= 4) {
      alloc_fast_staged<4><<<sgrid((const void*)alloc_fast_staged<4>), sthreads, smem, st>>>(s, md, out, q, tile_sets,
                                                                                           fast.stages);
    } else if (chunk >= 2) {
      alloc_fast_staged<2><<<sgrid((const void*)alloc_fast_staged<2>), sthreads, smem, st>>>(s, md, out, q, tile_sets,
                                                                                           fast.stages);
    } else {
      alloc_fast_staged<1><<<sgrid((const void*)alloc_fast_staged<1>), sthreads, smem, st>>>(s, md, out, q, tile_sets,
                                                                                           fast.stages);
    }
  } else if (chunk >= 8) {
    alloc_fast<8, 2><<<grid((const void*)alloc_fast<8, 2>), threads, 0, st>>>(s, md, out, q);
  } else if (chunk >= 4) {
    alloc_fast<4, 3><<<grid((const void*)alloc_fast<4, 3>), threads, 0, st>>>(s, md, out, q);
  } else if (chunk == 3) {
    alloc_fast<2, 3><<<grid((const void*)alloc_fast<2, 3>), threads, 0, st>>>(s, md, out, q);
  } else if (chunk >= 2) {
    alloc_fast<2, 2><<<grid((const void*)alloc_fast<2, 2>), threads, 0, st>>>(s, md, out, q);
  } else {
    alloc_fast<1, 1><<<grid((const void*)alloc_fast<1, 1>), threads, 0, st>>>(s, md, out, q);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  prof_mark(prof, st);
  // programmatic dependent launch: the merge grid may be scheduled while the
  // fast grid drains; it waits (griddepcontrol.wait) for the fast grid's
  // completion and memory before it reads the queue
  // merge grid: slow.warps_per_block warps per CTA in groups of slow.chunk
  // warps, one set per group at a time
  const int gw = slow.chunk >= 1 && slow.chunk <= kGrpWarpsMax ? slow.chunk : 1;
  const int wpb = max(gw, min(slow.warps_per_block, 8) / gw * gw);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)slow.blocks);
  cfg.blockDim = dim3((unsigned)(wpb * 32));
  cfg.dynamicSmemBytes = slow_smem_bytes(wpb, gw);
  if (cfg.dynamicSmemBytes > 232448) return cudaErrorInvalidConfiguration;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  // slow.stages == 2: the SMS top-size round (see merge_set)
  e = cudaLaunchKernelEx(&cfg, alloc_merge, s, md, p, out, q, reinterpret_cast<const MagicDiv*>(mdiv), gw,
                         slow.stages == 2 ? 1 : 0);
  if (e != cudaSuccess) return e;
  e = cudaGetLastError();
  prof_mark(prof, st);
  *launches += 2;
  return e;
}

cudaError_t launch_one_gpu(const DevSets& s, const DevModel& md, const AllocOut& out, const AllocQueue& q,
                           const MagicDivHost* mdiv, const LaunchShape& shape, cudaStream_t st, long long* launches,
                           Prof* prof) {
  // tickets, deferred count and the interference-term counter start at zero
  cudaError_t e = cudaMemsetAsync(q.counters, 0, 5 * sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  prof_mark(prof, st);
  // first kernel: as many eight-warp CTAs as fit on every SM at once
  const size_t fsmem = sizeof(PreSmem) * 8;
  int per_sm = 0, dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, one_gpu_fast, 256, fsmem);
  const long long want = (long long)(per_sm > 0 ? per_sm : 1) * (sms > 0 ? sms : 1) * 8;  // warps
  const long long fblocks = (std::min(want, s.nsets > 0 ? s.nsets : 1) + 7) / 8;
  one_gpu_fast<<<(unsigned)fblocks, 256, fsmem, st>>>(s, md, out, q, reinterpret_cast<const MagicDiv*>(mdiv));
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  prof_mark(prof, st);
  // second kernel: programmatic dependent launch (it waits for the first
  // grid's completion and memory before it reads the queue)
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)shape.blocks);
  cfg.blockDim = dim3((unsigned)(shape.warps_per_block * 32));
  cfg.dynamicSmemBytes = one_gpu_smem_bytes(shape.warps_per_block);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  e = cudaLaunchKernelEx(&cfg, one_gpu, s, md, out, q, reinterpret_cast<const MagicDiv*>(mdiv));
  if (e != cudaSuccess) return e;
  e = cudaGetLastError();
  prof_mark(prof, st);
  *launches += 2;
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
  cudaError_t e = cudaFuncSetAttribute(alloc_merge, cudaFuncAttributeMaxDynamicSharedMemorySize, 232448);
  if (e != cudaSuccess) return e;
  const int staged = (int)staged_smem_bytes(kStagesMax);
  if ((e = cudaFuncSetAttribute(alloc_fast_staged<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, staged)) !=
          cudaSuccess ||
      (e = cudaFuncSetAttribute(alloc_fast_staged<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, staged)) !=
          cudaSuccess ||
      (e = cudaFuncSetAttribute(alloc_fast_staged<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, staged)) !=
          cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(one_gpu_fast, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(sizeof(PreSmem) * 8))) != cudaSuccess)
    return e;
  return cudaFuncSetAttribute(one_gpu, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)one_gpu_smem_bytes(8));
}

GPA_NS_END
