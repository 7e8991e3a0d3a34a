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
#include "gpa_device.cuh"
#include "gpa_internal.h"

namespace gpa {

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
