// k_test.cu — WCET tables (§3.3 two-curve model in the §7.1 integer form)
// and the per-partition test over a flat batch of explicit candidates
// (a split of the SMs into parts plus a task-to-part map, §4.1-§4.2, §5.5).
#include <cuda_runtime.h>

#include "gpa_device.cuh"
#include "gpa_internal.h"

GPA_NS_BEGIN

namespace {

// One warp per task set; for every size m = g (mi + 1) the lanes write the
// set's row of n tasks (layout [set][mi][task]: coalesced int64 stores).
__global__ void __launch_bounds__(256) wcet_tables(DevSets S, DevModel md, long long* __restrict__ Cn,
                                                   long long* __restrict__ Cc, unsigned int* err,
                                                   const MagicDiv* __restrict__ mdiv) {
  const int lane = threadIdx.x & 31;
  const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
  const int Mu = md.M / md.g;
  for (long long s = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); s < S.nsets; s += warps) {
    const long long o = S.set_off[s];
    const long long n = S.set_off[s + 1] - o;
    if (n < 0 || n > kNmax || o < 0 || o > S.set_off[S.nsets] - n) {
      if (lane == 0) atomicOr(err, kErrRange);
      continue;
    }
    unsigned long long A[kWords], B[kWords];
    unsigned int kx[kWords];
    bool ok = true;
#pragma unroll
    for (int c = 0; c < kWords; c++) {
      const int t = c * 32 + lane;
      A[c] = B[c] = 0;
      kx[c] = 1000;
      if (t < n) {
        long long Tt = S.T[o + t], Dt = S.D[o + t], At = S.A[o + t], Bt = S.B[o + t];
        unsigned int yt = S.type[o + t];
        ok = ok && task_valid(Tt, Dt, At, Bt, S.u ? S.u[o + t] : 0, yt);
        A[c] = (unsigned long long)At;
        B[c] = (unsigned long long)Bt;
        kx[c] = yt == 1u ? (unsigned)md.km : (unsigned)md.kc;
      }
    }
    ok = __all_sync(kFull, ok);
    long long* cn = Cn + o * Mu;
    long long* cc = Cc + o * Mu;
    for (int mi = 0; mi < Mu; mi++) {
      const unsigned int m = (unsigned)md.g * (unsigned)(mi + 1);
      const MagicDiv d = mdiv[m];
#pragma unroll
      for (int c = 0; c < kWords; c++) {
        const int t = c * 32 + lane;
        if (t < n) {
          cn[(long long)mi * n + t] = ok ? (long long)wcet(A[c], B[c], 1000u, m, d) : -1LL;
          cc[(long long)mi * n + t] = ok ? (long long)wcet(A[c], B[c], kx[c], m, d) : -1LL;
        }
      }
    }
    if (!ok && lane == 0) atomicOr(err, kErrRange);
  }
}

struct TestSmem {
  SetSmem st;
  RtaScratch sc;
  long long R[kNmax];          // per row
  unsigned char part[kNmax];   // per row
  unsigned int err;            // error bits of the candidate being tested
};

// One warp per candidate: stage its set, then test every non-empty part at
// its size.  The candidate is schedulable iff the part sizes fit in M and
// every part passes.
__global__ void __launch_bounds__(256) test_candidates(DevSets S, DevModel md, Cands C, unsigned char* verdict,
                                                       long long* Rout, unsigned int* err,
                                                       const MagicDiv* __restrict__ mdiv) {
  const Sizes zs{(unsigned int)md.M, (unsigned int)md.g, md.zlist, md.zrank, md.nz};  // admissible part sizes
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  TestSmem& sm = reinterpret_cast<TestSmem*>(smem_raw)[warp];
  const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
  for (long long c = (long long)blockIdx.x * (blockDim.x >> 5) + warp; c < C.ncands; c += warps) {
    const long long s = C.set[c];
    bool bad = s < 0 || s >= S.nsets;
    long long o = 0;
    int n = 0;
    if (!bad) {
      o = S.set_off[s];
      long long nn = S.set_off[s + 1] - o;
      bad = nn < 0 || nn > kNmax || nn > C.map_stride || o < 0 || o > S.set_off[S.nsets] - nn;
      n = bad ? 0 : (int)nn;
    }
    const unsigned char* map = C.part_of_task + c * C.map_stride;
    const int* size = C.size_of_part + c * (long long)C.kparts;
    // part sizes: each 0 or a multiple of g in [g, M]; their sum against M
    long long total = 0;
    bool bad_size = false;
    for (int p = lane; p < C.kparts; p += 32) {
      int z = size[p];
      bad_size = bad_size || (z != 0 && !zs.admissible((unsigned int)z)) || z < 0;
      total += z;
    }
    bad = __any_sync(kFull, bad || bad_size);
    if (!bad) {
      // the staging validates the set's tasks
      bad = !stage_set(sm.st, o, n, S.T, S.D, S.A, S.B, S.u, S.type);
    }
    if (!bad) {
      bool bad_map = false;
      for (int r = lane; r < n; r += 32) {
        unsigned char pr = map[sm.st.orig[r]];
        bad_map = bad_map || pr >= C.kparts;
        sm.part[r] = pr;
        sm.R[r] = -1;
      }
      bad = __any_sync(kFull, bad_map);
    }
    if (bad) {
      if (lane == 0) {
        verdict[c] = 0;
        atomicOr(err, kErrRange);
      }
      if (Rout)
        for (int t = lane; t < C.map_stride; t += 32) Rout[c * C.map_stride + t] = -1;
      continue;
    }
    for (int off = 16; off > 0; off >>= 1) total += __shfl_xor_sync(kFull, total, off);
    bool ok = total <= md.M;
    if (lane == 0) sm.err = 0u;
    __syncwarp();
    // ok: no part fails for certain; undecided: a part's test hit its step
    // limit (the candidate is then undecided, 2, unless another part fails)
    bool undecided = false;
    for (int p = 0; p < C.kparts; p++) {
      unsigned int Sp[kWords];
      unsigned int any = 0u;
#pragma unroll
      for (int w = 0; w < kWords; w++) {
        const int r = w * 32 + lane;
        Sp[w] = __ballot_sync(kFull, r < n && sm.part[r] == p);
        any |= Sp[w];
      }
      if (!any) continue;
      const int z = size[p];
      if (z == 0) {
        ok = false;
        if (!Rout) break;
        continue;
      }
      const unsigned int e0 = sm.err;
      const bool pass = warp_test(sm.st, Sp, (unsigned)z, (unsigned)md.kc, (unsigned)md.km, md.sched, mdiv, sm.sc,
                                  Rout ? sm.R : nullptr, Rout == nullptr, &sm.err);
      if (!pass) {
        if (sm.err != e0) undecided = true;
        else ok = false;
      }
      if (!ok && !Rout) break;
    }
    __syncwarp();
    if (lane == 0) {
      verdict[c] = ok ? (undecided ? 2 : 1) : 0;
      if (sm.err) atomicOr(err, sm.err);
    }
    if (Rout) {
      for (int r = lane; r < n; r += 32) Rout[c * C.map_stride + sm.st.orig[r]] = sm.R[r];
      for (int t = n + lane; t < C.map_stride; t += 32) Rout[c * C.map_stride + t] = -1;
    }
    __syncwarp();
  }
}

// Bounds of a staged host batch (the same as task_valid and the set sizes
// in [0, n_max]): *flag becomes nonzero if any set or task violates them.
// Grid-stride and coalesced; the first offending set is looked up on the
// host only when the flag is set.
__global__ void __launch_bounds__(256) validate_batch(DevSets S, unsigned int* flag) {
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long ntasks = S.set_off[S.nsets];
  bool bad = false;
  for (long long s = tid; s < S.nsets; s += stride) {
    const long long n = S.set_off[s + 1] - S.set_off[s];
    bad = bad || n < 0 || n > S.n_max;
  }
  for (long long t = tid; t < ntasks; t += stride)
    bad = bad || !task_valid(__ldg(S.T + t), __ldg(S.D + t), __ldg(S.A + t), __ldg(S.B + t),
                             S.u ? __ldg(S.u + t) : 0ll, __ldg(S.type + t));
  if (__any_sync(kFull, bad) && (threadIdx.x & 31) == 0) atomicOr(flag, 1u);
}

}  // namespace

cudaError_t launch_validate_batch(const DevSets& s, unsigned int* flag, int sm_count, cudaStream_t st,
                                  long long* launches) {
  cudaError_t e = cudaMemsetAsync(flag, 0, sizeof(unsigned int), st);
  if (e != cudaSuccess) return e;
  validate_batch<<<sm_count * 4, 256, 0, st>>>(s, flag);
  *launches += 1;
  return cudaGetLastError();
}

cudaError_t launch_wcet_tables(const DevSets& s, const DevModel& md, long long* Cn, long long* Cc, unsigned int* err,
                               const MagicDivHost* mdiv, int sm_count, cudaStream_t st, long long* launches,
                               Prof* prof) {
  const int warps = 8;
  long long need = (s.nsets + warps - 1) / warps;
  int blocks = (int)(need < (long long)sm_count * 8 ? need : (long long)sm_count * 8);
  if (blocks < 1) blocks = 1;
  prof_mark(prof, st);
  wcet_tables<<<blocks, warps * 32, 0, st>>>(s, md, Cn, Cc, err, reinterpret_cast<const MagicDiv*>(mdiv));
  cudaError_t e = cudaGetLastError();
  prof_mark(prof, st);
  *launches += 1;
  return e;
}

static size_t test_smem_bytes(int warps) { return sizeof(TestSmem) * (size_t)warps; }

cudaError_t launch_test_schedulable(const DevSets& s, const DevModel& md, const Cands& c, unsigned char* verdict,
                                    long long* R, unsigned int* err, const MagicDivHost* mdiv, int sm_count,
                                    cudaStream_t st, long long* launches, Prof* prof) {
  const int warps = kNmax > 128 ? 2 : 4;  // warps x sizeof(TestSmem) stays below the 48 KB default
  long long need = (c.ncands + warps - 1) / warps;
  int blocks = (int)(need < (long long)sm_count * 4 ? need : (long long)sm_count * 4);
  if (blocks < 1) blocks = 1;
  prof_mark(prof, st);
  test_candidates<<<blocks, warps * 32, test_smem_bytes(warps), st>>>(s, md, c, verdict, R, err,
                                                                      reinterpret_cast<const MagicDiv*>(mdiv));
  cudaError_t e = cudaGetLastError();
  prof_mark(prof, st);
  *launches += 1;
  return e;
}

GPA_NS_END
