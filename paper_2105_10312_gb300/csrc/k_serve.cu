// k_serve.cu — the device side of the serving loop: one warp per request of
// a micro-batch, each request on a different tenant.  A tenant's tasks and
// its current allocation live in a device slot; the warp stages the tenant
// in shared memory in deadline-monotonic order, applies the operation and
// writes the new state back to the slot and to the request's response.
//
//  ADMIT   Alg. 1 on the new task set (the batch allocate path, merge_set).
//  ADD     first fit at the current sizes, then growth into the spare SMs
//          (Alg. 2), then a new Lemma 2 partition, then Alg. 1 on all tasks.
//  REMOVE  drop a task, shrink its partition to its minimum size, renumber
//          partitions by their lowest task index.
//  EVICT   nothing on the device (the host frees the slot).
#include <cuda_runtime.h>

#include "alloc_dev.cuh"
#include "gpa_device.cuh"
#include "gpa_internal.h"
#include "serve_types.h"

namespace gpa {

namespace {

struct ServeSmem {
  MergeSmem m;                  // staged tenant (m.st), test scratch, Alg. 1 state
  unsigned char prow[kNmax];    // partition of each row
  int cntc[kNmax], cntm[kNmax]; // tasks of each type per partition
};

__device__ __forceinline__ TenantSlot* slot_ptr(TenantSlot* const* chunks, int slot) {
  return chunks[slot / kSlotsPerChunkMax] + (slot % kSlotsPerChunkMax);
}

// Pi and W of the state (rows staged in st, prow = partition of each row).
__device__ void summarise_state(ServeSmem& sm, int n, const short* size, int np, const DevModel& md, int* Pi,
                                unsigned long long* W) {
  const int lane = threadIdx.x & 31;
  for (int p = lane; p < kNmax; p += 32) sm.cntc[p] = sm.cntm[p] = 0;
  __syncwarp();
  for (int r = lane; r < n; r += 32) {
    const bool mem = (sm.m.st.memmask[r >> 5] >> (r & 31)) & 1u;
    atomicAdd(mem ? &sm.cntm[sm.prow[r]] : &sm.cntc[sm.prow[r]], 1);
  }
  __syncwarp();
  unsigned long long w = 0;
  for (int r = lane; r < n; r += 32) {
    const bool mem = (sm.m.st.memmask[r >> 5] >> (r & 31)) & 1u;
    const int same = mem ? sm.cntm[sm.prow[r]] : sm.cntc[sm.prow[r]];
    const unsigned k = same >= 2 ? (unsigned)(mem ? md.km : md.kc) : 1000u;
    w += (unsigned long long)k * sm.m.st.u[r];
  }
  int pi = 0;
  for (int p = lane; p < np; p += 32) pi += size[p];
  *W = warp_sum_u64(w);
  *Pi = warp_sum_i32(pi);
}

// Partition p's rows as a task mask.
__device__ __forceinline__ void rows_of(const ServeSmem& sm, int n, int p, unsigned int* S) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int w = 0; w < kWords; w++) {
    const int r = w * 32 + lane;
    S[w] = __ballot_sync(kFull, r < n && sm.prow[r] == p);
  }
}

__device__ void copy_state_to_resp(const TenantSlot* t, ServeResp* rs) {
  const int lane = threadIdx.x & 31;
  for (int i = lane; i < kNmax; i += 32) {
    rs->part[i] = i < t->n ? t->part[i] : 255;
    rs->size[i] = i < t->n_parts ? t->size[i] : 0;
  }
  if (lane == 0) {
    rs->n_tasks = t->n;
    rs->n_parts = t->n_parts;
    rs->Pi = t->Pi;
    rs->W = t->W;
  }
}

// Alg. 1 on the staged n tasks; results into the response, and into the slot
// if accepted.  Returns the verdict on all lanes.
__device__ bool run_alg1(ServeSmem& sm, TenantSlot* t, ServeResp* rs, int n, const DevModel& md, const gpa_params& p,
                         const MagicDiv* mdiv, unsigned int* err) {
  const int lane = threadIdx.x & 31;
  AllocOut out{&rs->verdict, &rs->reason, &rs->n_parts, &rs->Pi, (long long*)&rs->W, &rs->n_tests, rs->part,
               rs->size};
  merge_set(warp_group(), sm.m, nullptr, 0, 0, n, md, p, out, mdiv, err, false);
  __syncwarp();
  const bool ok = rs->verdict != 0;
  if (ok) {
    for (int i = lane; i < kNmax; i += 32) {
      t->part[i] = i < n ? rs->part[i] : 255;
      t->size[i] = i < n ? rs->size[i] : 0;
      if (i >= n) rs->part[i] = 255;
      if (i >= rs->n_parts) rs->size[i] = 0;
    }
    if (lane == 0) {
      t->n = n;
      t->n_parts = rs->n_parts;
      t->Pi = rs->Pi;
      t->W = rs->W;
      rs->n_tasks = n;
    }
  }
  __syncwarp();
  return ok;
}

// One request by one warp.  err receives the request's error bits.
__device__ void serve_one(ServeSmem& sm, const ServeReq rq, ServeResp* rs, TenantSlot* const* __restrict__ chunks,
                          const ServePayload& pay, const DevModel& md, const gpa_params& prm,
                          const MagicDiv* __restrict__ mdiv, unsigned int* err) {
  const int lane = threadIdx.x & 31;
  if (lane == 0) {
    rs->verdict = 0;
    rs->reason = GPA_REASON_OK;
    rs->path = GPA_PATH_NONE;
    rs->status = 0;
    rs->n_tests = 0;
  }
  __syncwarp();
  if (rq.op == GPA_SERVE_EVICT) {
    if (lane == 0) {
      rs->verdict = 1;
      rs->n_tasks = rs->n_parts = rs->Pi = 0;
      rs->W = 0;
    }
    for (int i = lane; i < kNmax; i += 32) {
      rs->part[i] = 255;
      rs->size[i] = 0;
    }
    return;
  }
  TenantSlot* t = slot_ptr(chunks, rq.slot);
  const unsigned g = (unsigned)md.g;
  const Sizes z = sizes_of(md);

  if (rq.op == GPA_SERVE_ADMIT) {
    const int n = rq.n;
    for (int i = lane; i < n; i += 32) {
      const long long o = rq.payload + i;
      t->T[i] = pay.T[o];
      t->D[i] = pay.D[o];
      t->A[i] = pay.A[o];
      t->B[i] = pay.B[o];
      t->u[i] = pay.u[o];
      t->type[i] = pay.type[o];
    }
    __syncwarp();
    if (!stage_set(sm.m.st, 0, n, t->T, t->D, t->A, t->B, t->u, t->type)) {
      if (lane == 0) {
        rs->status = 1;
        atomicOr(err, kErrRange);
      }
      return;
    }
    if (!run_alg1(sm, t, rs, n, md, prm, mdiv, err)) {
      // not admitted: the tenant does not exist (empty state in the response)
      if (lane == 0) {
        rs->n_tasks = rs->n_parts = rs->Pi = 0;
        rs->W = 0;
      }
      for (int i = lane; i < kNmax; i += 32) {
        rs->part[i] = 255;
        rs->size[i] = 0;
      }
    }
    return;
  }

  if (rq.op == GPA_SERVE_ADD) {
    const int n = t->n;
    const int np = t->n_parts;
    if (lane == 0) {
      const long long o = rq.payload;
      t->T[n] = pay.T[o];
      t->D[n] = pay.D[o];
      t->A[n] = pay.A[o];
      t->B[n] = pay.B[o];
      t->u[n] = pay.u[o];
      t->type[n] = pay.type[o];
    }
    __syncwarp();
    if (!stage_set(sm.m.st, 0, n + 1, t->T, t->D, t->A, t->B, t->u, t->type)) {
      if (lane == 0) {
        rs->status = 1;
        atomicOr(err, kErrRange);
      }
      copy_state_to_resp(t, rs);
      return;
    }
    int rnew = 0;
    for (int r = lane; r <= n; r += 32) {
      const int orig = sm.m.st.orig[r];
      sm.prow[r] = orig < n ? t->part[orig] : 255;
      if (orig == n) rnew = r;
    }
    rnew = __reduce_max_sync(kFull, (unsigned)rnew);
    __syncwarp();
    const int spare = md.M - t->Pi;
    int path = GPA_PATH_NONE, where = -1, newsize = 0;
    unsigned int S[kWords];
    // fit at the current size, first partition in order
    for (int p = 0; p < np && path == GPA_PATH_NONE; p++) {
      rows_of(sm, n + 1, p, S);
      S[rnew >> 5] |= 1u << (rnew & 31);
      if (warp_test(sm.m.st, S, (unsigned)t->size[p], md.kc, md.km, md.sched, mdiv, sm.m.sc, nullptr, true, err)) {
        path = GPA_PATH_FIT;
        where = p;
        newsize = t->size[p];
      }
    }
    // grow into the spare SMs
    for (int p = 0; p < np && path == GPA_PATH_NONE && spare >= md.g; p++) {
      rows_of(sm, n + 1, p, S);
      S[rnew >> 5] |= 1u << (rnew & 31);
      const unsigned m = warp_minm(sm.m.st, S, (unsigned)t->size[p] + 1u, (unsigned)t->size[p] + (unsigned)spare, z,
                                   true, md.kc, md.km, md.sched, mdiv, sm.m.sc, err);
      if (m) {
        path = GPA_PATH_GROW;
        where = p;
        newsize = (int)m;
      }
    }
    // a new partition of the task's Lemma 2 size
    if (path == GPA_PATH_NONE) {
      const unsigned z1 = lemma2_size(sm.m.st.A[rnew], sm.m.st.B[rnew], sm.m.st.D[rnew], z);
      if (z1 && (int)z1 <= spare) {
        path = GPA_PATH_NEW;
        where = np;
        newsize = (int)z1;
      }
    }
    if (path != GPA_PATH_NONE) {
      __syncwarp();
      if (lane == 0) {
        t->part[n] = (unsigned char)where;
        t->size[where] = (short)newsize;
        t->n = n + 1;
        if (path == GPA_PATH_NEW) t->n_parts = np + 1;
        rs->verdict = 1;
        rs->path = (unsigned char)path;
        sm.prow[rnew] = (unsigned char)where;
      }
      __syncwarp();
      int Pi;
      unsigned long long W;
      summarise_state(sm, n + 1, t->size, t->n_parts, md, &Pi, &W);
      if (lane == 0) {
        t->Pi = Pi;
        t->W = (long long)W;
      }
      __syncwarp();
      copy_state_to_resp(t, rs);
      return;
    }
    // Alg. 1 on every task; on failure the state is unchanged
    if (run_alg1(sm, t, rs, n + 1, md, prm, mdiv, err)) {
      if (lane == 0) rs->path = GPA_PATH_REALLOC;
    } else {
      const unsigned char reason = rs->reason;
      copy_state_to_resp(t, rs);
      if (lane == 0) {
        rs->verdict = 0;
        rs->reason = reason;
      }
    }
    return;
  }

  if (rq.op == GPA_SERVE_REMOVE) {
    const int n = t->n, idx = rq.index;
    const int pr = t->part[idx];
    // shift the later tasks down by one (read everything first)
    long long vT[kWords], vD[kWords], vA[kWords], vB[kWords], vu[kWords];
    unsigned char vy[kWords], vp[kWords];
#pragma unroll
    for (int c = 0; c < kWords; c++) {
      const int i = c * 32 + lane;
      const int src = i < idx ? i : i + 1;
      if (src < n) {
        vT[c] = t->T[src];
        vD[c] = t->D[src];
        vA[c] = t->A[src];
        vB[c] = t->B[src];
        vu[c] = t->u[src];
        vy[c] = t->type[src];
        vp[c] = t->part[src];
      }
    }
    __syncwarp();
    const int n2 = n - 1;
    bool still = false;
#pragma unroll
    for (int c = 0; c < kWords; c++) {
      const int i = c * 32 + lane;
      if (i < n2) {
        t->T[i] = vT[c];
        t->D[i] = vD[c];
        t->A[i] = vA[c];
        t->B[i] = vB[c];
        t->u[i] = vu[c];
        t->type[i] = vy[c];
        unsigned char pp = vp[c];
        still = still || pp == pr;
        t->part[i] = pp;
      }
    }
    still = __any_sync(kFull, still);
    __syncwarp();
    int np = t->n_parts;
    if (!still) {
      // the partition disappears: close the gap in the numbering
      for (int i = lane; i < n2; i += 32)
        if (t->part[i] > pr) t->part[i]--;
      short sz[kWords];
#pragma unroll
      for (int c = 0; c < kWords; c++) {
        const int p = c * 32 + lane;
        sz[c] = (p + 1 < np) ? t->size[p + 1] : 0;
      }
      __syncwarp();
#pragma unroll
      for (int c = 0; c < kWords; c++) {
        const int p = c * 32 + lane;
        if (p >= pr && p + 1 < np) t->size[p] = sz[c];
      }
      np--;
    }
    __syncwarp();
    if (!stage_set(sm.m.st, 0, n2, t->T, t->D, t->A, t->B, t->u, t->type)) {
      if (lane == 0) {
        rs->status = 1;
        atomicOr(err, kErrRange);
      }
      return;
    }
    for (int r = lane; r < n2; r += 32) sm.prow[r] = t->part[sm.m.st.orig[r]];
    __syncwarp();
    if (still) {
      // its partition shrinks to its minimum size (the search of Alg. 2)
      unsigned int S[kWords];
      rows_of(sm, n2, pr, S);
      const unsigned m =
          warp_minm(sm.m.st, S, g, (unsigned)t->size[pr], z, false, md.kc, md.km, md.sched, mdiv, sm.m.sc, err);
      if (lane == 0) t->size[pr] = (short)m;
    }
    __syncwarp();
    // renumber partitions by their lowest task index
    for (int p = lane; p < kNmax; p += 32) sm.cntc[p] = n2;
    __syncwarp();
    for (int i = lane; i < n2; i += 32) atomicMin(&sm.cntc[t->part[i]], i);
    __syncwarp();
    short szv[kWords];
#pragma unroll
    for (int c = 0; c < kWords; c++) {
      const int p = c * 32 + lane;
      szv[c] = 0;
      if (p < np) {
        int rr = 0;
        for (int q2 = 0; q2 < np; q2++) rr += sm.cntc[q2] < sm.cntc[p];
        sm.cntm[p] = rr;
        szv[c] = t->size[p];
      }
    }
    __syncwarp();
#pragma unroll
    for (int c = 0; c < kWords; c++) {
      const int p = c * 32 + lane;
      if (p < np) t->size[sm.cntm[p]] = szv[c];
      else if (p < kNmax) t->size[p] = 0;
    }
    for (int i = lane; i < n2; i += 32) t->part[i] = (unsigned char)sm.cntm[t->part[i]];
    __syncwarp();
    for (int r = lane; r < n2; r += 32) sm.prow[r] = t->part[sm.m.st.orig[r]];
    __syncwarp();
    int Pi;
    unsigned long long W;
    summarise_state(sm, n2, t->size, np, md, &Pi, &W);
    if (lane == 0) {
      t->n = n2;
      t->n_parts = np;
      t->Pi = Pi;
      t->W = (long long)W;
      rs->verdict = 1;
    }
    __syncwarp();
    copy_state_to_resp(t, rs);
    return;
  }
}

// One warp per request.  A request whose analysis hit a test's step limit
// (kErrIter) answers status 2 (GPA_ERR_TIMEOUT): the tenant's state is still
// an allocation whose every partition passes, but the choice among them may
// differ from that of the exact analysis.
__global__ void __launch_bounds__(128, 1) serve_batch(const ServeReq* __restrict__ reqs, int nreq,
                                                   TenantSlot* const* __restrict__ chunks, ServePayload pay,
                                                   ServeResp* __restrict__ resps, DevModel md, gpa_params prm,
                                                   const MagicDiv* __restrict__ mdiv, unsigned int* err) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int q = blockIdx.x * (blockDim.x >> 5) + warp;
  if (q >= nreq) return;
  ServeSmem& sm = reinterpret_cast<ServeSmem*>(smem_raw)[warp];
  if (lane == 0) sm.m.err = 0u;
  __syncwarp();
  serve_one(sm, reqs[q], resps + q, chunks, pay, md, prm, mdiv, &sm.m.err);
  __syncwarp();
  const unsigned int e = sm.m.err;
  if (lane == 0 && e) {
    if ((e & kErrIter) && resps[q].status == 0) resps[q].status = 2;
    atomicOr(err, e);
  }
}

}  // namespace

size_t serve_smem_bytes(int warps) { return sizeof(ServeSmem) * (size_t)warps; }

cudaError_t serve_kernels_init() {
  return cudaFuncSetAttribute(serve_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)serve_smem_bytes(4));
}

cudaError_t launch_serve_batch(const ServeReq* reqs, int nreq, TenantSlot* const* chunks, const ServePayload& pay,
                               ServeResp* resps, const DevModel& md, const gpa_params& p, const MagicDivHost* mdiv,
                               unsigned int* err, cudaStream_t st) {
  if (nreq <= 0) return cudaSuccess;
  const int warps = 4;
  serve_batch<<<(nreq + warps - 1) / warps, warps * 32, serve_smem_bytes(warps), st>>>(
      reqs, nreq, chunks, pay, resps, md, p, reinterpret_cast<const MagicDiv*>(mdiv), err);
  return cudaGetLastError();
}

}  // namespace gpa
