// serve_types.h — records shared by the serving host loop (serve.cpp) and
// its kernel (k_serve.cu).  Not part of the ABI.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "gpa.h"
#include "gpa_internal.h"

namespace gpa {

constexpr int kSlotsPerChunkMax = 256;  // tenant slots per device allocation
constexpr int kMaxChunks = 4096;        // chunk table entries

// One tenant: its tasks (structure of arrays, original order) and its
// allocation (partition of each task, size of each partition).
struct TenantSlot {
  long long T[GPA_SERVE_NMAX], D[GPA_SERVE_NMAX], A[GPA_SERVE_NMAX], B[GPA_SERVE_NMAX], u[GPA_SERVE_NMAX];
  unsigned char type[GPA_SERVE_NMAX];
  unsigned char part[GPA_SERVE_NMAX];
  short size[GPA_SERVE_NMAX];
  int n, n_parts, Pi, pad;
  long long W;
};

struct ServeReq {
  int op;
  int slot;
  int index;         // REMOVE
  int n;             // ADMIT
  long long payload; // first task of the request in the batch payload
};

// Tasks carried by a batch's ADMIT / ADD requests (structure of arrays).
struct ServePayload {
  const long long* T;
  const long long* D;
  const long long* A;
  const long long* B;
  const long long* u;
  const unsigned char* type;
};

struct ServeResp {
  unsigned char verdict, reason, path, status;
  int n_tasks, n_parts, Pi;
  long long W;
  int n_tests, pad;
  unsigned char part[GPA_SERVE_NMAX];
  short size[GPA_SERVE_NMAX];
};

size_t serve_smem_bytes(int warps);
cudaError_t serve_kernels_init();
cudaError_t launch_serve_batch(const ServeReq* reqs, int nreq, TenantSlot* const* chunks, const ServePayload& pay,
                               ServeResp* resps, const DevModel& md, const gpa_params& p, const MagicDivHost* mdiv,
                               unsigned int* err, cudaStream_t st);

}  // namespace gpa
