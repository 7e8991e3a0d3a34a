// gpa_ctx.h — the library-owned context behind gpa_ctx* (host side only).
#pragma once

#include <cuda_runtime.h>

#include <cstdarg>
#include <map>
#include <string>
#include <vector>

#include "gpa.h"
#include "gpa_internal.h"

struct CtxBuf {
  void* ptr = nullptr;
  size_t bytes = 0;
};

struct CachedGraph {
  cudaGraphExec_t exec;
  long long kernels;  // kernel nodes in the graph
  gpa::Prof prof;     // timing events captured as graph nodes (prof.used == 0 without profiling)
};

struct ServeState;

struct gpa_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  int sm_count = 0;
  gpa::MagicDivHost* d_mdiv = nullptr;      // [GPA_MMAX + 1] reciprocals of 10^6 m
  unsigned long long* d_counters = nullptr; // [8] work-queue tickets, [4] interference terms of the last call
  unsigned int* d_err = nullptr;            // sticky error word
  long long* d_slow = nullptr;              // deferred-set queue of the allocate kernels
  long long slow_cap = 0;
  std::vector<CtxBuf> bufs;                 // host-path staging, by slot
  long long launches = 0;                   // kernels launched through this context
  bool autotune = false;
  bool use_graph = false;
  bool per_set_launch = false;
  bool graphs_dirty = false;
  bool profile = false;
  gpa::Prof prof{};                          // timing events of direct (non-graph) calls
  const gpa::Prof* last_prof = nullptr;      // events of the last profiled call
  gpa::LaunchShape force_fast{0, 0, 0, 0};
  gpa::LaunchShape force_merge{0, 0, 0, 0};  // GPA_OPT_MERGE_*: warps per CTA, warps per set, CTAs
  int force_test_warps = 0;                   // GPA_OPT_TEST_WARPS
  int host_slices = 0;                       // GPA_OPT_HOST_SLICES
  int host_copy = 0;                         // GPA_OPT_HOST_COPY
  cudaStream_t copy_in = nullptr;            // sliced host path: host-to-device copies
  cudaStream_t copy_out = nullptr;           // sliced host path: device-to-host copies
  cudaEvent_t pipe_ev[3] = {nullptr, nullptr, nullptr};  // start, slice copied in, slice computed
  unsigned int* h_err = nullptr;             // page-locked copy of the error word read at the end of a call
  std::vector<unsigned short> size_table;   // last admissible-size table copied to the device
  void* size_table_ptr = nullptr;
  std::map<std::string, gpa::AllocShapes> tuned;  // autotuned shapes per batch signature
  std::map<std::string, CachedGraph> graphs;
  ServeState* serve = nullptr;
};

// Makes `dev` the current device for the scope, then restores the previous one.
struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

int32_t gpa_fail(int32_t code, const char* fmt, ...);
int32_t gpa_cuda_fail(cudaError_t e, const char* what);
void* ctx_buffer(gpa_ctx* c, int slot, size_t bytes);
std::string tune_key(const gpa::DevSets& ds, const gpa::DevModel& md, const gpa_params& p);
void gpa_serve_teardown(gpa_ctx* c);
