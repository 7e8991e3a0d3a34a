// gpa_internal.h — host-side interface between the C ABI (host.cpp) and the
// kernel launchers (*.cu).  Not installed; not part of the ABI.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "gpa.h"

namespace gpa {

// Granlund-Montgomery reciprocal of 10^6 m, one per m in [0, GPA_MMAX]
// (layout identical to MagicDiv in gpa_device.cuh).
struct MagicDivHost {
  unsigned long long magic;
  unsigned int shift;
  unsigned int pad;
};

// Fills table[0 .. GPA_MMAX] (entry 0 unused): for d = 10^6 m and
// l = ceil(log2 d), magic = ceil(2^(60+l) / d) and shift = l - 4.  Every
// context and the allocation-free entry point build their table with it.
void build_reciprocals(MagicDivHost* table);

struct DevSets {
  long long nsets;
  int n_max;
  const long long* set_off;
  const long long* T;
  const long long* D;
  const long long* A;
  const long long* B;
  const long long* u;
  const unsigned char* type;
};

struct DevModel {
  int M, g, kc, km;
  int sched;  // GPA_SCHED_DM or GPA_SCHED_EDF
  // admissible partition sizes (device arrays): zlist[k] the k-th, zrank[m]
  // (m in [0, M + 1]) how many are < m; zlist == nullptr: every multiple of g
  int nz;
  const unsigned short* zlist;
  const unsigned short* zrank;
};

struct AllocOut {
  unsigned char* verdict;
  unsigned char* reason;
  int* n_parts;
  int* Pi;
  long long* W;
  int* n_tests;
  unsigned char* part_of_task;
  short* size_of_part;
};

// Byte ranges copied by one launch of the staging kernel (k_stage.cu); one
// side of each is page-locked host memory mapped into the device's address
// space, the other a device buffer.
constexpr int kStageRangesMax = 12;
struct StageRange {
  const void* src;
  void* dst;
  unsigned long long bytes;
};
struct StageList {
  StageRange r[kStageRangesMax];
  int n;
};
cudaError_t launch_stage_copy(const StageList& L, int blocks_per_range, cudaStream_t st, long long* launches);

// Measured WCET curves (k_probe.cu): the buffers of the kernel under test,
// the blocker that holds sm_count - m SMs, and the kernels' launchers.
struct ProbeBuffers {
  float* a;
  float* b;
  float* c;
};
size_t probe_blocker_smem();
cudaError_t probe_kernels_init();
cudaError_t launch_probe_blocker(int ctas, unsigned long long window_ns, const void* buf, unsigned long long buf_bytes,
                                 unsigned int* smid, unsigned long long* t_end, float* sink, cudaStream_t st);
cudaError_t launch_probe_kernel(int kernel, int ctas, const ProbeBuffers& b, unsigned long long n,
                                unsigned int* smid, unsigned long long* t_done, cudaStream_t st);

// Work-queue state of the persistent allocate kernels.
struct AllocQueue {
  unsigned long long* counters;  // [5]: fast ticket, slow count, slow ticket, 1G / search ticket,
                                 // interference terms evaluated by the call's kernels
  long long* slow_sets;          // [nsets] sets deferred to the merge kernel
  unsigned int* err;             // sticky error word
};

// Optional timing events recorded around kernels (see GPA_OPT_PROFILE).
struct Prof {
  cudaEvent_t ev[4];
  int used;       // events recorded by the last call
  bool capture;   // recording into a stream capture (graph node)
};

void prof_mark(Prof* p, cudaStream_t st);

struct LaunchShape {
  int warps_per_block;  // warps per CTA
  int chunk;            // sets per ticket (fast kernel); warps per set (merge kernel)
  int blocks;           // CTAs of the persistent grid
  int stages;           // fast kernel: 1 = direct loads, 2..5 = shared-memory stages fed by bulk copies;
                        // merge kernel: 2 = SMS steps open with the top-size round, else not
};

// The launch shapes of one gpa_allocate call: the fast kernel, the merge
// kernel (chunk = warps per set) and the 1G kernel.
struct AllocShapes {
  LaunchShape fast;
  LaunchShape slow;
  LaunchShape one;
};

struct BestOut {
  unsigned char* feasible;
  long long* W;
  int* sum_minm;
  int* n_blocks;
  int* spare;
  unsigned char* rgs;
  short* minm_block;
};

struct Cands {
  long long ncands;
  int map_stride;
  int kparts;
  const long long* set;
  const unsigned char* part_of_task;
  const int* size_of_part;
};

// Kernel launchers; each returns the CUDA error of its launches and adds the
// number of kernels it launched to *launches.
cudaError_t launch_allocate(const DevSets& s, const DevModel& md, const gpa_params& p, const AllocOut& out,
                            const AllocQueue& q, const MagicDivHost* mdiv, const LaunchShape& fast,
                            const LaunchShape& slow, cudaStream_t st, long long* launches, Prof* prof);
cudaError_t launch_one_gpu(const DevSets& s, const DevModel& md, const AllocOut& out, const AllocQueue& q,
                           const MagicDivHost* mdiv, const LaunchShape& shape, cudaStream_t st, long long* launches,
                           Prof* prof);
// Per-process kernel attribute set-up (dynamic shared memory opt-in).
cudaError_t alloc_kernels_init();
cudaError_t search_kernels_init();
cudaError_t launch_validate_batch(const DevSets& s, unsigned int* flag, int sm_count, cudaStream_t st,
                                  long long* launches);
cudaError_t launch_wcet_tables(const DevSets& s, const DevModel& md, long long* Cn, long long* Cc, unsigned int* err,
                               const MagicDivHost* mdiv, int sm_count, cudaStream_t st, long long* launches,
                               Prof* prof);
cudaError_t launch_test_schedulable(const DevSets& s, const DevModel& md, const Cands& c, unsigned char* verdict,
                                    long long* R, unsigned int* err, const MagicDivHost* mdiv, int sm_count,
                                    cudaStream_t st, long long* launches, Prof* prof);
cudaError_t launch_search_best(const DevSets& s, const DevModel& md, int kmin, int kmax, const BestOut& out,
                               const AllocQueue& q, const MagicDivHost* mdiv, int sm_count, cudaStream_t st,
                               long long* launches, Prof* prof);
// The explicit candidates (every composition x map) of each set; cverdict
// (nullable) receives each candidate's verdict at cstride bytes per set.
cudaError_t launch_search_explicit(const DevSets& s, const DevModel& md, int kmin, int kmax, const BestOut& out,
                                   unsigned char* cverdict, long long cstride, const AllocQueue& q,
                                   const MagicDivHost* mdiv, int sm_count, cudaStream_t st, long long* launches,
                                   Prof* prof);
// Measured throughput of the integer work the tests are made of (k_peak.cu).
cudaError_t measure_alu_peak(int sm_count, cudaStream_t st, double* terms_per_s, double* imad_per_s,
                             double* term_ms, long long* terms);

// Largest dynamic shared memory (bytes) the allocate merge kernel needs per CTA.
size_t slow_smem_bytes(int warps_per_block, int warps_per_set);
// CTAs per SM of the merge kernel (wpb warps per CTA in groups of gw) and of
// the 1G kernel (wpb warps per CTA), by occupancy; 0 when none fits.
int merge_ctas_per_sm(int wpb, int gw);
int one_gpu_ctas_per_sm(int wpb);
size_t staged_smem_bytes(int stages);
size_t one_gpu_smem_bytes(int warps_per_block);

// The same allocate kernels built for sets of up to 64 tasks
// (k_alloc_small.cu), used when a batch's n_max is at most kSmallNmax, and
// the allocate and candidate-test kernels built for up to 256 tasks
// (k_alloc_wide.cu, k_test_wide.cu), used when it exceeds kNarrowNmax.
constexpr int kSmallNmax = 64;
constexpr int kNarrowNmax = 128;
namespace small {
int merge_ctas_per_sm(int wpb, int gw);
int one_gpu_ctas_per_sm(int wpb);
cudaError_t launch_allocate(const DevSets& s, const DevModel& md, const gpa_params& p, const AllocOut& out,
                            const AllocQueue& q, const MagicDivHost* mdiv, const LaunchShape& fast,
                            const LaunchShape& slow, cudaStream_t st, long long* launches, Prof* prof);
cudaError_t launch_one_gpu(const DevSets& s, const DevModel& md, const AllocOut& out, const AllocQueue& q,
                           const MagicDivHost* mdiv, const LaunchShape& shape, cudaStream_t st, long long* launches,
                           Prof* prof);
cudaError_t alloc_kernels_init();
}  // namespace small
namespace wide {
int merge_ctas_per_sm(int wpb, int gw);
int one_gpu_ctas_per_sm(int wpb);
cudaError_t launch_allocate(const DevSets& s, const DevModel& md, const gpa_params& p, const AllocOut& out,
                            const AllocQueue& q, const MagicDivHost* mdiv, const LaunchShape& fast,
                            const LaunchShape& slow, cudaStream_t st, long long* launches, Prof* prof);
cudaError_t launch_one_gpu(const DevSets& s, const DevModel& md, const AllocOut& out, const AllocQueue& q,
                           const MagicDivHost* mdiv, const LaunchShape& shape, cudaStream_t st, long long* launches,
                           Prof* prof);
cudaError_t alloc_kernels_init();
cudaError_t launch_test_schedulable(const DevSets& s, const DevModel& md, const Cands& c, unsigned char* verdict,
                                    long long* R, unsigned int* err, const MagicDivHost* mdiv, int sm_count,
                                    cudaStream_t st, long long* launches, Prof* prof);
}  // namespace wide

}  // namespace gpa
