// k_noalloc.cu — gpa_allocate_noalloc: the allocate path for callers that
// cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at all: code that runs where the
// allocator is owned by someone else (a host application with its own
// memory pool or a fixed memory budget, a plug-in loaded into such an
// application, a real-time process that must not allocate after start-up).
// gpa_allocate needs a context, and creating one allocates device memory
// for its reciprocal table, its work-queue counters and its deferred-set
// queue.  This entry point needs no context: that scratch lives in the
// file-scope device arrays below, which every GPU that loads the library
// holds until the process exits.  The caller still passes every input and
// output array (device memory only).
//
// Limits and sharing: at most kNoAllocMaxSets task sets per call.  All calls
// share the arrays, which keep the last call's contents; each call clears
// the counters that must start at zero before its kernels run.  Calls whose
// work overlaps on the GPU (on different streams, or from different threads)
// race on the shared arrays and must be serialised by the caller.  The
// kernels record problems (an invalid set, a test that hit its step limit)
// in the arrays' error word, which gpa_allocate_noalloc_status reads and
// clears.
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>

#include "gpa.h"
#include "gpa_ctx.h"
#include "gpa_internal.h"

namespace {

constexpr long long kNoAllocMaxSets = GPA_NOALLOC_MAX_SETS;
constexpr int kMaxDevices = 64;

// work-queue counters [0..3], interference-term counter [4], error word,
// deferred-set queue
struct NoAllocScratch {
  unsigned long long counters[8];
  unsigned int err;
  unsigned int pad[7];
  long long slow_sets[kNoAllocMaxSets];
};

static __device__ __align__(256) NoAllocScratch g_scratch;
static __device__ __align__(256) gpa::MagicDivHost g_mdiv[GPA_MMAX + 1];

// Device addresses of the arrays above, looked up once per device.  In host
// code the names g_scratch / g_mdiv are host-side stand-ins, not device
// addresses: only the addresses from cudaGetSymbolAddress may reach a kernel.
struct DeviceSetup {
  bool ready = false;
  NoAllocScratch* scratch = nullptr;
  gpa::MagicDivHost* mdiv = nullptr;
  int sm_count = 0;
};

std::mutex g_setup_mutex;
DeviceSetup g_setup[kMaxDevices];

// One-time set-up of the current device (synchronous): fills the reciprocal
// table, clears the error word, looks up the device addresses of the arrays.
int32_t setup_current_device(DeviceSetup** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return gpa_cuda_fail(e, "gpa_allocate_noalloc: cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return gpa_fail(GPA_ERR_ARG, "gpa_allocate_noalloc: device %d unsupported", dev);
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  DeviceSetup& d = g_setup[dev];
  if (!d.ready) {
    gpa::MagicDivHost table[GPA_MMAX + 1];
    gpa::build_reciprocals(table);
    void* p = nullptr;
    if ((e = cudaGetSymbolAddress(&p, g_scratch)) != cudaSuccess)
      return gpa_cuda_fail(e, "gpa_allocate_noalloc: cudaGetSymbolAddress(scratch)");
    d.scratch = static_cast<NoAllocScratch*>(p);
    if ((e = cudaGetSymbolAddress(&p, g_mdiv)) != cudaSuccess)
      return gpa_cuda_fail(e, "gpa_allocate_noalloc: cudaGetSymbolAddress(reciprocals)");
    d.mdiv = static_cast<gpa::MagicDivHost*>(p);
    if ((e = cudaMemcpyToSymbol(g_mdiv, table, sizeof table)) != cudaSuccess)
      return gpa_cuda_fail(e, "gpa_allocate_noalloc: reciprocal table upload");
    if ((e = cudaMemset(&d.scratch->err, 0, sizeof(unsigned int))) != cudaSuccess)
      return gpa_cuda_fail(e, "gpa_allocate_noalloc: clearing the error word");
    if ((e = gpa::alloc_kernels_init()) != cudaSuccess)
      return gpa_cuda_fail(e, "gpa_allocate_noalloc: kernel attributes");
    if ((e = cudaDeviceGetAttribute(&d.sm_count, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
      return gpa_cuda_fail(e, "gpa_allocate_noalloc: SM count");
    d.ready = true;
  }
  *out = &d;
  return GPA_OK;
}

// The work goes onto the caller's stream, the scratch addresses are the
// current device's: the two must be the same device.
int32_t check_stream_device(cudaStream_t stream, const char* who) {
  int cur = 0, sdev = 0;
  cudaError_t e = cudaGetDevice(&cur);
  if (e != cudaSuccess) return gpa_cuda_fail(e, who);
  e = cudaStreamGetDevice(stream, &sdev);
  if (e != cudaSuccess) return gpa_cuda_fail(e, who);
  if (sdev != cur)
    return gpa_fail(GPA_ERR_ARG, "%s: the stream belongs to device %d, the current device is %d", who, sdev, cur);
  return GPA_OK;
}

}  // namespace

extern "C" int32_t gpa_allocate_noalloc_status(void* stream) {
  int32_t st = check_stream_device((cudaStream_t)stream, "gpa_allocate_noalloc_status");
  if (st != GPA_OK) return st;
  DeviceSetup* d = nullptr;
  if ((st = setup_current_device(&d)) != GPA_OK) return st;
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return gpa_cuda_fail(e, "gpa_allocate_noalloc_status: cudaStreamSynchronize");
  unsigned int err = 0;
  if ((e = cudaMemcpy(&err, &d->scratch->err, sizeof err, cudaMemcpyDeviceToHost)) != cudaSuccess)
    return gpa_cuda_fail(e, "gpa_allocate_noalloc_status: reading the error word");
  if (!err) return GPA_OK;
  if ((e = cudaMemset(&d->scratch->err, 0, sizeof err)) != cudaSuccess)
    return gpa_cuda_fail(e, "gpa_allocate_noalloc_status: clearing the error word");
  if (err & 2u)
    return gpa_fail(GPA_ERR_TIMEOUT,
                    "gpa_allocate_noalloc: a per-partition test hit its step limit (sets with GPA_REASON_UNDECIDED)");
  return gpa_fail(GPA_ERR_RANGE, "gpa_allocate_noalloc: a set failed validation (sets with GPA_REASON_INVALID)");
}

extern "C" int32_t gpa_allocate_noalloc(void* stream, const gpa_tasksets* sets, const gpa_model* model,
                                        const gpa_params* params, gpa_alloc_result* r) {
  if (!sets || !sets->set_off || !model || !params || !r)
    return gpa_fail(GPA_ERR_ARG, "gpa_allocate_noalloc: NULL argument");
  if (sets->mem != GPA_DEVICE || r->mem != GPA_DEVICE)
    return gpa_fail(GPA_ERR_ARG, "gpa_allocate_noalloc: device arrays only (mem = GPA_DEVICE)");
  if (sets->nsets < 0 || sets->nsets > kNoAllocMaxSets)
    return gpa_fail(GPA_ERR_RANGE, "gpa_allocate_noalloc: %lld task sets exceed the limit of %lld per call",
                    (long long)sets->nsets, kNoAllocMaxSets);
  if (sets->n_max < 0 || sets->n_max > GPA_SERVE_NMAX)
    return gpa_fail(GPA_ERR_RANGE, "gpa_allocate_noalloc: n_max above %d", GPA_SERVE_NMAX);
  if (model->g < 1 || model->M < 1 || model->M > GPA_MMAX || model->M % model->g != 0 || model->k_c_pm < 1000 ||
      model->k_c_pm > 16000 || model->k_m_pm < 1000 || model->k_m_pm > 16000 ||
      (model->sched != GPA_SCHED_DM && model->sched != GPA_SCHED_EDF))
    return gpa_fail(GPA_ERR_RANGE, "gpa_allocate_noalloc: model out of range");
  if (model->nsizes != 0) return gpa_fail(GPA_ERR_ARG, "gpa_allocate_noalloc: admissible size lists need a context");
  if (params->policy != GPA_POLICY_SMS && params->policy != GPA_POLICY_BF)
    return gpa_fail(GPA_ERR_ARG, "gpa_allocate_noalloc: policy must be GPA_POLICY_SMS or GPA_POLICY_BF");
  if (sets->nsets == 0) return GPA_OK;
  if (!sets->T || !sets->D || !sets->A || !sets->B || !sets->u_ppm || !sets->type || !r->verdict || !r->reason ||
      !r->n_parts || !r->Pi || !r->W || !r->part_of_task || !r->size_of_part)
    return gpa_fail(GPA_ERR_ARG, "gpa_allocate_noalloc: NULL array");
  int32_t st = check_stream_device((cudaStream_t)stream, "gpa_allocate_noalloc");
  if (st != GPA_OK) return st;
  DeviceSetup* d = nullptr;
  st = setup_current_device(&d);
  if (st != GPA_OK) return st;
  gpa::DevSets ds{sets->nsets,
                  sets->n_max,
                  (const long long*)sets->set_off,
                  (const long long*)sets->T,
                  (const long long*)sets->D,
                  (const long long*)sets->A,
                  (const long long*)sets->B,
                  (const long long*)sets->u_ppm,
                  (const unsigned char*)sets->type};
  gpa::DevModel md{model->M, model->g, model->k_c_pm, model->k_m_pm, model->sched};
  gpa::AllocOut out{r->verdict, r->reason, r->n_parts, r->Pi, (long long*)r->W, r->n_tests, r->part_of_task,
                    r->size_of_part};
  gpa::AllocQueue q{d->scratch->counters, d->scratch->slow_sets, &d->scratch->err};
  const gpa::LaunchShape fast{8, 2, 0};
  const gpa::LaunchShape slow{4, 1, d->sm_count * 2};
  long long launches = 0;
  cudaError_t e = gpa::launch_allocate(ds, md, *params, out, q, d->mdiv, fast, slow, (cudaStream_t)stream,
                                       &launches, nullptr);
  return e == cudaSuccess ? GPA_OK : gpa_cuda_fail(e, "gpa_allocate_noalloc: launch");
}
