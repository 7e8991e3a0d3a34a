// host.cpp — the C ABI of libgpa (gpa.h): context, validation, the
// host-memory path (stage in, run, copy back), the launch shapes of the
// persistent kernels with their autotuner and CUDA-graph cache, and the
// combinatorial helpers (ranking of SM splits and of set partitions).
#include <cuda_runtime.h>

#include <chrono>
#include <cstdio>
#include <cstring>
#include <map>
#include <algorithm>
#include <atomic>
#include <condition_variable>
#include <functional>
#include <mutex>
#include <thread>
#include <string>
#include <vector>

#include "gpa.h"
#include "gpa_internal.h"
#include "gpa_ctx.h"

using namespace gpa;

// ------------------------------------------------------------------ errors

static thread_local std::string g_last_error;

int32_t gpa_fail(int32_t code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}

int32_t gpa_cuda_fail(cudaError_t e, const char* what) {
  return gpa_fail(GPA_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

extern "C" int32_t gpa_last_error(char* buf, int32_t len) {
  if (!buf || len <= 0) return GPA_ERR_ARG;
  std::snprintf(buf, (size_t)len, "%s", g_last_error.c_str());
  return GPA_OK;
}

// ------------------------------------------------------------- validation

static bool model_valid(const gpa_model* m) {
  if (!(m && m->g >= 1 && m->M >= 1 && m->M <= GPA_MMAX && m->M % m->g == 0 && m->k_c_pm >= 1000 &&
        m->k_c_pm <= 16000 && m->k_m_pm >= 1000 && m->k_m_pm <= 16000 &&
        (m->sched == GPA_SCHED_DM || m->sched == GPA_SCHED_EDF)))
    return false;
  if (m->nsizes < 0 || m->nsizes > GPA_MMAX || (m->nsizes > 0 && !m->sizes)) return false;
  for (int k = 0; k < m->nsizes; k++) {
    const int z = m->sizes[k];
    if (z < m->g || z > m->M || z % m->g != 0 || (k > 0 && z <= m->sizes[k - 1])) return false;
  }
  return true;
}

// The model's admissible partition sizes on the device: nothing for the
// default (every multiple of g), else the list and its rank table (how many
// listed sizes lie below each m in [0, M + 1]) in context buffers, copied on
// the context stream when they change.
static int32_t device_model(gpa_ctx* c, const gpa_model* model, DevModel* md) {
  *md = DevModel{model->M, model->g, model->k_c_pm, model->k_m_pm, model->sched, 0, nullptr, nullptr};
  if (model->nsizes == 0) return GPA_OK;
  const int M = model->M;
  std::vector<unsigned short> host((size_t)model->nsizes + (size_t)M + 2);
  for (int k = 0; k < model->nsizes; k++) host[(size_t)k] = (unsigned short)model->sizes[k];
  int below = 0;
  for (int m = 0; m <= M + 1; m++) {
    host[(size_t)model->nsizes + (size_t)m] = (unsigned short)below;
    if (below < model->nsizes && model->sizes[below] == m) below++;
  }
  unsigned short* dev = (unsigned short*)ctx_buffer(c, 30, sizeof(unsigned short) * host.size());
  if (!dev) return gpa_fail(GPA_ERR_NOMEM, "size table allocation failed");
  if (c->size_table != host || c->size_table_ptr != dev) {
    cudaError_t e = cudaMemcpyAsync(dev, host.data(), sizeof(unsigned short) * host.size(), cudaMemcpyHostToDevice,
                                    c->stream);
    if (e != cudaSuccess) return gpa_cuda_fail(e, "size table copy");
    c->size_table = host;
    c->size_table_ptr = dev;
  }
  md->nz = model->nsizes;
  md->zlist = dev;
  md->zrank = dev + model->nsizes;
  return GPA_OK;
}

static bool host_task_valid(int64_t T, int64_t D, int64_t A, int64_t B, int64_t u, uint8_t type) {
  return D >= 1 && D <= T && T <= 2147483647LL && A >= 0 && B >= 0 && A + B >= 1 && A + B <= (1LL << 36) &&
         u >= 0 && u <= 4294967295LL && type <= 1;
}

// The same bounds without branches (unsigned compares), so that a loop over
// a column range vectorises.
static inline bool task_in_bounds(int64_t T, int64_t D, int64_t A, int64_t B, int64_t u, uint8_t type) {
  const uint64_t uT = (uint64_t)T, uD = (uint64_t)D, uA = (uint64_t)A, uB = (uint64_t)B, uu = (uint64_t)u;
  return (uT <= 0x7fffffffull) & (uD - 1ull < uT) & (uA <= (1ull << 36)) & (uB <= (1ull << 36)) &
         (uA + uB - 1ull < (1ull << 36)) & (uu <= 0xffffffffull) & (type <= 1);
}

// A fixed pool of host worker threads (created on first use, never torn
// down; calls are serialised) for the batch validation of host inputs.
namespace {
class HostPool {
 public:
  static HostPool& get() {
    static HostPool* pool = new HostPool();
    return *pool;
  }
  int workers() const { return (int)threads_.size(); }
  // fn(k) for k in [0, parts), on the workers and the calling thread.
  void run(int parts, const std::function<void(int)>& fn) {
    std::lock_guard<std::mutex> call(call_mu_);
    {
      std::lock_guard<std::mutex> lk(mu_);
      fn_ = &fn;
      parts_ = parts;
      next_.store(0);
      done_ = 0;
      gen_++;
    }
    cv_.notify_all();
    work();
    std::unique_lock<std::mutex> lk(mu_);
    done_cv_.wait(lk, [&] { return done_ == (int)threads_.size(); });
    fn_ = nullptr;
  }

 private:
  HostPool() {
    int n = (int)std::min<unsigned>(std::max(1u, std::thread::hardware_concurrency()), 32u) - 1;
    for (int i = 0; i < n; i++) threads_.emplace_back([this] { loop(); });
    for (auto& t : threads_) t.detach();
  }
  void work() {
    for (int k = next_.fetch_add(1); k < parts_; k = next_.fetch_add(1)) (*fn_)(k);
  }
  void loop() {
    unsigned long long seen = 0;
    for (;;) {
      {
        std::unique_lock<std::mutex> lk(mu_);
        cv_.wait(lk, [&] { return gen_ != seen; });
        seen = gen_;
      }
      work();
      std::lock_guard<std::mutex> lk(mu_);
      if (++done_ == (int)threads_.size()) done_cv_.notify_one();
    }
  }
  std::vector<std::thread> threads_;
  std::mutex call_mu_, mu_;
  std::condition_variable cv_, done_cv_;
  const std::function<void(int)>* fn_ = nullptr;
  int parts_ = 0, done_ = 0;
  std::atomic<int> next_{0};
  unsigned long long gen_ = 0;
};
}  // namespace

extern "C" int32_t gpa_validate(const gpa_tasksets* sets, const gpa_model* model, int64_t* bad_set) {
  if (bad_set) *bad_set = -1;
  if (!sets || !sets->set_off) return gpa_fail(GPA_ERR_ARG, "gpa_validate: NULL task sets");
  if (sets->mem != GPA_HOST) return gpa_fail(GPA_ERR_ARG, "gpa_validate: host arrays only");
  if (model && !model_valid(model)) return gpa_fail(GPA_ERR_RANGE, "gpa_validate: model out of range");
  if (sets->nsets < 0 || sets->n_max < 0 || sets->n_max > GPA_NMAX)
    return gpa_fail(GPA_ERR_RANGE, "gpa_validate: nsets/n_max out of range");
  if (sets->set_off[0] != 0) return gpa_fail(GPA_ERR_RANGE, "gpa_validate: set_off[0] != 0");
  if (sets->nsets > 0 && sets->set_off[sets->nsets] > 0 &&
      (!sets->T || !sets->D || !sets->A || !sets->B || !sets->type))
    return gpa_fail(GPA_ERR_ARG, "gpa_validate: NULL task column");
  const int64_t ns = sets->nsets;
  const int64_t* off = sets->set_off;
  // fast pass: every set size in [0, n_max], then (the offsets being
  // monotone) every task in bounds, in parallel ranges of sets
  const int64_t ntasks_hint = ns > 0 ? off[ns] : 0;
  const int parts = ntasks_hint >= 200000 ? 64 : 1;
  std::atomic<bool> bad{false};
  auto sizes_ok = [&](int64_t s0, int64_t s1) {
    bool ok = true;
    for (int64_t s = s0; s < s1; s++) {
      const int64_t n = off[s + 1] - off[s];
      ok &= (n >= 0) & (n <= sets->n_max);
    }
    return ok;
  };
  auto tasks_ok = [&](int64_t t0, int64_t t1) {
    bool ok = true;
    const int64_t *T = sets->T, *D = sets->D, *A = sets->A, *B = sets->B, *u = sets->u_ppm;
    const uint8_t* ty = sets->type;
    if (u) {
      for (int64_t t = t0; t < t1; t++) ok &= task_in_bounds(T[t], D[t], A[t], B[t], u[t], ty[t]);
    } else {
      for (int64_t t = t0; t < t1; t++) ok &= task_in_bounds(T[t], D[t], A[t], B[t], 0, ty[t]);
    }
    return ok;
  };
  std::function<void(int)> size_pass = [&](int k) {
    if (!sizes_ok(ns * k / parts, ns * (k + 1) / parts)) bad.store(true);
  };
  std::function<void(int)> task_pass = [&](int k) {
    const int64_t s0 = ns * k / parts, s1 = ns * (k + 1) / parts;
    if (!tasks_ok(off[s0], off[s1])) bad.store(true);
  };
  if (parts > 1) HostPool::get().run(parts, size_pass);
  else size_pass(0);
  if (!bad.load()) {
    if (parts > 1) HostPool::get().run(parts, task_pass);
    else task_pass(0);
  }
  if (!bad.load()) return GPA_OK;
  // slow path: the first invalid set
  for (int64_t s = 0; s < ns; s++) {
    const int64_t o = off[s], n = off[s + 1] - o;
    bool ok = n >= 0 && n <= sets->n_max;
    for (int64_t t = 0; ok && t < n; t++)
      ok = host_task_valid(sets->T[o + t], sets->D[o + t], sets->A[o + t], sets->B[o + t],
                           sets->u_ppm ? sets->u_ppm[o + t] : 0, sets->type[o + t]);
    if (!ok) {
      if (bad_set) *bad_set = s;
      return gpa_fail(GPA_ERR_RANGE, "gpa_validate: set %lld violates the bounds", (long long)s);
    }
  }
  return GPA_OK;
}

// ----------------------------------------------------------------- context

namespace gpa {
void build_reciprocals(MagicDivHost* t) {
  t[0] = MagicDivHost{0, 0, 0};
  for (int m = 1; m <= GPA_MMAX; m++) {
    unsigned long long d = 1000000ull * (unsigned long long)m;
    unsigned int l = 0;
    while ((1ull << l) < d) l++;
    unsigned __int128 num = ((unsigned __int128)1 << (60 + l)) + d - 1;
    t[m] = MagicDivHost{(unsigned long long)(num / d), l - 4, 0};
  }
}
}  // namespace gpa

static void build_mdiv(std::vector<MagicDivHost>& t) {
  t.assign(GPA_MMAX + 1, MagicDivHost{0, 0, 0});
  build_reciprocals(t.data());
}

extern "C" int32_t gpa_ctx_create(int32_t device, void* stream, gpa_ctx** out) {
  if (!out) return gpa_fail(GPA_ERR_ARG, "gpa_ctx_create: out is NULL");
  *out = nullptr;
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess) return gpa_cuda_fail(e, "cudaGetDeviceCount");
  if (device < 0 || device >= ndev) return gpa_fail(GPA_ERR_ARG, "gpa_ctx_create: no CUDA device %d", device);
  DeviceGuard guard(device);
  gpa_ctx* c = new gpa_ctx();
  c->device = device;
  c->stream = (cudaStream_t)stream;
  cudaDeviceProp prop;
  e = cudaGetDeviceProperties(&prop, device);
  if (e != cudaSuccess) { delete c; return gpa_cuda_fail(e, "cudaGetDeviceProperties"); }
  c->sm_count = prop.multiProcessorCount;
  std::vector<MagicDivHost> t;
  build_mdiv(t);
  if ((e = cudaMalloc(&c->d_mdiv, sizeof(MagicDivHost) * t.size())) != cudaSuccess ||
      (e = cudaMemcpy(c->d_mdiv, t.data(), sizeof(MagicDivHost) * t.size(), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (e = cudaMalloc(&c->d_counters, 8 * sizeof(unsigned long long))) != cudaSuccess ||
      (e = cudaMemset(c->d_counters, 0, 8 * sizeof(unsigned long long))) != cudaSuccess ||
      (e = cudaMalloc(&c->d_err, sizeof(unsigned int))) != cudaSuccess ||
      (e = cudaMemset(c->d_err, 0, sizeof(unsigned int))) != cudaSuccess) {
    gpa_ctx_destroy(c);
    return gpa_cuda_fail(e, "gpa_ctx_create: device allocation");
  }
  for (int i = 0; i < 4 && e == cudaSuccess; i++) e = cudaEventCreate(&c->prof.ev[i]);
  if (e != cudaSuccess) {
    gpa_ctx_destroy(c);
    return gpa_cuda_fail(e, "gpa_ctx_create: events");
  }
  static std::once_flag once;
  static cudaError_t init_err = cudaSuccess;
  std::call_once(once, [] {
    init_err = alloc_kernels_init();
    if (init_err == cudaSuccess) init_err = wide::alloc_kernels_init();
    if (init_err == cudaSuccess) init_err = small::alloc_kernels_init();
    if (init_err == cudaSuccess) init_err = search_kernels_init();
  });
  if (init_err != cudaSuccess) {
    gpa_ctx_destroy(c);
    return gpa_cuda_fail(init_err, "kernel attribute set-up");
  }
  *out = c;
  return GPA_OK;
}

static void destroy_graph(CachedGraph& g) {
  cudaGraphExecDestroy(g.exec);
  for (int i = 0; i < 4; i++)
    if (g.prof.ev[i]) cudaEventDestroy(g.prof.ev[i]);
}

// The timing events for the next call (nullptr when profiling is off).
static Prof* begin_prof(gpa_ctx* c) {
  if (!c->profile) return nullptr;
  c->prof.used = 0;
  c->prof.capture = false;
  c->last_prof = &c->prof;
  return &c->prof;
}

extern "C" int32_t gpa_ctx_last_timing(gpa_ctx* c, float* ms, int32_t n, int32_t* count) {
  if (!c || !count || (n > 0 && !ms)) return gpa_fail(GPA_ERR_ARG, "gpa_ctx_last_timing: NULL argument");
  *count = 0;
  const Prof* p = c->last_prof;
  if (!p || p->used < 2) return GPA_OK;
  DeviceGuard guard(c->device);
  cudaError_t e = cudaEventSynchronize(p->ev[p->used - 1]);
  if (e != cudaSuccess) return gpa_cuda_fail(e, "cudaEventSynchronize");
  int k = 0;
  for (int i = 0; i + 1 < p->used && k < n; i++, k++) {
    e = cudaEventElapsedTime(&ms[k], p->ev[i], p->ev[i + 1]);
    if (e != cudaSuccess) return gpa_cuda_fail(e, "cudaEventElapsedTime");
  }
  *count = k;
  return GPA_OK;
}

extern "C" int32_t gpa_ctx_last_terms(gpa_ctx* c, int64_t* terms) {
  if (!c || !terms) return gpa_fail(GPA_ERR_ARG, "gpa_ctx_last_terms: NULL argument");
  DeviceGuard guard(c->device);
  cudaError_t e = cudaStreamSynchronize(c->stream);
  unsigned long long v = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&v, c->d_counters + 4, sizeof v, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return gpa_cuda_fail(e, "gpa_ctx_last_terms");
  *terms = (int64_t)v;
  return GPA_OK;
}

extern "C" int32_t gpa_measure_alu_peak(gpa_ctx* c, gpa_alu_peak* out) {
  if (!c || !out) return gpa_fail(GPA_ERR_ARG, "gpa_measure_alu_peak: NULL argument");
  DeviceGuard guard(c->device);
  long long terms = 0;
  cudaError_t e = measure_alu_peak(c->sm_count, c->stream, &out->terms_per_s, &out->imad_per_s, &out->term_ms,
                                   &terms);
  if (e != cudaSuccess) return gpa_cuda_fail(e, "gpa_measure_alu_peak");
  out->terms = terms;
  return GPA_OK;
}

extern "C" int32_t gpa_ctx_destroy(gpa_ctx* c) {
  if (!c) return GPA_OK;
  DeviceGuard guard(c->device);
  gpa_serve_teardown(c);
  for (auto& kv : c->graphs) destroy_graph(kv.second);
  for (int i = 0; i < 4; i++)
    if (c->prof.ev[i]) cudaEventDestroy(c->prof.ev[i]);
  for (auto& b : c->bufs) cudaFree(b.ptr);
  for (cudaEvent_t ev : c->pipe_ev)
    if (ev) cudaEventDestroy(ev);
  if (c->h_err) cudaFreeHost(c->h_err);
  if (c->copy_in) cudaStreamDestroy(c->copy_in);
  if (c->copy_out) cudaStreamDestroy(c->copy_out);
  cudaFree(c->d_mdiv);
  cudaFree(c->d_counters);
  cudaFree(c->d_err);
  cudaFree(c->d_slow);
  delete c;
  return GPA_OK;
}

extern "C" int32_t gpa_ctx_set_stream(gpa_ctx* c, void* stream) {
  if (!c) return gpa_fail(GPA_ERR_ARG, "gpa_ctx_set_stream: NULL context");
  c->stream = (cudaStream_t)stream;
  return GPA_OK;
}

extern "C" int32_t gpa_ctx_launch_count(gpa_ctx* c, int64_t* out) {
  if (!c || !out) return gpa_fail(GPA_ERR_ARG, "gpa_ctx_launch_count: NULL argument");
  *out = c->launches;
  return GPA_OK;
}

extern "C" int32_t gpa_ctx_set_option(gpa_ctx* c, int32_t opt, int64_t value) {
  if (!c) return gpa_fail(GPA_ERR_ARG, "gpa_ctx_set_option: NULL context");
  switch (opt) {
    case GPA_OPT_AUTOTUNE: c->autotune = value != 0; break;
    case GPA_OPT_GRAPH: c->use_graph = value != 0; break;
    case GPA_OPT_FAST_WARPS:
      if (value != 0 && value != 1 && value != 2 && value != 4 && value != 8) return gpa_fail(GPA_ERR_RANGE, "warps");
      c->force_fast.warps_per_block = (int)value;
      break;
    case GPA_OPT_FAST_CHUNK:
      if (value < 0 || value > 64) return gpa_fail(GPA_ERR_RANGE, "chunk (task sets per tile, <= 64)");
      c->force_fast.chunk = (int)value;
      break;
    case GPA_OPT_FAST_BLOCKS:
      if (value < 0 || value > (1 << 20)) return gpa_fail(GPA_ERR_RANGE, "blocks");
      c->force_fast.blocks = (int)value;
      break;
    case GPA_OPT_FAST_STAGES:
      if (value < 0 || value > 5) return gpa_fail(GPA_ERR_RANGE, "stages (0 = tuned, 1 = direct loads, 2..5)");
      c->force_fast.stages = (int)value;
      break;
    case GPA_OPT_HOST_SLICES:
      if (value < 0 || value > 64) return gpa_fail(GPA_ERR_RANGE, "host slices (0 = by size, 1 = whole, <= 64)");
      c->host_slices = (int)value;
      break;
    case GPA_OPT_HOST_COPY:
      if (value < 0 || value > 256) return gpa_fail(GPA_ERR_RANGE, "host copy (0 = by kernel where page-locked, 1 = copies, <= 256)");
      c->host_copy = (int)value;
      break;
    case GPA_OPT_MERGE_WARPS:
      if (value < 0 || value > 8) return gpa_fail(GPA_ERR_RANGE, "merge warps per CTA (0 = tuned, 1..8)");
      c->force_merge.warps_per_block = (int)value;
      break;
    case GPA_OPT_MERGE_GROUP:
      if (value != 0 && value != 1 && value != 2 && value != 4 && value != 8)
        return gpa_fail(GPA_ERR_RANGE, "merge warps per set (0 = tuned, 1, 2, 4, 8)");
      c->force_merge.chunk = (int)value;
      break;
    case GPA_OPT_MERGE_BLOCKS:
      if (value < 0 || value > (1 << 20)) return gpa_fail(GPA_ERR_RANGE, "merge blocks");
      c->force_merge.blocks = (int)value;
      break;
    case GPA_OPT_MERGE_TOPFIRST:
      if (value < 0 || value > 2) return gpa_fail(GPA_ERR_RANGE, "merge top-size round (0 = tuned, 1 = off, 2 = on)");
      c->force_merge.stages = (int)value;
      break;
    case GPA_OPT_TEST_WARPS:
      if (value < 0 || value > 8) return gpa_fail(GPA_ERR_RANGE, "1G warps per CTA (0 = tuned, 1..8)");
      c->force_test_warps = (int)value;
      break;
    case GPA_OPT_PER_SET_LAUNCH: c->per_set_launch = value != 0; break;
    case GPA_OPT_PROFILE:
      c->profile = value != 0;
      if (!c->profile) c->last_prof = nullptr;
      break;
    default: return gpa_fail(GPA_ERR_ARG, "gpa_ctx_set_option: unknown option %d", opt);
  }
  return GPA_OK;
}

// The status a nonzero error word stands for; clears the word on the device.
static int32_t err_word_status(gpa_ctx* c, unsigned int err) {
  if (!err) return GPA_OK;
  cudaMemset(c->d_err, 0, sizeof(unsigned int));
  if (err & 2u)
    return gpa_fail(GPA_ERR_TIMEOUT, "a per-partition test hit its step limit: the sets concerned are undecided");
  if (err & 4u) return gpa_fail(GPA_ERR_TIMEOUT, "a pipeline barrier wait exceeded its time limit");
  return gpa_fail(GPA_ERR_RANGE, "a device-resident set failed validation");
}

extern "C" int32_t gpa_ctx_sync(gpa_ctx* c) {
  if (!c) return gpa_fail(GPA_ERR_ARG, "gpa_ctx_sync: NULL context");
  DeviceGuard guard(c->device);
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return gpa_cuda_fail(e, "cudaStreamSynchronize");
  unsigned int err = 0;
  e = cudaMemcpy(&err, c->d_err, sizeof err, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return gpa_cuda_fail(e, "read error word");
  return err_word_status(c, err);
}

// --------------------------------------------------------- scratch buffers

void* ctx_buffer(gpa_ctx* c, int slot, size_t bytes) {
  if (slot >= (int)c->bufs.size()) c->bufs.resize((size_t)slot + 1);
  CtxBuf& b = c->bufs[(size_t)slot];
  if (b.bytes < bytes) {
    if (b.ptr) cudaFree(b.ptr);
    b.ptr = nullptr;
    b.bytes = 0;
    size_t want = bytes < 256 ? 256 : bytes;
    if (cudaMalloc(&b.ptr, want) != cudaSuccess) return nullptr;
    b.bytes = want;
    c->graphs_dirty = true;  // cached graphs may hold the old pointer
  }
  return b.ptr;
}

static int32_t ensure_slow(gpa_ctx* c, long long nsets) {
  if (c->slow_cap >= nsets && c->d_slow) return GPA_OK;
  if (c->d_slow) cudaFree(c->d_slow);
  c->d_slow = nullptr;
  long long cap = nsets < 1024 ? 1024 : nsets;
  cudaError_t e = cudaMalloc(&c->d_slow, sizeof(long long) * (size_t)cap);
  if (e != cudaSuccess) {
    c->slow_cap = 0;
    return gpa_fail(GPA_ERR_NOMEM, "slow-queue allocation of %lld sets failed", cap);
  }
  c->slow_cap = cap;
  c->graphs_dirty = true;
  return GPA_OK;
}

// --------------------------------------------------- host <-> device staging

// The device address of host range [p, p + bytes) when both its first and its
// last byte lie in page-locked memory mapped for the current device (then the
// staging kernel may read or write it), else nullptr.  A caller's array is one
// allocation, page-locked as a whole or not at all.
static void* mapped_host(const void* p, size_t bytes) {
  if (!p || bytes == 0) return nullptr;
  cudaPointerAttributes a{}, b{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (a.type != cudaMemoryTypeHost || !a.devicePointer) return nullptr;
  const char* last = static_cast<const char*>(p) + bytes - 1;
  if (cudaPointerGetAttributes(&b, last) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (b.type != cudaMemoryTypeHost || static_cast<char*>(b.devicePointer) != static_cast<char*>(a.devicePointer) + (bytes - 1))
    return nullptr;
  return a.devicePointer;
}

// The copies of one direction on one stream: ranges whose host side is
// page-locked are gathered into one launch of the staging kernel, the others
// go to cudaMemcpyAsync (GPA_OPT_HOST_COPY = 1 sends every range there).
struct Mover {
  gpa_ctx* c;
  cudaStream_t st;
  bool to_device;
  bool engine;  // copy engine only
  StageList L{};
  unsigned long long widest = 0;
  cudaError_t e = cudaSuccess;

  Mover(gpa_ctx* ctx, cudaStream_t s, bool in, bool engine_only = false)
      : c(ctx), st(s), to_device(in), engine(engine_only || ctx->host_copy == 1) {}

  void add(void* dst, const void* src, size_t bytes) {
    if (e != cudaSuccess || bytes == 0) return;
    void* mapped = engine ? nullptr : mapped_host(to_device ? src : dst, bytes);
    if (mapped) {
      if (L.n == kStageRangesMax) flush();
      if (e != cudaSuccess) return;
      L.r[L.n++] = to_device ? StageRange{mapped, dst, bytes} : StageRange{src, mapped, bytes};
      if (bytes > widest) widest = bytes;
      return;
    }
    e = cudaMemcpyAsync(dst, src, bytes, to_device ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToHost, st);
  }
  // CTAs per range: one per 256 KB of the widest range, at most 16 (or the
  // count GPA_OPT_HOST_COPY forces)
  cudaError_t flush() {
    if (e == cudaSuccess && L.n > 0) {
      int blocks = c->host_copy >= 2 ? c->host_copy : (int)std::min<unsigned long long>(16, 1 + (widest >> 18));
      e = launch_stage_copy(L, blocks, st, &c->launches);
    }
    L.n = 0;
    widest = 0;
    return e;
  }
};

struct HostStage {
  DevSets ds{};
  long long ntasks = 0;
};

// Copy a host batch into context buffers (slots 0..6).
static int32_t stage_in(gpa_ctx* c, const gpa_tasksets* sets, HostStage* hs) {
  const long long ns = sets->nsets;
  const long long nt = sets->set_off[ns];
  hs->ntasks = nt;
  const size_t b8 = sizeof(long long) * (size_t)(nt > 0 ? nt : 1);
  long long* off = (long long*)ctx_buffer(c, 0, sizeof(long long) * (size_t)(ns + 1));
  long long* T = (long long*)ctx_buffer(c, 1, b8);
  long long* D = (long long*)ctx_buffer(c, 2, b8);
  long long* A = (long long*)ctx_buffer(c, 3, b8);
  long long* B = (long long*)ctx_buffer(c, 4, b8);
  long long* u = (long long*)ctx_buffer(c, 5, b8);
  unsigned char* ty = (unsigned char*)ctx_buffer(c, 6, (size_t)(nt > 0 ? nt : 1));
  if (!off || !T || !D || !A || !B || !u || !ty) return gpa_fail(GPA_ERR_NOMEM, "staging allocation failed");
  cudaStream_t st = c->stream;
  Mover mv(c, st, true);
  mv.add(off, sets->set_off, sizeof(long long) * (size_t)(ns + 1));
  if (nt > 0) {
    mv.add(T, sets->T, b8);
    mv.add(D, sets->D, b8);
    mv.add(A, sets->A, b8);
    mv.add(B, sets->B, b8);
    if (sets->u_ppm) mv.add(u, sets->u_ppm, b8);
    mv.add(ty, sets->type, (size_t)nt);
  }
  cudaError_t e = mv.flush();
  if (e == cudaSuccess && nt > 0 && !sets->u_ppm) e = cudaMemsetAsync(u, 0, b8, st);
  if (e != cudaSuccess) return gpa_cuda_fail(e, "host-to-device copy of task sets");
  hs->ds = DevSets{ns, sets->n_max, off, T, D, A, B, u, ty};
  return GPA_OK;
}

static DevSets dev_sets(const gpa_tasksets* s) {
  return DevSets{s->nsets, s->n_max, (const long long*)s->set_off, (const long long*)s->T, (const long long*)s->D,
                 (const long long*)s->A, (const long long*)s->B, (const long long*)s->u_ppm,
                 (const unsigned char*)s->type};
}

static int32_t finish_host_call(gpa_ctx* c) { return gpa_ctx_sync(c); }

static int32_t common_checks(gpa_ctx* c, const gpa_tasksets* sets, const gpa_model* model, const char* who) {
  if (!c) return gpa_fail(GPA_ERR_ARG, "%s: NULL context", who);
  if (!sets || !sets->set_off) return gpa_fail(GPA_ERR_ARG, "%s: NULL task sets", who);
  if (sets->mem != GPA_HOST && sets->mem != GPA_DEVICE) return gpa_fail(GPA_ERR_ARG, "%s: bad mem tag", who);
  if (!model_valid(model)) return gpa_fail(GPA_ERR_RANGE, "%s: model out of range", who);
  if (sets->nsets < 0 || sets->n_max < 0 || sets->n_max > GPA_NMAX)
    return gpa_fail(GPA_ERR_RANGE, "%s: nsets/n_max out of range", who);
  if (sets->mem == GPA_HOST) {
    // cheap structural checks here; the bounds of every task are checked by
    // stage_in_validated while the copies run
    if (sets->set_off[0] != 0) return gpa_fail(GPA_ERR_RANGE, "%s: set_off[0] != 0", who);
    if (sets->nsets > 0 && sets->set_off[sets->nsets] < 0)
      return gpa_fail(GPA_ERR_RANGE, "%s: negative task count", who);
  }
  return GPA_OK;
}

// Host inputs: copy the batch into context buffers, check its bounds there
// with one grid-stride kernel, and launch no computation when they fail (the
// host then names the first offending set with gpa_validate).  The copies
// and the check are waited for before the call goes on, so no transfer reads
// the caller's arrays after an early return.
static int32_t stage_in_validated(gpa_ctx* c, const gpa_tasksets* sets, const gpa_model* model, HostStage* hs) {
  int32_t st = GPA_OK;
  if (sets->nsets > 0 && sets->set_off[sets->nsets] > 0 &&
      (!sets->T || !sets->D || !sets->A || !sets->B || !sets->type))
    return gpa_fail(GPA_ERR_ARG, "NULL task column");
  if ((st = stage_in(c, sets, hs)) != GPA_OK) return st;
  unsigned int* dflag = (unsigned int*)ctx_buffer(c, 29, sizeof(unsigned int));
  if (!dflag) return gpa_fail(GPA_ERR_NOMEM, "validation flag allocation failed");
  cudaError_t e = launch_validate_batch(hs->ds, dflag, c->sm_count, c->stream, &c->launches);
  unsigned int flag = 0u;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&flag, dflag, sizeof flag, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return gpa_cuda_fail(e, "batch validation");
  if (flag) {
    int64_t bad = -1;
    st = gpa_validate(sets, model, &bad);
    return st != GPA_OK ? st : gpa_fail(GPA_ERR_RANGE, "a set violates the bounds");
  }
  return GPA_OK;
}

// -------------------------------------------------------------- WCET tables

extern "C" int32_t gpa_build_wcet_tables(gpa_ctx* c, const gpa_tasksets* sets, const gpa_model* model, int64_t* Cn,
                                         int64_t* Cc) {
  int32_t st = common_checks(c, sets, model, "gpa_build_wcet_tables");
  if (st != GPA_OK) return st;
  if (sets->nsets == 0) return GPA_OK;
  if (!Cn || !Cc) return gpa_fail(GPA_ERR_ARG, "gpa_build_wcet_tables: NULL output");
  DeviceGuard guard(c->device);
  DevModel md;
  if ((st = device_model(c, model, &md)) != GPA_OK) return st;
  const long long Mu = model->M / model->g;
  if (sets->mem == GPA_DEVICE) {
    cudaError_t e = launch_wcet_tables(dev_sets(sets), md, (long long*)Cn, (long long*)Cc, c->d_err, c->d_mdiv,
                                       c->sm_count, c->stream, &c->launches, begin_prof(c));
    return e == cudaSuccess ? GPA_OK : gpa_cuda_fail(e, "wcet_tables launch");
  }
  HostStage hs;
  if ((st = stage_in_validated(c, sets, model, &hs)) != GPA_OK) return st;
  const size_t bytes = sizeof(long long) * (size_t)(hs.ntasks * Mu > 0 ? hs.ntasks * Mu : 1);
  long long* dCn = (long long*)ctx_buffer(c, 7, bytes);
  long long* dCc = (long long*)ctx_buffer(c, 8, bytes);
  if (!dCn || !dCc) return gpa_fail(GPA_ERR_NOMEM, "table allocation failed");
  cudaError_t e = launch_wcet_tables(hs.ds, md, dCn, dCc, c->d_err, c->d_mdiv, c->sm_count, c->stream, &c->launches,
                                     begin_prof(c));
  if (e == cudaSuccess && hs.ntasks * Mu > 0) {
    e = cudaMemcpyAsync(Cn, dCn, sizeof(long long) * (size_t)(hs.ntasks * Mu), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(Cc, dCc, sizeof(long long) * (size_t)(hs.ntasks * Mu), cudaMemcpyDeviceToHost, c->stream);
  }
  if (e != cudaSuccess) return gpa_cuda_fail(e, "wcet_tables");
  return finish_host_call(c);
}

// ------------------------------------------------------- explicit candidates

extern "C" int32_t gpa_test_schedulable(gpa_ctx* c, const gpa_tasksets* sets, const gpa_model* model,
                                        const gpa_candidates* cands, uint8_t* verdict, int64_t* R) {
  int32_t st = common_checks(c, sets, model, "gpa_test_schedulable");
  if (st != GPA_OK) return st;
  if (!cands) return gpa_fail(GPA_ERR_ARG, "gpa_test_schedulable: NULL candidates");
  if (cands->mem != sets->mem) return gpa_fail(GPA_ERR_ARG, "gpa_test_schedulable: candidates and sets differ in mem");
  if (cands->ncands < 0 || cands->kparts < 1 || cands->kparts > 255 || cands->map_stride < 1 ||
      cands->map_stride > 65536)
    return gpa_fail(GPA_ERR_RANGE, "gpa_test_schedulable: candidate shape out of range");
  if (cands->ncands == 0) return GPA_OK;
  if (!verdict || !cands->set || !cands->part_of_task || !cands->size_of_part)
    return gpa_fail(GPA_ERR_ARG, "gpa_test_schedulable: NULL array");
  DeviceGuard guard(c->device);
  DevModel md;
  if ((st = device_model(c, model, &md)) != GPA_OK) return st;
  const long long nc = cands->ncands;
  if (sets->mem == GPA_DEVICE) {
    Cands cc{nc, cands->map_stride, cands->kparts, (const long long*)cands->set, cands->part_of_task,
             cands->size_of_part};
    cudaError_t e = (sets->n_max > kNarrowNmax ? wide::launch_test_schedulable : launch_test_schedulable)(
        dev_sets(sets), md, cc, verdict, (long long*)R, c->d_err, c->d_mdiv, c->sm_count, c->stream, &c->launches,
        begin_prof(c));
    return e == cudaSuccess ? GPA_OK : gpa_cuda_fail(e, "test_schedulable launch");
  }
  // host path: validate candidates on the host too
  for (long long i = 0; i < nc; i++) {
    long long s = cands->set[i];
    if (s < 0 || s >= sets->nsets) return gpa_fail(GPA_ERR_RANGE, "candidate %lld: bad set index", i);
    long long n = sets->set_off[s + 1] - sets->set_off[s];
    if (n > cands->map_stride) return gpa_fail(GPA_ERR_RANGE, "candidate %lld: map_stride < tasks", i);
    for (long long t = 0; t < n; t++)
      if (cands->part_of_task[i * cands->map_stride + t] >= cands->kparts)
        return gpa_fail(GPA_ERR_RANGE, "candidate %lld: part index out of range", i);
    for (int p = 0; p < cands->kparts; p++) {
      int z = cands->size_of_part[i * cands->kparts + p];
      bool ok = z == 0 || (z >= model->g && z <= model->M && z % model->g == 0);
      if (ok && z != 0 && model->nsizes > 0) ok = std::binary_search(model->sizes, model->sizes + model->nsizes, z);
      if (!ok) return gpa_fail(GPA_ERR_RANGE, "candidate %lld: part size not admissible", i);
    }
  }
  HostStage hs;
  if ((st = stage_in_validated(c, sets, model, &hs)) != GPA_OK) return st;
  long long* dset = (long long*)ctx_buffer(c, 9, sizeof(long long) * (size_t)nc);
  unsigned char* dmap = (unsigned char*)ctx_buffer(c, 10, (size_t)(nc * cands->map_stride));
  int* dsize = (int*)ctx_buffer(c, 11, sizeof(int) * (size_t)(nc * cands->kparts));
  unsigned char* dver = (unsigned char*)ctx_buffer(c, 12, (size_t)nc);
  long long* dR = R ? (long long*)ctx_buffer(c, 13, sizeof(long long) * (size_t)(nc * cands->map_stride)) : nullptr;
  if (!dset || !dmap || !dsize || !dver || (R && !dR)) return gpa_fail(GPA_ERR_NOMEM, "candidate staging failed");
  cudaStream_t s = c->stream;
  cudaError_t e = cudaMemcpyAsync(dset, cands->set, sizeof(long long) * (size_t)nc, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(dmap, cands->part_of_task, (size_t)(nc * cands->map_stride), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(dsize, cands->size_of_part, sizeof(int) * (size_t)(nc * cands->kparts),
                        cudaMemcpyHostToDevice, s);
  Cands cc{nc, cands->map_stride, cands->kparts, dset, dmap, dsize};
  if (e == cudaSuccess)
    e = (hs.ds.n_max > kNarrowNmax ? wide::launch_test_schedulable : launch_test_schedulable)(
        hs.ds, md, cc, dver, dR, c->d_err, c->d_mdiv, c->sm_count, s, &c->launches, begin_prof(c));
  if (e == cudaSuccess) e = cudaMemcpyAsync(verdict, dver, (size_t)nc, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && R)
    e = cudaMemcpyAsync(R, dR, sizeof(long long) * (size_t)(nc * cands->map_stride), cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return gpa_cuda_fail(e, "test_schedulable");
  return finish_host_call(c);
}

// --------------------------------------------------------------- allocate

// blocks = 0: the launcher sizes the grid to the kernel's occupancy x SMs
static LaunchShape default_fast(const gpa_ctx* c) {
  (void)c;
  return LaunchShape{4, 2, 0, 1};
}

std::string tune_key(const DevSets& ds, const DevModel& md, const gpa_params& p) {
  char buf[160];
  std::snprintf(buf, sizeof buf, "alloc:%lld:%d:%d:%d:%d:%d:%d:%d:%d", ds.nsets, ds.n_max, md.M, md.g, p.policy,
                p.act, md.sched, md.nz, p.linear_merge);
  return buf;
}

// The launchers of the batch's task capacity: the 64-task build when n_max
// is at most 64, the 256-task build when it exceeds 128, else the 128-task
// build.
using AllocLauncher = cudaError_t (*)(const DevSets&, const DevModel&, const gpa_params&, const AllocOut&,
                                      const AllocQueue&, const MagicDivHost*, const LaunchShape&, const LaunchShape&,
                                      cudaStream_t, long long*, Prof*);
static AllocLauncher allocate_launcher(int n_max) {
  return n_max > kNarrowNmax ? wide::launch_allocate : n_max <= kSmallNmax ? small::launch_allocate : launch_allocate;
}
static int merge_ctas(int n_max, int wpb, int gw) {
  return n_max > kNarrowNmax ? wide::merge_ctas_per_sm(wpb, gw)
                             : n_max <= kSmallNmax ? small::merge_ctas_per_sm(wpb, gw) : merge_ctas_per_sm(wpb, gw);
}
static int one_gpu_ctas(int n_max, int wpb) {
  return n_max > kNarrowNmax ? wide::one_gpu_ctas_per_sm(wpb)
                             : n_max <= kSmallNmax ? small::one_gpu_ctas_per_sm(wpb) : one_gpu_ctas_per_sm(wpb);
}

// Merge kernel: wpb warps per CTA in groups of gw warps per set, as many
// CTAs per SM as fit (at most `cap`).
static LaunchShape merge_shape(const gpa_ctx* c, int n_max, int wpb, int gw, int cap) {
  int per_sm = merge_ctas(n_max, wpb, gw);
  if (cap > 0 && per_sm > cap) per_sm = cap;
  return LaunchShape{wpb, gw, c->sm_count * (per_sm > 0 ? per_sm : 1), 1};
}

// Library defaults per capacity build: one warp per set; the 256-task build
// keeps 58 KB of shared memory per set (one-warp CTAs, up to three per SM),
// the 64-task build 10 KB and 128 registers (four-warp CTAs), the 128-task
// build 22 KB (two-warp CTAs, up to five per SM), as many as the registers
// and shared memory allow; the 64-task build opens SMS steps with the
// top-size round (merge_set).  The 1G kernel: eight-warp CTAs, as many as fit.
static AllocShapes default_shapes(const gpa_ctx* c, const DevSets& ds) {
  AllocShapes sh;
  sh.fast = default_fast(c);
  const bool wide_sets = ds.n_max > kNarrowNmax, small_sets = ds.n_max <= kSmallNmax;
  sh.slow = wide_sets ? merge_shape(c, ds.n_max, 1, 1, 3)
                      : small_sets ? merge_shape(c, ds.n_max, 4, 1, 0) : merge_shape(c, ds.n_max, 2, 1, 5);
  if (small_sets) sh.slow.stages = 2;  // the SMS top-size round
  const int per_sm = one_gpu_ctas(ds.n_max, 8);
  sh.one = LaunchShape{8, 1, c->sm_count * (per_sm > 0 ? per_sm : 1), 1};
  return sh;
}

// The shapes of a call: tuned for its signature when the autotuner ran,
// else the defaults; forced options override either.
static AllocShapes call_shapes(gpa_ctx* c, const DevSets& ds, const DevModel& md, const gpa_params& p) {
  AllocShapes sh = default_shapes(c, ds);
  auto it = c->tuned.find(tune_key(ds, md, p));
  if (it != c->tuned.end()) sh = it->second;
  if (c->force_fast.warps_per_block) sh.fast.warps_per_block = c->force_fast.warps_per_block;
  if (c->force_fast.chunk) sh.fast.chunk = c->force_fast.chunk;
  if (c->force_fast.blocks) sh.fast.blocks = c->force_fast.blocks;
  if (c->force_fast.stages) sh.fast.stages = c->force_fast.stages;
  if (c->force_merge.warps_per_block || c->force_merge.chunk || c->force_merge.blocks) {
    const int gw = c->force_merge.chunk ? c->force_merge.chunk : sh.slow.chunk;
    int wpb = c->force_merge.warps_per_block ? c->force_merge.warps_per_block : sh.slow.warps_per_block;
    if (wpb < gw || wpb % gw) wpb = gw;
    // the largest multiple of the group width up to wpb whose CTA fits an SM
    while (wpb > gw && merge_ctas(ds.n_max, wpb, gw) <= 0) wpb -= gw;
    const int stages = sh.slow.stages;
    sh.slow = merge_shape(c, ds.n_max, wpb, gw, 0);
    sh.slow.stages = stages;
    if (c->force_merge.blocks) sh.slow.blocks = c->force_merge.blocks;
  }
  if (c->force_merge.stages) sh.slow.stages = c->force_merge.stages;
  if (c->force_test_warps) {
    const int w = c->force_test_warps;
    const int per_sm = one_gpu_ctas(ds.n_max, w);
    sh.one = LaunchShape{w, 1, c->sm_count * (per_sm > 0 ? per_sm : 1), 1};
  }
  return sh;
}

static cudaError_t run_allocate(gpa_ctx* c, const DevSets& ds, const DevModel& md, const gpa_params& p,
                                const AllocOut& out, const AllocShapes& sh, Prof* prof) {
  AllocQueue q{c->d_counters, c->d_slow, c->d_err};
  const bool wide_sets = ds.n_max > kNarrowNmax, small_sets = ds.n_max <= kSmallNmax;
  if (p.policy == GPA_POLICY_ONE_GPU)
    return (wide_sets ? wide::launch_one_gpu : small_sets ? small::launch_one_gpu : launch_one_gpu)(
        ds, md, out, q, c->d_mdiv, sh.one, c->stream, &c->launches, prof);
  return allocate_launcher(ds.n_max)(ds, md, p, out, q, c->d_mdiv, sh.fast, sh.slow, c->stream, &c->launches, prof);
}

// Mean device time (ms) of `reps` runs after one untimed run.
static float time_allocate(gpa_ctx* c, const DevSets& ds, const DevModel& md, const gpa_params& p, const AllocOut& out,
                           const AllocShapes& sh, int reps, cudaEvent_t e0, cudaEvent_t e1) {
  run_allocate(c, ds, md, p, out, sh, nullptr);
  cudaEventRecord(e0, c->stream);
  for (int r = 0; r < reps; r++) run_allocate(c, ds, md, p, out, sh, nullptr);
  cudaEventRecord(e1, c->stream);
  if (cudaEventSynchronize(e1) != cudaSuccess) return 1e30f;
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  return ms / (float)reps;
}

// Autotuner: on the first call of a batch signature, time the candidate
// launch shapes of the kernels the call runs on this batch (every shape
// computes the same result) and keep the fastest for the signature:
//  * 1G: warps per CTA of the test kernel (1, 2, 4, 8; CTAs per SM by
//    occupancy);
//  * heuristic: the fast kernel (direct loads: warps {4, 8} x sets per
//    ticket {1, 2, 3, 4, 8}; staged: compute warps {4, 8} x sets {1, 2, 4} x
//    stages {2, 3}), then the merge kernel with the best of those: warps per
//    set {1, 2, 4, 8} x warps per CTA (multiples of it, up to 8) x CTAs per
//    SM (as many as fit, or half of that), then the SMS top-size round on
//    and off.
// The merge kernel's shapes are tried while the time spent tuning stays
// below max(50 ms, 8 x the default run): a batch whose merges take seconds
// keeps the shapes tried by then.
static void autotune_allocate(gpa_ctx* c, const DevSets& ds, const DevModel& md, const gpa_params& p,
                              const AllocOut& out) {
  const std::string key = tune_key(ds, md, p);
  if (c->tuned.count(key)) return;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  AllocShapes best = default_shapes(c, ds);
  float best_ms = time_allocate(c, ds, md, p, out, best, 2, e0, e1);
  if (p.policy == GPA_POLICY_ONE_GPU) {
    for (int w : {1, 2, 4, 8}) {
      AllocShapes t = best;
      const int per_sm = one_gpu_ctas(ds.n_max, w);
      if (per_sm <= 0) continue;
      t.one = LaunchShape{w, 1, c->sm_count * per_sm, 1};
      const float ms = time_allocate(c, ds, md, p, out, t, 2, e0, e1);
      if (ms < best_ms) {
        best_ms = ms;
        best = t;
      }
    }
  } else {
    std::vector<LaunchShape> shapes;
    for (int w : {4, 8})
      for (int ch : {1, 2, 3, 4, 8}) shapes.push_back(LaunchShape{w, ch, 0, 1});
    for (int w : {4, 8})
      for (int ch : {1, 2, 4})
        for (int stg : {2, 3}) shapes.push_back(LaunchShape{w, ch, 0, stg});
    for (const LaunchShape& f : shapes) {
      AllocShapes t = best;
      t.fast = f;
      const float ms = time_allocate(c, ds, md, p, out, t, 2, e0, e1);
      if (ms < best_ms) {
        best_ms = ms;
        best = t;
      }
    }
    const float budget = std::max(50.f, 8.f * best_ms);
    float spent = 0.f;
    for (int gw : {1, 2, 4, 8})
      for (int wpb = gw; wpb <= 8 && spent < budget; wpb += gw) {
        const int full = merge_ctas(ds.n_max, wpb, gw);
        if (full <= 0) continue;
        for (int cap : {full, full / 2}) {
          if (cap <= 0 || spent >= budget || (cap == full / 2 && cap == full)) continue;
          AllocShapes t = best;
          t.slow = merge_shape(c, ds.n_max, wpb, gw, cap);
          if (t.slow.warps_per_block == best.slow.warps_per_block && t.slow.chunk == best.slow.chunk &&
              t.slow.blocks == best.slow.blocks)
            continue;
          const float ms = time_allocate(c, ds, md, p, out, t, 1, e0, e1);
          spent += 2.f * ms;
          if (ms < best_ms) {
            best_ms = ms;
            best = t;
          }
        }
      }
    // the SMS top-size round on or off, with the best of those shapes
    AllocShapes t = best;
    t.slow.stages = best.slow.stages == 2 ? 1 : 2;
    const float ms = time_allocate(c, ds, md, p, out, t, 1, e0, e1);
    if (ms < best_ms) {
      best_ms = ms;
      best = t;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c->tuned[key] = best;
}

static std::string graph_key(const DevSets& ds, const DevModel& md, const gpa_params& p, const AllocOut& o,
                             const AllocShapes& sh) {
  char buf[640];
  std::snprintf(buf, sizeof buf, "%lld|%d|%p|%p|%p|%p|%p|%p|%p|%d|%d|%d|%d|%d|%d|%p|%d|%d|%d|%p|%p|%p|%p|%p|%p|%p|%p|%d|%d|%d|%d|%d|%d|%d|%d|%d|%d",
                ds.nsets, ds.n_max, (const void*)ds.set_off, (const void*)ds.T, (const void*)ds.D,
                (const void*)ds.A, (const void*)ds.B, (const void*)ds.u, (const void*)ds.type, md.M, md.g, md.kc,
                md.km, md.sched, md.nz, (const void*)md.zlist, p.policy, p.act, p.linear_merge, (void*)o.verdict, (void*)o.reason, (void*)o.n_parts,
                (void*)o.Pi, (void*)o.W, (void*)o.n_tests, (void*)o.part_of_task, (void*)o.size_of_part,
                sh.fast.warps_per_block, sh.fast.chunk, sh.fast.blocks, sh.fast.stages, sh.slow.warps_per_block,
                sh.slow.chunk, sh.slow.blocks, sh.one.warps_per_block, sh.one.blocks, sh.slow.stages);
  return buf;
}

static int32_t allocate_device(gpa_ctx* c, const DevSets& ds, const DevModel& md, const gpa_params& p,
                               const AllocOut& out) {
  int32_t st = ensure_slow(c, ds.nsets);
  if (st != GPA_OK) return st;
  if (c->per_set_launch && p.policy != GPA_POLICY_ONE_GPU) {
    // the plain form: one launch sequence per task set
    for (long long s = 0; s < ds.nsets; s++) {
      DevSets one = ds;
      one.nsets = 1;
      one.set_off = ds.set_off + s;
      AllocOut o1 = out;
      o1.verdict += s;
      o1.reason += s;
      o1.n_parts += s;
      o1.Pi += s;
      o1.W += s;
      if (o1.n_tests) o1.n_tests += s;
      LaunchShape one_shape{1, 1, 1, 1};
      AllocQueue q{c->d_counters, c->d_slow, c->d_err};
      LaunchShape slow1{1, 1, 1, 1};
      cudaError_t e = allocate_launcher(one.n_max)(one, md, p, o1, q, c->d_mdiv, one_shape, slow1, c->stream,
                                                   &c->launches, nullptr);
      if (e != cudaSuccess) return gpa_cuda_fail(e, "per-set allocate launch");
    }
    return GPA_OK;
  }
  if (c->autotune) autotune_allocate(c, ds, md, p, out);
  const AllocShapes shapes = call_shapes(c, ds, md, p);
  if (c->use_graph) {
    if (c->graphs_dirty) {
      for (auto& kv : c->graphs) destroy_graph(kv.second);
      c->graphs.clear();
      c->last_prof = nullptr;
      c->graphs_dirty = false;
    }
    const std::string key = graph_key(ds, md, p, out, shapes) + (c->profile ? "|prof" : "");
    auto it = c->graphs.find(key);
    if (it == c->graphs.end()) {
      Prof gp{};
      gp.capture = true;
      if (c->profile)
        for (int i = 0; i < 4; i++) {
          cudaError_t ee = cudaEventCreate(&gp.ev[i]);
          if (ee != cudaSuccess) return gpa_cuda_fail(ee, "graph timing events");
        }
      cudaGraph_t g = nullptr;
      cudaError_t e = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal);
      if (e != cudaSuccess) return gpa_cuda_fail(e, "cudaStreamBeginCapture (graphs need a non-default stream)");
      long long before = c->launches;
      cudaError_t le = run_allocate(c, ds, md, p, out, shapes, c->profile ? &gp : nullptr);
      long long kernels = c->launches - before;
      c->launches = before;
      e = cudaStreamEndCapture(c->stream, &g);
      if (le != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return gpa_cuda_fail(le, "allocate capture");
      }
      if (e != cudaSuccess) return gpa_cuda_fail(e, "cudaStreamEndCapture");
      cudaGraphExec_t exec = nullptr;
      e = cudaGraphInstantiate(&exec, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) return gpa_cuda_fail(e, "cudaGraphInstantiate");
      it = c->graphs.emplace(key, CachedGraph{exec, kernels, gp}).first;
    }
    cudaError_t e = cudaGraphLaunch(it->second.exec, c->stream);
    if (e != cudaSuccess) return gpa_cuda_fail(e, "cudaGraphLaunch");
    c->launches += it->second.kernels;
    c->last_prof = it->second.prof.used ? &it->second.prof : nullptr;
    return GPA_OK;
  }
  cudaError_t e = run_allocate(c, ds, md, p, out, shapes, begin_prof(c));
  return e == cudaSuccess ? GPA_OK : gpa_cuda_fail(e, "allocate launch");
}

// ------------------------------------------- allocate on host buffers, sliced

// gpa_allocate on host buffers.  The batch's sets are checked by the kernels
// that compute them (as for device inputs), so no pass over the batch
// precedes the computation and the call waits for the GPU once, at its end.
// A batch with more than 3/4 of kSliceBytes of task columns is split into
// max(2, ceil(bytes / kSliceBytes)) slices (at most kAutoSlicesMax): slice j's
// copy in, its kernels and its copy out run on three streams, so the host
// link carries slice j + 1 in while slice j computes and slice j - 1 goes
// out.  Each slice costs a few launches and waits, and the two directions of
// the link share its bandwidth, so a few large slices do best.  GPA_OPT_HOST_SLICES = 1 selects the
// whole-batch form instead: copy, check on the device, then compute only if
// every set passed.
static const long long kSliceBytes = 64ll << 20;
static const int kAutoSlicesMax = 16;

// Set boundaries 0 = b[0] < b[1] < ... < b[S] = nsets balancing the task
// count (S = 1 for a batch that is not split); an empty vector selects the
// whole-batch form.  set_off is not yet checked, so every boundary's task
// offset is checked to lie in [0, ntasks] and not to decrease (a batch that
// fails this takes the whole-batch form, whose check rejects it).
static std::vector<long long> slice_bounds(const gpa_ctx* c, const gpa_tasksets* sets) {
  const long long ns = sets->nsets, nt = sets->set_off[ns];
  long long S = c->host_slices;
  if (S == 1) return {};
  if (S == 0) {
    const long long bytes = 41 * nt + 8 * ns;
    S = 4 * bytes <= 3 * kSliceBytes
            ? 1
            : std::min<long long>(std::max(2ll, (bytes + kSliceBytes - 1) / kSliceBytes), kAutoSlicesMax);
  }
  S = std::max(1ll, std::min(S, ns));
  std::vector<long long> b{0};
  for (long long j = 1; j < S; j++) {
    const long long target = nt / S * j + nt % S * j / S;
    long long lo = b.back() + 1, hi = ns - 1;  // first set index in [lo, hi] whose offset reaches target
    if (lo > hi) break;
    while (lo < hi) {
      const long long mid = lo + (hi - lo) / 2;
      if (sets->set_off[mid] < target) lo = mid + 1;
      else hi = mid;
    }
    b.push_back(lo);
  }
  b.push_back(ns);
  for (size_t j = 0; j + 1 < b.size(); j++) {
    const long long t0 = sets->set_off[b[j]], t1 = sets->set_off[b[j + 1]];
    if (b[j + 1] <= b[j] || t0 < 0 || t1 < t0 || t1 > nt) return {};
  }
  return b;
}

static int32_t ensure_pipe(gpa_ctx* c) {
  cudaError_t e = cudaSuccess;
  if (!c->copy_in) e = cudaStreamCreateWithFlags(&c->copy_in, cudaStreamNonBlocking);
  if (e == cudaSuccess && !c->copy_out) e = cudaStreamCreateWithFlags(&c->copy_out, cudaStreamNonBlocking);
  for (int i = 0; i < 3 && e == cudaSuccess; i++)
    if (!c->pipe_ev[i]) e = cudaEventCreateWithFlags(&c->pipe_ev[i], cudaEventDisableTiming);
  if (e == cudaSuccess && !c->h_err) e = cudaHostAlloc((void**)&c->h_err, 64, cudaHostAllocDefault);
  return e == cudaSuccess ? GPA_OK : gpa_cuda_fail(e, "copy streams");
}

// Device buffers that receive policy k's results on the host path: slots
// 14..21 for the first policy of a call, 40 + 8 (k - 1) .. 47 + 8 (k - 1)
// for the others.
static int32_t host_out_bufs(gpa_ctx* c, int k, long long ns, long long nt, bool tests, AllocOut* out) {
  const int b = k == 0 ? 14 : 40 + 8 * (k - 1);
  const size_t nsb = (size_t)(ns > 0 ? ns : 1), ntb = (size_t)(nt > 0 ? nt : 1);
  *out = AllocOut{(unsigned char*)ctx_buffer(c, b, nsb), (unsigned char*)ctx_buffer(c, b + 1, nsb),
                  (int*)ctx_buffer(c, b + 2, sizeof(int) * nsb), (int*)ctx_buffer(c, b + 3, sizeof(int) * nsb),
                  (long long*)ctx_buffer(c, b + 4, sizeof(long long) * nsb),
                  tests ? (int*)ctx_buffer(c, b + 5, sizeof(int) * nsb) : nullptr,
                  (unsigned char*)ctx_buffer(c, b + 6, ntb), (short*)ctx_buffer(c, b + 7, sizeof(short) * ntb)};
  if (!out->verdict || !out->reason || !out->n_parts || !out->Pi || !out->W || (tests && !out->n_tests) ||
      !out->part_of_task || !out->size_of_part)
    return gpa_fail(GPA_ERR_NOMEM, "result staging failed");
  return GPA_OK;
}

// Queue the copies of sets [s0, s1) (tasks [t0, t1)) of one policy's results
// from its device buffers to the caller's arrays.
static void copy_out_range(Mover& mo, const gpa_alloc_result& r, const AllocOut& out, long long s0, long long s1,
                           long long t0, long long t1) {
  const size_t m = (size_t)(s1 - s0), n = (size_t)(t1 - t0);
  mo.add(r.verdict + s0, out.verdict + s0, m);
  mo.add(r.reason + s0, out.reason + s0, m);
  mo.add(r.n_parts + s0, out.n_parts + s0, sizeof(int) * m);
  mo.add(r.Pi + s0, out.Pi + s0, sizeof(int) * m);
  mo.add(r.W + s0, out.W + s0, sizeof(long long) * m);
  if (r.n_tests) mo.add(r.n_tests + s0, out.n_tests + s0, sizeof(int) * m);
  mo.add(r.part_of_task + t0, out.part_of_task + t0, n);
  mo.add(r.size_of_part + t0, out.size_of_part + t0, sizeof(short) * n);
}

// Host arrays in slices b[j] .. b[j + 1]: slice j + 1's columns are copied in
// while slice j is decided, under each of the np policies in turn, and slice
// j's results of every policy are copied out while slice j + 1 is decided.
static int32_t allocate_host_sliced(gpa_ctx* c, const gpa_tasksets* sets, const gpa_model* model,
                                    const DevModel& md, const gpa_params* p, int np, gpa_alloc_result* r,
                                    const std::vector<long long>& b) {
  const long long ns = sets->nsets, nt = sets->set_off[ns];
  if (nt > 0 && (!sets->T || !sets->D || !sets->A || !sets->B || !sets->type))
    return gpa_fail(GPA_ERR_ARG, "NULL task column");
  int32_t st = ensure_pipe(c);
  if (st != GPA_OK) return st;
  if ((st = ensure_slow(c, ns)) != GPA_OK) return st;
  const size_t b8 = sizeof(long long) * (size_t)(nt > 0 ? nt : 1);
  long long* off = (long long*)ctx_buffer(c, 0, sizeof(long long) * (size_t)(ns + 1));
  long long* T = (long long*)ctx_buffer(c, 1, b8);
  long long* D = (long long*)ctx_buffer(c, 2, b8);
  long long* A = (long long*)ctx_buffer(c, 3, b8);
  long long* B = (long long*)ctx_buffer(c, 4, b8);
  long long* u = (long long*)ctx_buffer(c, 5, b8);
  unsigned char* ty = (unsigned char*)ctx_buffer(c, 6, (size_t)(nt > 0 ? nt : 1));
  if (!off || !T || !D || !A || !B || !u || !ty) return gpa_fail(GPA_ERR_NOMEM, "staging allocation failed");
  AllocOut outs[GPA_MULTI_MAX_POLICIES];
  bool one_gpu = false;
  for (int k = 0; k < np; k++) {
    if ((st = host_out_bufs(c, k, ns, nt, r[k].n_tests != nullptr, &outs[k])) != GPA_OK) return st;
    one_gpu = one_gpu || p[k].policy == GPA_POLICY_ONE_GPU;
  }
  cudaStream_t in = c->copy_in, cs = c->stream, ot = c->copy_out;
  cudaEvent_t ev_start = c->pipe_ev[0], ev_in = c->pipe_ev[1], ev_done = c->pipe_ev[2];
  // Every wait below is issued right after the record it waits for, so the
  // three events serve all slices.
  cudaError_t e = cudaEventRecord(ev_start, cs);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(in, ev_start, 0);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(ot, ev_start, 0);
  // The staging kernel needs SM slots while the previous slice computes; the
  // 1G kernel holds every SM for its whole slice, so its slices move by copy
  // engine (unless GPA_OPT_HOST_COPY forces the kernel).
  const bool engine = one_gpu && c->host_copy < 2 && b.size() > 2;
  Mover mi(c, in, true, engine), mo(c, ot, false, engine);
  mi.add(off, sets->set_off, sizeof(long long) * (size_t)(ns + 1));
  st = GPA_OK;
  for (size_t j = 0; j + 1 < b.size() && e == cudaSuccess && st == GPA_OK; j++) {
    const long long s0 = b[j], s1 = b[j + 1], t0 = sets->set_off[s0], t1 = sets->set_off[s1];
    const size_t n = (size_t)(t1 - t0), n8 = sizeof(long long) * n;
    mi.add(T + t0, sets->T + t0, n8);
    mi.add(D + t0, sets->D + t0, n8);
    mi.add(A + t0, sets->A + t0, n8);
    mi.add(B + t0, sets->B + t0, n8);
    mi.add(u + t0, sets->u_ppm + t0, n8);
    mi.add(ty + t0, sets->type + t0, n);
    if ((e = mi.flush()) != cudaSuccess) break;
    e = cudaEventRecord(ev_in, in);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, ev_in, 0);
    if (e != cudaSuccess) break;
    // the slice's sets index the full task columns (their offsets are absolute)
    DevSets ds{s1 - s0, sets->n_max, off + s0, T, D, A, B, u, ty};
    for (int k = 0; k < np && st == GPA_OK; k++) {
      AllocOut o = outs[k];
      o.verdict += s0;
      o.reason += s0;
      o.n_parts += s0;
      o.Pi += s0;
      o.W += s0;
      if (o.n_tests) o.n_tests += s0;
      st = allocate_device(c, ds, md, p[k], o);
    }
    if (st != GPA_OK) break;
    e = cudaEventRecord(ev_done, cs);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ot, ev_done, 0);
    if (e != cudaSuccess) break;
    for (int k = 0; k < np; k++) copy_out_range(mo, r[k], outs[k], s0, s1, t0, t1);
    // after the last slice, the error word comes out with the results
    if (j + 2 == b.size()) mo.add(c->h_err, c->d_err, sizeof(unsigned int));
    e = mo.flush();
  }
  if (st != GPA_OK || e != cudaSuccess) {
    // No copy may touch the caller's arrays after the call returns: wait for
    // all three streams whatever happened above.
    cudaStreamSynchronize(in);
    cudaStreamSynchronize(cs);
    cudaStreamSynchronize(ot);
    return st != GPA_OK ? st : gpa_cuda_fail(e, "allocate on host buffers");
  }
  // the copy-out stream's last work waited for the last slice's kernels,
  // which waited for the last copy in: one wait covers all three streams
  if ((e = cudaStreamSynchronize(ot)) != cudaSuccess) return gpa_cuda_fail(e, "allocate on host buffers");
  st = err_word_status(c, *c->h_err);
  if (st == GPA_ERR_RANGE) {
    // the kernels flagged an invalid set: name the first one
    int64_t bad = -1;
    const int32_t vs = gpa_validate(sets, model, &bad);
    if (vs != GPA_OK) return vs;
  }
  return st;
}

// gpa_allocate and gpa_allocate_multi: the batch decided under np policies,
// its host columns (if any) copied to the device once for all of them.
static int32_t allocate_policies(gpa_ctx* c, const gpa_tasksets* sets, const gpa_model* model,
                                 const gpa_params* params, int np, gpa_alloc_result* r, const char* who) {
  int32_t st = common_checks(c, sets, model, who);
  if (st != GPA_OK) return st;
  if (!params || !r) return gpa_fail(GPA_ERR_ARG, "%s: NULL params/result", who);
  if (np < 1 || np > GPA_MULTI_MAX_POLICIES)
    return gpa_fail(GPA_ERR_RANGE, "%s: %d policies (1 to %d)", who, np, GPA_MULTI_MAX_POLICIES);
  for (int k = 0; k < np; k++) {
    if (params[k].policy < GPA_POLICY_SMS || params[k].policy > GPA_POLICY_ONE_GPU)
      return gpa_fail(GPA_ERR_ARG, "%s: unknown policy %d", who, params[k].policy);
    if (r[k].mem != sets->mem) return gpa_fail(GPA_ERR_ARG, "%s: result and sets differ in mem", who);
  }
  if (sets->nsets == 0) return GPA_OK;
  for (int k = 0; k < np; k++)
    if (!r[k].verdict || !r[k].reason || !r[k].n_parts || !r[k].Pi || !r[k].W || !r[k].part_of_task ||
        !r[k].size_of_part)
      return gpa_fail(GPA_ERR_ARG, "%s: NULL result array", who);
  if (!sets->u_ppm) return gpa_fail(GPA_ERR_ARG, "%s: u_ppm is required", who);
  DeviceGuard guard(c->device);
  DevModel md;
  if ((st = device_model(c, model, &md)) != GPA_OK) return st;
  if (sets->mem == GPA_DEVICE) {
    for (int k = 0; k < np && st == GPA_OK; k++) {
      AllocOut out{r[k].verdict, r[k].reason, r[k].n_parts, r[k].Pi, (long long*)r[k].W, r[k].n_tests,
                   r[k].part_of_task, r[k].size_of_part};
      st = allocate_device(c, dev_sets(sets), md, params[k], out);
    }
    return st;
  }
  const std::vector<long long> bounds = slice_bounds(c, sets);
  if (!bounds.empty()) return allocate_host_sliced(c, sets, model, md, params, np, r, bounds);
  HostStage hs;
  if ((st = stage_in_validated(c, sets, model, &hs)) != GPA_OK) return st;
  const long long ns = sets->nsets;
  AllocOut outs[GPA_MULTI_MAX_POLICIES];
  for (int k = 0; k < np; k++)
    if ((st = host_out_bufs(c, k, ns, hs.ntasks, r[k].n_tests != nullptr, &outs[k])) != GPA_OK) return st;
  for (int k = 0; k < np; k++)
    if ((st = allocate_device(c, hs.ds, md, params[k], outs[k])) != GPA_OK) return st;
  Mover mv(c, c->stream, false);
  for (int k = 0; k < np; k++) copy_out_range(mv, r[k], outs[k], 0, ns, 0, hs.ntasks);
  cudaError_t e = mv.flush();
  if (e != cudaSuccess) return gpa_cuda_fail(e, "allocate result copy");
  return finish_host_call(c);
}

extern "C" int32_t gpa_allocate(gpa_ctx* c, const gpa_tasksets* sets, const gpa_model* model,
                                const gpa_params* params, gpa_alloc_result* r) {
  return allocate_policies(c, sets, model, params, 1, r, "gpa_allocate");
}

extern "C" int32_t gpa_allocate_multi(gpa_ctx* c, const gpa_tasksets* sets, const gpa_model* model,
                                      const gpa_params* params, int32_t npolicies, gpa_alloc_result* results) {
  return allocate_policies(c, sets, model, params, npolicies, results, "gpa_allocate_multi");
}

// ------------------------------------------------------- exhaustive optimum

extern "C" int32_t gpa_search_best(gpa_ctx* c, const gpa_tasksets* sets, const gpa_model* model, int32_t kmin,
                                   int32_t kmax, gpa_best_result* r) {
  int32_t st = common_checks(c, sets, model, "gpa_search_best");
  if (st != GPA_OK) return st;
  if (!r) return gpa_fail(GPA_ERR_ARG, "gpa_search_best: NULL result");
  if (kmin < 1 || kmax < kmin || kmax > GPA_SEARCH_KMAX)
    return gpa_fail(GPA_ERR_RANGE, "gpa_search_best: need 1 <= kmin <= kmax <= %d", GPA_SEARCH_KMAX);
  if (sets->n_max > GPA_SEARCH_NMAX)
    return gpa_fail(GPA_ERR_RANGE, "gpa_search_best: n_max %d exceeds %d", sets->n_max, GPA_SEARCH_NMAX);
  if (r->mem != sets->mem) return gpa_fail(GPA_ERR_ARG, "gpa_search_best: result and sets differ in mem");
  if (sets->nsets == 0) return GPA_OK;
  if (!sets->u_ppm) return gpa_fail(GPA_ERR_ARG, "gpa_search_best: u_ppm is required");
  if (!r->feasible || !r->W || !r->sum_minm || !r->n_blocks || !r->spare || !r->rgs || !r->minm_block)
    return gpa_fail(GPA_ERR_ARG, "gpa_search_best: NULL result array");
  DeviceGuard guard(c->device);
  DevModel md;
  if ((st = device_model(c, model, &md)) != GPA_OK) return st;
  AllocQueue q{c->d_counters, c->d_slow, c->d_err};
  if (sets->mem == GPA_DEVICE) {
    BestOut out{r->feasible, (long long*)r->W, r->sum_minm, r->n_blocks, r->spare, r->rgs, r->minm_block};
    cudaError_t e = launch_search_best(dev_sets(sets), md, kmin, kmax, out, q, c->d_mdiv, c->sm_count, c->stream,
                                       &c->launches, begin_prof(c));
    return e == cudaSuccess ? GPA_OK : gpa_cuda_fail(e, "search_best launch");
  }
  HostStage hs;
  if ((st = stage_in_validated(c, sets, model, &hs)) != GPA_OK) return st;
  const long long ns = sets->nsets, nt = hs.ntasks > 0 ? hs.ntasks : 1;
  BestOut out{(unsigned char*)ctx_buffer(c, 22, (size_t)ns), (long long*)ctx_buffer(c, 23, 8 * (size_t)ns),
              (int*)ctx_buffer(c, 24, 4 * (size_t)ns), (int*)ctx_buffer(c, 25, 4 * (size_t)ns),
              (int*)ctx_buffer(c, 26, 4 * (size_t)ns), (unsigned char*)ctx_buffer(c, 27, (size_t)nt),
              (short*)ctx_buffer(c, 28, 2 * (size_t)(ns * kmax))};
  if (!out.feasible || !out.W || !out.sum_minm || !out.n_blocks || !out.spare || !out.rgs || !out.minm_block)
    return gpa_fail(GPA_ERR_NOMEM, "result staging failed");
  cudaStream_t s = c->stream;
  cudaError_t e =
      launch_search_best(hs.ds, md, kmin, kmax, out, q, c->d_mdiv, c->sm_count, s, &c->launches, begin_prof(c));
  if (e == cudaSuccess) e = cudaMemcpyAsync(r->feasible, out.feasible, (size_t)ns, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(r->W, out.W, 8 * (size_t)ns, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(r->sum_minm, out.sum_minm, 4 * (size_t)ns, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(r->n_blocks, out.n_blocks, 4 * (size_t)ns, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(r->spare, out.spare, 4 * (size_t)ns, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && hs.ntasks > 0)
    e = cudaMemcpyAsync(r->rgs, out.rgs, (size_t)hs.ntasks, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(r->minm_block, out.minm_block, 2 * (size_t)(ns * kmax), cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return gpa_cuda_fail(e, "search_best");
  return finish_host_call(c);
}

extern "C" int32_t gpa_search_explicit(gpa_ctx* c, const gpa_tasksets* sets, const gpa_model* model, int32_t kmin,
                                       int32_t kmax, gpa_best_result* r, uint8_t* cand_verdict, int64_t* ncand) {
  int32_t st = common_checks(c, sets, model, "gpa_search_explicit");
  if (st != GPA_OK) return st;
  if (!r) return gpa_fail(GPA_ERR_ARG, "gpa_search_explicit: NULL result");
  if (kmin < 1 || kmax < kmin || kmax > GPA_SEARCH_KMAX)
    return gpa_fail(GPA_ERR_RANGE, "gpa_search_explicit: need 1 <= kmin <= kmax <= %d", GPA_SEARCH_KMAX);
  if (sets->n_max > GPA_SEARCH_NMAX)
    return gpa_fail(GPA_ERR_RANGE, "gpa_search_explicit: n_max %d exceeds %d", sets->n_max, GPA_SEARCH_NMAX);
  if (model->nsizes != 0) return gpa_fail(GPA_ERR_ARG, "gpa_search_explicit: admissible size lists are not supported");
  if (r->mem != sets->mem) return gpa_fail(GPA_ERR_ARG, "gpa_search_explicit: result and sets differ in mem");
  // candidates of a set of n_max tasks: sum over k of C(Mu - 1, k - 1) k^n_max
  const int Mu = model->M / model->g;
  const int nmax = sets->n_max < 0 ? 0 : sets->n_max;
  unsigned __int128 total = 0;
  for (int k = kmin; k <= kmax && k <= Mu; k++) {
    unsigned __int128 maps = 1;
    for (int i = 0; i < nmax && maps <= (unsigned __int128)GPA_EXPLICIT_MAX; i++) maps *= (unsigned)k;
    unsigned __int128 comps = 1;
    for (int i = 1; i <= k - 1 && comps <= (unsigned __int128)GPA_EXPLICIT_MAX; i++)
      comps = comps * (unsigned)(Mu - 1 - (k - 1) + i) / (unsigned)i;
    total += comps * maps;
    if (total > (unsigned __int128)GPA_EXPLICIT_MAX) break;
  }
  if (total > (unsigned __int128)GPA_EXPLICIT_MAX)
    return gpa_fail(GPA_ERR_RANGE, "gpa_search_explicit: more than %lld candidates per set", (long long)GPA_EXPLICIT_MAX);
  const long long stride = (long long)total;
  if (ncand) *ncand = stride;
  if (sets->nsets == 0) return GPA_OK;
  if (!sets->u_ppm) return gpa_fail(GPA_ERR_ARG, "gpa_search_explicit: u_ppm is required");
  if (!r->feasible || !r->W || !r->sum_minm || !r->n_blocks || !r->spare || !r->rgs || !r->minm_block)
    return gpa_fail(GPA_ERR_ARG, "gpa_search_explicit: NULL result array");
  DeviceGuard guard(c->device);
  DevModel md;
  if ((st = device_model(c, model, &md)) != GPA_OK) return st;
  AllocQueue q{c->d_counters, c->d_slow, c->d_err};
  if (sets->mem == GPA_DEVICE) {
    BestOut out{r->feasible, (long long*)r->W, r->sum_minm, r->n_blocks, r->spare, r->rgs, r->minm_block};
    cudaError_t e = launch_search_explicit(dev_sets(sets), md, kmin, kmax, out, cand_verdict, stride, q, c->d_mdiv,
                                           c->sm_count, c->stream, &c->launches, begin_prof(c));
    return e == cudaSuccess ? GPA_OK : gpa_cuda_fail(e, "search_explicit launch");
  }
  HostStage hs;
  if ((st = stage_in_validated(c, sets, model, &hs)) != GPA_OK) return st;
  const long long ns = sets->nsets, nt = hs.ntasks > 0 ? hs.ntasks : 1;
  BestOut out{(unsigned char*)ctx_buffer(c, 22, (size_t)ns), (long long*)ctx_buffer(c, 23, 8 * (size_t)ns),
              (int*)ctx_buffer(c, 24, 4 * (size_t)ns), (int*)ctx_buffer(c, 25, 4 * (size_t)ns),
              (int*)ctx_buffer(c, 26, 4 * (size_t)ns), (unsigned char*)ctx_buffer(c, 27, (size_t)nt),
              (short*)ctx_buffer(c, 28, 2 * (size_t)(ns * kmax))};
  unsigned char* dcv = cand_verdict ? (unsigned char*)ctx_buffer(c, 29, (size_t)(ns * stride)) : nullptr;
  if (!out.feasible || !out.W || !out.sum_minm || !out.n_blocks || !out.spare || !out.rgs || !out.minm_block ||
      (cand_verdict && !dcv))
    return gpa_fail(GPA_ERR_NOMEM, "result staging failed");
  cudaStream_t s = c->stream;
  cudaError_t e = launch_search_explicit(hs.ds, md, kmin, kmax, out, dcv, stride, q, c->d_mdiv, c->sm_count, s,
                                         &c->launches, begin_prof(c));
  if (e == cudaSuccess) e = cudaMemcpyAsync(r->feasible, out.feasible, (size_t)ns, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(r->W, out.W, 8 * (size_t)ns, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(r->sum_minm, out.sum_minm, 4 * (size_t)ns, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(r->n_blocks, out.n_blocks, 4 * (size_t)ns, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(r->spare, out.spare, 4 * (size_t)ns, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && hs.ntasks > 0)
    e = cudaMemcpyAsync(r->rgs, out.rgs, (size_t)hs.ntasks, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(r->minm_block, out.minm_block, 2 * (size_t)(ns * kmax), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && cand_verdict)
    e = cudaMemcpyAsync(cand_verdict, dcv, (size_t)(ns * stride), cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return gpa_cuda_fail(e, "search_explicit");
  return finish_host_call(c);
}

// --------------------------------------------- compositions and set partitions

static unsigned __int128 binom128(long long n, long long k) {
  if (k < 0 || n < 0 || k > n) return 0;
  if (k > n - k) k = n - k;
  unsigned __int128 r = 1;
  for (long long i = 1; i <= k; i++) {
    r = r * (unsigned __int128)(n - k + i) / (unsigned __int128)i;
    if (r > (((unsigned __int128)1) << 100)) return r;  // saturates; callers check against 2^64
  }
  return r;
}

extern "C" int32_t gpa_enumerate_partitions(int32_t Mu, int32_t kmin, int32_t kmax, uint64_t* count) {
  if (!count) return gpa_fail(GPA_ERR_ARG, "gpa_enumerate_partitions: NULL count");
  if (Mu < 1 || Mu > GPA_MMAX || kmin < 1 || kmax < kmin) return gpa_fail(GPA_ERR_RANGE, "bad Mu/kmin/kmax");
  unsigned __int128 total = 0;
  for (int k = kmin; k <= kmax && k <= Mu; k++) total += binom128(Mu - 1, k - 1);
  if (total >> 64) return gpa_fail(GPA_ERR_RANGE, "count exceeds 2^64");
  *count = (uint64_t)total;
  return GPA_OK;
}

extern "C" int32_t gpa_unrank_composition(int32_t Mu, int32_t k, uint64_t rank, int32_t* parts) {
  if (!parts) return gpa_fail(GPA_ERR_ARG, "NULL parts");
  if (Mu < 1 || Mu > GPA_MMAX || k < 1 || k > Mu) return gpa_fail(GPA_ERR_RANGE, "bad Mu/k");
  unsigned __int128 total = binom128(Mu - 1, k - 1);
  if ((unsigned __int128)rank >= total) return gpa_fail(GPA_ERR_RANGE, "rank out of range");
  unsigned __int128 r = rank;
  int left = Mu;
  for (int i = 0; i < k; i++) {
    const int rest = k - i - 1;  // parts after this one
    if (rest == 0) {
      parts[i] = left;
      break;
    }
    for (int p = 1; p <= left - rest; p++) {
      // completions with parts[i] = p: compositions of left - p into rest parts
      unsigned __int128 c = binom128(left - p - 1, rest - 1);
      if (r < c) {
        parts[i] = p;
        left -= p;
        break;
      }
      r -= c;
    }
  }
  return GPA_OK;
}

// completions[i][j]: ways to label positions i..n-1 given j open blocks
static void rgs_counts(int n, int kmax, std::vector<std::vector<unsigned __int128>>& cnt) {
  cnt.assign((size_t)n + 1, std::vector<unsigned __int128>((size_t)kmax + 2, 0));
  for (int j = 0; j <= kmax + 1; j++) cnt[(size_t)n][(size_t)j] = 1;
  for (int i = n - 1; i >= 0; i--)
    for (int j = 0; j <= kmax; j++) {
      unsigned __int128 c = (unsigned __int128)j * cnt[(size_t)i + 1][(size_t)j];
      if (j < kmax) c += cnt[(size_t)i + 1][(size_t)j + 1];
      cnt[(size_t)i][(size_t)j] = c;
    }
}

extern "C" int32_t gpa_count_rgs(int32_t n, int32_t kmax, uint64_t* count) {
  if (!count) return gpa_fail(GPA_ERR_ARG, "NULL count");
  if (n < 0 || n > GPA_NMAX || kmax < 1 || kmax > GPA_NMAX) return gpa_fail(GPA_ERR_RANGE, "bad n/kmax");
  if (n == 0) {
    *count = 1;
    return GPA_OK;
  }
  std::vector<std::vector<unsigned __int128>> cnt;
  rgs_counts(n, kmax, cnt);
  unsigned __int128 t = cnt[1][1];
  if (t >> 64) return gpa_fail(GPA_ERR_RANGE, "count exceeds 2^64");
  *count = (uint64_t)t;
  return GPA_OK;
}

extern "C" int32_t gpa_unrank_rgs(int32_t n, int32_t kmax, uint64_t rank, uint8_t* rgs) {
  if (!rgs && n > 0) return gpa_fail(GPA_ERR_ARG, "NULL rgs");
  if (n < 0 || n > GPA_NMAX || kmax < 1 || kmax > GPA_NMAX) return gpa_fail(GPA_ERR_RANGE, "bad n/kmax");
  if (n == 0) return rank == 0 ? GPA_OK : gpa_fail(GPA_ERR_RANGE, "rank out of range");
  std::vector<std::vector<unsigned __int128>> cnt;
  rgs_counts(n, kmax, cnt);
  if ((unsigned __int128)rank >= cnt[1][1]) return gpa_fail(GPA_ERR_RANGE, "rank out of range");
  unsigned __int128 r = rank;
  rgs[0] = 0;
  int used = 1;
  for (int i = 1; i < n; i++) {
    const int top = used < kmax ? used : kmax - 1;
    for (int b = 0; b <= top; b++) {
      const int nu = b + 1 > used ? b + 1 : used;
      unsigned __int128 c = cnt[(size_t)i + 1][(size_t)nu];
      if (r < c) {
        rgs[i] = (uint8_t)b;
        used = nu;
        break;
      }
      r -= c;
    }
  }
  return GPA_OK;
}
