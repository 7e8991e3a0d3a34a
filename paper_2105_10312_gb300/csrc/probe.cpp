// probe.cpp — gpa_measure_wcet and gpa_fit_wcet: a kernel's execution time
// against the number of SMs it may use, measured with the blocker method of
// §3 (Fig. 1), and the least-squares fit of §3.3's C(m) = a / m + b.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <climits>
#include <mutex>
#include <set>
#include <thread>
#include <vector>

#include "gpa.h"
#include "gpa_ctx.h"
#include "gpa_internal.h"

using namespace gpa;

namespace {

constexpr unsigned long long kWindowMaxNs = 1000000000ull;  // the blocker never holds SMs longer than 1 s
constexpr size_t kInterfereBytes = size_t(1) << 30;          // the co-runner's buffer (8 x L2)
constexpr int kAttempts = 3;                                 // placement retries per repetition

// The call's device buffers, streams and events, released on every return.
struct ProbeState {
  ProbeBuffers b{};
  void* ibuf = nullptr;
  unsigned int* smid_block = nullptr;
  unsigned int* smid_test = nullptr;
  unsigned long long* times = nullptr;  // [0] earliest blocker end, [1] latest end of the kernel under test
  float* sink = nullptr;
  cudaStream_t sb = nullptr, st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  ~ProbeState() {
    if (sb) cudaStreamSynchronize(sb);
    if (st) cudaStreamSynchronize(st);
    cudaFree(b.a);
    cudaFree(b.b);
    cudaFree(b.c);
    cudaFree(ibuf);
    cudaFree(smid_block);
    cudaFree(smid_test);
    cudaFree(times);
    cudaFree(sink);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (sb) cudaStreamDestroy(sb);
    if (st) cudaStreamDestroy(st);
  }
};

double median(std::vector<double> v) {
  std::sort(v.begin(), v.end());
  const size_t k = v.size();
  return k % 2 ? v[k / 2] : 0.5 * (v[k / 2 - 1] + v[k / 2]);
}

}  // namespace

extern "C" int32_t gpa_fit_wcet(const int32_t* m, const double* ms, int32_t n, double* a, double* b) {
  if (!m || !ms || !a || !b || n < 2) return gpa_fail(GPA_ERR_ARG, "gpa_fit_wcet: NULL argument or fewer than 2 points");
  // ms = a x + b with x = 1 / m, by the normal equations
  double sx = 0, sy = 0, sxx = 0, sxy = 0;
  int k = 0, m0 = 0;
  bool spread = false;
  for (int i = 0; i < n; i++) {
    if (ms[i] < 0 || m[i] < 1) continue;
    const double x = 1.0 / m[i], y = ms[i];
    sx += x;
    sy += y;
    sxx += x * x;
    sxy += x * y;
    if (k == 0) m0 = m[i];
    spread = spread || m[i] != m0;
    k++;
  }
  if (k < 2 || !spread) return gpa_fail(GPA_ERR_ARG, "gpa_fit_wcet: need usable points at two or more m");
  const double den = k * sxx - sx * sx;
  *a = (k * sxy - sx * sy) / den;
  *b = (sy - *a * sx) / k;
  return GPA_OK;
}

extern "C" int32_t gpa_measure_wcet(gpa_ctx* c, const gpa_probe_cfg* cfg, const int32_t* m, int32_t nm, double* ms,
                                    int32_t* sms_used) {
  if (!c || !cfg || !m || !ms || !sms_used || nm < 1)
    return gpa_fail(GPA_ERR_ARG, "gpa_measure_wcet: NULL argument or no m");
  const int kernel = cfg->kernel;
  if (kernel < GPA_PROBE_VADD || kernel > GPA_PROBE_COMPUTE)
    return gpa_fail(GPA_ERR_ARG, "gpa_measure_wcet: unknown kernel %d", kernel);
  const bool square = kernel == GPA_PROBE_TRANSPOSE || kernel == GPA_PROBE_STENCIL;
  if (square ? (cfg->n < 32 || cfg->n > 16384) : (cfg->n < 1 || cfg->n > (1ll << 28)))
    return gpa_fail(GPA_ERR_RANGE, "gpa_measure_wcet: problem size %lld out of range", (long long)cfg->n);
  if (cfg->reps < 1 || cfg->reps > 100) return gpa_fail(GPA_ERR_RANGE, "gpa_measure_wcet: reps in 1..100");
  if (cfg->ctas < 0 || cfg->ctas > (1 << 20)) return gpa_fail(GPA_ERR_RANGE, "gpa_measure_wcet: ctas");
  for (int i = 0; i < nm; i++)
    if (m[i] < 1 || m[i] > c->sm_count)
      return gpa_fail(GPA_ERR_RANGE, "gpa_measure_wcet: m = %d outside [1, %d]", m[i], c->sm_count);
  DeviceGuard guard(c->device);
  static std::once_flag once;
  static cudaError_t init_err = cudaSuccess;
  std::call_once(once, [] { init_err = probe_kernels_init(); });
  if (init_err != cudaSuccess) return gpa_cuda_fail(init_err, "probe kernel set-up");

  const size_t elems = square ? (size_t)cfg->n * (size_t)cfg->n : (size_t)cfg->n;
  const int ctas = cfg->ctas ? cfg->ctas : 4 * c->sm_count;
  const int sms = c->sm_count;
  ProbeState S;
  cudaError_t e = cudaSuccess;
  auto ok = [&](cudaError_t x) { return (e = x) == cudaSuccess; };
  if (!ok(cudaMalloc(&S.b.a, elems * sizeof(float))) || !ok(cudaMalloc(&S.b.b, elems * sizeof(float))) ||
      !ok(cudaMalloc(&S.b.c, elems * sizeof(float))) ||
      !ok(cudaMalloc(&S.smid_block, sizeof(unsigned int) * (size_t)sms)) ||
      !ok(cudaMalloc(&S.smid_test, sizeof(unsigned int) * (size_t)ctas)) ||
      !ok(cudaMalloc(&S.times, 2 * sizeof(unsigned long long))) || !ok(cudaMalloc(&S.sink, sizeof(float))) ||
      (cfg->interfere && !ok(cudaMalloc(&S.ibuf, kInterfereBytes))))
    return e == cudaErrorMemoryAllocation ? gpa_fail(GPA_ERR_NOMEM, "gpa_measure_wcet: device buffers")
                                          : gpa_cuda_fail(e, "gpa_measure_wcet: device buffers");
  if (!ok(cudaStreamCreateWithFlags(&S.sb, cudaStreamNonBlocking)) ||
      !ok(cudaStreamCreateWithFlags(&S.st, cudaStreamNonBlocking)) || !ok(cudaEventCreate(&S.e0)) ||
      !ok(cudaEventCreate(&S.e1)))
    return gpa_cuda_fail(e, "gpa_measure_wcet: streams");
  // inputs: bytes 0x3c make every float 0.0115
  if (!ok(cudaMemsetAsync(S.b.a, 0x3c, elems * sizeof(float), S.st)) ||
      !ok(cudaMemsetAsync(S.b.b, 0x3c, elems * sizeof(float), S.st)) ||
      (S.ibuf && !ok(cudaMemsetAsync(S.ibuf, 0x3c, kInterfereBytes, S.st))) || !ok(cudaStreamSynchronize(S.st)))
    return gpa_cuda_fail(e, "gpa_measure_wcet: input set-up");

  auto time_test = [&](float* out_ms) -> cudaError_t {
    cudaError_t x = cudaEventRecord(S.e0, S.st);
    if (x == cudaSuccess) x = launch_probe_kernel(kernel, ctas, S.b, (unsigned long long)cfg->n, S.smid_test, S.times + 1, S.st);
    if (x == cudaSuccess) x = cudaEventRecord(S.e1, S.st);
    if (x == cudaSuccess) x = cudaEventSynchronize(S.e1);
    if (x == cudaSuccess) x = cudaEventElapsedTime(out_ms, S.e0, S.e1);
    return x;
  };
  // the kernel alone on the whole GPU sizes the blocker's window
  std::vector<double> full;
  for (int r = 0; r < 5; r++) {
    float t = 0.f;
    if (!ok(time_test(&t))) return gpa_cuda_fail(e, "gpa_measure_wcet: kernel under test");
    if (r >= 2) full.push_back(t);
  }
  const double t_full_ms = median(full);

  std::vector<unsigned int> hb((size_t)sms), ht((size_t)ctas);
  for (int i = 0; i < nm; i++) {
    const int blk = sms - m[i];
    // room for the kernel on m SMs, slowed by a co-runner, plus the host's
    // wait for the blocker to become resident
    const double want_ns = 1e6 * (8.0 * t_full_ms * sms / m[i] + 2.0);
    const unsigned long long window = blk > 0 ? std::min<unsigned long long>(kWindowMaxNs, (unsigned long long)want_ns) : 0;
    std::vector<double> good;
    int used = -1;
    for (int r = 0; r < cfg->reps; r++) {
      for (int attempt = 0; attempt < kAttempts; attempt++) {
        const unsigned long long init[2] = {ULLONG_MAX, 0ull};
        if (!ok(cudaMemcpyAsync(S.times, init, sizeof init, cudaMemcpyHostToDevice, S.st)) ||
            !ok(cudaMemsetAsync(S.smid_block, 0xff, sizeof(unsigned int) * (size_t)sms, S.st)) ||
            !ok(cudaMemsetAsync(S.smid_test, 0xff, sizeof(unsigned int) * (size_t)ctas, S.st)) ||
            !ok(cudaStreamSynchronize(S.st)))
          return gpa_cuda_fail(e, "gpa_measure_wcet: reset");
        if (blk > 0) {
          if (!ok(launch_probe_blocker(blk, window, cfg->interfere ? S.ibuf : nullptr, kInterfereBytes, S.smid_block,
                                       S.times, S.sink, S.sb)))
            return gpa_cuda_fail(e, "gpa_measure_wcet: blocker");
          // every blocker CTA is resident long before this (launch latency is microseconds)
          std::this_thread::sleep_for(std::chrono::microseconds(300));
        }
        float t = 0.f;
        if (!ok(time_test(&t)) || !ok(cudaStreamSynchronize(S.sb)))
          return gpa_cuda_fail(e, "gpa_measure_wcet: measurement");
        unsigned long long tm[2] = {0, 0};
        if (!ok(cudaMemcpy(hb.data(), S.smid_block, sizeof(unsigned int) * (size_t)sms, cudaMemcpyDeviceToHost)) ||
            !ok(cudaMemcpy(ht.data(), S.smid_test, sizeof(unsigned int) * (size_t)ctas, cudaMemcpyDeviceToHost)) ||
            !ok(cudaMemcpy(tm, S.times, sizeof tm, cudaMemcpyDeviceToHost)))
          return gpa_cuda_fail(e, "gpa_measure_wcet: placement read-back");
        const std::set<unsigned int> B(hb.begin(), hb.begin() + blk), T(ht.begin(), ht.end());
        bool placed = (int)B.size() == blk && B.count(0xffffffffu) == 0 && T.count(0xffffffffu) == 0;
        for (unsigned int s : T) placed = placed && B.count(s) == 0;
        if (ctas >= m[i]) placed = placed && (int)T.size() == m[i];
        placed = placed && (int)T.size() <= m[i] && (blk == 0 || tm[1] <= tm[0]);
        if (placed) {
          good.push_back(t);
          used = (int)T.size();
          break;
        }
      }
    }
    ms[i] = good.empty() ? -1.0 : median(good);
    sms_used[i] = good.empty() ? -1 : used;
  }
  return GPA_OK;
}

extern "C" int32_t gpa_probe_run(gpa_ctx* c, int32_t kernel, int64_t n, int32_t ctas, const float* a, const float* b,
                                 float* out) {
  if (!c || !a || !out || (kernel == GPA_PROBE_VADD && !b)) return gpa_fail(GPA_ERR_ARG, "gpa_probe_run: NULL argument");
  if (kernel < GPA_PROBE_VADD || kernel > GPA_PROBE_COMPUTE) return gpa_fail(GPA_ERR_ARG, "gpa_probe_run: bad kernel");
  const bool square = kernel == GPA_PROBE_TRANSPOSE || kernel == GPA_PROBE_STENCIL;
  if (square ? (n < 32 || n > 16384) : (n < 1 || n > (1ll << 28)))
    return gpa_fail(GPA_ERR_RANGE, "gpa_probe_run: problem size %lld out of range", (long long)n);
  if (ctas < 0 || ctas > (1 << 20)) return gpa_fail(GPA_ERR_RANGE, "gpa_probe_run: ctas");
  DeviceGuard guard(c->device);
  const size_t elems = square ? (size_t)n * (size_t)n : (size_t)n;
  const int nctas = ctas ? ctas : 4 * c->sm_count;
  ProbeState S;
  cudaError_t e = cudaSuccess;
  auto ok = [&](cudaError_t x) { return (e = x) == cudaSuccess; };
  if (!ok(cudaMalloc(&S.b.a, elems * sizeof(float))) || !ok(cudaMalloc(&S.b.b, elems * sizeof(float))) ||
      !ok(cudaMalloc(&S.b.c, elems * sizeof(float))) ||
      !ok(cudaMalloc(&S.smid_test, sizeof(unsigned int) * (size_t)nctas)) ||
      !ok(cudaMalloc(&S.times, 2 * sizeof(unsigned long long))))
    return e == cudaErrorMemoryAllocation ? gpa_fail(GPA_ERR_NOMEM, "gpa_probe_run: device buffers")
                                          : gpa_cuda_fail(e, "gpa_probe_run: device buffers");
  if (!ok(cudaMemcpy(S.b.a, a, elems * sizeof(float), cudaMemcpyHostToDevice)) ||
      (b && !ok(cudaMemcpy(S.b.b, b, elems * sizeof(float), cudaMemcpyHostToDevice))) ||
      !ok(cudaMemset(S.times, 0, 2 * sizeof(unsigned long long))) ||
      !ok(launch_probe_kernel(kernel, nctas, S.b, (unsigned long long)n, S.smid_test, S.times + 1, c->stream)) ||
      !ok(cudaStreamSynchronize(c->stream)) ||
      !ok(cudaMemcpy(out, S.b.c, elems * sizeof(float), cudaMemcpyDeviceToHost)))
    return gpa_cuda_fail(e, "gpa_probe_run");
  return GPA_OK;
}
