// k_peak.cu — the integer throughput ceiling the test kernels are measured
// against (gpa_measure_alu_peak).
//
// The unit of work of the per-partition test (§5.5) is one interference
// term ceil(R / T_j) C_j of the response-time iteration.  The test kernels
// evaluate it as: the period's reciprocal and shift and C_j read from shared
// memory (the same address for every lane of a warp), the high word of a
// 32 x 32-bit product and a shift (floor_div_T2), and a 32 x 32 -> 64-bit
// multiply-add into the sum (the +1 of the ceiling is added once per step,
// as a sum of WCETs).  term_peak runs exactly that sequence with four
// independent iterations per thread over a 64-entry table, on every SM with
// every warp slot it can fill, so its rate is what the device can sustain on
// this arithmetic when nothing (dependences, divergence, idle warps) holds
// it back.  imad_peak gives, for context, the rate of independent 32-bit
// integer multiply-adds.
#include <cuda_runtime.h>

#include <algorithm>

#include "gpa_device.cuh"
#include "gpa_internal.h"

namespace gpa {

namespace {

constexpr int kPeakThreads = 256;
constexpr int kPeakTab = 64;
constexpr int kPeakChains = 4;
constexpr int kImadChains = 8;
constexpr int kImadUnroll = 16;

__global__ void __launch_bounds__(kPeakThreads) term_peak(int reps, unsigned long long base, unsigned int seed,
                                                          unsigned long long* sink) {
  __shared__ unsigned int sC[kPeakTab], sM[kPeakTab];
  __shared__ unsigned char sS[kPeakTab];
  const int t = threadIdx.x;
  if (t < kPeakTab) {
    const unsigned int T = 1000u + 37u * (unsigned)t + (seed & 7u);
    unsigned int mg, sh;
    magic_for_period(T, &mg, &sh);
    sM[t] = mg;
    sS[t] = (unsigned char)sh;
    sC[t] = 1u + ((unsigned)t * 13u) % 97u;
  }
  __syncthreads();
  unsigned int R[kPeakChains];
#pragma unroll
  for (int c = 0; c < kPeakChains; c++) R[c] = 100000u + 1000u * (unsigned)c + threadIdx.x + blockIdx.x;
  unsigned long long chk = 0ull;
  for (int rep = 0; rep < reps; rep++) {
    unsigned long long nx[kPeakChains];
    unsigned int R2[kPeakChains];
#pragma unroll
    for (int c = 0; c < kPeakChains; c++) {
      nx[c] = base;  // stands for the step's sum of WCETs
      R2[c] = 2u * (R[c] - 1u);
    }
#pragma unroll 4
    for (int j = 0; j < kPeakTab; j++) {
      const unsigned int mg = sM[j], sh = sS[j], C = sC[j];
#pragma unroll
      for (int c = 0; c < kPeakChains; c++) nx[c] += (unsigned long long)floor_div_T2(R2[c], mg, sh) * C;
    }
#pragma unroll
    for (int c = 0; c < kPeakChains; c++) {
      R[c] = ((unsigned int)nx[c] & 0x3fffffffu) | 1u;  // next iterate: in [1, 2^30)
      chk += nx[c];
    }
  }
  if (chk == 0x0123456789abcdefull) *sink = chk;  // keeps the work observable
}

__device__ __forceinline__ unsigned int mad_u32(unsigned int x, unsigned int a, unsigned int b) {
  unsigned int r;
  asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(r) : "r"(x), "r"(a), "r"(b));
  return r;
}

__global__ void __launch_bounds__(kPeakThreads) imad_peak(int reps, unsigned int a, unsigned int b,
                                                          unsigned long long* sink) {
  unsigned int x[kImadChains];
#pragma unroll
  for (int i = 0; i < kImadChains; i++) x[i] = threadIdx.x + 77u * (unsigned)i + blockIdx.x;
  for (int rep = 0; rep < reps; rep++) {
#pragma unroll
    for (int k = 0; k < kImadUnroll; k++)
#pragma unroll
      for (int i = 0; i < kImadChains; i++) x[i] = mad_u32(x[i], a, b);
  }
  unsigned int s = 0u;
#pragma unroll
  for (int i = 0; i < kImadChains; i++) s ^= x[i];
  if (s == 0x9e3779b9u) *sink = s;
}

// Best of `timed` launches (ms) after one warm-up, each launch `reps` deep.
template <class Launch>
cudaError_t best_ms(Launch launch, cudaStream_t st, int timed, float* best) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) {
    launch();
    e = cudaGetLastError();
  }
  *best = 1e30f;
  for (int i = 0; i < timed && e == cudaSuccess; i++) {
    cudaEventRecord(e0, st);
    launch();
    cudaEventRecord(e1, st);
    e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess) *best = std::min(*best, ms);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  return e;
}

}  // namespace

cudaError_t measure_alu_peak(int sm_count, cudaStream_t st, double* terms_per_s, double* imad_per_s,
                             double* term_ms, long long* terms) {
  unsigned long long* sink = nullptr;
  cudaError_t e = cudaMalloc(&sink, sizeof(unsigned long long));
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, term_peak, kPeakThreads, 0);
  const int blocks_t = std::max(1, per_sm) * sm_count;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, imad_peak, kPeakThreads, 0);
  const int blocks_i = std::max(1, per_sm) * sm_count;
  // calibrate the depth so that a launch takes about 3 ms
  int reps = 8;
  float ms = 0.f;
  for (int round = 0; round < 2 && e == cudaSuccess; round++) {
    e = best_ms([&] { term_peak<<<blocks_t, kPeakThreads, 0, st>>>(reps, 4321ull, 3u, sink); }, st, 1, &ms);
    if (e == cudaSuccess && ms > 0.f) reps = std::max(1, (int)std::min(1048576.0f, reps * 3.0f / ms));
  }
  if (e == cudaSuccess)
    e = best_ms([&] { term_peak<<<blocks_t, kPeakThreads, 0, st>>>(reps, 4321ull, 3u, sink); }, st, 5, &ms);
  if (e == cudaSuccess) {
    const double n = (double)blocks_t * kPeakThreads * kPeakChains * kPeakTab * (double)reps;
    *terms_per_s = n / (ms * 1e-3);
    *term_ms = ms;
    *terms = (long long)n;
  }
  int ireps = 64;
  for (int round = 0; round < 2 && e == cudaSuccess; round++) {
    e = best_ms([&] { imad_peak<<<blocks_i, kPeakThreads, 0, st>>>(ireps, 0x9e3779b1u, 7u, sink); }, st, 1, &ms);
    if (e == cudaSuccess && ms > 0.f) ireps = std::max(1, (int)std::min(4194304.0f, ireps * 3.0f / ms));
  }
  if (e == cudaSuccess)
    e = best_ms([&] { imad_peak<<<blocks_i, kPeakThreads, 0, st>>>(ireps, 0x9e3779b1u, 7u, sink); }, st, 5, &ms);
  if (e == cudaSuccess)
    *imad_per_s = (double)blocks_i * kPeakThreads * kImadChains * kImadUnroll * (double)ireps / (ms * 1e-3);
  cudaFree(sink);
  return e;
}

}  // namespace gpa
