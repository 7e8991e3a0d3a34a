// k_stage.cu — byte-range copies between page-locked host memory and device
// buffers done by one kernel per list of ranges.
//
// The host entry points move a batch's task columns in and its results out.
// With cudaMemcpyAsync each column is one transfer with a fixed cost of about
// a microsecond on the copy engine; a kernel whose loads (or stores) go
// straight to the mapped host pages moves every column of a slice in one
// launch at the same link bandwidth.  Ranges are copied 16 bytes at a time
// where source and destination share their alignment modulo 16, else 8, else
// byte by byte.
#include <cuda_runtime.h>

#include "gpa_internal.h"

namespace gpa {
namespace {

constexpr int kStageThreads = 512;
constexpr int kUnroll = 4;

template <typename V>
__device__ __forceinline__ void copy_words(const V* __restrict__ s, V* __restrict__ d, unsigned long long n) {
  const unsigned long long step = (unsigned long long)gridDim.x * blockDim.x;
  unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
  // kUnroll loads in flight per thread before their stores
  for (; i + (kUnroll - 1) * step < n; i += kUnroll * step) {
    V v[kUnroll];
#pragma unroll
    for (int k = 0; k < kUnroll; k++) v[k] = s[i + k * step];
#pragma unroll
    for (int k = 0; k < kUnroll; k++) d[i + k * step] = v[k];
  }
  for (; i < n; i += step) d[i] = s[i];
}

__global__ void __launch_bounds__(kStageThreads) stage_copy(StageList L) {
  if ((int)blockIdx.y >= L.n) return;
  const StageRange r = L.r[blockIdx.y];
  const unsigned char* s = static_cast<const unsigned char*>(r.src);
  unsigned char* d = static_cast<unsigned char*>(r.dst);
  const unsigned long long bytes = r.bytes;
  const unsigned long long sa = (unsigned long long)(size_t)s, da = (unsigned long long)(size_t)d;
  const unsigned long long w = ((sa ^ da) & 15ull) == 0 ? 16ull : ((sa ^ da) & 7ull) == 0 ? 8ull : 1ull;
  unsigned long long head = (w - (sa & (w - 1))) & (w - 1);
  if (head > bytes) head = bytes;
  const unsigned long long nw = (bytes - head) / w, tail0 = head + nw * w;
  // the unaligned head and the tail, byte by byte, by the first CTA
  if (blockIdx.x == 0) {
    for (unsigned long long i = threadIdx.x; i < head; i += blockDim.x) d[i] = s[i];
    for (unsigned long long i = tail0 + threadIdx.x; i < bytes; i += blockDim.x) d[i] = s[i];
  }
  if (w == 16)
    copy_words(reinterpret_cast<const uint4*>(s + head), reinterpret_cast<uint4*>(d + head), nw);
  else if (w == 8)
    copy_words(reinterpret_cast<const unsigned long long*>(s + head), reinterpret_cast<unsigned long long*>(d + head),
               nw);
  else
    copy_words(s + head, d + head, nw);
}

}  // namespace

cudaError_t launch_stage_copy(const StageList& L, int blocks_per_range, cudaStream_t st, long long* launches) {
  if (L.n <= 0) return cudaSuccess;
  if (L.n > kStageRangesMax || blocks_per_range < 1) return cudaErrorInvalidValue;
  stage_copy<<<dim3((unsigned)blocks_per_range, (unsigned)L.n), kStageThreads, 0, st>>>(L);
  *launches += 1;
  return cudaGetLastError();
}

}  // namespace gpa
