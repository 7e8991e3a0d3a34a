// k_probe.cu — execution time of a kernel as a function of the number of SMs
// it may use, measured the way §3 describes (Fig. 1): a blocker kernel takes
// sm_count - m SMs, and the kernel under test, launched on another stream,
// runs on the m SMs left.
//
// The blocker holds an SM by asking for the whole opt-in shared memory of a
// CTA (227 KB), so that no second CTA of any kernel fits beside it; its
// sm_count - m CTAs therefore sit on sm_count - m distinct SMs.  Each blocker
// CTA spins for a fixed time window read from %globaltimer (it never waits
// on another kernel) and, in the interference mode, streams a large buffer
// from HBM meanwhile, like the memory-intensive co-runner of §3.3.  Every
// CTA of both kernels records its %smid and the kernel under test its end
// time, so the host can check that the placement was disjoint, that exactly
// m SMs ran the kernel under test, and that it ended inside the window.
//
// Kernels under test (§3 used vector add, transpose, hotspot and pathfinder
// from the CUDA samples and Rodinia; these are written here from those
// kernels' published definitions):
//   vadd       c[i] = a[i] + b[i] over n floats, 16-byte accesses (memory-bound)
//   transpose  an n x n float matrix through 32 x 32 shared-memory tiles
//   stencil    one 5-point Jacobi sweep of an n x n grid (hotspot-like)
//   compute    64 dependent FMAs per element of n floats (compute-bound)
#include <cuda_runtime.h>

#include "gpa_internal.h"

namespace gpa {

namespace {

__device__ __forceinline__ unsigned long long probe_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned int probe_smid() {
  unsigned int s;
  asm volatile("mov.u32 %0, %%smid;" : "=r"(s));
  return s;
}

// One CTA per held SM (the dynamic shared memory request keeps any other CTA
// off it).  Spins until start + window_ns; with `buf`, reads it meanwhile.
__global__ void __launch_bounds__(1024, 1) probe_blocker(unsigned long long window_ns, const float4* __restrict__ buf,
                                                        unsigned long long buf_n, unsigned int* smid,
                                                        unsigned long long* t_end, float* sink) {
  extern __shared__ float4 hold[];
  const unsigned long long t0 = probe_ns();
  if (threadIdx.x == 0) {
    smid[blockIdx.x] = probe_smid();
    hold[0] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  const unsigned long long stop = t0 + window_ns;
  float acc = 0.f;
  // Eight coalesced 16-byte loads per thread per check of the clock (128 KB
  // in flight per SM): load k of thread t reads buf[i + k * nth], i = t + a
  // multiple of 8 nth kept below buf_n - 8 nth, so every index is < buf_n.
  const unsigned long long nth = (unsigned long long)gridDim.x * blockDim.x, tid = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x;
  const unsigned long long limit = buf && buf_n > 16 * nth ? buf_n - 8 * nth : 0ull;
  unsigned long long i = tid;
  while (probe_ns() < stop) {
    if (limit) {
      float4 v[8];
#pragma unroll
      for (int k = 0; k < 8; k++) v[k] = buf[i + k * nth];
#pragma unroll
      for (int k = 0; k < 8; k++) acc += v[k].x + v[k].y + v[k].z + v[k].w;
      i += 8 * nth;
      if (i >= limit) i = tid;
    }
  }
  if (threadIdx.x == 0) atomicMin(t_end, probe_ns());
  if (acc == 123456.f) sink[0] = acc;  // keeps the loads
}

__device__ __forceinline__ void probe_mark(unsigned int* smid, unsigned long long* t_done) {
  __syncthreads();
  if (threadIdx.x == 0) {
    smid[blockIdx.x] = probe_smid();
    atomicMax(t_done, probe_ns());
  }
}

// 16-byte accesses (the buffers come from cudaMalloc, so 16-byte aligned);
// the last n % 4 elements by the first CTA.
__global__ void __launch_bounds__(256) probe_vadd(const float* __restrict__ a, const float* __restrict__ b,
                                                  float* __restrict__ c, unsigned long long n, unsigned int* smid,
                                                  unsigned long long* t_done) {
  const unsigned long long step = (unsigned long long)gridDim.x * blockDim.x, n4 = n / 4;
  const float4* a4 = reinterpret_cast<const float4*>(a);
  const float4* b4 = reinterpret_cast<const float4*>(b);
  float4* c4 = reinterpret_cast<float4*>(c);
  for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += step) {
    const float4 x = a4[i], y = b4[i];
    c4[i] = make_float4(x.x + y.x, x.y + y.y, x.z + y.z, x.w + y.w);
  }
  if (blockIdx.x == 0)
    for (unsigned long long i = 4 * n4 + threadIdx.x; i < n; i += blockDim.x) c[i] = a[i] + b[i];
  probe_mark(smid, t_done);
}

// 32 x 32 tiles, 32 x 8 threads, padded shared tile (no bank conflicts).
__global__ void __launch_bounds__(256) probe_transpose(const float* __restrict__ in, float* __restrict__ out,
                                                       unsigned int n, unsigned int* smid,
                                                       unsigned long long* t_done) {
  __shared__ float tile[32][33];
  const unsigned int tiles = (n + 31) / 32;
  for (unsigned long long t = blockIdx.x; t < (unsigned long long)tiles * tiles; t += gridDim.x) {
    const unsigned int bx = (unsigned int)(t % tiles) * 32, by = (unsigned int)(t / tiles) * 32;
    for (unsigned int r = threadIdx.y; r < 32; r += 8) {
      const unsigned int x = bx + threadIdx.x, y = by + r;
      if (x < n && y < n) tile[r][threadIdx.x] = in[(unsigned long long)y * n + x];
    }
    __syncthreads();
    for (unsigned int r = threadIdx.y; r < 32; r += 8) {
      const unsigned int x = by + threadIdx.x, y = bx + r;
      if (x < n && y < n) out[(unsigned long long)y * n + x] = tile[threadIdx.x][r];
    }
    __syncthreads();
  }
  probe_mark(smid, t_done);
}

__global__ void __launch_bounds__(256) probe_stencil(const float* __restrict__ in, float* __restrict__ out,
                                                     unsigned int n, unsigned int* smid,
                                                     unsigned long long* t_done) {
  const unsigned long long cells = (unsigned long long)n * n;
  const unsigned long long step = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < cells; i += step) {
    const unsigned int x = (unsigned int)(i % n), y = (unsigned int)(i / n);
    const float c = in[i];
    const float l = x > 0 ? in[i - 1] : c, r = x + 1 < n ? in[i + 1] : c;
    const float u = y > 0 ? in[i - n] : c, d = y + 1 < n ? in[i + n] : c;
    out[i] = c + 0.1f * (l + r + u + d - 4.f * c);
  }
  probe_mark(smid, t_done);
}

__global__ void __launch_bounds__(256) probe_compute(const float* __restrict__ a, float* __restrict__ c,
                                                     unsigned long long n, unsigned int* smid,
                                                     unsigned long long* t_done) {
  const unsigned long long step = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += step) {
    float x = a[i], y = 1.0f;
#pragma unroll 16
    for (int k = 0; k < 64; k++) y = fmaf(y, x, 0.5f);
    c[i] = y;
  }
  probe_mark(smid, t_done);
}

}  // namespace

size_t probe_blocker_smem() { return 232448; }  // 227 KB: the opt-in maximum per CTA

cudaError_t probe_kernels_init() {
  return cudaFuncSetAttribute(probe_blocker, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)probe_blocker_smem());
}

cudaError_t launch_probe_blocker(int ctas, unsigned long long window_ns, const void* buf, unsigned long long buf_bytes,
                                 unsigned int* smid, unsigned long long* t_end, float* sink, cudaStream_t st) {
  if (ctas <= 0) return cudaSuccess;
  probe_blocker<<<ctas, 1024, probe_blocker_smem(), st>>>(window_ns, static_cast<const float4*>(buf), buf_bytes / 16,
                                                         smid, t_end, sink);
  return cudaGetLastError();
}

cudaError_t launch_probe_kernel(int kernel, int ctas, const ProbeBuffers& b, unsigned long long n,
                                unsigned int* smid, unsigned long long* t_done, cudaStream_t st) {
  switch (kernel) {
    case GPA_PROBE_VADD:
      probe_vadd<<<ctas, 256, 0, st>>>(b.a, b.b, b.c, n, smid, t_done);
      break;
    case GPA_PROBE_TRANSPOSE:
      probe_transpose<<<ctas, dim3(32, 8), 0, st>>>(b.a, b.c, (unsigned int)n, smid, t_done);
      break;
    case GPA_PROBE_STENCIL:
      probe_stencil<<<ctas, 256, 0, st>>>(b.a, b.c, (unsigned int)n, smid, t_done);
      break;
    case GPA_PROBE_COMPUTE:
      probe_compute<<<ctas, 256, 0, st>>>(b.a, b.c, n, smid, t_done);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace gpa
