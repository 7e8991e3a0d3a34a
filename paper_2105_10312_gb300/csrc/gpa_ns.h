// gpa_ns.h — task capacity and namespace of the kernel code.
//
// The allocate and candidate-test kernels keep per-set state in shared memory
// and per-lane task masks in registers, both sized by the task capacity.
// They are compiled for sets of up to 128 tasks in namespace gpa; the
// allocate kernels also, with GPA_SMALL defined (k_alloc_small.cu), for up to
// 64 tasks in namespace gpa::small, and both, with GPA_WIDE defined
// (k_alloc_wide.cu, k_test_wide.cu), for up to GPA_NMAX = 256 tasks in
// namespace gpa::wide.  The host picks the build by the batch's n_max, so a
// batch pays only for the capacity it uses: more merge warps fit on an SM
// with the 64-task state, and batches of at most 128 tasks never carry the
// 256-task state.
#pragma once

// GPA_MERGE_MINB: CTAs of 256 threads the merge kernel's registers must
// allow per SM; the 64-task build keeps its state in 128 registers (more
// sets in flight: paper50 2.7 -> 2.2 ms), the larger builds in up to 255
// (fewer spills: 200-task sets 126 -> 114 ms).  GPA_ONEGPU_MINB: the same
// for the 1G kernel (64-task build: 64 registers, 1 000 000 sets 2.43 ->
// 1.96 ms against no limit).
#if defined(GPA_WIDE)
#define GPA_KNMAX 256
#define GPA_MERGE_MINB 1
#define GPA_ONEGPU_MINB 1
#define GPA_NS_BEGIN \
  namespace gpa {    \
  namespace wide {
#define GPA_NS_END \
  }                \
  }
#elif defined(GPA_SMALL)
#define GPA_KNMAX 64
#define GPA_MERGE_MINB 2
#define GPA_ONEGPU_MINB 4
#define GPA_NS_BEGIN \
  namespace gpa {    \
  namespace small {
#define GPA_NS_END \
  }                \
  }
#else
#define GPA_KNMAX 128
#define GPA_MERGE_MINB 1
#define GPA_ONEGPU_MINB 1
#define GPA_NS_BEGIN namespace gpa {
#define GPA_NS_END }
#endif
