// gpa_ns.h — task capacity and namespace of the kernel code.
//
// The allocate and candidate-test kernels keep per-set state in shared memory
// and per-lane task masks in registers, both sized by the task capacity.
// They are compiled twice: for sets of up to 128 tasks in namespace gpa, and,
// with GPA_WIDE defined (k_alloc_wide.cu, k_test_wide.cu), for up to
// GPA_NMAX = 256 tasks in namespace gpa::wide.  The host picks the build by
// the batch's n_max, so batches of at most 128 tasks keep the smaller
// register and shared-memory budget.
#pragma once

#ifdef GPA_WIDE
#define GPA_KNMAX 256
#define GPA_NS_BEGIN \
  namespace gpa {    \
  namespace wide {
#define GPA_NS_END \
  }                \
  }
#else
#define GPA_KNMAX 128
#define GPA_NS_BEGIN namespace gpa {
#define GPA_NS_END }
#endif
