// k_alloc_wide.cu — the allocate kernels (k_alloc.cu) built for sets of up to
// 256 tasks, in namespace gpa::wide (see gpa_ns.h).
#define GPA_WIDE 1
#include "k_alloc.cu"
