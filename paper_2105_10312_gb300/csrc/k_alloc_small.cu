// k_alloc_small.cu — the allocate kernels (k_alloc.cu) built for sets of up
// to 64 tasks, in namespace gpa::small (see gpa_ns.h).
#define GPA_SMALL 1
#include "k_alloc.cu"
