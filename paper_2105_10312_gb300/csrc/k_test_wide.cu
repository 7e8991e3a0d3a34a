// k_test_wide.cu — the candidate-test kernels (k_test.cu) built for sets of up
// to 256 tasks, in namespace gpa::wide (see gpa_ns.h).
#define GPA_WIDE 1
#include "k_test.cu"
