// serve.cpp — continuous-batching admission-control server (filled in below).
#include "gpa_ctx.h"

void gpa_serve_teardown(gpa_ctx* c) { (void)c; }
