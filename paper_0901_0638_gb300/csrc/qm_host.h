// qm_host.h -- host-side helpers shared by the library's translation units.
#pragma once

#include <cstddef>

#include "qm.h"

namespace qm {

qm_status fail(qm_status s, const char* fmt, ...);
qm_status check_launch(const char* what);
int sm_count();
bool bad_overlap(const void* a, size_t abytes, const void* b, size_t bbytes);

// FP64 normal quantile, fixed-point segment evaluation (qm_fixed.cu); u and z
// device arrays of n doubles, in place allowed; stream is a cudaStream_t.
qm_status launch_f64_fixed(const double* u, double* z, size_t n, void* stream);

}  // namespace qm
