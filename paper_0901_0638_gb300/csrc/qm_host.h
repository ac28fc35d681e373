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
// The paper's own kernels from its printed coefficients (qm_paper.cu):
// Appendix A in FP32; Appendix C (with_vote = 1) or Appendix B in FP64.
qm_status launch_paper_f32(const float* u, float* z, size_t n, void* stream);
qm_status launch_paper_f64(const double* u, double* z, size_t n, int with_vote, void* stream);
// Device address of the fixed-point FP64 table (fxt::SEG_FX) on the current
// device, or NULL with *st set.
const void* fx_table_device(qm_status* st);

// Normal -> Student t tables for nu in [QM_T_NU_MIN, QM_T_NU_MAX] (qm_tdyn.cu):
// host build (seg: NSEG x 10 coefficients, tail: nu, log kappa, degree, R_k)
// and the current device's copy, built and uploaded at first use.
qm_status t_table_build(double nu, double* seg, double* tail);
qm_status t_table_device(double nu, const void** seg_dev, const double** tail_dev);
// Index of nu in the tabulated set (or -1) and, for other nu in range, the
// run-time tables: fills k, seg, tail of a TSel-shaped record (qm_device.cuh).
qm_status t_select(double nu, int* k, const void** seg_dev, const double** tail_dev);

// t-copula recycling tables for nu (qm_tcop_tables.cu): host build (layout of
// qm_tcopula_table_build) and the current device's copy, built at first use.
qm_status tcop_table_build(double nu, double* chi_seg, double* g_seg, int* ne);
// Device layout: 64-byte rows (coefficients 0..4 double, 5..9 float, the
// Student-t segment layout) followed by one double per row (centre or 1 / m_c).
qm_status tcop_table_device(double nu, const void** chi, const void** g, const void** fx, int* ne);

}  // namespace qm
