// qm_paper.cu -- QM_VAR_PAPER_EXACT and QM_VAR_PAPER_EXACT_B: the paper's
// own normal quantiles, evaluated from its printed coefficients
// (qm_paper_coeffs.h) with the arithmetic it specifies, so that its accuracy
// and speed claims can be reproduced on GB300 beside this library's forms.
//
//   FP32 (Sec. 6.1, Appendix A): x = 2 min(u, 1-u) (exact), v = -log(x) by
//     the fast single-precision logarithm (__logf), the (5,6) rational by
//     Horner with FMA, |z| = (p / q) v with the fast division (__fdividef).
//   FP64, PAPER_EXACT_B (Sec. 7.2, Appendix B): the same steps in double with
//     the (13,13) rational, log, and the rounded reciprocal of q (__drcp_rn):
//     |z| = (p rcp(q)) v.  One branch-free form for the whole range.
//   FP64, PAPER_EXACT (Sec. 7.3, Appendix C): v = |u - 1/2| rsqrt(u - u^2)
//     (u - u^2 as one fused multiply-add, as the printed expression compiles
//     under nvcc's default contraction); if every lane of the warp has
//     v < 15.5 the warp takes the (14,15) t_2 rational, otherwise the whole
//     warp takes the Appendix B form.  Lanes past the end vote "inside".
//     Warps cover aligned groups of 32 consecutive elements, one per lane.
//
// The paper certifies these forms on v <= 25 (FP32) and v <= 42 (FP64,
// u >= 2.875e-19); further out the printed rationals are extrapolated as
// printed, with no deep-tail piece.  The library's IEEE contract replaces only
// what the printed forms leave undefined: u = 0 -> -inf, u = 1 -> +inf,
// u = 1/2 -> +0, u outside [0, 1] or NaN -> NaN.  (The FP32 form flushes
// x below 2^-126, u below 2^-127, to zero in __logf and returns NaN there,
// as printed.)
#include <cuda_runtime.h>
#include <stdint.h>

#include "qm.h"
#include "qm_host.h"
#include "qm_paper_coeffs.h"

namespace qm {
namespace {

constexpr int kBlock = 256;

__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }

// sum_k c[k] v^k by Horner's rule with one FMA per step (c[k]: v^k coefficient)
template <typename T, int N>
__device__ __forceinline__ T poly(const T (&c)[N], T v)
{
    T acc = c[N - 1];
#pragma unroll
    for (int k = N - 2; k >= 0; --k) acc = fma_rn(acc, v, c[k]);
    return acc;
}

__device__ __forceinline__ float paper_a(float u)
{
    const bool upper = u >= 0.5f;
    const float x = upper ? __fadd_rn(2.0f, -2.0f * u) : 2.0f * u;     // 2 min(u, 1-u), exact
    const float v = -__logf(x);
    const float mag = fabsf(__fmul_rn(__fdividef(poly(paper::A_P, v), poly(paper::A_Q, v)), v));
    float r = (x == 0.0f) ? __int_as_float(0x7f800000) : mag;
    r = (u >= 0.0f && u <= 1.0f) ? r : __int_as_float(0x7fffffff);
    return upper ? r : -r;
}

// |Phi^{-1}| of the Appendix B form at x = 2 min(u, 1-u)
__device__ __forceinline__ double paper_b_mag(double x)
{
    const double v = -log(x);
    return fabs(__dmul_rn(__dmul_rn(poly(paper::B_P, v), __drcp_rn(poly(paper::B_Q, v))), v));
}

__device__ __forceinline__ double paper_edges(double u, double x, double mag)
{
    double r = (x == 0.0) ? __longlong_as_double(0x7ff0000000000000ll) : mag;
    r = (u >= 0.0 && u <= 1.0) ? r : __longlong_as_double(0x7ff8000000000000ll);
    return (u >= 0.5) ? r : -r;
}

__device__ __forceinline__ double paper_b(double u)
{
    const double x = (u >= 0.5) ? __dadd_rn(2.0, -2.0 * u) : 2.0 * u;
    return paper_edges(u, x, paper_b_mag(x));
}

// Appendix C for one element; `valid` false for lanes past the end
__device__ __forceinline__ double paper_c(double u, bool valid)
{
    const double x = (u >= 0.5) ? __dadd_rn(2.0, -2.0 * u) : 2.0 * u;
    const double v = fabs(__dmul_rn(__dadd_rn(u, -0.5), rsqrt(__fma_rn(-u, u, u))));
    double mag;
    if (__all_sync(0xffffffffu, v < paper::C_VOTE_MAX || !valid))
        mag = fabs(__dmul_rn(__dmul_rn(poly(paper::C_P, v), __drcp_rn(poly(paper::C_Q, v))), v));
    else
        mag = paper_b_mag(x);
    return paper_edges(u, x, mag);
}

__global__ void __launch_bounds__(kBlock)
k_paper_a(const float* __restrict__ in, float* out, size_t n)
{
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t nv = ((uintptr_t)in % 16 == 0 && (uintptr_t)out % 16 == 0) ? n / 4 : 0;
    for (size_t i = t; i < nv; i += stride) {
        const float4 a = __ldcs(reinterpret_cast<const float4*>(in) + i);
        __stcs(reinterpret_cast<float4*>(out) + i,
               make_float4(paper_a(a.x), paper_a(a.y), paper_a(a.z), paper_a(a.w)));
    }
    for (size_t i = nv * 4 + t; i < n; i += stride) out[i] = paper_a(in[i]);
}

__global__ void __launch_bounds__(kBlock)
k_paper_b(const double* __restrict__ in, double* out, size_t n)
{
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t nv = ((uintptr_t)in % 16 == 0 && (uintptr_t)out % 16 == 0) ? n / 2 : 0;
    for (size_t i = t; i < nv; i += stride) {
        const double2 a = __ldcs(reinterpret_cast<const double2*>(in) + i);
        __stcs(reinterpret_cast<double2*>(out) + i, make_double2(paper_b(a.x), paper_b(a.y)));
    }
    for (size_t i = nv * 2 + t; i < n; i += stride) out[i] = paper_b(in[i]);
}

// One element per lane; the grid stride is a multiple of 32, so every warp
// covers an aligned group of 32 consecutive elements on every pass.
__global__ void __launch_bounds__(kBlock)
k_paper_c(const double* __restrict__ in, double* out, size_t n)
{
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t n_warps = (n + 31) / 32 * 32;        // every lane of a started warp joins the vote
    for (size_t i = t; i < n_warps; i += stride) {
        const bool valid = i < n;
        const double u = valid ? __ldcs(in + i) : 0.5;
        const double z = paper_c(u, valid);
        if (valid) __stcs(out + i, z);
    }
}

template <class Kern>
int persistent_grid(Kern k, size_t items)
{
    int bps = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k, kBlock, 0) != cudaSuccess || bps < 1)
        bps = 1;
    const int sms = sm_count() > 0 ? sm_count() : 1;
    size_t g = (items + kBlock - 1) / kBlock;
    const size_t cap = (size_t)sms * bps;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (int)g;
}

}  // namespace

qm_status launch_paper_f32(const float* u, float* z, size_t n, void* stream)
{
    k_paper_a<<<persistent_grid(k_paper_a, (n + 3) / 4), kBlock, 0, (cudaStream_t)stream>>>(u, z, n);
    return check_launch("f32 paper exact (Appendix A)");
}

qm_status launch_paper_f64(const double* u, double* z, size_t n, int with_vote, void* stream)
{
    cudaStream_t s = (cudaStream_t)stream;
    if (with_vote)
        k_paper_c<<<persistent_grid(k_paper_c, n), kBlock, 0, s>>>(u, z, n);
    else
        k_paper_b<<<persistent_grid(k_paper_b, (n + 1) / 2), kBlock, 0, s>>>(u, z, n);
    return check_launch(with_vote ? "f64 paper exact (Appendix C)" : "f64 paper exact (Appendix B)");
}

}  // namespace qm
