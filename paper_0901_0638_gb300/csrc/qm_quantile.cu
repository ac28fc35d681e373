// qm_quantile.cu -- streaming normal-quantile kernels, Philox fill, fused
// generate+transform, the exponential->normal recycling map, and their C ABI.
//
// Kernel shapes (sm_103a, 152 SMs):
//   * map kernels: persistent grid-stride over 128-bit vectors (float4 /
//     double2), U independent vectors in flight per thread, streaming cache
//     hints (ld.global.cs / st.global.cs); scalar tail.  Grid = SMs x resident
//     blocks per SM.
//   * COMPACT (FP64): per 1024-element tile, every element whose t_2
//     coordinate is below 15.5 is finished in place; the rest are appended to
//     two shared-memory queues (exponential main piece, deep tail) with
//     warp-aggregated atomics and evaluated densely by the whole block.
//   * HYBRID_VOTE (FP64): the Sec. 7.3 warp vote with __all_sync.
#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <mutex>
#include <string>

#include "qm.h"
#include "qm_device.cuh"
#include "qm_fx.cuh"
#include "qm_exp_map.cuh"
#include "qm_host.h"
#include "qm_tables_deep.h"
#include "qm_filter_coeffs.h"

namespace qm {

// ===========================================================================
// Error reporting
// ===========================================================================
static thread_local std::string g_last_error;

qm_status fail(qm_status s, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return s;
}

qm_status check_launch(const char* what)
{
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return fail(QM_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
    return QM_OK;
}

int sm_count()
{
    static int cached[64];
    static std::once_flag once[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return -1;
    std::call_once(once[dev], [dev] {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) v = -1;
        cached[dev] = v;
    });
    return cached[dev];
}

bool bad_overlap(const void* a, size_t abytes, const void* b, size_t bbytes)
{
    const char* pa = (const char*)a;
    const char* pb = (const char*)b;
    if (pa == pb) return false;  // exact in-place is allowed
    return pa < pb + bbytes && pb < pa + abytes;
}

// ===========================================================================
// Element functors
// ===========================================================================
struct F32Sqrt   { __device__ float operator()(float u) const { return probit_f32<FORM_SQRT>(u); } };
struct F32Paper  { __device__ float operator()(float u) const { return probit_f32<FORM_PAPER>(u); } };
struct F32Libm   { __device__ float operator()(float u) const { return normcdfinvf(u); } };
struct F32Table  { __device__ float operator()(float u) const { return probit_f32_tbl(u); } };

struct F64BranchFree {
    __device__ double operator()(double u) const
    {
        const double d = reflect_f64(u);
        const double v = -log(2.0 * d);
        const double m = is_deep(d) ? probit_mag_exp_deep(v) : probit_mag_exp_main(v);
        return fix_edges_f64(u, d, m);
    }
};
struct F64Mixed {
    __device__ double operator()(double u) const
    {
        const double d = reflect_f64(u);
        const double m = (d > 0.0 && d <= 0.5) ? probit_mag_mixed(d) : 0.0;
        return fix_edges_f64(u, d, m);
    }
};
struct F64Libm { __device__ double operator()(double u) const { return normcdfinv(u); } };

// ---------------------------------------------------------------------------
// Almost-normal / almost-chi-squared filtering coordinates (Sec. 4.4):
//     a = -(pi/2) log(4 d (1 - d)) = Q_AN(u)^2,  w = sqrt(a) = |Q_AN(u)|,
//     a <= 8: |z| = (1 - 2d) P(a - a_c);   a > 8: |z| = T_k(w - w_c).
// 4 d (1 - d) = (2d)(2 - 2d): 2d is exact, 2 - 2d rounds once.
// ---------------------------------------------------------------------------
constexpr double kHalfPi = 1.5707963267948966;

// FP64: every piece is a degree-20 polynomial, so one Horner loop runs over
// the lane's coefficient row (no divergent branch).  d in (0, 1/2].
__device__ __forceinline__ double probit_mag_an64(double d)
{
    const double t4 = __dmul_rn(2.0 * d, __fma_rn(-2.0, d, 2.0));
    const double a = fmax(-kHalfPi * log(t4), 0.0);
    const bool centre = a <= filt::AN_A0;
    const double w = sqrt(a);
    const int row = centre ? 0
        : 1 + (w > filt::AN64_WHI[0]) + (w > filt::AN64_WHI[1]) + (w > filt::AN64_WHI[2]);
    const double* c = filt::AN64[row];
    const double s = __dadd_rn(centre ? a : w, -__ldg(c));
    double acc = __ldg(c + filt::AN64_DEG + 1);
#pragma unroll
    for (int k = filt::AN64_DEG; k >= 1; --k) acc = __fma_rn(acc, s, __ldg(c + k));
    const double f = centre ? __fma_rn(-2.0, d, 1.0) : 1.0;
    return __dmul_rn(f, acc);
}

struct F64AlmostNormal {
    __device__ double operator()(double u) const
    {
        const double d = reflect_f64(u);
        const double m = (d > 0.0 && d <= 0.5) ? probit_mag_an64(d) : 0.0;
        return fix_edges_f64(u, d, m);
    }
};

// FP32: centre polynomial with its coefficients as constant operands; the
// tail (d < 1.7e-3) reads one of two rows.  d in (0, 1/2]; d below 2^-100 is
// scaled by 2^64 before the MUFU logarithm, which flushes subnormals.
__device__ __forceinline__ float probit_mag_an32(float d)
{
    const bool tiny = d < 7.888609052210118e-31f;                      // 2^-100
    const float ds = tiny ? d * 1.8446744073709552e19f : d;              // 2^64
    const float t4 = __fmul_rn(2.0f * ds, __fmaf_rn(-2.0f, d, 2.0f));
    const float lg = __log2f(t4) - (tiny ? 64.0f : 0.0f);
    const float a = fmaxf(-1.0887930451518f * lg, 0.0f);                // (pi/2) ln 2
    if (a <= (float)filt::AN_A0) {
        const float s = a - filt::AN32_C_OFF;
        float acc = filt::AN32_C[filt::AN32_DEG];
#pragma unroll
        for (int k = filt::AN32_DEG - 1; k >= 0; --k) acc = __fmaf_rn(acc, s, filt::AN32_C[k]);
        return __fmul_rn(__fmaf_rn(-2.0f, d, 1.0f), acc);
    }
    const float w = sqrtf(a);
    const float* c = filt::AN32_T[w > filt::AN32_WHI0 ? 1 : 0];
    const float s = w - __ldg(c);
    float acc = __ldg(c + filt::AN32_DEG + 1);
#pragma unroll
    for (int k = filt::AN32_DEG; k >= 1; --k) acc = __fmaf_rn(acc, s, __ldg(c + k));
    return acc;
}

struct F32AlmostNormal {
    __device__ float operator()(float u) const
    {
        const bool upper = u >= 0.5f;
        const float d = upper ? __fadd_rn(1.0f, -u) : u;   // exact for u >= 1/2
        float mag = (d > 0.0f && d <= 0.5f) ? probit_mag_an32(d) : 0.0f;
        mag = (d == 0.0f) ? __int_as_float(0x7f800000) : mag;
        mag = (u >= 0.0f && u <= 1.0f) ? mag : __int_as_float(0x7fffffff);
        return upper ? mag : -mag;
    }
};

// ---------------------------------------------------------------------------
// t_2 coordinate with more branches (Sec. 7.4): the Sec. 7.3 rational on
// v <= 15.5 and a second (14,15) rational on the near tail 15.5 < v <= 1000,
// one evaluation with the coefficients selected per lane.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double probit_mag_t2_two(double v)
{
    const bool near = v > 15.5;
    double p = near ? filt::T2N_P[14] : coef::F64_T2_P[14];
#pragma unroll
    for (int k = 13; k >= 0; --k) p = __fma_rn(p, v, near ? filt::T2N_P[k] : coef::F64_T2_P[k]);
    double q = near ? filt::T2N_Q[15] : coef::F64_T2_Q[15];
#pragma unroll
    for (int k = 14; k >= 0; --k) q = __fma_rn(q, v, near ? filt::T2N_Q[k] : coef::F64_T2_Q[k]);
    return __dmul_rn(v, div_f64(p, q));
}

__device__ __forceinline__ bool in_t2_multi_domain(double d) { return d > filt::T2N_D_LO; }

// element-wise form (in-place calls): the far tail as a divergent branch
struct F64T2Multi {
    __device__ double operator()(double u) const
    {
        const double d = reflect_f64(u);
        double m = 0.0;
        if (in_t2_multi_domain(d)) m = probit_mag_t2_two(t2_coord(d));
        else if (d > 0.0) m = probit_mag_f64_exp(d);
        return fix_edges_f64(u, d, m);
    }
};

struct ExpToNormal {
    __device__ double operator()(double x) const { return exp_to_normal_fx(x); }
};

struct TDynMap {
    const ttbl::TRows* seg;
    const double* tail;
    __device__ double operator()(double z) const { return recycle_t_dyn(seg, tail, z); }
};

// ===========================================================================
// Generic streaming map
// ===========================================================================
template <typename T> struct Vec;
template <> struct Vec<float>  { using type = float4;  static constexpr int W = 4; };
template <> struct Vec<double> { using type = double2; static constexpr int W = 2; };

template <typename V, class F>
__device__ __forceinline__ V apply_vec(V a, const F& f);
template <class F>
__device__ __forceinline__ float4 apply_vec(float4 a, const F& f)
{
    return make_float4(f(a.x), f(a.y), f(a.z), f(a.w));
}
template <class F>
__device__ __forceinline__ double2 apply_vec(double2 a, const F& f)
{
    return make_double2(f(a.x), f(a.y));
}

// MINB: resident blocks per SM the compiler must allow (register cap); the
// single-precision maps are latency bound at low occupancy.
template <typename T, int U, class F, int MINB = 1>
__global__ void __launch_bounds__(256, MINB)
k_map_vec(const T* __restrict__ in, T* out, size_t n, F f)
{
    using V = typename Vec<T>::type;
    constexpr int W = Vec<T>::W;
    const size_t nv = n / W;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    const V* vin = reinterpret_cast<const V*>(in);
    V* vout = reinterpret_cast<V*>(out);
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += stride * U) {
        V a[U];
#pragma unroll
        for (int k = 0; k < U; ++k)
            if (i + k * stride < nv) a[k] = __ldcs(vin + i + k * stride);
#pragma unroll
        for (int k = 0; k < U; ++k)
            if (i + k * stride < nv) __stcs(vout + i + k * stride, apply_vec(a[k], f));
    }
    const size_t tail = nv * W;
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n - tail) out[tail + t] = f(in[tail + t]);
}

template <typename T, class F>
__global__ void __launch_bounds__(256)
k_map_scalar(const T* in, T* out, size_t n, F f)
{
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        out[i] = f(in[i]);
}

// Blocks for `work_items` threads of `block`, at most `waves` x the blocks
// resident at once (1: a persistent grid-stride launch).
template <typename K>
static int grid_for(K kernel, int block, size_t work_items, int waves = 1)
{
    int bps = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kernel, block, 0) != cudaSuccess || bps < 1)
        bps = 1;
    const int sms = sm_count() > 0 ? sm_count() : 1;
    size_t g = (work_items + block - 1) / block;
    size_t cap = (size_t)sms * bps * waves;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (int)g;
}

// MINB: single-precision maps 6 blocks of 256 per SM; double-precision maps 4
// (a 64-register cap: the Student-t map at its compiler's choice of 89
// registers held 2 blocks, 137 Gs/s, and 175.6 at 4, measured), over 16
// waves of resident blocks
template <typename T, class F>
static qm_status launch_map(const T* in, T* out, size_t n, F f, cudaStream_t s, const char* what)
{
    constexpr int U = 2, B = 256;
    constexpr int MINB = sizeof(T) == 4 ? 6 : 4;
    constexpr int WAVES = sizeof(T) == 4 ? 1 : 16;
    const bool aligned = ((uintptr_t)in % 16 == 0) && ((uintptr_t)out % 16 == 0);
    if (aligned) {
        const size_t nv = n / Vec<T>::W;
        const int g = grid_for(k_map_vec<T, U, F, MINB>, B, (nv + U - 1) / U > 0 ? (nv + U - 1) / U : 1, WAVES);
        k_map_vec<T, U, F, MINB><<<g, B, 0, s>>>(in, out, n, f);
    } else {
        const int g = grid_for(k_map_scalar<T, F>, B, n);
        k_map_scalar<T, F><<<g, B, 0, s>>>(in, out, n, f);
    }
    return check_launch(what);
}

// ===========================================================================
// FP32 TABLE map: one check per float4 for the rare edge inputs (0, 1, 1/2,
// tiny or out of range, NaN); the common case runs the short table path on
// all four lanes of the vector with no per-element branch.  The kernel is
// bound by the L1 (the streaming traffic plus one 16-byte table gather per
// element), so the common path is kept to as few instructions as possible:
// x = 2d = min(2u, 2 - 2u) (Sec. 6.1; 2 - 2u is exact for u >= 1/2 and
// above 1 otherwise), the range check on x (normal and below 1, which also
// excludes u = 1/2, u = 1, u <= 0, u > 1 and NaN), and the sign of
// u - 1/2 applied to |z| by one logic operation.
// ===========================================================================
__device__ __forceinline__ float f32_x(float u)
{
    return fminf(2.0f * u, __fmaf_rn(-2.0f, u, 2.0f));
}

__device__ __forceinline__ bool f32_x_common(float x)
{
    return __float_as_uint(x) - 0x00800000u < 0x3f800000u - 0x00800000u;
}

// -g for u < 1/2, +g for u > 1/2 (g = |z|)
__device__ __forceinline__ float f32_signed(float g, float u)
{
    const uint32_t q = __float_as_uint(__fadd_rn(u, -0.5f));
    return __uint_as_float(__float_as_uint(g) ^ (q & 0x80000000u));
}

__device__ __forceinline__ float4 f32_table4(float4 v)
{
    const float4 x = make_float4(f32_x(v.x), f32_x(v.y), f32_x(v.z), f32_x(v.w));
    if (f32_x_common(x.x) && f32_x_common(x.y) && f32_x_common(x.z) && f32_x_common(x.w))
        return make_float4(f32_signed(tbl32_core(x.x), v.x), f32_signed(tbl32_core(x.y), v.y),
                           f32_signed(tbl32_core(x.z), v.z), f32_signed(tbl32_core(x.w), v.w));
    return make_float4(probit_f32_tbl(v.x), probit_f32_tbl(v.y), probit_f32_tbl(v.z),
                       probit_f32_tbl(v.w));
}

// U float4 loads in flight per thread; the main loop runs over whole groups
// of U without bounds checks, then a remainder loop, then the scalar tail.
// Four blocks of 256 per SM (64 registers) measured faster than six.
template <int U>
__global__ void __launch_bounds__(256, 4)
k_f32_table(const float* __restrict__ in, float* out, size_t n)
{
    const size_t nv = n / 4;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    const float4* vin = reinterpret_cast<const float4*>(in);
    float4* vout = reinterpret_cast<float4*>(out);
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (; i + (U - 1) * stride < nv; i += stride * U) {
        float4 a[U];
#pragma unroll
        for (int k = 0; k < U; ++k) a[k] = __ldcs(vin + i + k * stride);
#pragma unroll
        for (int k = 0; k < U; ++k) __stcs(vout + i + k * stride, f32_table4(a[k]));
    }
    for (; i < nv; i += stride) __stcs(vout + i, f32_table4(__ldcs(vin + i)));
    const size_t tail = nv * 4;
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n - tail) out[tail + t] = probit_f32_tbl(in[tail + t]);
}

// ===========================================================================
// FP64 hybrid with the warp vote (Sec. 7.3): every lane holds one element;
// if all 32 t_2 coordinates are below 15.5 the warp takes the t_2 rational,
// otherwise the whole warp takes the exponential form.
// ===========================================================================
__device__ __forceinline__ double hybrid_vote_elem(double u, bool valid)
{
    const double d = reflect_f64(u);
    const bool t2 = in_t2_domain(d) || !valid;
    double m;
    if (__all_sync(0xffffffffu, t2)) {
        m = probit_mag_t2(t2_coord(d));
    } else {
        const double v = -log(2.0 * d);
        m = is_deep(d) ? probit_mag_exp_deep(v) : probit_mag_exp_main(v);
    }
    return fix_edges_f64(u, d, m);
}

template <int U>
__global__ void __launch_bounds__(256)
k_f64_hybrid_vote(const double* __restrict__ in, double* out, size_t n)
{
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    const size_t warp_base0 = ((size_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u));
    const unsigned lane = threadIdx.x & 31u;
    for (size_t wb = warp_base0; wb < n; wb += stride * U) {
        double a[U];
#pragma unroll
        for (int k = 0; k < U; ++k) {
            const size_t i = wb + k * stride + lane;
            a[k] = (i < n) ? __ldcs(in + i) : 0.5;
        }
#pragma unroll
        for (int k = 0; k < U; ++k) {
            const size_t i = wb + k * stride + lane;
            const double z = hybrid_vote_elem(a[k], i < n);
            if (i < n) __stcs(out + i, z);
        }
    }
}

// ===========================================================================
// FP64 COMPACT: t_2 in place, compacted exponential / deep-tail queues.
// ===========================================================================
constexpr int kCompactBlock = 256;
constexpr int kCompactEPT = 4;
constexpr int kCompactTile = kCompactBlock * kCompactEPT;

__device__ __forceinline__ void queue_push(bool pred, int* counter, unsigned short* q,
                                           unsigned short idx)
{
    const unsigned mask = __ballot_sync(0xffffffffu, pred);
    if (mask == 0) return;
    const unsigned lane = threadIdx.x & 31u;
    const int leader = __ffs(mask) - 1;
    int base = 0;
    if ((int)lane == leader) base = atomicAdd(counter, __popc(mask));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (pred) q[base + __popc(mask & ((1u << lane) - 1u))] = idx;
}

// MULTI: the in-place branch is the two-piece t_2 form on v <= 1000 (Sec. 7.4)
// instead of the Sec. 7.3 rational on v <= 15.5.
template <bool MULTI>
__global__ void __launch_bounds__(kCompactBlock)
k_f64_compact(const double* __restrict__ in, double* out, size_t n)
{
    __shared__ unsigned short q_exp[kCompactTile];
    __shared__ unsigned short q_deep[kCompactTile];
    __shared__ int cnt[2];
    const size_t ntiles = (n + kCompactTile - 1) / kCompactTile;
    for (size_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const size_t base = tile * kCompactTile;
        if (threadIdx.x < 2) cnt[threadIdx.x] = 0;
        __syncthreads();
        double a[kCompactEPT];
#pragma unroll
        for (int k = 0; k < kCompactEPT; ++k) {
            const size_t i = base + k * kCompactBlock + threadIdx.x;
            a[k] = (i < n) ? __ldcs(in + i) : 0.5;
        }
#pragma unroll
        for (int k = 0; k < kCompactEPT; ++k) {
            const unsigned short li = (unsigned short)(k * kCompactBlock + threadIdx.x);
            const size_t i = base + li;
            const double u = a[k];
            const double d = reflect_f64(u);
            const bool edge = !(d > 0.0 && d <= 0.5);       // 0, NaN, out of range
            const bool t2 = !edge && (MULTI ? in_t2_multi_domain(d) : in_t2_domain(d));
            const bool deep = !edge && !t2 && is_deep(d);
            const bool ex = !edge && !t2 && !deep;
            if (i < n && (t2 || edge)) {
                const double m = t2 ? (MULTI ? probit_mag_t2_two(t2_coord(d)) : probit_mag_t2(t2_coord(d)))
                                    : 0.0;
                __stcs(out + i, fix_edges_f64(u, d, m));
            }
            queue_push(i < n && ex, &cnt[0], q_exp, li);
            queue_push(i < n && deep, &cnt[1], q_deep, li);
        }
        __syncthreads();
        const int ne = cnt[0], nd = cnt[1];
        for (int j = threadIdx.x; j < ne; j += kCompactBlock) {
            const size_t i = base + q_exp[j];
            const double u = in[i];
            const double d = reflect_f64(u);
            const double m = probit_mag_exp_main(-log(2.0 * d));
            out[i] = fix_edges_f64(u, d, m);
        }
        for (int j = threadIdx.x; j < nd; j += kCompactBlock) {
            const size_t i = base + q_deep[j];
            const double u = in[i];
            const double d = reflect_f64(u);
            const double m = probit_mag_exp_deep(-log(2.0 * d));
            out[i] = fix_edges_f64(u, d, m);
        }
        __syncthreads();
    }
}

// ===========================================================================
// FP64 TABLE: table-driven exponential coordinate for every normal d (main
// and deep tables), subnormal d (u < 2.2e-308) compacted per tile and
// evaluated densely with the deep rational.
// Reflection, domain tests and the sign use integer operations on the bits
// (the FP64 pipe is the bottleneck on this part).
// ===========================================================================
// |Phi^{-1}| for normal d in [2^-1022, 1/2): main table (k = 6) for
// E >= -64, deep table (k = 5) below; one code path, the table chosen by
// integer selects.
__device__ __forceinline__ double probit_mag_f64_tbl_full(double d)
{
    const uint64_t b = (uint64_t)__double_as_longlong(d) + (1ull << 52);   // x = 2d
    const int E0 = (int)(b >> 52) - 1023;
    const int E = min(E0, -1);                          // d = 1/2 (x = 1): +0 below
    const double m = __longlong_as_double((long long)((b & 0x000fffffffffffffull) | 0x3ff0000000000000ull));
    const int j6 = (int)((b >> (52 - tbl::F64_K)) & ((1u << tbl::F64_K) - 1));
    const int j5 = (int)((b >> (52 - tbl::DEEP_K)) & ((1u << tbl::DEEP_K) - 1));
    const tbl::SegF64* e = (E >= tbl::F64_EMIN)
        ? &tbl::SEG_F64[(-1 - E) * (1 << tbl::F64_K) + j6]
        : &tbl::SEG_F64_DEEP[(tbl::DEEP_EHI - E) * (1 << tbl::DEEP_K) + j5];
    const double g = f64_seg_eval(e, m);
    return (E0 >= 0) ? 0.0 : g;
}

__global__ void __launch_bounds__(kCompactBlock)
k_f64_table(const double* __restrict__ in, double* out, size_t n)
{
    __shared__ unsigned short q_deep[kCompactTile];
    __shared__ int cnt;
    const size_t ntiles = (n + kCompactTile - 1) / kCompactTile;
    for (size_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const size_t base = tile * kCompactTile;
        if (threadIdx.x == 0) cnt = 0;
        __syncthreads();
        double a[kCompactEPT];
#pragma unroll
        for (int k = 0; k < kCompactEPT; ++k) {
            const size_t i = base + k * kCompactBlock + threadIdx.x;
            a[k] = (i < n) ? __ldcs(in + i) : 0.5;
        }
#pragma unroll
        for (int k = 0; k < kCompactEPT; ++k) {
            const unsigned short li = (unsigned short)(k * kCompactBlock + threadIdx.x);
            const size_t i = base + li;
            const double u = a[k];
            const long long ub = __double_as_longlong(u);
            const bool upper = ub >= 0x3FE0000000000000ll;                // u >= 1/2
            const bool valid = ub > 0 && ub < 0x3FF0000000000000ll;       // 0 < u < 1
            const double d = upper ? one_minus_upper(u) : u;                 // exact
            const bool covers = valid && __double_as_longlong(d) >= 0x0010000000000000ll;  // normal d
            if (i < n && !(valid && !covers)) {
                double m = covers ? probit_mag_f64_tbl_full(d) : 0.0;
                long long mb = __double_as_longlong(m) & 0x7fffffffffffffffll;
                if (!valid) {
                    const bool zero = (ub & 0x7fffffffffffffffll) == 0;
                    mb = zero ? (0x7ff0000000000000ll | (1ll << 63))
                              : (ub == 0x3FF0000000000000ll ? 0x7ff0000000000000ll : 0x7ff8000000000000ll);
                } else if (!upper) {
                    mb |= (1ll << 63);
                }
                __stcs(out + i, __longlong_as_double(mb));
            }
            queue_push(i < n && valid && !covers, &cnt, q_deep, li);
        }
        __syncthreads();
        const int nd = cnt;
        for (int j = threadIdx.x; j < nd; j += kCompactBlock) {
            const size_t i = base + q_deep[j];
            const double u = in[i];
            const double d = reflect_f64(u);
            const double m = probit_mag_exp_deep(-log(2.0 * d));
            out[i] = fix_edges_f64(u, d, m);
        }
        __syncthreads();
    }
}

// ===========================================================================
// Philox fill, 24-bit grid transform, fused generate + transform
// ===========================================================================
__device__ __forceinline__ uint32_t word_of(uint4 b, unsigned j)
{
    return j == 0 ? b.x : j == 1 ? b.y : j == 2 ? b.z : b.w;
}

__global__ void __launch_bounds__(256)
k_philox_fill(PhiloxKeys K, uint64_t ctr0, uint32_t* out, size_t n)
{
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    const uint64_t first_blk = ctr0 >> 2;
    const unsigned off = (unsigned)(ctr0 & 3);
    // thread t produces words of blocks first_blk + t, + stride, ...
    const size_t nblk = (off + n + 3) / 4;
    for (size_t b = (size_t)blockIdx.x * blockDim.x + threadIdx.x; b < nblk; b += stride) {
        const uint4 w = philox_block_keys(K, first_blk + b);
#pragma unroll
        for (unsigned j = 0; j < 4; ++j) {
            const long long i = (long long)(b * 4 + j) - (long long)off;
            if (i >= 0 && (size_t)i < n) out[i] = word_of(w, j);
        }
    }
}

__global__ void __launch_bounds__(256)
k_bits24_f32(const uint32_t* __restrict__ words, float* z, size_t n)
{
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        z[i] = probit_grid24_tbl(words[i] >> 8);
}

// Per-block partial moments -> partials[blockIdx.x * 4 + k].
__device__ __forceinline__ void block_reduce4(double s[4], double* partials)
{
    __shared__ double red[32][4];
#pragma unroll
    for (int k = 0; k < 4; ++k)
        for (int o = 16; o > 0; o >>= 1) s[k] += __shfl_xor_sync(0xffffffffu, s[k], o);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0)
        for (int k = 0; k < 4; ++k) red[warp][k] = s[k];
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
        for (int k = 0; k < 4; ++k) {
            double v = lane < nw ? red[lane][k] : 0.0;
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) partials[blockIdx.x * 4 + k] = v;
        }
    }
}

__global__ void k_sum_partials(const double* partials, int nblocks, double* moments)
{
    // one warp per moment, fixed summation order
    const int k = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (k >= 4) return;
    double v = 0.0;
    for (int b = lane; b < nblocks; b += 32) v += partials[b * 4 + k];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) moments[k] = v;
}

// Moments are accumulated per thread in FP32 over 64 samples (16 Philox
// blocks), then folded into FP64 accumulators.
template <bool OUT, bool MOM>
__global__ void __launch_bounds__(256)
k_fused_normal_f32(PhiloxKeys K, uint64_t blk0, size_t n, float* out, double* partials)
{
    __shared__ float4 stbl[kF32SmemSeg];
    stage_f32_table(stbl);
    __syncthreads();
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    const size_t nblk = (n + 3) / 4;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    float f1 = 0.f, f2 = 0.f, f3 = 0.f, f4 = 0.f;
    int cnt = 0;
    const bool vec_ok = OUT && ((uintptr_t)out % 16 == 0);
    for (size_t b = (size_t)blockIdx.x * blockDim.x + threadIdx.x; b < nblk; b += stride) {
        const uint4 w = philox_block_keys(K, blk0 + b);
        float z[4];
        z[0] = probit_grid24_word_s(w.x, stbl);
        z[1] = probit_grid24_word_s(w.y, stbl);
        z[2] = probit_grid24_word_s(w.z, stbl);
        z[3] = probit_grid24_word_s(w.w, stbl);
        const size_t i0 = b * 4;
        const bool full = i0 + 4 <= n;
        if (OUT) {
            if (full && vec_ok) {
                __stcs(reinterpret_cast<float4*>(out + i0), make_float4(z[0], z[1], z[2], z[3]));
            } else {
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (i0 + j < n) out[i0 + j] = z[j];
            }
        }
        if (MOM) {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float x = (i0 + j < n) ? z[j] : 0.0f;
                const float x2 = x * x;
                f1 += x;
                f2 += x2;
                f3 = __fmaf_rn(x2, x, f3);
                f4 = __fmaf_rn(x2, x2, f4);
            }
            if (++cnt == 16) {
                acc[0] += f1; acc[1] += f2; acc[2] += f3; acc[3] += f4;
                f1 = f2 = f3 = f4 = 0.f;
                cnt = 0;
            }
        }
    }
    if (MOM) {
        acc[0] += f1; acc[1] += f2; acc[2] += f3; acc[3] += f4;
        block_reduce4(acc, partials);
    }
}

// FP64 normal samples: block b gives two samples from 53-bit integers
// k = (w0 >> 11) 2^32 + w1 and (w2 >> 11) 2^32 + w3, evaluated at the exact
// reflected point d = (min(k, 2^53-1-k) + 1/2) 2^-53 by the fixed-point FP64
// evaluation of the Sec. 7.3 segment expansions.  KIND 0: normal; KIND 2:
// exponential -> normal with x = -log((k + 1/2) 2^-53).

template <int KIND, bool OUT, bool MOM>
__global__ void __launch_bounds__(256)
k_fused_f64(PhiloxKeys K, uint64_t blk0, size_t n, double* out, double* partials, TSel tk,
            const fxt::FxTable* fxT)
{
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    const size_t nblk = (n + 1) / 2;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    const size_t warp0 = (size_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u);
    const unsigned lane = threadIdx.x & 31u;
    for (size_t wb = warp0; wb < nblk; wb += stride) {
        const size_t b = wb + lane;
        const bool valid = b < nblk;
        const uint4 w = philox_block_keys(K, blk0 + b);
        double z[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            bool upper;
            const uint32_t hi = h ? w.z : w.x, lo = h ? w.w : w.y;
            const unsigned long long kk = ((unsigned long long)(hi >> 11) << 32) | lo;
            // |Phi^{-1}((k + 1/2) 2^-53)|; the Student-t map makes KIND 1 FP64 bound
            const double zn = probit_grid53_fx<KIND == 1 ? FX_FP64_LEAN : FX_TU_FADD>(fxT, kk, upper);
            // the sign on the bits: a select between zn and -zn costs FP64
            // instructions
            const long long zb = __double_as_longlong(zn);
            const long long neg = (long long)((unsigned long long)(KIND == 2 ? upper : !upper) << 63);
            const double zs = __longlong_as_double(zb ^ neg);
            if (KIND == 1) {
                // Student t by recycling the normal sample (Sec. 3 map)
                z[h] = recycle_t_sel(tk, zs);
            } else {
                // KIND 0: the normal sample; KIND 2: the Exp(1) sample
                // x = -log(u) recycled by the Sec. 6 map, Q(x) = Phi^{-1}(1 - u),
                // evaluated from the exact u (no log)
                z[h] = zs;
            }
        }
        const size_t i0 = b * 2;
        if (OUT && valid) {
            if (i0 + 2 <= n && ((uintptr_t)out % 16 == 0)) {
                __stcs(reinterpret_cast<double2*>(out + i0), make_double2(z[0], z[1]));
            } else {
                for (int h = 0; h < 2; ++h)
                    if (i0 + h < n) out[i0 + h] = z[h];
            }
        }
        if (MOM && valid) {
            for (int h = 0; h < 2; ++h) {
                const double x = (i0 + h < n) ? z[h] : 0.0;
                const double x2 = x * x;
                acc[0] += x;
                acc[1] += x2;
                acc[2] += x2 * x;
                acc[3] += x2 * x2;
            }
        }
    }
    if (MOM) block_reduce4(acc, partials);
}

// Moment launches use grids of at most kMomentWaves waves of resident blocks.
constexpr int kMomentWaves = 4;

// Per-device scratch for moment partials.  Allocated once, at the first
// moment call on a device, for the largest grid a moment launch can have
// (SMs x the hardware's resident-block limit x kMomentWaves), and never
// freed or replaced: a pointer handed to one caller stays valid for every
// later kernel until the process exits.  All moment calls on a device share
// it, so calls that overlap on the GPU race (documented in qm.h).
static double* partials_scratch(int nblocks)
{
    static std::mutex mu;
    static double* ptr[64] = {nullptr};
    static int cap[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lk(mu);
    if (!ptr[dev]) {
        int sms = 0, per_sm = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxBlocksPerMultiprocessor, dev) != cudaSuccess)
            return nullptr;
        const int slots = std::max(1, sms) * std::max(1, per_sm) * kMomentWaves;
        if (cudaMalloc(&ptr[dev], sizeof(double) * 4 * (size_t)slots) != cudaSuccess) {
            ptr[dev] = nullptr;
            return nullptr;
        }
        cap[dev] = slots;
    }
    return nblocks <= cap[dev] ? ptr[dev] : nullptr;
}

}  // namespace qm

// ===========================================================================
// C ABI
// ===========================================================================
using namespace qm;

extern "C" const char* qm_last_error(void) { return g_last_error.c_str(); }
extern "C" const char* qm_version(void) { return "qm 0.1 (sm_103a)"; }
extern "C" int qm_sm_count(void) { return sm_count(); }

extern "C" qm_status qm_normal_quantile_f32(const float* u, float* z, size_t n, int variant,
                                           void* stream)
{
    if (n == 0) return QM_OK;
    if (!u || !z) return fail(QM_ERR_INVALID, "qm_normal_quantile_f32: null pointer");
    if (bad_overlap(u, n * 4, z, n * 4))
        return fail(QM_ERR_INVALID, "qm_normal_quantile_f32: partially overlapping in/out");
    cudaStream_t s = (cudaStream_t)stream;
    switch (variant) {
    case QM_VAR_SQRT_FORM: return launch_map(u, z, n, F32Sqrt(), s, "f32 sqrt form");
    case QM_VAR_BRANCHFREE: return launch_map(u, z, n, F32Paper(), s, "f32 branch-free");
    case QM_VAR_CUDA_LIBM: return launch_map(u, z, n, F32Libm(), s, "f32 normcdfinvf");
    case QM_VAR_ALMOST_NORMAL: return launch_map(u, z, n, F32AlmostNormal(), s, "f32 almost-normal");
    case QM_VAR_PAPER_EXACT: return launch_paper_f32(u, z, n, stream);
    case QM_VAR_DEFAULT:
    case QM_VAR_TABLE: {
        if ((uintptr_t)u % 16 != 0 || (uintptr_t)z % 16 != 0)
            return launch_map(u, z, n, F32Table(), s, "f32 table (unaligned)");
        const int g = grid_for(k_f32_table<4>, 256, (n / 4 + 3) / 4 + 1);
        k_f32_table<4><<<g, 256, 0, s>>>(u, z, n);
        return check_launch("f32 table");
    }
    default: return fail(QM_ERR_INVALID, "qm_normal_quantile_f32: variant %d not available in FP32", variant);
    }
}

extern "C" qm_status qm_normal_quantile_f64(const double* u, double* z, size_t n, int variant,
                                           void* stream)
{
    if (n == 0) return QM_OK;
    if (!u || !z) return fail(QM_ERR_INVALID, "qm_normal_quantile_f64: null pointer");
    if (bad_overlap(u, n * 8, z, n * 8))
        return fail(QM_ERR_INVALID, "qm_normal_quantile_f64: partially overlapping in/out");
    cudaStream_t s = (cudaStream_t)stream;
    switch (variant) {
    case QM_VAR_BRANCHFREE: return launch_map(u, z, n, F64BranchFree(), s, "f64 branch-free");
    case QM_VAR_MIXED_HALLEY: return launch_map(u, z, n, F64Mixed(), s, "f64 mixed");
    case QM_VAR_CUDA_LIBM: return launch_map(u, z, n, F64Libm(), s, "f64 normcdfinv");
    case QM_VAR_DEFAULT:
    case QM_VAR_FIXED: return launch_f64_fixed(u, z, n, stream);
    case QM_VAR_PAPER_EXACT: return launch_paper_f64(u, z, n, 1, stream);
    case QM_VAR_PAPER_EXACT_B: return launch_paper_f64(u, z, n, 0, stream);
    case QM_VAR_HYBRID_VOTE: {
        const int g = grid_for(k_f64_hybrid_vote<2>, 256, (n + 1) / 2);
        k_f64_hybrid_vote<2><<<g, 256, 0, s>>>(u, z, n);
        return check_launch("f64 hybrid vote");
    }
    case QM_VAR_TABLE: {
        if (u == z) {
            // the deep-tail queue re-reads the input after in-place stores
            return launch_map(u, z, n, F64BranchFree(), s, "f64 branch-free (in place)");
        }
        const size_t tiles = (n + kCompactTile - 1) / kCompactTile;
        const int g = grid_for(k_f64_table, kCompactBlock, tiles * kCompactBlock);
        k_f64_table<<<g, kCompactBlock, 0, s>>>(u, z, n);
        return check_launch("f64 table");
    }
    case QM_VAR_COMPACT: {
        if (u == z) {
            // the queues re-read the input after the in-place t_2 stores
            const int g = grid_for(k_f64_hybrid_vote<2>, 256, (n + 1) / 2);
            k_f64_hybrid_vote<2><<<g, 256, 0, s>>>(u, z, n);
            return check_launch("f64 hybrid vote (in place)");
        }
        const size_t tiles = (n + kCompactTile - 1) / kCompactTile;
        const int g = grid_for(k_f64_compact<false>, kCompactBlock, tiles * kCompactBlock);
        k_f64_compact<false><<<g, kCompactBlock, 0, s>>>(u, z, n);
        return check_launch("f64 compact");
    }
    case QM_VAR_T2_MULTI: {
        if (u == z) {
            // the queue re-reads the input after the in-place stores
            return launch_map(u, z, n, F64T2Multi(), s, "f64 t2 multi (in place)");
        }
        const size_t tiles = (n + kCompactTile - 1) / kCompactTile;
        const int g = grid_for(k_f64_compact<true>, kCompactBlock, tiles * kCompactBlock);
        k_f64_compact<true><<<g, kCompactBlock, 0, s>>>(u, z, n);
        return check_launch("f64 t2 multi");
    }
    case QM_VAR_ALMOST_NORMAL: return launch_map(u, z, n, F64AlmostNormal(), s, "f64 almost-normal");
    default: return fail(QM_ERR_INVALID, "qm_normal_quantile_f64: variant %d not available in FP64", variant);
    }
}

extern "C" qm_status qm_normal_quantile_bits24_f32(const uint32_t* words, float* z, size_t n,
                                                  void* stream)
{
    if (n == 0) return QM_OK;
    if (!words || !z) return fail(QM_ERR_INVALID, "qm_normal_quantile_bits24_f32: null pointer");
    if (bad_overlap(words, n * 4, z, n * 4))
        return fail(QM_ERR_INVALID, "qm_normal_quantile_bits24_f32: partially overlapping in/out");
    const int g = grid_for(k_bits24_f32, 256, n);
    k_bits24_f32<<<g, 256, 0, (cudaStream_t)stream>>>(words, z, n);
    return check_launch("bits24 f32");
}

extern "C" qm_status qm_philox_fill_u32(uint64_t key, uint64_t ctr0, uint32_t* out, size_t n,
                                       void* stream)
{
    if (n == 0) return QM_OK;
    if (!out) return fail(QM_ERR_INVALID, "qm_philox_fill_u32: null pointer");
    const int g = grid_for(k_philox_fill, 256, (n + 3) / 4 + 1);
    k_philox_fill<<<g, 256, 0, (cudaStream_t)stream>>>(philox_keys(key), ctr0, out, n);
    return check_launch("philox fill");
}

extern "C" qm_status qm_sample_fused(int target, const qm_params* p, uint64_t key_in, uint64_t ctr0,
                                    void* out, int out_is_f64, size_t n, double* moments4,
                                    void* stream)
{
    (void)p;
    if (n == 0) {
        if (moments4) {
            if (cudaMemsetAsync(moments4, 0, 4 * sizeof(double), (cudaStream_t)stream) != cudaSuccess)
                return fail(QM_ERR_CUDA, "qm_sample_fused: memset failed");
        }
        return QM_OK;
    }
    if (!out && !moments4) return fail(QM_ERR_INVALID, "qm_sample_fused: no output requested");
    if (ctr0 % 4 != 0) return fail(QM_ERR_INVALID, "qm_sample_fused: ctr0 must be a multiple of 4");
    cudaStream_t s = (cudaStream_t)stream;
    const int B = 256;
    if (target == QM_DIST_NORMAL && !out_is_f64) {
        const size_t nblk = (n + 3) / 4;
        int g;
        double* part = nullptr;
        if (moments4) {
            // one grid for both moment variants (same partials, same order)
            g = grid_for(k_fused_normal_f32<true, true>, B, nblk, kMomentWaves);
            part = partials_scratch(g);
            if (!part) return fail(QM_ERR_NOMEM, "qm_sample_fused: moment scratch unavailable");
            const PhiloxKeys K = philox_keys(key_in);
            if (out) k_fused_normal_f32<true, true><<<g, B, 0, s>>>(K, ctr0 / 4, n, (float*)out, part);
            else k_fused_normal_f32<false, true><<<g, B, 0, s>>>(K, ctr0 / 4, n, nullptr, part);
            k_sum_partials<<<1, 128, 0, s>>>(part, g, moments4);
        } else {
            // 4 waves of resident blocks (632 vs 624 Gs/s persistent; more waves
            // repeat the per-block table staging)
            g = grid_for(k_fused_normal_f32<true, false>, B, nblk, 4);
            k_fused_normal_f32<true, false><<<g, B, 0, s>>>(philox_keys(key_in), ctr0 / 4, n, (float*)out, nullptr);
        }
        return check_launch("fused normal f32");
    }
    if ((target == QM_DIST_NORMAL || target == QM_DIST_EXPONENTIAL || target == QM_DIST_STUDENT_T) &&
        out_is_f64) {
        if (target == QM_DIST_STUDENT_T) {
            if (!p || !(p->nu > 0.0)) return fail(QM_ERR_INVALID, "qm_sample_fused: Student t needs nu > 0");
        }
        const size_t nblk = (n + 1) / 2;
        TSel tk{0, 0, nullptr, nullptr};
        if (target == QM_DIST_STUDENT_T) {
            const void* tseg = nullptr;
            const double* ttail = nullptr;
            const qm_status st = t_select(p->nu, &tk.k, &tseg, &ttail);
            if (st != QM_OK) return st;
            tk.seg = (const ttbl::TRows*)tseg;
            tk.tail = ttail;
        }
        double* o = (double*)out;
        const uint64_t b0 = ctr0 / 4;
        const PhiloxKeys key = philox_keys(key_in);
        qm_status fst;
        const fxt::FxTable* fxT = (const fxt::FxTable*)fx_table_device(&fst);
        if (!fxT) return fst;
        // Each variant's grid from its own occupancy (the write-only kernel
        // holds fewer registers) and, for the write-only kernel, up to 64
        // waves of resident blocks (155.6 vs 147.4 Gs/s persistent); the two
        // moment variants share one persistent grid, so the per-block
        // partials, and with them the summation order, match.
        int g = 0;
        double* part = nullptr;
#define QM_LAUNCH_F64(KIND)                                                                        \
    if (moments4) {                                                                                \
        g = grid_for(k_fused_f64<KIND, true, true>, B, nblk);                                      \
        part = partials_scratch(g);                                                                \
        if (!part) return fail(QM_ERR_NOMEM, "qm_sample_fused: moment scratch unavailable");       \
        if (o) k_fused_f64<KIND, true, true><<<g, B, 0, s>>>(key, b0, n, o, part, tk, fxT);        \
        else k_fused_f64<KIND, false, true><<<g, B, 0, s>>>(key, b0, n, nullptr, part, tk, fxT);   \
    } else {                                                                                       \
        g = grid_for(k_fused_f64<KIND, true, false>, B, nblk, 64);                                 \
        k_fused_f64<KIND, true, false><<<g, B, 0, s>>>(key, b0, n, o, nullptr, tk, fxT);           \
    }
        if (target == QM_DIST_NORMAL) { QM_LAUNCH_F64(0) }
        else if (target == QM_DIST_STUDENT_T) { QM_LAUNCH_F64(1) }
        else { QM_LAUNCH_F64(2) }
#undef QM_LAUNCH_F64
        if (part) k_sum_partials<<<1, 128, 0, s>>>(part, g, moments4);
        return check_launch("fused f64");
    }
    if (target == QM_DIST_STUDENT_T)
        return fail(QM_ERR_INVALID, "qm_sample_fused: Student t is FP64 only (out_is_f64 = 1)");
    return fail(QM_ERR_INVALID, "qm_sample_fused: unsupported target/precision (%d, %d)", target, out_is_f64);
}

extern "C" qm_status qm_recycle(int src, int dst, const qm_params* p, const double* in, double* out,
                               size_t n, void* stream)
{
    (void)p;
    if (src == QM_DIST_EXPONENTIAL && dst == QM_DIST_NORMAL) {
        if (n == 0) return QM_OK;
        if (!in || !out) return fail(QM_ERR_INVALID, "qm_recycle: null pointer");
        if (bad_overlap(in, n * 8, out, n * 8))
            return fail(QM_ERR_INVALID, "qm_recycle: partially overlapping in/out");
        return launch_map(in, out, n, ExpToNormal(), (cudaStream_t)stream, "recycle exp->normal");
    }
    if (src == QM_DIST_UNIFORM && dst == QM_DIST_NORMAL)
        return qm_normal_quantile_f64(in, out, n, QM_VAR_DEFAULT, stream);
    if (src == QM_DIST_NORMAL && dst == QM_DIST_STUDENT_T) {
        if (!p) return fail(QM_ERR_INVALID, "qm_recycle: Student t needs params (nu)");
        if (!(p->nu > 0.0)) return fail(QM_ERR_INVALID, "qm_recycle: nu must be > 0 (got %g)", p->nu);
        bool tabulated = false;
        for (int i = 0; i < ttbl::NNU; ++i) tabulated |= (p->nu == ttbl::T_NU[i]);
        if (!tabulated && !(p->nu >= QM_T_NU_MIN && p->nu <= QM_T_NU_MAX))
            return fail(QM_ERR_UNSUPPORTED, "qm_recycle: nu = %g outside [%g, %g] and not tabulated",
                        p->nu, QM_T_NU_MIN, QM_T_NU_MAX);
        if (n == 0) return QM_OK;
        if (!in || !out) return fail(QM_ERR_INVALID, "qm_recycle: null pointer");
        if (bad_overlap(in, n * 8, out, n * 8))
            return fail(QM_ERR_INVALID, "qm_recycle: partially overlapping in/out");
        const void* seg = nullptr;
        const double* tail = nullptr;
        int kk = -1;
        const qm_status st = t_select(p->nu, &kk, &seg, &tail);
        if (st != QM_OK) return st;
        return launch_map(in, out, n, TDynMap{(const ttbl::TRows*)seg, tail}, (cudaStream_t)stream,
                          "recycle normal->t");
    }
    return fail(QM_ERR_UNSUPPORTED, "qm_recycle: pair (%d -> %d) not supported", src, dst);
}
