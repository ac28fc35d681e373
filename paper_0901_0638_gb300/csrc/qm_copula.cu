// qm_copula.cu -- Gaussian-copula sampling with recycled marginals (Sec. 9).
//
// The paper's conclusion notes that for a Gaussian copula the two steps
// "map the correlated normals to the unit hypercube, then to the marginals"
// fold into one: each coordinate goes straight through the recycling map
// Q_j = F_j^{-1} o Phi.  One thread draws one d-dimensional sample:
//     eps_k = Phi^{-1}((m_k + 1/2) 2^-53),  m_k a 53-bit Philox integer
//             (two per Philox block, as the fused FP64 normal sampler;
//             fixed-point FP64 evaluation, one FP64 FMA),
//     y = L eps / sigma                      (L lower triangular, d <= 16,
//                                             sigma_j its row norms),
//     x_j = Q_j(y_j)                         (normal: identity; Student t:
//                                             the Sec. 3 map, any supported nu).
// Sample i uses the Philox blocks ctr0/4 + i ceil(d/2) + 0 .. ceil(d/2)-1.
// Output is column-major, x[j n + i], so the stores of a warp coalesce.
//
// The t copula (same handle): one more grid normal per sample gives the
// chi-squared mixing variable through its recycling map, W = exp(L(z)),
// T_j = y_j / sigma_j sqrt(nu / W), and each T_j goes to its margin: itself
// (Student t with the copula's nu), G(T_j) (normal; the Student t -> normal
// map) or the normal -> t_mu map after G.  The two maps are the host-built
// tables of qm_tcop_tables.cu.
#include <cuda_runtime.h>

#include <cmath>
#include <utility>
#include <vector>

#include "qm.h"
#include "qm_device.cuh"
#include "qm_fx.cuh"
#include "qm_host.h"

namespace qm {
namespace {

constexpr int kMaxD = QM_COPULA_MAX_DIM;

enum { MARGIN_NORMAL = 0, MARGIN_T = 1, MARGIN_SAME_T = 2 };

static_assert(sizeof(ttbl::SegT) == 64, "t-copula rows share the Student-t segment layout");

struct CopulaDev {
    int d;
    int tcop;                             // 0: Gaussian copula, 1: t copula
    double L[kMaxD * (kMaxD + 1) / 2];   // packed rows of the lower triangle, each
                                          // divided by its norm (L L^T -> correlation)
    int kind[kMaxD];                      // MARGIN_*
    TSel t[kMaxD];
    // t copula
    double half_log_nu;
    const ttbl::SegT* chi;                // log W(z) rows (QM_TC_NZ)
    const double* chi_c;                  //   and their centres
    const ttbl::SegT* g;                  // G rows (1 + ne 2^QM_TC_G_K)
    const double* g_c;                    //   and their 1 / m_c (row 0: unused)
    const ttbl::SegTX* chi_fx;            // the same maps as biased fixed-point rows:
    const ttbl::SegTX* g_fx;              //   QM_TC_NZ log W rows, 1 + ne 2^QM_TC_G_K G rows
    int ne;
    int pad;
};

// log W for the normal score z from the FP64 rows (z outside the table, NaN)
static __device__ __noinline__ double tc_log_w_rare(const CopulaDev& c, double z)
{
    int j = (int)(__fma_rn(z, (double)QM_TC_HZ_INV, QM_TC_Z_MAX * QM_TC_HZ_INV));
    j = min(max(j, 0), QM_TC_NZ - 1);
    return seg_poly(c.chi[j], z - __ldg(c.chi_c + j));
}

// log W for the normal score z (|z| <= 8.3 on the 53-bit grid): in
// u = z + z_max, segment j = floor(16 u) and the offset sigma = u - j/16
// (exact) from the bits of u, tau = 8 sigma, one biased fixed-point row
__device__ __forceinline__ double tc_log_w(const CopulaDev& c, double z)
{
    const double u = __dadd_rn(z, QM_TC_Z_MAX);
    const uint64_t ub = (uint64_t)__double_as_longlong(u);
    // 0 <= u < 2 z_max = 17 on the bits (+0 included; -0, negative values and
    // NaN fail)
    static_assert(QM_TC_Z_MAX == 8.5, "the bit pattern below is that of 17.0");
    if (ub >= 0x4031000000000000ull) return tc_log_w_rare(c, z);
    const int Eu = (int)(ub >> 52) - 1023;                           // u < 17: Eu <= 4
    const uint64_t M = (ub & 0x000FFFFFFFFFFFFFull) | (1ull << 52);
    const int q = 48 - Eu;                                            // bits of M below 1/16
    const bool first = q >= 53;                                       // u < 1/16: segment 0
    const uint64_t low = first ? M : (M & ((1ull << q) - 1ull));
    const int j = first ? 0 : (int)(M >> q);
    const double start = first ? 0.0 : __longlong_as_double((long long)(ub & ~((1ull << q) - 1ull)));
    const double sig = __dadd_rn(u, -start);
    const int sh = Eu + 15;                                           // sigma 2^67 = low 2^(Eu + 15)
    const uint64_t Sig = sh >= 0 ? (low << sh) : (sh > -64 ? (low >> -sh) : 0ull);
    return segts_eval(c.chi_fx + j, Sig, sig);
}

// G(t) from the FP64 rows (|t| past the table, inf, NaN): |t| = 2^E m
// selects the row by E and the top QM_TC_G_K bits of m, r = m / m_c - 1 is
// one FMA (the last binade's rows continue beyond it)
static __device__ __noinline__ double tc_g_rare(const CopulaDev& c, double t)
{
    const double a = fabs(t);
    const unsigned long long b = (unsigned long long)__double_as_longlong(a);
    const int E = (int)(b >> 52) - 1023;
    const bool small = E < QM_TC_G_EMIN;
    const int e = min(E - QM_TC_G_EMIN, c.ne - 1);
    const int j = (int)(b >> (52 - QM_TC_G_K)) & ((1 << QM_TC_G_K) - 1);
    const int row = small ? 0 : 1 + (e << QM_TC_G_K) + j;
    const double m = __longlong_as_double((long long)((b & 0x000FFFFFFFFFFFFFull) | 0x3FF0000000000000ull));
    const double v = small ? a : __fma_rn(m, __ldg(c.g_c + row), -1.0);
    return copysign(seg_poly(c.g[row], v), t);
}

// G(t) = Phi^{-1}(F_nu(t)) from the biased fixed-point rows, no logarithm:
// |t| >= 2^QM_TC_G_EMIN takes segment j of binade E (sigma = |t| - start
// exact, tau = the significand's low 47 bits 2^-48); below, row 0 (the
// series about 0: sigma = |t|, tau = 16 |t|).  Odd in t.
__device__ __forceinline__ double tc_g(const CopulaDev& c, double t)
{
    const uint64_t tb = (uint64_t)__double_as_longlong(t);
    const uint64_t b = tb & 0x7fffffffffffffffull;
    const int E = (int)(b >> 52) - 1023;
    const int e = E - QM_TC_G_EMIN;
    if (e >= c.ne) return tc_g_rare(c, t);
    const double a = __longlong_as_double((long long)b);
    const bool small = e < 0;
    const uint64_t low = b & ((1ull << 47) - 1ull);
    const uint64_t M = (b & 0x000FFFFFFFFFFFFFull) | (1ull << 52);
    const int sh = E + 16;                                            // |t| 2^68 = M 2^(E + 16)
    const uint64_t Sig0 = sh >= 0 ? ((M << sh) & 0x7fffffffffffffffull) : (sh > -64 ? (M >> -sh) : 0ull);
    const int row = small ? 0 : 1 + (e << QM_TC_G_K) + (int)((b >> 47) & 31u);
    const double start = small ? 0.0 : __longlong_as_double((long long)(b - low));
    const double r = segts_eval(c.g_fx + row, small ? Sig0 : (low << 16), __dadd_rn(a, -start));
    return with_sign_of(r, tb);
}

// normal from two Philox words (53-bit integer, exact reflected grid point,
// the fixed-point FP64 evaluation)
__device__ __forceinline__ double normal_from_words(const fxt::FxTable* fxT, uint32_t hi, uint32_t lo)
{
    const uint64_t k = ((uint64_t)(hi >> 11) << 32) | lo;
    bool upper;
    const double m = probit_grid53_fx<FX_FP64_LEAN>(fxT, k, upper);
    // the sign on the bits (a select between m and -m costs FP64 instructions)
    return __longlong_as_double(__double_as_longlong(m) ^ (long long)((unsigned long long)!upper << 63));
}

// D: the dimension at compile time, so that y = L eps unrolls to exactly the
// D(D+1)/2 products of the lower triangle
template <int D>
__global__ void __launch_bounds__(128)
k_copula(const CopulaDev* __restrict__ cp, PhiloxKeys K, uint64_t blk0, double* out, size_t n,
         const fxt::FxTable* fxT)
{
    __shared__ CopulaDev c;
    {
        const int* src = reinterpret_cast<const int*>(cp);
        int* dst = reinterpret_cast<int*>(&c);
        for (int i = threadIdx.x; i < (int)(sizeof(CopulaDev) / sizeof(int)); i += blockDim.x) dst[i] = src[i];
    }
    __syncthreads();
    constexpr int nb = (D + 1) / 2;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        double y[D];
#pragma unroll
        for (int j = 0; j < D; ++j) y[j] = 0.0;
#pragma unroll
        for (int b = 0; b < nb; ++b) {
            const uint4 w = philox_block_keys(K, blk0 + (uint64_t)i * nb + b);
            const double e0 = normal_from_words(fxT, w.x, w.y);
            const double e1 = normal_from_words(fxT, w.z, w.w);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int k = 2 * b + h;
                if (k >= D) break;
                const double e = h ? e1 : e0;
#pragma unroll
                for (int j = k; j < D; ++j) y[j] = __fma_rn(c.L[j * (j + 1) / 2 + k], e, y[j]);
            }
        }
#pragma unroll
        for (int j = 0; j < D; ++j) {
            double x = y[j];
            if (c.kind[j] == MARGIN_T) x = recycle_t_call(c.t[j], x);
            __stcs(out + (size_t)j * n + i, x);
        }
    }
}

// t copula: sample i draws ceil((D+1)/2) Philox blocks; normal 0 is the
// mixing variable's score, normals 1..D are eps
template <int D>
__global__ void __launch_bounds__(128)
k_tcopula(const CopulaDev* __restrict__ cp, PhiloxKeys K, uint64_t blk0, double* out, size_t n,
          const fxt::FxTable* fxT)
{
    __shared__ CopulaDev c;
    {
        const int* src = reinterpret_cast<const int*>(cp);
        int* dst = reinterpret_cast<int*>(&c);
        for (int i = threadIdx.x; i < (int)(sizeof(CopulaDev) / sizeof(int)); i += blockDim.x) dst[i] = src[i];
    }
    __syncthreads();
    constexpr int nb = (D + 2) / 2;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        double y[D];
#pragma unroll
        for (int j = 0; j < D; ++j) y[j] = 0.0;
        double zw = 0.0;
#pragma unroll
        for (int b = 0; b < nb; ++b) {
            const uint4 w = philox_block_keys(K, blk0 + (uint64_t)i * nb + b);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int q = 2 * b + h;               // normal index in the sample
                if (q > D) break;
                const double e = h ? normal_from_words(fxT, w.z, w.w) : normal_from_words(fxT, w.x, w.y);
                if (q == 0) {
                    zw = e;
                } else {
                    const int k = q - 1;
#pragma unroll
                    for (int j = k; j < D; ++j) y[j] = __fma_rn(c.L[j * (j + 1) / 2 + k], e, y[j]);
                }
            }
        }
        const double S = exp(c.half_log_nu - 0.5 * tc_log_w(c, zw));       // sqrt(nu / W)
#pragma unroll
        for (int j = 0; j < D; ++j) {
            const double T = y[j] * S;
            double x = T;
            if (c.kind[j] != MARGIN_SAME_T) {
                x = tc_g(c, T);
                if (c.kind[j] == MARGIN_T) x = recycle_t_call(c.t[j], x);
            }
            __stcs(out + (size_t)j * n + i, x);
        }
    }
}

template <int D>
qm_status launch_d(const CopulaDev* dev, bool tcop, PhiloxKeys K, uint64_t blk0, double* out, size_t n,
                   cudaStream_t s)
{
    qm_status fst;
    const fxt::FxTable* fxT = (const fxt::FxTable*)fx_table_device(&fst);
    if (!fxT) return fst;
    int bps = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, tcop ? k_tcopula<D> : k_copula<D>, 128, 0);
    // up to 8 waves of resident blocks (each sample's output depends only on
    // its index; 7.04 vs 6.98 G samples/s persistent at d = 8)
    const size_t cap = (size_t)(sm_count() > 0 ? sm_count() : 1) * (bps > 0 ? bps : 1) * 8;
    size_t g = (n + 127) / 128;
    if (g > cap) g = cap;
    if (tcop) k_tcopula<D><<<(int)g, 128, 0, s>>>(dev, K, blk0, out, n, fxT);
    else k_copula<D><<<(int)g, 128, 0, s>>>(dev, K, blk0, out, n, fxT);
    return check_launch("copula sample");
}

template <int... Ds>
qm_status launch_dispatch(int d, const CopulaDev* dev, bool tcop, PhiloxKeys K, uint64_t blk0, double* out,
                          size_t n, cudaStream_t s, std::integer_sequence<int, Ds...>)
{
    qm_status st = QM_ERR_INVALID;
    ((d == Ds + 1 ? (st = launch_d<Ds + 1>(dev, tcop, K, blk0, out, n, s), 0) : 0), ...);
    return st;
}

qm_status launch_copula(int d, const CopulaDev* dev, bool tcop, PhiloxKeys K, uint64_t blk0, double* out,
                        size_t n, cudaStream_t s)
{
    return launch_dispatch(d, dev, tcop, K, blk0, out, n, s, std::make_integer_sequence<int, kMaxD>{});
}

}  // namespace
}  // namespace qm

using namespace qm;

struct qm_copula {
    CopulaDev host;
    CopulaDev* dev;
};

namespace {

// validation and the parts common to both copulas; tcop_nu > 0 for the t copula
qm_status fill_copula(int d, const double* chol, const qm_margin* margins, double tcop_nu, qm_copula& c,
                      const char* who)
{
    if (!chol || !margins) return fail(QM_ERR_INVALID, "%s: null argument", who);
    if (d < 1 || d > kMaxD) return fail(QM_ERR_INVALID, "%s: d = %d outside [1, %d]", who, d, kMaxD);
    c.host.d = d;
    c.host.tcop = tcop_nu > 0.0;
    for (int j = 0; j < d; ++j) {
        double ss = 0.0;
        for (int k = 0; k < d; ++k) {
            const double v = chol[j * d + k];
            if (!std::isfinite(v)) return fail(QM_ERR_INVALID, "%s: L[%d][%d] not finite", who, j, k);
            if (k > j && v != 0.0)
                return fail(QM_ERR_INVALID, "%s: L must be lower triangular (L[%d][%d] = %g)", who, j, k, v);
            if (k <= j) {
                c.host.L[j * (j + 1) / 2 + k] = v;
                ss += v * v;
            }
        }
        if (!(chol[j * d + j] > 0.0)) return fail(QM_ERR_INVALID, "%s: L[%d][%d] must be > 0", who, j, j);
        const double inv_sigma = 1.0 / std::sqrt(ss);         // the copula of L L^T is its correlation's
        for (int k = 0; k <= j; ++k) c.host.L[j * (j + 1) / 2 + k] *= inv_sigma;
        const qm_margin& m = margins[j];
        c.host.t[j] = TSel{0, 0, nullptr, nullptr};
        if (m.kind == QM_DIST_STUDENT_T) {
            if (tcop_nu > 0.0 && m.nu == tcop_nu) {
                c.host.kind[j] = MARGIN_SAME_T;
                continue;
            }
            c.host.kind[j] = MARGIN_T;
            const void* seg = nullptr;
            const double* tail = nullptr;
            const qm_status st = t_select(m.nu, &c.host.t[j].k, &seg, &tail);
            if (st != QM_OK) return st;
            c.host.t[j].seg = (const ttbl::TRows*)seg;
            c.host.t[j].tail = tail;
        } else if (m.kind == QM_DIST_NORMAL) {
            c.host.kind[j] = MARGIN_NORMAL;
        } else {
            return fail(QM_ERR_UNSUPPORTED, "%s: margin %d: kind %d not supported (normal or Student t)", who, j,
                        m.kind);
        }
    }
    return QM_OK;
}

qm_status upload(qm_copula& c, qm_copula** out, const char* who)
{
    if (cudaMalloc(&c.dev, sizeof(CopulaDev)) != cudaSuccess) return fail(QM_ERR_NOMEM, "%s: allocation failed", who);
    if (cudaMemcpy(c.dev, &c.host, sizeof(CopulaDev), cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaFree(c.dev);
        return fail(QM_ERR_CUDA, "%s: upload failed", who);
    }
    *out = new qm_copula(c);
    return QM_OK;
}

}  // namespace

extern "C" qm_status qm_copula_create(int d, const double* chol, const qm_margin* margins, qm_copula** out)
{
    if (!out) return fail(QM_ERR_INVALID, "qm_copula_create: null argument");
    *out = nullptr;
    qm_copula c{};
    const qm_status st = fill_copula(d, chol, margins, 0.0, c, "qm_copula_create");
    if (st != QM_OK) return st;
    return upload(c, out, "qm_copula_create");
}

extern "C" qm_status qm_tcopula_create(int d, double nu, const double* chol, const qm_margin* margins,
                                       qm_copula** out)
{
    if (!out) return fail(QM_ERR_INVALID, "qm_tcopula_create: null argument");
    *out = nullptr;
    if (!(nu >= QM_T_NU_MIN && nu <= QM_T_NU_MAX))
        return fail(QM_ERR_UNSUPPORTED, "qm_tcopula_create: nu = %g outside [%g, %g]", nu, QM_T_NU_MIN, QM_T_NU_MAX);
    qm_copula c{};
    qm_status st = fill_copula(d, chol, margins, nu, c, "qm_tcopula_create");
    if (st != QM_OK) return st;
    c.host.half_log_nu = 0.5 * std::log(nu);
    const void* chi = nullptr;
    const void* g = nullptr;
    const void* fx = nullptr;
    st = tcop_table_device(nu, &chi, &g, &fx, &c.host.ne);
    if (st != QM_OK) return st;
    c.host.chi_fx = static_cast<const ttbl::SegTX*>(fx);
    c.host.g_fx = c.host.chi_fx + QM_TC_NZ;
    c.host.chi = static_cast<const ttbl::SegT*>(chi);
    c.host.chi_c = reinterpret_cast<const double*>(c.host.chi + QM_TC_NZ);
    c.host.g = static_cast<const ttbl::SegT*>(g);
    c.host.g_c = reinterpret_cast<const double*>(c.host.g + 1 + (c.host.ne << QM_TC_G_K));
    return upload(c, out, "qm_tcopula_create");
}

extern "C" qm_status qm_copula_sample(const qm_copula* c, uint64_t key, uint64_t ctr0, double* out, size_t n,
                                      void* stream)
{
    if (!c) return fail(QM_ERR_INVALID, "qm_copula_sample: null handle");
    if (ctr0 % 4 != 0) return fail(QM_ERR_INVALID, "qm_copula_sample: ctr0 must be a multiple of 4");
    if (n == 0) return QM_OK;
    if (!out) return fail(QM_ERR_INVALID, "qm_copula_sample: null output");
    return launch_copula(c->host.d, c->dev, c->host.tcop != 0, philox_keys(key), ctr0 / 4, out, n,
                         (cudaStream_t)stream);
}

extern "C" qm_status qm_copula_destroy(qm_copula* c)
{
    if (!c) return QM_OK;
    cudaFree(c->dev);
    delete c;
    return QM_OK;
}
