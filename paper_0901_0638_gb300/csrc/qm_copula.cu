// qm_copula.cu -- Gaussian-copula sampling with recycled marginals (Sec. 9).
//
// The paper's conclusion notes that for a Gaussian copula the two steps
// "map the correlated normals to the unit hypercube, then to the marginals"
// fold into one: each coordinate goes straight through the recycling map
// Q_j = F_j^{-1} o Phi.  One thread draws one d-dimensional sample:
//     eps_k = Phi^{-1}((m_k + 1/2) 2^-53),  m_k a 53-bit Philox integer
//             (two per Philox block, as the fused FP64 normal sampler;
//             fixed-point FP64 evaluation, one FP64 FMA),
//     y = L eps                              (L lower triangular, d <= 16),
//     x_j = Q_j(y_j)                         (normal: identity; Student t:
//                                             the Sec. 3 map, any supported nu).
// Sample i uses the Philox blocks ctr0/4 + i ceil(d/2) + 0 .. ceil(d/2)-1.
// Output is column-major, x[j n + i], so the stores of a warp coalesce.
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

struct CopulaDev {
    int d;
    int pad;
    double L[kMaxD * (kMaxD + 1) / 2];   // packed rows of the lower triangle
    int kind[kMaxD];                      // QM_DIST_NORMAL or QM_DIST_STUDENT_T
    TSel t[kMaxD];
};

// normal from two Philox words (53-bit integer, exact reflected grid point,
// the fixed-point FP64 evaluation)
__device__ __forceinline__ double normal_from_words(const fxt::FxTable* fxT, uint32_t hi, uint32_t lo)
{
    const uint64_t k = ((uint64_t)(hi >> 11) << 32) | lo;
    bool upper;
    const double m = probit_grid53_fx<FX_FP64_LEAN>(fxT, k, upper);
    return upper ? m : -m;
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
            if (c.kind[j] == QM_DIST_STUDENT_T) x = recycle_t_call(c.t[j], x);
            __stcs(out + (size_t)j * n + i, x);
        }
    }
}

template <int D>
qm_status launch_d(const CopulaDev* dev, PhiloxKeys K, uint64_t blk0, double* out, size_t n, cudaStream_t s)
{
    qm_status fst;
    const fxt::FxTable* fxT = (const fxt::FxTable*)fx_table_device(&fst);
    if (!fxT) return fst;
    int bps = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_copula<D>, 128, 0);
    const size_t cap = (size_t)(sm_count() > 0 ? sm_count() : 1) * (bps > 0 ? bps : 1);
    size_t g = (n + 127) / 128;
    if (g > cap) g = cap;
    k_copula<D><<<(int)g, 128, 0, s>>>(dev, K, blk0, out, n, fxT);
    return check_launch("copula sample");
}

template <int... Ds>
qm_status launch_dispatch(int d, const CopulaDev* dev, PhiloxKeys K, uint64_t blk0, double* out, size_t n,
                          cudaStream_t s, std::integer_sequence<int, Ds...>)
{
    qm_status st = QM_ERR_INVALID;
    ((d == Ds + 1 ? (st = launch_d<Ds + 1>(dev, K, blk0, out, n, s), 0) : 0), ...);
    return st;
}

qm_status launch_copula(int d, const CopulaDev* dev, PhiloxKeys K, uint64_t blk0, double* out, size_t n,
                        cudaStream_t s)
{
    return launch_dispatch(d, dev, K, blk0, out, n, s, std::make_integer_sequence<int, kMaxD>{});
}

}  // namespace
}  // namespace qm

using namespace qm;

struct qm_copula {
    CopulaDev host;
    CopulaDev* dev;
};

extern "C" qm_status qm_copula_create(int d, const double* chol, const qm_margin* margins, qm_copula** out)
{
    if (!out || !chol || !margins) return fail(QM_ERR_INVALID, "qm_copula_create: null argument");
    *out = nullptr;
    if (d < 1 || d > kMaxD) return fail(QM_ERR_INVALID, "qm_copula_create: d = %d outside [1, %d]", d, kMaxD);
    qm_copula c{};
    c.host.d = d;
    for (int j = 0; j < d; ++j) {
        for (int k = 0; k < d; ++k) {
            const double v = chol[j * d + k];
            if (!std::isfinite(v)) return fail(QM_ERR_INVALID, "qm_copula_create: L[%d][%d] not finite", j, k);
            if (k > j && v != 0.0)
                return fail(QM_ERR_INVALID, "qm_copula_create: L must be lower triangular (L[%d][%d] = %g)", j, k, v);
            if (k <= j) c.host.L[j * (j + 1) / 2 + k] = v;
        }
        if (!(chol[j * d + j] > 0.0))
            return fail(QM_ERR_INVALID, "qm_copula_create: L[%d][%d] must be > 0", j, j);
        const qm_margin& m = margins[j];
        c.host.kind[j] = m.kind;
        c.host.t[j] = TSel{0, 0, nullptr, nullptr};
        if (m.kind == QM_DIST_STUDENT_T) {
            const void* seg = nullptr;
            const double* tail = nullptr;
            const qm_status st = t_select(m.nu, &c.host.t[j].k, &seg, &tail);
            if (st != QM_OK) return st;
            c.host.t[j].seg = (const ttbl::SegT*)seg;
            c.host.t[j].tail = tail;
        } else if (m.kind != QM_DIST_NORMAL) {
            return fail(QM_ERR_UNSUPPORTED, "qm_copula_create: margin %d: kind %d not supported "
                        "(normal or Student t)", j, m.kind);
        }
    }
    if (cudaMalloc(&c.dev, sizeof(CopulaDev)) != cudaSuccess)
        return fail(QM_ERR_NOMEM, "qm_copula_create: allocation failed");
    if (cudaMemcpy(c.dev, &c.host, sizeof(CopulaDev), cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaFree(c.dev);
        return fail(QM_ERR_CUDA, "qm_copula_create: upload failed");
    }
    *out = new qm_copula(c);
    return QM_OK;
}

extern "C" qm_status qm_copula_sample(const qm_copula* c, uint64_t key, uint64_t ctr0, double* out, size_t n,
                                      void* stream)
{
    if (!c) return fail(QM_ERR_INVALID, "qm_copula_sample: null handle");
    if (ctr0 % 4 != 0) return fail(QM_ERR_INVALID, "qm_copula_sample: ctr0 must be a multiple of 4");
    if (n == 0) return QM_OK;
    if (!out) return fail(QM_ERR_INVALID, "qm_copula_sample: null output");
    return launch_copula(c->host.d, c->dev, philox_keys(key), ctr0 / 4, out, n, (cudaStream_t)stream);
}

extern "C" qm_status qm_copula_destroy(qm_copula* c)
{
    if (!c) return QM_OK;
    cudaFree(c->dev);
    delete c;
    return QM_OK;
}
