// qm_hyp.cu -- exponential -> hyperbolic recycling (Sec. 8.1).
//
// Target: the hyperbolic density (location 0)
//     f(x) = exp(g(x)) / Z,  g(x) = -alpha sqrt(delta^2 + x^2) + beta x,
//     |beta| < alpha, delta > 0.
// Base: the two-sided exponential with the same mass split at 0,
//     f_0(v) = p_+ (alpha - beta) e^{-(alpha-beta) v} (v > 0),
//              p_- (alpha + beta) e^{(alpha+beta) v}  (v < 0),  p_+ = int_0^inf f.
// The map Q(v) = F^{-1}(G_0(v)) solves the right and left recycling ODEs
//     Q'' + (alpha - beta) Q' = H(Q) Q'^2   (v > 0),
//     Q'' - (alpha + beta) Q' = H(Q) Q'^2   (v < 0),   H(Q) = alpha Q / sqrt(delta^2 + Q^2) - beta,
// with Q(0) = 0 and Q'(0+-) = f_0(0+-) / f(0).  The left problem is the right
// one for -beta reflected: Q(v; beta) = -Q(-v; -beta), so one builder serves
// both sides.
//
// Tables (built on the host in long double at qm_hyp_create): for each side,
// segments of |v| on a binade grid -- binade [2^E, 2^(E+1)) cut into 32
// segments, E_MIN <= E <= E_max -- each with the degree-9 Taylor expansion of
// Q about its centre, plus the series about v = 0 for |v| < 2^E_MIN.  The
// expansions come from the ODE itself (matching powers of s in
// Q(v0 + s) = sum b_k s^k gives b_{k+2} from b_0..b_{k+1}), integrated with
// steps of at most 1/(4 rate).  Perturbations of Q grow like 1/f(Q) towards
// larger |v|, so the outer binades come from a pass BACKWARDS from the tail
// (the start value at the outermost centre solves P(X > Q) =
// p_+ e^{-(alpha-beta) v} by Newton's method on tail integrals of f, exp-sinh
// quadrature, and Q' = f_0(v)/f(Q)), the inner ones (|v| < ~0.5/rate) from a
// pass forwards from Q(0) = 0, Q'(0+), which keeps Q's relative accuracy as
// v -> 0; the two passes must agree where they meet.
//
// On the device each segment is a biased fixed-point row (pack_fx_biased,
// qm_t_fx.h: the coefficients have no common sign, so the Horner accumulators
// carry a bias that each step removes) evaluated by segts_eval with one DFMA;
// the FP64 rows serve |v| < 2^E_MIN, |v| past the table, 0, inf and NaN.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "qm.h"
#include "qm_device.cuh"
#include "qm_host.h"

namespace qm {
namespace {

using LD = long double;
constexpr int K_SEG = 5;                 // 32 segments per binade
constexpr int E_MIN = QM_HYP_E_MIN;      // |v| < 2^E_MIN: series about 0
constexpr int DEG_INT = 22;
constexpr LD PI_L = 3.14159265358979323846264338327950288L;

struct HypParams {
    LD alpha, beta, delta;
};

LD g_of(const HypParams& P, LD x) { return -P.alpha * std::hypot(P.delta, x) + P.beta * x; }

// g(x + u) - g(x) without cancellation
LD dg_of(const HypParams& P, LD x, LD u)
{
    return u * (P.beta - P.alpha * (2 * x + u) / (std::hypot(P.delta, x + u) + std::hypot(P.delta, x)));
}

// exp-sinh quadrature of int_0^inf h(u) du (h smooth, decaying at infinity)
template <class F>
LD exp_sinh(F h)
{
    const LD step = 1.0L / 64;
    LD sum = 0.0L;
    for (int k = -448; k <= 448; ++k) {
        const LD t = k * step;
        const LD u = std::exp(PI_L / 2 * std::sinh(t));
        if (!(u > 0) || !std::isfinite(u)) continue;
        const LD w = PI_L / 2 * std::cosh(t) * u;
        const LD val = h(u);
        if (std::isfinite(val)) sum += w * val;
    }
    return sum * step;
}

// log of int_x^inf exp(g) for x >= 0
LD log_tail(const HypParams& P, LD x)
{
    const LD I = exp_sinh([&](LD u) { return std::exp(dg_of(P, x, u)); });
    return g_of(P, x) + std::log(I);
}

// b_0..b_D of Q(v0 + s) for the right-side ODE Q'' + r Q' = H(Q) Q'^2
void taylor_hyp(const HypParams& P, LD r, LD q0, LD q1, int D, LD* b)
{
    b[0] = q0;
    b[1] = q1;
    std::vector<LD> S(D + 1), Pw(D + 1), QP(D + 1), H(D + 1), d1(D + 1), d1sq(D + 1);
    const LD d2 = P.delta * P.delta;
    for (int n = 0; n + 2 <= D; ++n) {
        // S = delta^2 + Q^2 and Pw = S^{-1/2}, coefficient n (needs b_0..b_n)
        LD q2 = 0.0L;
        for (int j = 0; j <= n; ++j) q2 += b[j] * b[n - j];
        S[n] = q2 + (n == 0 ? d2 : 0.0L);
        if (n == 0) {
            Pw[0] = 1.0L / std::sqrt(S[0]);
        } else {
            LD acc = 0.0L;       // n Pw_n S_0 = sum_{k=1}^n (p k - (n-k)) S_k Pw_{n-k}, p = -1/2
            for (int k = 1; k <= n; ++k) acc += (-0.5L * k - (n - k)) * S[k] * Pw[n - k];
            Pw[n] = acc / (n * S[0]);
        }
        LD qp = 0.0L;
        for (int j = 0; j <= n; ++j) qp += b[j] * Pw[n - j];
        QP[n] = qp;
        H[n] = P.alpha * QP[n] - (n == 0 ? P.beta : 0.0L);
        d1[n] = (n + 1) * b[n + 1];
        LD dd = 0.0L;
        for (int j = 0; j <= n; ++j) dd += d1[j] * d1[n - j];
        d1sq[n] = dd;
        LD rhs = 0.0L;
        for (int j = 0; j <= n; ++j) rhs += H[j] * d1sq[n - j];
        b[n + 2] = (rhs - r * (n + 1) * b[n + 1]) / ((n + 2) * (n + 1));
    }
}

LD horner(const LD* b, int D, LD s)
{
    LD v = b[D];
    for (int k = D - 1; k >= 0; --k) v = v * s + b[k];
    return v;
}

LD horner_d(const LD* b, int D, LD s)
{
    LD v = D * b[D];
    for (int k = D - 1; k >= 1; --k) v = v * s + k * b[k];
    return v;
}

// centre of segment j of binade E: 2^E (1 + (2j+1)/64)
LD centre(int E, int j) { return std::ldexp(1.0L + (2 * j + 1) / 64.0L, E); }

// One side (v >= 0 of parameters P).  seg: (1 + 32 nb) x 10 coefficients,
// entry 0 the series about 0, entry 1 + 32 (E - E_MIN) + j segment (E, j).
// info: p (mass of the side), slope Q'(0+), E_max.
qm_status build_side(const HypParams& P, LD logZ, double* seg, int* e_max_out, LD* p_side, LD* slope)
{
    const LD r = P.alpha - P.beta;
    const LD lp = log_tail(P, 0.0L) - logZ;                 // log p_side
    *p_side = std::exp(lp);
    *slope = std::exp(lp + logZ - g_of(P, 0.0L)) * r;       // f_0(0+)/f(0) = p r Z e^{-g(0)}
    // largest |v| a double sample of the base can reach: p e^{-r v} >= 2^-1074
    const LD vmax = (lp + 745.2L) / r;
    int e_max = (int)std::floor(std::log2(vmax));
    if (e_max < E_MIN) e_max = E_MIN;
    if (e_max - E_MIN + 1 > QM_HYP_MAX_BINADES)
        return fail(QM_ERR_UNSUPPORTED, "hyperbolic: parameter range needs %d binades (max %d)",
                    e_max - E_MIN + 1, QM_HYP_MAX_BINADES);
    *e_max_out = e_max;
    // binades below E_join come from a forward pass from v = 0 (exact Q(0) = 0
    // and Q'(0+): relative accuracy as Q -> 0, errors grow at most ~e), the
    // others from a backward pass from the tail (errors decay towards 0)
    int e_join = (int)std::floor(std::log2(0.5L / r));
    e_join = std::min(std::max(e_join, E_MIN + 1), e_max);
    auto store = [&](int E, int j, const LD* b) {
        double* e = seg + 10 * (1 + 32 * (E - E_MIN) + j);
        for (int k = 0; k < 10; ++k) e[k] = (double)b[k];
    };
    // advance (q, qp) from v to c with the series b, in sub-steps of at most
    // 1/(4 r) (the series must also resolve the ODE's mode e^{r (v - v0)})
    LD b[DEG_INT + 1];
    auto advance = [&](LD& v, LD c, LD& q, LD& qp) {
        const int nsub = std::max(1, (int)std::ceil(std::fabs(c - v) * 4 * r));
        const LD h = (c - v) / nsub;
        for (int k = 0; k < nsub; ++k) {
            if (k > 0) taylor_hyp(P, r, q, qp, DEG_INT, b);
            q = horner(b, DEG_INT, h);
            qp = horner_d(b, DEG_INT, h);
            v += h;
        }
        v = c;
    };
    // backward pass: start at the outermost centre, P(X > Q) = p e^{-r v}
    LD v = centre(e_max, 31);
    const LD target = lp - r * v + logZ;                    // log int_Q^inf exp(g)
    LD q = v;
    for (int it = 0; it < 200; ++it) {
        const LD lt = log_tail(P, q);
        // d/dq log int_q^inf exp(g) = -exp(g(q) - lt)
        const LD dq = (lt - target) / std::exp(g_of(P, q) - lt);
        q += dq;
        if (q < 0) q = 0;
        if (std::fabs(dq) <= 1e-19L * (1 + std::fabs(q))) break;
    }
    LD qp = std::exp(lp + logZ - r * v - g_of(P, q)) * r;   // f_0(v)/f(Q)
    LD q_join = 0;
    for (int E = e_max; E >= e_join; --E) {
        for (int j = 31; j >= 0; --j) {
            const LD c = centre(E, j);
            if (c != v) advance(v, c, q, qp);
            taylor_hyp(P, r, q, qp, DEG_INT, b);
            if (!std::isfinite(b[DEG_INT]))
                return fail(QM_ERR_INVALID, "hyperbolic: integration overflow at v = %Lg", v);
            store(E, j, b);
            q_join = q;
        }
    }
    // forward pass from 0
    taylor_hyp(P, r, 0.0L, *slope, DEG_INT, b);
    for (int k = 0; k < 10; ++k) seg[k] = (double)b[k];
    v = 0;
    q = 0;
    qp = *slope;
    for (int E = E_MIN; E <= e_join; ++E) {
        for (int j = 0; j < 32; ++j) {
            const LD c = centre(E, j);
            advance(v, c, q, qp);
            if (E == e_join) {                              // the join: both passes must agree
                if (std::fabs(q / q_join - 1) > 1e-12L)
                    return fail(QM_ERR_INVALID, "hyperbolic: forward and backward integrations "
                                "disagree at v = %Lg (%Lg)", c, q / q_join - 1);
                return QM_OK;
            }
            taylor_hyp(P, r, q, qp, DEG_INT, b);
            if (!std::isfinite(b[DEG_INT]))
                return fail(QM_ERR_INVALID, "hyperbolic: integration overflow at v = %Lg", v);
            store(E, j, b);
        }
    }
    return QM_OK;
}

}  // namespace

qm_status hyp_table_build(double alpha, double beta, double delta, double* seg_right, double* seg_left,
                          int* e_max, double* info)
{
    if (!(alpha > 0 && std::fabs(beta) < alpha && delta > 0) || !std::isfinite(alpha) || !std::isfinite(delta))
        return fail(QM_ERR_INVALID, "hyperbolic: need alpha > 0, |beta| < alpha, delta > 0");
    if (alpha - std::fabs(beta) < 1e-3 * alpha || alpha * delta < 1e-4 || alpha * delta > 1e4)
        return fail(QM_ERR_UNSUPPORTED, "hyperbolic: (alpha, beta, delta) = (%g, %g, %g) outside the "
                    "supported range (alpha - |beta| >= 1e-3 alpha, 1e-4 <= alpha delta <= 1e4)",
                    alpha, beta, delta);
    const HypParams R{alpha, beta, delta}, L{alpha, -beta, delta};
    // Z = int exp(g): both half-lines by exp-sinh
    const LD zr = std::exp(log_tail(R, 0.0L)), zl = std::exp(log_tail(L, 0.0L));
    const LD logZ = std::log(zr + zl);
    LD pr, sr, pl, sl;
    qm_status st = build_side(R, logZ, seg_right, &e_max[0], &pr, &sr);
    if (st != QM_OK) return st;
    st = build_side(L, logZ, seg_left, &e_max[1], &pl, &sl);
    if (st != QM_OK) return st;
    info[0] = (double)pr;
    info[1] = (double)pl;
    info[2] = (double)sr;
    info[3] = (double)sl;
    info[4] = (double)logZ;
    return QM_OK;
}

// ---------------------------------------------------------------------------
// device side
// ---------------------------------------------------------------------------
namespace {

struct HypSide {
    const ttbl::SegT* seg;     // 1 + 32 nb FP64 rows (the series about 0, then the segments)
    const ttbl::SegTX* fx;     // 32 nb fixed-point rows (binades E_MIN .. e_max)
    int e_max;
};

// |Q| on one side from the FP64 rows: |v| < 2^E_MIN (the series about 0),
// |v| beyond the last binade (its last segment continued), 0, inf and NaN
static __device__ __noinline__ double hyp_side_rare(const ttbl::SegT* seg, int e_max, double a)
{
    const uint64_t ab = (uint64_t)__double_as_longlong(a);
    const int E = (int)(ab >> 52) - 1023;
    double s;
    int idx;
    if (E < E_MIN) {                                        // series about 0
        idx = 0;
        s = a;
    } else {
        const int Ec = min(E, e_max);
        const uint32_t j = (E > e_max) ? 31u : (uint32_t)(ab >> 47) & 31u;
        const uint64_t cb = ((uint64_t)(Ec + 1023) << 52) | ((uint64_t)j << 47) | (1ull << 46);
        s = __dadd_rn(a, -__longlong_as_double((long long)cb));     // exact within the binade
        idx = 1 + 32 * (Ec - E_MIN) + (int)j;
    }
    return seg_poly(seg[idx], s);
}

// |Q| on one side for a = |v|: segment j of binade E from the bits, the
// offset sigma = a - start exact (Sterbenz), tau = sigma / (2 w) =
// (low 47 bits of the significand) 2^-48, and the biased fixed-point row
// (returns the bits of the value: see hyp_eval)
__device__ __forceinline__ uint64_t hyp_side_eval(const HypSide& S, double a)
{
    const uint64_t ab = (uint64_t)__double_as_longlong(a);
    const int E = (int)(ab >> 52) - 1023;
    if (E < E_MIN || E > S.e_max) return (uint64_t)__double_as_longlong(hyp_side_rare(S.seg, S.e_max, a));
    const uint64_t low = ab & ((1ull << 47) - 1ull);
    // sigma = a - (segment start) = low 2^(E - 52) as a double without an FP64
    // instruction: low < 2^47 normalised (significand (low << lz) >> 11,
    // exponent E + 11 - lz); the exact subtraction issued FP64 instructions
    // on a pipe that bound the map
    const int lz = __clzll(low | 1ull);
    const uint64_t sb = low == 0 ? 0ull : ((low << lz) >> 11) + ((uint64_t)(E + 1033 - lz) << 52);
    return (uint64_t)__double_as_longlong(segts_eval(S.fx + 32 * (E - E_MIN) + (int)((ab >> 47) & 31u), low << 16,
                                                     __longlong_as_double((long long)sb)));
}

__device__ __forceinline__ double hyp_eval(const HypSide& R, const HypSide& L, double v)
{
    const uint64_t vb = (uint64_t)__double_as_longlong(v);
    const double a = __longlong_as_double((long long)(vb & 0x7fffffffffffffffull));
    // pick the side's table first and evaluate once (selecting between two
    // evaluations would run both)
    const bool neg = (vb >> 63) != 0;
    const HypSide S{neg ? L.seg : R.seg, neg ? L.fx : R.fx, neg ? L.e_max : R.e_max};
    // the inf/NaN case and the sign on the bits (no select between doubles)
    const uint64_t ab = vb & 0x7fffffffffffffffull;
    const uint64_t xb = ab >= 0x7ff0000000000000ull ? ab                                 // inf, NaN
                                                    : hyp_side_eval(S, a);
    return __longlong_as_double((long long)((xb & 0x7fffffffffffffffull) | (vb & 0x8000000000000000ull)));
}

// VEC: two elements per thread through 16-byte loads and stores (in and out
// 16-byte aligned), the odd last element by thread 0 of block 0.
template <bool VEC>
__global__ void __launch_bounds__(256)
k_hyp(HypSide R, HypSide L, const double* __restrict__ in, double* out, size_t n)
{
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    if (VEC) {
        const size_t nv = n / 2;
        const double2* vin = reinterpret_cast<const double2*>(in);
        double2* vout = reinterpret_cast<double2*>(out);
        for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += stride) {
            const double2 v = __ldcs(vin + i);
            __stcs(vout + i, make_double2(hyp_eval(R, L, v.x), hyp_eval(R, L, v.y)));
        }
        if (blockIdx.x == 0 && threadIdx.x == 0 && (n & 1)) out[n - 1] = hyp_eval(R, L, in[n - 1]);
    } else {
        for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
            __stcs(out + i, hyp_eval(R, L, __ldcs(in + i)));
    }
}

}  // namespace
}  // namespace qm

using namespace qm;

struct qm_hyp {
    int device;
    HypSide right, left;
    ttbl::SegT* mem;       // FP64 rows of both sides
    ttbl::SegTX* fxmem;    // fixed-point rows of both sides
    double info[5];
};

namespace qm {
namespace {

// The fixed-point rows of both sides from the FP64 tables (binade E,
// segment j: width 2^(E-5), expanded about its centre), 32 per binade from
// E_MIN; rows past e_max stay zero and unused.
qm_status hyp_pack_rows(const double* sr, const double* sl, const int* e_max, ttbl::SegTX* fr, ttbl::SegTX* fl)
{
    for (int side = 0; side < 2; ++side) {
        const double* tab = side ? sl : sr;
        ttbl::SegTX* out = side ? fl : fr;
        for (int E = E_MIN; E <= e_max[side]; ++E)
            for (int j = 0; j < 32; ++j) {
                const size_t i = (size_t)(32 * (E - E_MIN) + j);
                const qm_status st = pack_fx_biased(&tab[10 * (1 + i)], std::ldexp(1.0, E - 5),
                                                    std::ldexp(1.0, E - 6), &out[i]);
                if (st != QM_OK) {
                    const std::string why = qm_last_error();      // fail() rewrites that buffer
                    return fail(QM_ERR_UNSUPPORTED, "hyperbolic: %s side, binade %d, segment %d: %s",
                                side ? "left" : "right", E, j, why.c_str());
                }
            }
    }
    return QM_OK;
}

}  // namespace
}  // namespace qm

extern "C" qm_status qm_hyp_rows_build(double alpha, double beta, double delta, void* rows_right, void* rows_left,
                                       int* e_max)
{
    if (!rows_right || !rows_left || !e_max) return fail(QM_ERR_INVALID, "qm_hyp_rows_build: null pointer");
    const size_t per = (size_t)(1 + 32 * QM_HYP_MAX_BINADES);
    std::vector<double> sr(10 * per), sl(10 * per);
    double info[5];
    qm_status st = hyp_table_build(alpha, beta, delta, sr.data(), sl.data(), e_max, info);
    if (st != QM_OK) return st;
    const size_t fper = (size_t)(32 * QM_HYP_MAX_BINADES);
    std::memset(rows_right, 0, sizeof(ttbl::SegTX) * fper);
    std::memset(rows_left, 0, sizeof(ttbl::SegTX) * fper);
    return hyp_pack_rows(sr.data(), sl.data(), e_max, static_cast<ttbl::SegTX*>(rows_right),
                         static_cast<ttbl::SegTX*>(rows_left));
}

extern "C" qm_status qm_hyp_table_build(double alpha, double beta, double delta, double* seg_right,
                                        double* seg_left, int* e_max, double* info)
{
    if (!seg_right || !seg_left || !e_max || !info) return fail(QM_ERR_INVALID, "qm_hyp_table_build: null pointer");
    return hyp_table_build(alpha, beta, delta, seg_right, seg_left, e_max, info);
}

extern "C" qm_status qm_hyp_create(double alpha, double beta, double delta, qm_hyp** out)
{
    if (!out) return fail(QM_ERR_INVALID, "qm_hyp_create: null handle pointer");
    *out = nullptr;
    const size_t per = (size_t)(1 + 32 * QM_HYP_MAX_BINADES);
    std::vector<double> sr(10 * per), sl(10 * per);
    int e_max[2];
    qm_hyp h{};
    qm_status st = hyp_table_build(alpha, beta, delta, sr.data(), sl.data(), e_max, h.info);
    if (st != QM_OK) return st;
    std::vector<ttbl::SegT> packed(2 * per);
    for (size_t i = 0; i < 2 * per; ++i) {
        const double* c = (i < per) ? &sr[10 * i] : &sl[10 * (i - per)];
        for (int k = 0; k < 5; ++k) packed[i].a[k] = c[k];
        for (int k = 0; k < 5; ++k) packed[i].b[k] = (float)c[5 + k];
        packed[i].pad = 0.0f;
    }
    const size_t fper = (size_t)(32 * QM_HYP_MAX_BINADES);
    std::vector<ttbl::SegTX> fx(2 * fper);
    st = hyp_pack_rows(sr.data(), sl.data(), e_max, fx.data(), fx.data() + fper);
    if (st != QM_OK) return st;
    if (cudaGetDevice(&h.device) != cudaSuccess) return fail(QM_ERR_CUDA, "qm_hyp_create: no device");
    if (cudaMalloc(&h.mem, sizeof(ttbl::SegT) * packed.size()) != cudaSuccess)
        return fail(QM_ERR_NOMEM, "qm_hyp_create: table allocation failed");
    if (cudaMalloc(&h.fxmem, sizeof(ttbl::SegTX) * fx.size()) != cudaSuccess) {
        cudaFree(h.mem);
        return fail(QM_ERR_NOMEM, "qm_hyp_create: table allocation failed");
    }
    if (cudaMemcpy(h.mem, packed.data(), sizeof(ttbl::SegT) * packed.size(), cudaMemcpyHostToDevice) !=
            cudaSuccess ||
        cudaMemcpy(h.fxmem, fx.data(), sizeof(ttbl::SegTX) * fx.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaFree(h.mem);
        cudaFree(h.fxmem);
        return fail(QM_ERR_CUDA, "qm_hyp_create: table upload failed");
    }
    h.right = HypSide{h.mem, h.fxmem, e_max[0]};
    h.left = HypSide{h.mem + per, h.fxmem + fper, e_max[1]};
    *out = new qm_hyp(h);
    return QM_OK;
}

extern "C" qm_status qm_hyp_info(const qm_hyp* h, double* info)
{
    if (!h || !info) return fail(QM_ERR_INVALID, "qm_hyp_info: null argument");
    for (int k = 0; k < 5; ++k) info[k] = h->info[k];
    return QM_OK;
}

extern "C" qm_status qm_hyp_recycle(const qm_hyp* h, const double* v, double* x, size_t n, void* stream)
{
    if (!h) return fail(QM_ERR_INVALID, "qm_hyp_recycle: null handle");
    if (n == 0) return QM_OK;
    if (!v || !x) return fail(QM_ERR_INVALID, "qm_hyp_recycle: null pointer");
    if (bad_overlap(v, n * 8, x, n * 8)) return fail(QM_ERR_INVALID, "qm_hyp_recycle: partially overlapping in/out");
    const bool vec = (uintptr_t)v % 16 == 0 && (uintptr_t)x % 16 == 0;
    int bps = 0;
    if (vec) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_hyp<true>, 256, 0);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_hyp<false>, 256, 0);
    const size_t cap = (size_t)(sm_count() > 0 ? sm_count() : 1) * (bps > 0 ? bps : 1) * 8;
    size_t g = ((vec ? n / 2 : n) + 255) / 256;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    if (vec) k_hyp<true><<<(int)g, 256, 0, (cudaStream_t)stream>>>(h->right, h->left, v, x, n);
    else k_hyp<false><<<(int)g, 256, 0, (cudaStream_t)stream>>>(h->right, h->left, v, x, n);
    return check_launch("hyperbolic recycle");
}

extern "C" qm_status qm_hyp_destroy(qm_hyp* h)
{
    if (!h) return QM_OK;
    cudaFree(h->mem);
    cudaFree(h->fxmem);
    delete h;
    return QM_OK;
}
