/*
 * qm.h -- C ABI of the GB300 quantile library (libqm.so).
 *
 * Element-wise quantile evaluation over device arrays, after Shaw, Luu &
 * Brickman, "Quantile Mechanics II" (arXiv 0901.0638):
 *   - the normal quantile w(u) = Phi^{-1}(u) (Sec. 1, Eq. 1) through a change
 *     of variables to the exponential coordinate v = -log(2 min(u, 1-u))
 *     (Sec. 6, Sec. 7.2) or the scaled Student-t_2 coordinate
 *     v = |u - 1/2| / sqrt(u - u^2) (Sec. 7.3), each followed by one rational
 *     approximation;
 *   - the recycling maps Q(x) = F^{-1}(G(x)) of Sec. 2.1: normal -> Student t
 *     (Sec. 3), exponential -> normal (Sec. 2.3, Sec. 6) and two-sided
 *     exponential -> hyperbolic (Sec. 8.1);
 *   - fused counter-based generation (Philox4x32-10) + transform, and the
 *     Gaussian copula with recycled marginals (Sec. 9).
 *
 * Conventions (all entry points):
 *   - Data pointers are DEVICE pointers owned by the caller unless stated.
 *     The library owns only workspaces it allocates in *_create calls, a
 *     small per-device scratch for reductions, and the run-time Student-t
 *     tables of untabulated nu (both allocated on first use, kept until the
 *     process exits).
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Calls are asynchronous on it; argument errors are returned
 *     synchronously before any launch; launch failures return QM_ERR_CUDA.
 *   - n == 0 returns QM_OK with no launch.  In-place (in == out) is allowed;
 *     any other overlap of in and out is QM_ERR_INVALID.  Pointers of any
 *     alignment are accepted (16-byte aligned ones take the vector path).
 *   - Out-of-domain inputs give IEEE results, not errors: Phi^{-1}(0) = -inf,
 *     Phi^{-1}(1) = +inf, NaN for u outside [0, 1] or NaN.
 *   - qm_last_error() returns a thread-local message for the last failure.
 */
#ifndef QM_H
#define QM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    QM_OK = 0,
    QM_ERR_INVALID = 1,      /* bad argument: null pointer, overlap, bad enum */
    QM_ERR_UNSUPPORTED = 2,  /* valid request this library does not provide  */
    QM_ERR_CUDA = 3,         /* a CUDA runtime call or launch failed          */
    QM_ERR_NOMEM = 4,        /* device or host allocation failed              */
    QM_ERR_TIMEOUT = 5       /* a bounded device wait gave up                 */
} qm_status;

typedef enum {
    QM_DIST_UNIFORM = 0,
    QM_DIST_NORMAL = 1,
    QM_DIST_STUDENT_T = 2,
    QM_DIST_EXPONENTIAL = 3
} qm_dist;

/* Algorithm variants of the normal quantile. */
typedef enum {
    QM_VAR_DEFAULT = 0,      /* FP32: TABLE; FP64: FIXED                        */
    QM_VAR_BRANCHFREE = 1,   /* exponential coordinate, one rational for the
                                whole range (FP32: Sec. 6.1 form z = v P/Q on
                                v <= 25, a reproduction of the paper's form
                                that reaches 4.1 ulp, just outside the 4-ulp
                                FP32 bound that TABLE and SQRT_FORM meet;
                                FP64: Sec. 7.2 form on v <= 42 plus a
                                deep-tail rational on 42 < v <= 745)            */
    QM_VAR_HYBRID_VOTE = 2,  /* FP64: t_2 coordinate when the whole warp has
                                v < 15.5, else the exponential form (Sec. 7.3,
                                the warp vote)                                  */
    QM_VAR_MIXED_HALLEY = 3, /* FP64: FP32 rational + one FP64 Halley step     */
    QM_VAR_COMPACT = 4,      /* FP64: t_2 coordinate for every element it
                                covers; the others are compacted per block and
                                evaluated densely in the exponential form       */
    QM_VAR_SQRT_FORM = 5,    /* FP32: exponential coordinate with a two-float
                                logarithm, z = v sqrt(R(v)), R = (Q(v)/v)^2     */
    QM_VAR_CUDA_LIBM = 6,    /* comparator: CUDA's normcdfinvf / normcdfinv     */
    QM_VAR_TABLE = 7,        /* exponential coordinate without log or divide:
                                x = 2d = 2^E m, segment (E, top bits of m),
                                r = m c - 1, |z| = local expansion G(r) of Q(v)
                                from the recycling ODE (FP64: d >= 2^-65, the
                                deep tail compacted to the deep rational)       */
    QM_VAR_FIXED = 8,        /* FP64: the same segment expansions (Sec. 2.3,
                                Sec. 6) in an exact integer offset t from the
                                segment anchor, evaluated in 64-bit fixed
                                point with one FP64 FMA, |z| = a0 + t H(t);
                                every 0 < u < 1 (subnormal u too) takes the
                                same path.  The FP64 default.                   */
    QM_VAR_ALMOST_NORMAL = 9, /* FP32 and FP64: the almost-normal /
                                almost-chi-squared filtering coordinates
                                (Sec. 4.4): a = -(pi/2) log(4 d (1-d));
                                a <= 8: |z| = (1 - 2d) P(a); a > 8: |z| = T(sqrt a)
                                on pieces of the sqrt(a) axis; polynomials
                                only (no divide).  FP64: one Horner loop over a
                                per-lane coefficient row (no branch).           */
    QM_VAR_T2_MULTI = 10,    /* FP64: the hybrid with more branches (Sec. 7.4):
                                t_2 coordinate for v <= 1000 (the Sec. 7.3
                                rational on v <= 15.5, a second (14,15) t_2
                                rational on the near tail 15.5 < v <= 1000,
                                coefficients selected per lane), the rest
                                compacted per tile onto the exponential form.  */
    QM_VAR_PAPER_EXACT = 11, /* reproduction of the paper's own kernels from its
                                printed coefficients and arithmetic.  FP32: the
                                (5,6) rational of Sec. 6.1 / Appendix A, with
                                the fast logarithm and division.  FP64: the
                                Appendix C hybrid, t_2 (14,15) rational when the
                                whole warp (32 consecutive elements) has
                                v < 15.5 (Sec. 7.3), else the Appendix B
                                (13,13) exponential-coordinate rational.
                                Certified by the paper on v <= 25 (FP32) and
                                u >= 2.875e-19 (FP64); beyond, the printed
                                rationals are extrapolated as printed (no
                                deep-tail piece), and the FP32 form returns NaN
                                for u below 2^-127.  Edges as in the contract. */
    QM_VAR_PAPER_EXACT_B = 12 /* FP64: the branch-free Appendix B kernel alone
                                (Sec. 7.2), printed (13,13) coefficients, log,
                                rounded reciprocal; same domain as above.      */
} qm_variant;

typedef struct {
    double nu; /* Student-t degrees of freedom, nu > 0; ignored otherwise */
} qm_params;

/* ---- normal quantile ------------------------------------------------------
 * z[i] = Phi^{-1}(u[i]) for i < n (Sec. 1, Eq. 1).  FP32 variants: DEFAULT,
 * BRANCHFREE, SQRT_FORM, TABLE, ALMOST_NORMAL, CUDA_LIBM, PAPER_EXACT; FP64
 * variants: DEFAULT, BRANCHFREE, HYBRID_VOTE, MIXED_HALLEY, COMPACT, TABLE,
 * FIXED, ALMOST_NORMAL, T2_MULTI, CUDA_LIBM, PAPER_EXACT, PAPER_EXACT_B
 * (others: QM_ERR_INVALID).
 * u, z: contiguous arrays of n elements, in device memory or in page-locked
 * host memory (cudaHostAlloc / cudaHostRegister; with unified addressing its
 * pointer is a device pointer): the kernel then streams the data over the
 * host link itself, with no staging copy.  Pageable host memory is not
 * accepted (the kernel cannot address it).
 * In place (u == z), three FP64 variants whose kernels read some inputs a
 * second time after storing others switch algorithm, with results still
 * within the FP64 bound but not bit-identical to the out-of-place call:
 * TABLE runs as BRANCHFREE (about 14x slower), COMPACT as HYBRID_VOTE, and
 * T2_MULTI as its per-element form without the compaction.  The default
 * (FIXED) and every other variant run the same kernel in place.            */
qm_status qm_normal_quantile_f32(const float* u, float* z, size_t n,
                                 int variant, void* stream);
qm_status qm_normal_quantile_f64(const double* u, double* z, size_t n,
                                 int variant, void* stream);

/* z[i] = Phi^{-1}((k + 1/2) 2^-24) with k = words[i] >> 8 (the top 24 bits),
 * evaluated in the exact reflected form d = (min(k, 2^24-1-k) + 1/2) 2^-24
 * (Sec. 6.1, the "better" reflection) with the TABLE form.
 * words: uint32[n], z: float[n].                                            */
qm_status qm_normal_quantile_bits24_f32(const uint32_t* words, float* z,
                                        size_t n, void* stream);

/* ---- Philox4x32-10 (Salmon et al., SC'11) ---------------------------------
 * out[i] = word (ctr0 + i) of the stream with 64-bit key `key`: output word
 * (j mod 4) of block floor(j/4), block b = counter (b lo32, b hi32, 0, 0),
 * key (key lo32, key hi32).  out: uint32[n] (device).                      */
qm_status qm_philox_fill_u32(uint64_t key, uint64_t ctr0, uint32_t* out,
                             size_t n, void* stream);

/* ---- fused generate + transform -------------------------------------------
 * Sample i (0 <= i < n) of `target` drawn from the key's stream starting at
 * word ctr0 (ctr0 must be a multiple of 4), uniforms kept in registers:
 *   QM_DIST_NORMAL, out_is_f64 = 0: word ctr0+i -> k = top 24 bits ->
 *       z = Phi^{-1}((k + 1/2) 2^-24), identical to
 *       qm_philox_fill_u32 + qm_normal_quantile_bits24_f32;
 *   QM_DIST_NORMAL, out_is_f64 = 1: words (ctr0+2i, ctr0+2i+1) -> 53-bit k
 *       -> z = Phi^{-1}((k + 1/2) 2^-53) (FP64 exponential form);
 *   QM_DIST_STUDENT_T (p->nu required): t = F_nu^{-1}(Phi(z)) of the FP64
 *       normal above (Sec. 3 map), FP64 only;
 *   QM_DIST_EXPONENTIAL: the Exp(1) sample x = -log(u), u = (k + 1/2) 2^-53,
 *       mapped to the normal by the Sec. 6 recycling map Q(x) =
 *       Phi^{-1}(1 - e^{-x}) = Phi^{-1}(1 - u), evaluated from the exact u
 *       (x itself is never rounded), FP64 only.
 * out: float[n] / double[n] (device) or NULL.  moments4: double[4] (device)
 * or NULL; if given it receives sum z, sum z^2, sum z^3, sum z^4 over the n
 * samples (overwritten, not accumulated).  At least one of out / moments4.
 * Moment calls keep their per-block partials in one library-owned scratch
 * buffer per device (one cudaMalloc at the first moment call on a device,
 * sized for the largest grid, never freed or replaced until exit).  Every
 * moment call on a device shares it: calls that overlap on the GPU
 * (different streams with no ordering between them) race and return wrong
 * moments; calls ordered on one stream are safe.                           */
qm_status qm_sample_fused(int target, const qm_params* p, uint64_t key,
                          uint64_t ctr0, void* out, int out_is_f64, size_t n,
                          double* moments4, void* stream);

/* ---- fused moments without allocation ---------------------------------------
 * Same sums as qm_sample_fused(QM_DIST_NORMAL, NULL, key, ctr0, NULL, 0, n,
 * moments4, stream) (up to the order of the FP64 additions), for callers that
 * must not allocate device memory at call time: cudaMalloc can synchronise
 * the device, which a latency-bound pipeline cannot afford; embedded runtimes
 * plan all device memory up front and have no allocator to call; code that
 * runs while a caching allocator holds its lock would deadlock on it.  The
 * paper has no counterpart; this is a property of the library interface.
 * Scratch is a file-scope device array of 16384 x 4 doubles (512 KiB) that
 * every device loading the library keeps until the process exits; a call
 * makes no cudaMalloc/cudaFree and no allocating library call.
 * n <= 2^32 (16384 blocks of 2^18 samples); larger n returns QM_ERR_INVALID
 * with a message.  ctr0 must be a multiple of 4.  moments4: double[4]
 * (device), overwritten.  The first call on a device looks up the array's
 * device address (cudaGetSymbolAddress) with that device current; make that
 * first call before any stream capture.  All calls share the one array:
 * calls that overlap on the GPU (different streams, no ordering) race and
 * give wrong moments; calls ordered on one stream are safe.  Each call
 * overwrites every scratch slot it reads, so nothing is cleared between calls. */
qm_status qm_sample_moments_noalloc(uint64_t key, uint64_t ctr0, size_t n,
                                    double* moments4, void* stream);

/* ---- recycling maps Q = F^{-1}(G(x)) (Sec. 2.1) -----------------------------
 * Supported (src, dst): (NORMAL, STUDENT_T): out = F_nu^{-1}(Phi(in))
 * (Sec. 3; p->nu required: nu in {1,2,3,4,5,8,10,30} from tables fitted
 * offline, any other real nu in [QM_T_NU_MIN, QM_T_NU_MAX] from tables built
 * on the host at the first call with that nu on a device -- the recurrence of
 * Sec. 3.2 integrated from the tail coordinate of Sec. 3.3, see
 * qm_t_table_build -- then uploaded (a synchronous cudaMalloc + copy of
 * QM_T_ROWS_BYTES, kept until exit; at most 256 distinct nu per process, then
 * QM_ERR_NOMEM); nu outside both: QM_ERR_UNSUPPORTED).  On upload every
 * segment is split into four rows of width 1/128, each re-expanded about its
 * start and stored for evaluation in 64-bit fixed point with one FP64 FMA
 * (the offline tables too, at the first use on a device; see
 * qm_t_rows_build); a table whose coefficients fail the conversion's sign,
 * range or accuracy checks is refused with QM_ERR_UNSUPPORTED;
 * (EXPONENTIAL, NORMAL): out = Phi^{-1}(1 - e^{-in}) (Sec. 2.3, Sec. 6);
 * (UNIFORM, NORMAL): out = Phi^{-1}(in) (FP64 default variant).
 * Anything else: QM_ERR_UNSUPPORTED.  in, out: double[n] (device).        */
qm_status qm_recycle(int src, int dst, const qm_params* p, const double* in,
                     double* out, size_t n, void* stream);

/* ---- normal -> Student t tables for any real nu (host only, no GPU) ---------
 * The tables qm_recycle builds for an untabulated nu, returned in host memory
 * for inspection and testing.  Q_nu(z) = F_nu^{-1}(Phi(z)) on 0 <= z < 8.75 is
 * cut into QM_T_NSEG segments of width 1/32; seg_coef[10 j + k] is the
 * coefficient of s^k of the expansion of Q_nu about z_j = (j + 1/2)/32
 * (z_0 = 0, the central series of Sec. 3.2), s = z - z_j.  The expansions come
 * from the Gaussian-background recycling ODE (Sec. 3.1), integrated in long
 * double backwards from the tail (the stable direction) and checked against
 * the central series.  tail[0] = nu, tail[1] = log kappa, kappa =
 * nu B(nu/2, 1/2), tail[2] = degree D = QM_T_TAIL_TERMS - 1, tail[3 + k] = R_k:
 * for z >= 8.75, Q = sqrt(nu) w^{-1/nu} R(w^{2/nu}), w = kappa (1 - Phi(z))
 * (Sec. 3.3), R from series reversion of the exact Student tail.
 * seg_coef: 10 QM_T_NSEG doubles; tail: 3 + QM_T_TAIL_TERMS doubles (host).
 * nu outside [QM_T_NU_MIN, QM_T_NU_MAX]: QM_ERR_UNSUPPORTED.                 */
#define QM_T_NSEG 280
#define QM_T_TAIL_TERMS 30
#define QM_T_NU_MIN 0.75
#define QM_T_NU_MAX 100.0
qm_status qm_t_table_build(double nu, double* seg_coef, double* tail);

/* qm_t_rows_build (host only, no GPU): the rows the device evaluates for nu,
 * QM_T_NROW rows of width 1/128 on 0 <= |z| < 8.75 (row r starts at
 * z_r = r/128; segment j of qm_t_table_build re-expanded about each of its
 * four row starts and truncated to degree 7), in QM_T_ROWS_BYTES of host
 * memory: first QM_T_NROW 32-byte rows {double a0; int64 B0, B1, B2e}, then
 * QM_T_NROW 16-byte rows {uint32 C3, C4, C5, C6s}.
 * |t| = a0 + sigma H(th), sigma = |z| - z_r, th = 64 sigma in [0, 1/2);
 * H = sum b'_k th^k with B_k = b'_k 2^-s0 (k <= 2; B2e = B_2 | e0 << 52,
 * e0 = 1080 + s0, H(0) 2^-s0 in [2^58, 2^59)) and C_k = b'_k 2^-(s0 + c)
 * (k = 3..6; C6s = C_6 | (32 - c) << 27), every b'_k >= 0.
 * Errors as qm_t_table_build; QM_ERR_UNSUPPORTED if a row does not fit the
 * form (signs, ranges, or off by more than 1e-12 from the segment's
 * degree-9 expansion after packing).  QM_FX_ROW_BYTES is the size of the
 * 64-byte rows of qm_hyp_rows_build.                                       */
#define QM_T_NROW 1120
#define QM_T_ROWS_BYTES (QM_T_NROW * 48)
#define QM_FX_ROW_BYTES 64
qm_status qm_t_rows_build(double nu, void* rows);

/* ---- exponential -> hyperbolic recycling (Sec. 8.1) --------------------------
 * Target: the hyperbolic density f(x) = exp(-alpha sqrt(delta^2 + x^2) +
 * beta x) / Z (location 0; Z = 2 alpha delta K_1(delta gamma) / gamma,
 * gamma = sqrt(alpha^2 - beta^2)).  Base: the two-sided exponential with the
 * same mass split at 0: density p_+ (alpha-beta) e^{-(alpha-beta) v} for v > 0
 * and p_- (alpha+beta) e^{(alpha+beta) v} for v < 0, p_+ = P(X > 0).
 * x = Q(v) = F^{-1}(G_0(v)) maps base samples to hyperbolic samples; Q solves
 * the paper's right/left recycling ODEs with Q(0) = 0 and
 * Q'(0+-) = f_0(0+-)/f(0).
 * qm_hyp_create builds the map for one parameter set on the host (long
 * double: Taylor series of the ODEs integrated backwards from the tails, on
 * segments of |v| with 32 per binade 2^E <= |v| < 2^(E+1), E >= QM_HYP_E_MIN,
 * degree 9 per segment, and the series about 0 below), uploads it (one
 * cudaMalloc of ~260 KB, owned by the handle) and returns the handle.
 * Errors: alpha <= 0, |beta| >= alpha, delta <= 0: QM_ERR_INVALID; alpha - |beta|
 * < 1e-3 alpha or alpha delta outside [1e-4, 1e4]: QM_ERR_UNSUPPORTED.
 * qm_hyp_recycle: x[i] = Q(v[i]) for device arrays of n doubles (in place
 * allowed); +-inf -> +-inf, NaN -> NaN; |v| beyond what a double sample of the
 * base can reach (p e^{-rate |v|} < 2^-1074) is extrapolated from the last
 * segment.  qm_hyp_info: p_+, p_-, Q'(0+), Q'(0-), log Z (host double[5]).
 * qm_hyp_table_build (host only, no GPU): the same tables in host memory --
 * seg_right / seg_left: (1 + 32 QM_HYP_MAX_BINADES) x 10 doubles each; entry 0
 * the series about 0 (coefficient k of v^k), entry 1 + 32 (E - QM_HYP_E_MIN)
 * + j the expansion about 2^E (1 + (2j+1)/64) for the right (v > 0) and left
 * (|v| for v < 0, values -Q(-|v|)) sides; e_max[2] the last binade per side;
 * info as qm_hyp_info.                                                       */
#define QM_HYP_E_MIN (-30)
#define QM_HYP_MAX_BINADES 64
typedef struct qm_hyp qm_hyp;
qm_status qm_hyp_create(double alpha, double beta, double delta, qm_hyp** out);
qm_status qm_hyp_recycle(const qm_hyp* h, const double* v, double* x, size_t n, void* stream);
qm_status qm_hyp_info(const qm_hyp* h, double* info);
qm_status qm_hyp_destroy(qm_hyp* h);
qm_status qm_hyp_table_build(double alpha, double beta, double delta, double* seg_right,
                             double* seg_left, int* e_max, double* info);

/* qm_hyp_rows_build (host only, no GPU): the fixed-point rows the device
 * evaluates, 32 QM_HYP_MAX_BINADES rows of QM_FX_ROW_BYTES per side (row
 * 32 (E - QM_HYP_E_MIN) + j for segment j of binade E, width 2^(E-5), up to
 * e_max[side]; later rows zero).  Layout as qm_t_rows_build, but biased for
 * coefficients of either sign: |Q| = a0 + sigma P(tau), sigma = |v| - start,
 * tau = sigma / 2^(E-4); D1..D3 hold d_k 2^-s0 + 2^60, D4e the low 52 bits
 * d_4 2^-s0 + 2^51 (e0 above), c[0..2] C_k + 2^29, c[3] (C_8 + 2^25) |
 * (32 - c) << 27.  Errors as qm_hyp_table_build.                           */
qm_status qm_hyp_rows_build(double alpha, double beta, double delta, void* rows_right, void* rows_left,
                            int* e_max);

/* ---- Gaussian copula with recycled marginals (Sec. 9) ------------------------
 * Samples x in R^d with a Gaussian copula of correlation L L^T and the given
 * marginals, folding "normal -> uniform -> marginal" into the recycling map
 * of each coordinate (the remark of the paper's conclusion): per sample,
 * eps_k = Phi^{-1}((m_k + 1/2) 2^-53) from 53-bit Philox integers (two per
 * Philox block; sample i uses blocks ctr0/4 + i ceil(d/2) + b), y = L eps,
 * x_j = Q_j(y_j) with Q_j the identity (QM_DIST_NORMAL) or the Sec. 3 map to
 * Student t with nu_j (QM_DIST_STUDENT_T; tabulated or run-time tables as in
 * qm_recycle).
 * qm_copula_create: chol = host d x d row-major lower-triangular Cholesky
 * factor with positive diagonal (1 <= d <= QM_COPULA_MAX_DIM) of a
 * correlation or covariance matrix (rows are divided by their norms: the
 * copula is that of the correlation), margins = host array of d; copies both
 * to the device (one cudaMalloc, owned by the handle).  Errors: bad d, non-finite or non-lower-triangular L, L[j][j] <= 0:
 * QM_ERR_INVALID; other margin kinds or out-of-range nu: QM_ERR_UNSUPPORTED.
 * qm_copula_sample: out = device double[d n], column-major (x_j of sample i
 * at out[j n + i]); ctr0 a multiple of 4.                                    */
#define QM_COPULA_MAX_DIM 16
typedef struct {
    int kind;            /* QM_DIST_NORMAL or QM_DIST_STUDENT_T */
    double nu;           /* Student-t degrees of freedom */
} qm_margin;
typedef struct qm_copula qm_copula;
qm_status qm_copula_create(int d, const double* chol, const qm_margin* margins, qm_copula** out);
qm_status qm_copula_sample(const qm_copula* c, uint64_t key, uint64_t ctr0, double* out, size_t n,
                           void* stream);
qm_status qm_copula_destroy(qm_copula* c);

/* ---- t copula (Sec. 9) ------------------------------------------------------
 * x_j = F_j^{-1}(F_nu(T_j)), T = (L eps) / sigma * sqrt(nu / W): eps iid
 * normal, W ~ chi-squared(nu) shared by the coordinates of a sample, sigma_j
 * the row norms of L (as for qm_copula_create).  The paper's folding (Sec. 9): W comes from one more
 * grid normal through the normal -> chi-squared recycling map, and each
 * coordinate goes straight to its margin: a Student-t margin with the
 * copula's nu is T_j itself, a normal margin is G(T_j) = Phi^{-1}(F_nu(T_j))
 * (the Student t -> normal recycling map), a Student-t margin with another
 * mu is the normal -> t_mu map after G.  Both maps are tables built on the
 * host from their recycling ODEs at the first use of a nu (cached per device
 * until exit).  Sample i uses the Philox blocks ctr0/4 + i ceil((d+1)/2) + b:
 * its first 53-bit normal is W's, the next d are eps.
 * qm_tcopula_create: as qm_copula_create plus nu in [QM_T_NU_MIN, QM_T_NU_MAX]
 * (QM_ERR_UNSUPPORTED outside); the handle is sampled and destroyed by
 * qm_copula_sample / qm_copula_destroy.
 * qm_tcopula_table_build (host only, no GPU): the two tables for nu, rows of
 * QM_TC_ROW doubles (coefficients 0..9, then one more value) --
 * chi_seg: QM_TC_NZ rows, log W(z) about the centre c_j = -QM_TC_Z_MAX +
 * (j + 1/2)/QM_TC_HZ_INV (stored as the row's last value);
 * g_seg: room for 1 + QM_TC_G_NE_MAX 2^QM_TC_G_K rows, *ne binades used:
 * row 0 is G(t) about t = 0 (for |t| < 2^QM_TC_G_EMIN); row
 * 1 + e 2^K + j covers |t| = 2^E m, E = QM_TC_G_EMIN + e, m in
 * [1 + j 2^-K, 1 + (j+1) 2^-K), as a series in r = m / m_c - 1,
 * m_c = 1 + (j + 1/2) 2^-K, with 1 / m_c as the row's last value.          */
#define QM_TC_Z_MAX 8.5
#define QM_TC_HZ_INV 16
#define QM_TC_NZ 272
#define QM_TC_ROW 11
#define QM_TC_G_EMIN (-5)
#define QM_TC_G_K 5
#define QM_TC_G_NE_MAX 128
qm_status qm_tcopula_create(int d, double nu, const double* chol, const qm_margin* margins, qm_copula** out);
qm_status qm_tcopula_table_build(double nu, double* chi_seg, double* g_seg, int* ne);

/* ---- ragged batches ---------------------------------------------------------
 * A batch is a table of independent recycling jobs evaluated by ONE
 * persistent launch over a device-resident segment table, replayed as a CUDA
 * graph.  Each segment is cut into tiles of block x ept elements that never
 * span two segments, so the target is uniform within a block.
 * Segment pairs: (NORMAL, STUDENT_T) with nu in [QM_T_NU_MIN, QM_T_NU_MAX]
 * (tabulated nu from the offline tables, others from tables built on the host
 * at first use), (EXPONENTIAL, NORMAL), (UNIFORM, NORMAL); in/out device
 * arrays of n doubles.
 * qm_batch_create validates everything before any launch: unsupported pairs
 * or out-of-range nu, null pointers, in/out partial overlap and overlapping
 * outputs of two segments are rejected (QM_ERR_INVALID / QM_ERR_UNSUPPORTED).
 * Tuning: block in {128, 256, 512}, ept in {1, 2, 4}, estrin in {0, 1}
 * (Estrin instead of Horner for the 32-bit inner part of the Student-t
 * segment polynomial; the two truncate differently, so bit-exact comparisons
 * need the same choice).  With
 * tuning == NULL the tuning cache ($QM_TUNE_CACHE, default
 * ~/.cache/qm_tune.txt) is consulted, else (256, 2, 0).  The batch owns its
 * device table and graph; the caller owns the data arrays.                  */
typedef struct {
    int src, dst;        /* distribution pair */
    double nu;           /* Student-t degrees of freedom */
    const double* in;    /* device, n doubles */
    double* out;         /* device, n doubles */
    size_t n;
} qm_segment;

typedef struct {
    int block, ept, estrin;
} qm_tuning;

typedef struct qm_batch qm_batch;

qm_status qm_batch_create(const qm_segment* segs, int nseg, const qm_tuning* tuning,
                          qm_batch** out);
/* One graph launch of the persistent kernel on `stream` (asynchronous). */
qm_status qm_batch_run(qm_batch* b, void* stream);
/* Baseline: one plain launch per segment on `stream`. */
qm_status qm_batch_run_separate(qm_batch* b, void* stream);
qm_status qm_batch_get_tuning(const qm_batch* b, qm_tuning* t);
/* Re-tiles the batch for tuning t and re-uploads its device table.  The call
 * first blocks the host until the batch's last qm_batch_run (on whatever
 * stream it was queued) has finished, so a run in flight never sees the
 * table change under it; qm_batch_destroy waits the same way before it
 * frees the table. */
qm_status qm_batch_set_tuning(qm_batch* b, const qm_tuning* t);
/* Autotuner: times every candidate tuning on this batch (reps graph launches
 * each, synchronising `stream`), keeps the fastest, appends it to the tuning
 * cache under the batch signature (segment count, size bucket, target mix). */
qm_status qm_batch_tune(qm_batch* b, int reps, void* stream, qm_tuning* best);
qm_status qm_batch_destroy(qm_batch* b);

/* ---- serving: continuous batching of Monte Carlo sample requests ------------
 * A request asks for n samples of one target from its own Philox key
 * (counters from 0): QM_REQ_NORMAL_F32 (24-bit grid, TABLE form),
 * QM_REQ_NORMAL_F64 (53-bit grid), QM_REQ_STUDENT_T (the FP64 normal
 * recycled by the Sec. 3 map, nu in [QM_T_NU_MIN, QM_T_NU_MAX]; an
 * untabulated nu has its tables built at submit), QM_REQ_EXP_NORMAL (Exp(1)
 * samples x = -log u recycled by the Sec. 6 map, evaluated from the exact u
 * as in qm_sample_fused).  Sample i of a request is the same value whether
 * it is computed alone or inside any batch.
 * The server owns a device arena of mem_budget bytes (one cudaMalloc at
 * create): a request is admitted, in FIFO order, only when its output fits;
 * its output stays on the device until qm_server_release(id) (or is freed
 * as soon as it completes when release_on_done = 1).  A worker thread packs
 * admitted requests into one launch per batch (<= max_batch requests) on one
 * of `streams` streams; requests arriving while batches run are admitted
 * into the next batch, and batches on different streams overlap.
 * max_batch = 1 with streams = 1 is the plain baseline (one launch per
 * request, FIFO on one stream).  Times are seconds on the server clock
 * (qm_server_now).  Waits are bounded; expiry returns QM_ERR_TIMEOUT.       */
enum { QM_REQ_NORMAL_F32 = 0, QM_REQ_NORMAL_F64 = 1, QM_REQ_STUDENT_T = 2, QM_REQ_EXP_NORMAL = 3 };

typedef struct {
    uint64_t id;
    size_t n;
    int kind;
    double nu;
    uint64_t key;
    double t_arrival;    /* server clock (replay: seconds from the replay call) */
} qm_request;

typedef struct {
    uint64_t id;
    int status;
    void* out;           /* device: n floats (NORMAL_F32) or doubles; NULL once released */
    size_t n;
    int is_f64;
    int kind;
    double nu;
    uint64_t key;
    double t_arrival, t_admit, t_launch, t_done;
} qm_completion;

typedef struct {
    size_t mem_budget;   /* bytes of device arena */
    int max_batch;       /* requests per launch (1 = plain) */
    int streams;         /* concurrent batches, 1..8 */
    int release_on_done; /* free outputs on completion (consumer-less replay) */
    int device;
} qm_server_config;

typedef struct {
    size_t launches, arena_used, arena_capacity;
} qm_server_stats_t;

typedef struct qm_server qm_server;

qm_status qm_server_create(const qm_server_config* cfg, qm_server** out);
qm_status qm_server_submit(qm_server* s, const qm_request* r);
qm_status qm_server_poll(qm_server* s, qm_completion* out, int max, int* got);
qm_status qm_server_release(qm_server* s, uint64_t id);
qm_status qm_server_stats(const qm_server* s, qm_server_stats_t* st);
double qm_server_now(const qm_server* s);
/* Submits trace[i] at t_arrival seconds after the call (real time), waits
 * for all nreq completions (at most timeout_s), stores them in out. */
qm_status qm_server_replay(qm_server* s, const qm_request* trace, int nreq, double timeout_s,
                           qm_completion* out);
qm_status qm_server_destroy(qm_server* s);

/* ---- diagnostics ----------------------------------------------------------- */
const char* qm_last_error(void);
const char* qm_version(void);
int qm_sm_count(void); /* SMs of the current device, or -1 */

#ifdef __cplusplus
}
#endif
#endif /* QM_H */
