/*
 * orc.h -- CPU FP64 oracle for the quantile hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may include, link or
 * call this library: only tests/, __graft_entry__.smoke() and the cpu_baseline
 * leg of bench.py use it.  It shares no code, header, constant table or helper
 * with the CUDA library under paper_0901_0638_gb300/csrc.
 *
 * Every routine is a plain, slow restatement of a definition:
 *   - Phi^{-1}(u) is the root w of F(w) = u for the normal CDF F (Sec. 1,
 *     Eq. 1), found by bracketed Newton iteration with a bisection safeguard.
 *   - The recycling maps are Q(x) = F^{-1}(G(x)) (abstract; Sec. 2.1): the
 *     normal->Student-t map of Sec. 3 and the exponential->normal map of
 *     Sec. 6, each solved the same way on its own CDF.
 *   - erf / erfc are the Maclaurin series (A&S 7.1.5) and the even
 *     contraction of the Laplace continued fraction (A&S 7.1.14).
 *   - I_x(a, b) is the continued fraction of DLMF 8.17.22 (modified Lentz).
 *   - Philox4x32-10 follows Salmon, Moraes, Dror & Shaw, SC'11.
 * All arithmetic is IEEE binary64 (libm exp, log, log1p, expm1, lgamma,
 * sqrt, fma only).
 */
#ifndef ORC_H
#define ORC_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- special functions ---------------------------------------------- */
double orc_erf(double x);
double orc_erfc(double x);
double orc_erfcx(double x);            /* exp(x^2) erfc(x), x >= 0            */
double orc_norm_cdf(double w);         /* Phi(w)                              */
double orc_norm_sf(double w);          /* 1 - Phi(w), relative-accurate       */
double orc_log_norm_sf(double w);      /* log(1 - Phi(w)), never underflows   */

/* ---- normal quantile (Sec. 1, Eq. 1) --------------------------------- */
double orc_probit(double u);           /* Phi^{-1}(u); 0 -> -inf, 1 -> +inf  */
double orc_probit_centre(double t);    /* w >= 0 with erf(w/sqrt2) = t        */
double orc_probit_tail_log(double L);  /* w >= 0 with log(1-Phi(w)) = L       */

/* ---- Student t (Sec. 3.1) -------------------------------------------- */
double orc_ibeta(double a, double b, double x);      /* I_x(a, b)            */
double orc_t_sf(double nu, double t);                /* P(T_nu > t)          */
double orc_t_gamma(double nu);                       /* Q'(0), Sec. 3.1      */
double orc_recycle_normal_to_t(double nu, double z); /* F_nu^{-1}(Phi(z))    */

/* ---- t copula (Sec. 9): chi-squared mixing variable, t -> normal ------- */
double orc_log_gamma_p(double a, double s);   /* log P(a, e^s), regularised    */
double orc_log_gamma_q(double a, double s);   /* log Q(a, e^s) = log(1 - P)    */
double orc_chi2_from_normal(double nu, double z); /* F_chi2(nu)^{-1}(Phi(z))   */
double orc_t_to_normal(double nu, double t);      /* Phi^{-1}(F_nu(t))         */

/* ---- exponential background (Sec. 2.3, Sec. 6) ------------------------ */
double orc_recycle_exp_to_normal(double x);          /* Phi^{-1}(1 - e^{-x}) */

/* ---- Philox4x32-10 ----------------------------------------------------- */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2],
                       uint32_t out[4]);
/* Word i of the stream (key, counter base c0): block (c0 + floor(i/4)) as a
 * 128-bit counter little-endian over (x, y, z, w), output word i mod 4.     */
void orc_philox_stream(uint64_t seed, uint64_t first, size_t n, uint32_t* out);

/* ---- array drivers (nthreads <= 0: all online cores) ------------------ */
int orc_probit_array(const double* u, double* z, size_t n, int nthreads);
int orc_recycle_t_array(double nu, const double* z, double* t, size_t n,
                        int nthreads);
int orc_recycle_exp_array(const double* x, double* z, size_t n, int nthreads);
int orc_threads_used(int nthreads);

#ifdef __cplusplus
}
#endif
#endif
