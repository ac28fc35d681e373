"""Local Taylor expansions from the recycling ODE (offline, mpmath).

Sec. 2.1 shows that Q = F^{-1} o G satisfies the recycling ODE
    Q'' + H0(v) Q' = H1(Q) (Q')^2,           H_i = -(log f_i)'.
For the normal target H1(Q) = Q.  Two backgrounds are used here:

* exponential background (Sec. 2.3), H0 = 1:     Q'' + Q' = Q (Q')^2,
  solved by Q(v) = Phi^{-1}(1 - e^{-v}/2), with Q'(v) = (e^{-v}/2) / phi(Q);
* Gaussian background (Sec. 2.2) with the Student-t target of Sec. 3,
  H0 = v, H1(Q) = (1 + 1/n) Q / (1 + Q^2/n):
      (1 + Q^2/n)(Q'' + v Q') = (1 + 1/n) Q (Q')^2.

Given Q and Q' at a point, matching powers of s in Q(v0 + s) = sum b_k s^k
gives each b_{k+2} from b_0..b_{k+1} -- the recurrence of Sec. 3.2 generalised
from the centre v0 = 0 to any expansion point.  These local series are the
coefficients of the table-driven kernels.
"""
from __future__ import annotations

import mpmath as mp


def _conv(a, b, n):
    """Coefficient n of the product of two power series."""
    return mp.fsum(a[i] * b[n - i] for i in range(n + 1) if i < len(a) and n - i < len(b))


def taylor_exp_background(v0, q0, q1, K):
    """b_0..b_K of Q(v0 + s) for Q'' + Q' = Q Q'^2, Q(v0) = q0, Q'(v0) = q1."""
    b = [mp.mpf(q0), mp.mpf(q1)]
    for n in range(0, K - 1):
        d1 = [(i + 1) * b[i + 1] for i in range(len(b) - 1)]        # Q'
        d1sq = [_conv(d1, d1, i) for i in range(n + 1)]            # Q'^2
        rhs = _conv(b, d1sq, n)                                    # Q Q'^2
        b.append((-(n + 1) * b[n + 1] + rhs) / ((n + 2) * (n + 1)))
    return b[: K + 1]


def taylor_gauss_background_t(nu, v0, q0, q1, K):
    """b_0..b_K of Q(v0 + s) for (1 + Q^2/n)(Q'' + v Q') = (1 + 1/n) Q Q'^2."""
    n_ = mp.mpf(nu)
    v0 = mp.mpf(v0)
    b = [mp.mpf(q0), mp.mpf(q1)]
    for n in range(0, K - 1):
        # series of the pieces up to degree n with b_{n+2} unknown (set 0)
        bb = b + [mp.mpf(0)]
        d1 = [(i + 1) * bb[i + 1] for i in range(len(bb) - 1)]
        d2 = [(i + 2) * (i + 1) * bb[i + 2] for i in range(len(bb) - 2)]
        # Q'' + (v0 + s) Q'
        L = [(d2[i] if i < len(d2) else 0) + v0 * d1[i] + (d1[i - 1] if i >= 1 else 0)
             for i in range(n + 1)]
        Q2 = [_conv(bb, bb, i) for i in range(n + 1)]
        A = [(1 if i == 0 else 0) + Q2[i] / n_ for i in range(n + 1)]   # 1 + Q^2/n
        lhs_known = _conv(A, L, n)           # includes A_0 * d2_n with b_{n+2} = 0
        d1sq = [_conv(d1, d1, i) for i in range(n + 1)]
        rhs = (1 + 1 / n_) * _conv(bb, d1sq, n)
        # A_0 (n+2)(n+1) b_{n+2} + lhs_known = rhs
        b.append((rhs - lhs_known) / (A[0] * (n + 2) * (n + 1)))
    return b[: K + 1]


def compose(b, s, K):
    """Coefficients (degree <= K) of sum_k b_k s(r)^k, s(0) = 0."""
    out = [mp.mpf(0)] * (K + 1)
    p = [mp.mpf(1)] + [mp.mpf(0)] * K           # s^0
    for k in range(K + 1):
        for i in range(K + 1):
            out[i] += b[k] * p[i]
        # p <- p * s
        p = [mp.fsum(p[j] * s[i - j] for j in range(i + 1) if i - j < len(s)) for i in range(K + 1)]
    return out


def neg_log1p_series(K):
    """-log(1 + r) = -r + r^2/2 - r^3/3 + ..."""
    return [mp.mpf(0)] + [mp.mpf((-1) ** k) / k for k in range(1, K + 1)]
