"""Near-minimax rational fits in relative error (offline coefficient builder).

The paper builds its approximations with a minimax rational generator in high
precision (Sec. 6, the fit of Q(v)/v with the series near v = 0).  This is the
builder's own equivalent: a Sanathanan-Koerner linearisation with Lawson
reweighting (Lawson 1961; Nakatsukasa & Trefethen, SIAM J. Sci. Comput. 2020)
on a dense Chebyshev grid, solved by Householder QR in x87 extended precision
(numpy longdouble, 64-bit significand), then converted to monomial
coefficients in multiprecision and checked against the target in mpmath.
Runs on the development machine only; its output is a generated header.
"""
from __future__ import annotations

import mpmath as mp
import numpy as np

LD = np.longdouble


def cheb_basis(t, deg):
    T = np.empty((t.size, deg + 1), dtype=LD)
    T[:, 0] = 1
    if deg >= 1:
        T[:, 1] = t
    for k in range(2, deg + 1):
        T[:, k] = 2 * t * T[:, k - 1] - T[:, k - 2]
    return T


def lstsq_qr(A, b):
    """Least squares by Householder QR in longdouble."""
    A = A.copy()
    b = b.copy()
    m, n = A.shape
    for j in range(n):
        x = A[j:, j]
        nx = np.sqrt(np.sum(x * x))
        if nx == 0:
            continue
        alpha = -nx if x[0] >= 0 else nx
        v = x.copy()
        v[0] -= alpha
        nv = np.sum(v * v)
        if nv == 0:
            continue
        A[j:, j:] -= np.outer(v, (2 / nv) * (v @ A[j:, j:]))
        b[j:] -= v * ((2 / nv) * (v @ b[j:]))
    R = A[:n, :n]
    y = b[:n].copy()
    for i in range(n - 1, -1, -1):
        y[i] = (y[i] - R[i, i + 1:] @ y[i + 1:]) / R[i, i]
    return y


def fit(t, f, n, m, iters=300, lawson_start=8, verbose=False):
    """Fit f(t) ~ P(t)/Q(t), deg P = n, deg Q = m, on nodes t in [-1, 1], in
    relative error.  Returns Chebyshev coefficients (p, q) with q[0] = 1 and
    the max relative error seen on the nodes."""
    Tp = cheb_basis(t, n)
    Tq = cheb_basis(t, m)
    w = np.ones_like(t) / t.size
    qprev = np.ones_like(t)
    best = None
    for it in range(iters):
        s = np.sqrt(w) / (f * qprev)
        A = np.concatenate([Tp * s[:, None], -(f * s)[:, None] * Tq[:, 1:]], axis=1)
        b = f * s * Tq[:, 0]
        c = lstsq_qr(A, b)
        p = c[: n + 1]
        q = np.concatenate([[LD(1)], c[n + 1:]])
        P = Tp @ p
        Q = Tq @ q
        e = (P / Q - f) / f
        emax = np.max(np.abs(e))
        if best is None or emax < best[2]:
            best = (p.copy(), q.copy(), emax)
        if verbose and it % 20 == 0:
            print(it, float(emax))
        qprev = Q
        if it >= lawson_start:
            w = w * np.abs(e)
            w = w / np.sum(w)
            w = np.maximum(w, 1e-30)
    return best


def cheb_to_monomial(c, a, b):
    """Chebyshev series in t = (2x - a - b)/(b - a) -> monomial in x (mpmath)."""
    a, b = mp.mpf(a), mp.mpf(b)
    deg = len(c) - 1
    # T_k as monomials in t
    Tm = [[mp.mpf(1)], [mp.mpf(0), mp.mpf(1)]]
    for k in range(2, deg + 1):
        prev, pp = Tm[k - 1], Tm[k - 2]
        cur = [mp.mpf(0)] * (k + 1)
        for i, v in enumerate(prev):
            cur[i + 1] += 2 * v
        for i, v in enumerate(pp):
            cur[i] -= v
        Tm.append(cur)
    tpoly = [mp.mpf(0)] * (deg + 1)
    for k, ck in enumerate(c):
        ck = mp.mpf(str(ck)) if not isinstance(ck, mp.mpf) else ck
        for i, v in enumerate(Tm[k]):
            tpoly[i] += ck * v
    # substitute t = alpha x + beta
    alpha, beta = 2 / (b - a), -(a + b) / (b - a)
    out = [mp.mpf(0)] * (deg + 1)
    # (alpha x + beta)^i expansion
    for i, ti in enumerate(tpoly):
        for j in range(i + 1):
            out[j] += ti * mp.binomial(i, j) * alpha**j * beta ** (i - j)
    return out


def horner(c, x):
    acc = mp.mpf(0)
    for ck in reversed(c):
        acc = acc * x + ck
    return acc


# ---------------------------------------------------------------------------
# Rational Remez exchange in relative error (multiprecision).  At a reference
# set x_0 < ... < x_{n+m+1} it solves
#     P(x_i) - f_i Q(x_i) = (-1)^i E f_i Q(x_i),   q_0 = 1,
# by fixed-point iteration on the E Q term (Q from the previous solve), then
# moves the reference to the alternating extrema of the error on a dense grid.
# Polynomials are kept in the Chebyshev basis of t in [-1, 1].
# ---------------------------------------------------------------------------
def _cheb_row(t, deg):
    row = [mp.mpf(1)]
    if deg >= 1:
        row.append(t)
    for k in range(2, deg + 1):
        row.append(2 * t * row[-1] - row[-2])
    return row


def _cheb_eval(c, t):
    return mp.fsum(ck * tk for ck, tk in zip(c, _cheb_row(t, len(c) - 1)))


def _alternating_extrema(ts, es, N):
    runs = []
    cur = None
    for t, e in zip(ts, es):
        s = 1 if e >= 0 else -1
        if cur is None or s != cur[2]:
            if cur is not None:
                runs.append(cur)
            cur = [t, e, s]
        elif abs(e) > abs(cur[1]):
            cur[0], cur[1] = t, e
    runs.append(cur)
    while len(runs) > N:
        # drop the smaller of the two ends, or merge away the weakest interior
        mags = [abs(r[1]) for r in runs]
        if len(runs) - N == 1 or True:
            if mags[0] < mags[-1]:
                cand_end = 0
            else:
                cand_end = len(runs) - 1
            i_min = min(range(1, len(runs) - 1), key=lambda i: mags[i]) if len(runs) > 2 else cand_end
            if len(runs) - N >= 2 and mags[i_min] < mags[cand_end] and 0 < i_min < len(runs) - 1:
                # remove an interior weak pair (keeps alternation)
                j = i_min + 1 if mags[i_min + 1] < mags[i_min - 1] else i_min - 1
                for k in sorted([i_min, j], reverse=True):
                    runs.pop(k)
            else:
                runs.pop(cand_end)
    return runs


def remez(fun, a, b, n, m, *, init=None, ngrid=3000, iters=40, tol=1e-3,
          verbose=False):
    """Minimax (n, m) rational in relative error for fun on [a, b].
    ``fun(x)`` returns an mpf.  Returns (p_cheb, q_cheb, E, ref)."""
    a, b = mp.mpf(a), mp.mpf(b)
    N = n + m + 2
    to_x = lambda t: (t * (b - a) + (a + b)) / 2
    # dense grid, Chebyshev-clustered, plus the end points
    G = [mp.cos(mp.pi * (ngrid - 1 - k) / (ngrid - 1)) for k in range(ngrid)]
    fG = [fun(to_x(t)) for t in G]
    if init is None:
        ref = [mp.cos(mp.pi * (N - 1 - k) / (N - 1)) for k in range(N)]
    else:
        ref = [mp.mpf(r) for r in init]
    fmap = {}
    p = q = None
    E = mp.mpf(0)
    for it in range(iters):
        fr = [fun(to_x(t)) for t in ref]
        Qprev = [mp.mpf(1)] * N if q is None else [_cheb_eval(q, t) for t in ref]
        for inner in range(30):
            A = mp.matrix(N, N)
            rhs = mp.matrix(N, 1)
            for i, t in enumerate(ref):
                rp = _cheb_row(t, n)
                rq = _cheb_row(t, m)
                for j in range(n + 1):
                    A[i, j] = rp[j]
                for j in range(1, m + 1):
                    A[i, n + j] = -fr[i] * rq[j]
                A[i, N - 1] = -((-1) ** i) * fr[i] * Qprev[i]
                rhs[i] = fr[i] * rq[0]
            sol = mp.lu_solve(A, rhs)
            p = [sol[j] for j in range(n + 1)]
            q = [mp.mpf(1)] + [sol[n + j] for j in range(1, m + 1)]
            Enew = sol[N - 1]
            Qnew = [_cheb_eval(q, t) for t in ref]
            done = abs(Enew - E) <= mp.mpf("1e-6") * abs(Enew)
            E = Enew
            Qprev = Qnew
            if done:
                break
        es = [(_cheb_eval(p, t) / _cheb_eval(q, t) - f) / f for t, f in zip(G, fG)]
        emax = max(abs(e) for e in es)
        runs = _alternating_extrema(G, es, N)
        if verbose:
            print(f"  remez it {it}: |E| {float(abs(E)):.4g} max {float(emax):.4g} nruns {len(runs)}")
        if len(runs) < N:
            break
        newref = [r[0] for r in runs]
        if abs(emax / abs(E) - 1) < tol:
            ref = newref
            break
        ref = newref
    return p, q, emax, ref


def to_monomial(p, q, a, b):
    P = cheb_to_monomial(p, a, b)
    Q = cheb_to_monomial(q, a, b)
    q0 = Q[0]
    return [c / q0 for c in P], [c / q0 for c in Q]
