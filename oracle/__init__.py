"""CPU FP64 oracle for the quantile hot path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` leg of
``bench.py`` may import this package.  The product library never does; the two
share no code.  The arithmetic lives in ``orc.c`` (plain C, IEEE binary64,
compiled with floating-point contraction off so that x86 and Arm builds agree);
this module only builds it and marshals numpy arrays through ctypes.

What each routine computes, and the passage it restates:

* ``probit``      -- Phi^{-1}(u), the normal quantile w(u) with F(w(u)) = u
                     (Sec. 1, Eq. 1), by bracketed Newton on erf (centre) or on
                     log(1 - Phi) (tails).
* ``recycle_t``   -- Q(z) = F_nu^{-1}(Phi(z)), normal -> Student t (Sec. 3),
                     through the regularised incomplete beta function.
* ``recycle_exp`` -- Q(x) = Phi^{-1}(1 - e^{-x}), exponential -> normal
                     (Sec. 2.3 and Sec. 6).
* ``chi2_from_normal`` -- W = F^{-1}(Phi(z)) for W ~ chi-squared(nu): the
                     mixing variable of the t copula (Sec. 9), through the
                     regularised incomplete gamma function (DLMF 8.7.1 series,
                     8.9.2 continued fraction) solved in log space.
* ``t_to_normal`` -- G(t) = Phi^{-1}(F_nu(t)), Student t -> normal (the
                     inverse of the Sec. 3 map), for t-copula margins.
* ``philox_stream`` -- Philox4x32-10 words (Salmon et al., SC'11).
* ``hyperbolic.recycle_hyperbolic`` -- Q(v) = F^{-1}(G_0(v)), two-sided
                     exponential -> hyperbolic (Sec. 8.1), by quadrature and
                     Brent's method (``oracle/hyperbolic.py``, numpy/scipy).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "orc.c")
_HDR = os.path.join(_HERE, "orc.h")
_LIB = os.path.join(_HERE, "liborc.so")

_lib = None


def build(force: bool = False) -> str:
    """Compile ``liborc.so`` with gcc (no GPU or CUDA needed)."""
    stale = (not os.path.exists(_LIB)) or any(
        os.path.getmtime(p) > os.path.getmtime(_LIB) for p in (_SRC, _HDR))
    if force or stale:
        tmp = _LIB + ".tmp.%d" % os.getpid()
        cmd = ["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-fno-fast-math",
               "-ffp-contract=off", "-o", tmp, _SRC, "-lm", "-lpthread"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
    return _LIB


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        d, p, sz, i = ctypes.c_double, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int
        for name in ("orc_erf", "orc_erfc", "orc_erfcx", "orc_norm_cdf",
                     "orc_norm_sf", "orc_log_norm_sf", "orc_probit",
                     "orc_probit_centre", "orc_probit_tail_log",
                     "orc_recycle_exp_to_normal"):
            getattr(L, name).restype = d
            getattr(L, name).argtypes = [d]
        for name in ("orc_t_sf", "orc_recycle_normal_to_t", "orc_log_gamma_p", "orc_log_gamma_q",
                     "orc_chi2_from_normal", "orc_t_to_normal"):
            getattr(L, name).restype = d
            getattr(L, name).argtypes = [d, d]
        L.orc_t_gamma.restype = d
        L.orc_t_gamma.argtypes = [d]
        L.orc_ibeta.restype = d
        L.orc_ibeta.argtypes = [d, d, d]
        L.orc_philox4x32_10.restype = None
        L.orc_philox4x32_10.argtypes = [p, p, p]
        L.orc_philox_stream.restype = None
        L.orc_philox_stream.argtypes = [ctypes.c_uint64, ctypes.c_uint64, sz, p]
        L.orc_probit_array.restype = i
        L.orc_probit_array.argtypes = [p, p, sz, i]
        L.orc_recycle_t_array.restype = i
        L.orc_recycle_t_array.argtypes = [d, p, p, sz, i]
        L.orc_recycle_exp_array.restype = i
        L.orc_recycle_exp_array.argtypes = [p, p, sz, i]
        L.orc_threads_used.restype = i
        L.orc_threads_used.argtypes = [i]
        _lib = L
    return _lib


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _vec(fn, x, *, nthreads: int = 0, extra=()):
    x = _f64(x)
    out = np.empty_like(x)
    fn(*extra, x.ctypes.data, out.ctypes.data, x.size, nthreads)
    return out


def probit(u, nthreads: int = 0) -> np.ndarray:
    return _vec(lib().orc_probit_array, u, nthreads=nthreads)


def recycle_t(nu: float, z, nthreads: int = 0) -> np.ndarray:
    return _vec(lib().orc_recycle_t_array, z, nthreads=nthreads,
                extra=(ctypes.c_double(nu),))


def recycle_exp(x, nthreads: int = 0) -> np.ndarray:
    return _vec(lib().orc_recycle_exp_array, x, nthreads=nthreads)


def chi2_from_normal(nu: float, z) -> np.ndarray:
    """W = F_{chi2(nu)}^{-1}(Phi(z)) element by element."""
    f = lib().orc_chi2_from_normal
    z = _f64(z)
    return np.array([f(nu, float(v)) for v in z.ravel()]).reshape(z.shape)


def t_to_normal(nu: float, t) -> np.ndarray:
    """G(t) = Phi^{-1}(F_nu(t)) element by element."""
    f = lib().orc_t_to_normal
    t = _f64(t)
    return np.array([f(nu, float(v)) for v in t.ravel()]).reshape(t.shape)


def scalar(name: str):
    """Scalar entry point ``orc_<name>`` as a Python callable."""
    return getattr(lib(), "orc_" + name)


def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32))
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint32))
    o = np.empty(4, dtype=np.uint32)
    lib().orc_philox4x32_10(c.ctypes.data, k.ctypes.data, o.ctypes.data)
    return o


def philox_stream(seed: int, first: int, n: int) -> np.ndarray:
    o = np.empty(n, dtype=np.uint32)
    lib().orc_philox_stream(seed, first, n, o.ctypes.data)
    return o


def threads_used(nthreads: int = 0) -> int:
    return lib().orc_threads_used(nthreads)
