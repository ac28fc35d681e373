"""Shared helpers of the GPU parity tests (tolerance measures)."""
import numpy as np


def ulp32(w):
    """Spacing of float32 at |w| (w given as float64)."""
    a = np.abs(np.asarray(w, dtype=np.float64)).astype(np.float32)
    return np.spacing(a).astype(np.float64)


def f32_violations(z, w, ulps=4.0, abs_small=2e-7):
    """Elements where the FP32 result z misses the exact w by more than
    `ulps` ulp of w, or by more than abs_small where |w| < 1e-2.  Infinite
    and NaN exact values must be reproduced exactly."""
    z = np.asarray(z, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    fin = np.isfinite(w)
    bad = np.zeros(w.shape, dtype=bool)
    bad[~fin] = ~((z[~fin] == w[~fin]) | (np.isnan(z[~fin]) & np.isnan(w[~fin])))
    err = np.abs(z[fin] - w[fin])
    ok = (err <= ulps * ulp32(w[fin])) | ((np.abs(w[fin]) < 1e-2) & (err <= abs_small))
    bad[fin] = ~ok
    return bad


def max_ulp(z, w):
    fin = np.isfinite(w) & (np.abs(w) >= 1e-2)
    return float(np.max(np.abs(np.asarray(z, np.float64)[fin] - w[fin]) / ulp32(w[fin]))) if fin.any() else 0.0


def rel_err(z, w):
    z = np.asarray(z, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    out = np.zeros(w.shape)
    m = np.isfinite(w) & (w != 0)
    out[m] = np.abs(z[m] / w[m] - 1.0)
    return out


def f64_violations(z, w, tol, u=None, lo=1e-300, hi=1.0 - 2.0**-53):
    """Relative error above `tol` where w is finite and non-zero (and, if u is
    given, u in [lo, hi]); exact agreement required for infinite/NaN/zero w."""
    z = np.asarray(z, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    bad = np.zeros(w.shape, dtype=bool)
    special = ~np.isfinite(w) | (w == 0)
    bad[special] = ~((z[special] == w[special]) | (np.isnan(z[special]) & np.isnan(w[special])))
    m = ~special
    if u is not None:
        u = np.asarray(u, dtype=np.float64)
        m &= (u >= lo) & (u <= hi)
    bad[m] = ~(np.abs(z[m] / w[m] - 1.0) <= tol)   # NaN counts as a miss
    return bad


_cudart = None


def cudart():
    """The CUDA runtime library (for raw device-to-host copies in tests)."""
    import ctypes
    global _cudart
    if _cudart is None:
        for name in ("libcudart.so.13", "libcudart.so.12", "libcudart.so",
                     "/usr/local/cuda/lib64/libcudart.so"):
            try:
                _cudart = ctypes.CDLL(name)
                break
            except OSError:
                continue
        if _cudart is None:
            raise RuntimeError("libcudart not found")
    return _cudart


def d2h(ptr, n, dtype):
    """Copy n elements of dtype from a raw device pointer to a numpy array."""
    import ctypes
    host = np.empty(n, dtype=dtype)
    rc = cudart().cudaMemcpy(ctypes.c_void_p(host.ctypes.data), ctypes.c_void_p(ptr),
                             ctypes.c_size_t(host.nbytes), 2)   # cudaMemcpyDeviceToHost
    assert rc == 0, rc
    return host
