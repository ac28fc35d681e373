"""GB300 quantile library: Python binding of the C ABI in include/qm.h.

Argument marshalling only.  Every computation runs in the CUDA kernels of
``libqm.so`` (built in-tree from ``csrc/`` by ``_build.build()``); there is no
CPU or PyTorch fallback, and a missing library raises at import of a binding.
Tensors are torch CUDA tensors used for device memory; the stream defaults to
torch's current stream on the tensor's device.
"""
from __future__ import annotations

import ctypes
import os

from . import _build


def _read_text(path):
    with open(path) as fh:
        return fh.read()


QM_OK, QM_ERR_INVALID, QM_ERR_UNSUPPORTED, QM_ERR_CUDA, QM_ERR_NOMEM, QM_ERR_TIMEOUT = range(6)
QM_DIST_UNIFORM, QM_DIST_NORMAL, QM_DIST_STUDENT_T, QM_DIST_EXPONENTIAL = range(4)
(QM_VAR_DEFAULT, QM_VAR_BRANCHFREE, QM_VAR_HYBRID_VOTE, QM_VAR_MIXED_HALLEY,
 QM_VAR_COMPACT, QM_VAR_SQRT_FORM, QM_VAR_CUDA_LIBM, QM_VAR_TABLE, QM_VAR_FIXED,
 QM_VAR_ALMOST_NORMAL, QM_VAR_T2_MULTI, QM_VAR_PAPER_EXACT, QM_VAR_PAPER_EXACT_B) = range(13)

LIB_PATH = _build.LIB

_lib = None


class QMError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"qm status {status}: {msg}")
        self.status = status


class qm_params(ctypes.Structure):
    _fields_ = [("nu", ctypes.c_double)]


class qm_segment(ctypes.Structure):
    _fields_ = [("src", ctypes.c_int), ("dst", ctypes.c_int), ("nu", ctypes.c_double),
                ("inp", ctypes.c_void_p), ("out", ctypes.c_void_p), ("n", ctypes.c_size_t)]


class qm_request(ctypes.Structure):
    _fields_ = [("id", ctypes.c_uint64), ("n", ctypes.c_size_t), ("kind", ctypes.c_int),
                ("nu", ctypes.c_double), ("key", ctypes.c_uint64), ("t_arrival", ctypes.c_double)]


class qm_completion(ctypes.Structure):
    _fields_ = [("id", ctypes.c_uint64), ("status", ctypes.c_int), ("out", ctypes.c_void_p),
                ("n", ctypes.c_size_t), ("is_f64", ctypes.c_int), ("kind", ctypes.c_int),
                ("nu", ctypes.c_double), ("key", ctypes.c_uint64), ("t_arrival", ctypes.c_double),
                ("t_admit", ctypes.c_double), ("t_launch", ctypes.c_double), ("t_done", ctypes.c_double)]


class qm_server_config(ctypes.Structure):
    _fields_ = [("mem_budget", ctypes.c_size_t), ("max_batch", ctypes.c_int), ("streams", ctypes.c_int),
                ("release_on_done", ctypes.c_int), ("device", ctypes.c_int)]


class qm_server_stats_t(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_size_t), ("arena_used", ctypes.c_size_t),
                ("arena_capacity", ctypes.c_size_t)]


QM_REQ_NORMAL_F32, QM_REQ_NORMAL_F64, QM_REQ_STUDENT_T, QM_REQ_EXP_NORMAL = range(4)


class qm_tuning(ctypes.Structure):
    _fields_ = [("block", ctypes.c_int), ("ept", ctypes.c_int), ("estrin", ctypes.c_int)]


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load libqm.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing:
        _build.build()
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"CUDA library {LIB_PATH} is missing; run __graft_entry__.build()")
    L = ctypes.CDLL(LIB_PATH)
    vp, sz, i, u64, d = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_uint64, ctypes.c_double
    sig = {
        "qm_normal_quantile_f32": [vp, vp, sz, i, vp],
        "qm_normal_quantile_f64": [vp, vp, sz, i, vp],
        "qm_normal_quantile_bits24_f32": [vp, vp, sz, vp],
        "qm_philox_fill_u32": [u64, u64, vp, sz, vp],
        "qm_sample_fused": [i, vp, u64, u64, vp, i, sz, vp, vp],
        "qm_recycle": [i, i, vp, vp, vp, sz, vp],
        "qm_t_table_build": [d, vp, vp],
        "qm_hyp_create": [d, d, d, vp],
        "qm_hyp_recycle": [vp, vp, vp, sz, vp],
        "qm_hyp_info": [vp, vp],
        "qm_hyp_destroy": [vp],
        "qm_hyp_table_build": [d, d, d, vp, vp, vp, vp],
        "qm_hyp_rows_build": [d, d, d, vp, vp, vp],
        "qm_t_rows_build": [d, vp],
        "qm_copula_create": [i, vp, vp, vp],
        "qm_tcopula_create": [i, d, vp, vp, vp],
        "qm_tcopula_table_build": [d, vp, vp, vp],
        "qm_copula_sample": [vp, u64, u64, vp, sz, vp],
        "qm_copula_destroy": [vp],
        "qm_sample_moments_noalloc": [u64, u64, sz, vp, vp],
        "qm_batch_create": [vp, i, vp, vp],
        "qm_batch_run": [vp, vp],
        "qm_batch_run_separate": [vp, vp],
        "qm_batch_get_tuning": [vp, vp],
        "qm_batch_set_tuning": [vp, vp],
        "qm_batch_tune": [vp, i, vp, vp],
        "qm_batch_destroy": [vp],
        "qm_server_create": [vp, vp],
        "qm_server_submit": [vp, vp],
        "qm_server_poll": [vp, vp, i, vp],
        "qm_server_release": [vp, u64],
        "qm_server_stats": [vp, vp],
        "qm_server_replay": [vp, vp, i, d, vp],
        "qm_server_destroy": [vp],
    }
    for name, args in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    L.qm_last_error.restype = ctypes.c_char_p
    L.qm_last_error.argtypes = []
    L.qm_version.restype = ctypes.c_char_p
    L.qm_sm_count.restype = ctypes.c_int
    L.qm_server_now.restype = ctypes.c_double
    L.qm_server_now.argtypes = [vp]
    _lib = L
    return L


def declared_symbols():
    """The entry points include/qm.h declares (parsed from the header)."""
    import re
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    names = []
    for h in sorted(os.listdir(os.path.join(root, "include"))):
        if not h.endswith(".h"):
            continue
        txt = _read_text(os.path.join(root, "include", h))
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        names += re.findall(r"\b(qm_[a-z0-9_]+)\s*\(", txt)
    return sorted(set(names))


def _check(status: int):
    if status != QM_OK:
        raise QMError(status, load().qm_last_error().decode())


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, int):
        return t
    return t.data_ptr()


def _stream(stream, t=None):
    if stream is None:
        import torch
        dev = t.device if (t is not None and getattr(getattr(t, "device", None), "type", "") == "cuda") else None
        return torch.cuda.current_stream(dev).cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _numel(t, n):
    return t.numel() if n is None else n


def _params(nu):
    return None if nu is None else ctypes.byref(qm_params(float(nu)))


# ---- bindings (same names as the C entry points) ---------------------------

def qm_normal_quantile_f32(u, z, variant: int = QM_VAR_DEFAULT, n=None, stream=None):
    _check(load().qm_normal_quantile_f32(_ptr(u), _ptr(z), _numel(u, n), variant, _stream(stream, u)))
    return z


def qm_normal_quantile_f64(u, z, variant: int = QM_VAR_DEFAULT, n=None, stream=None):
    _check(load().qm_normal_quantile_f64(_ptr(u), _ptr(z), _numel(u, n), variant, _stream(stream, u)))
    return z


def qm_normal_quantile_bits24_f32(words, z, n=None, stream=None):
    _check(load().qm_normal_quantile_bits24_f32(_ptr(words), _ptr(z), _numel(words, n),
                                                _stream(stream, words)))
    return z


def qm_philox_fill_u32(key: int, ctr0: int, out, n=None, stream=None):
    _check(load().qm_philox_fill_u32(key, ctr0, _ptr(out), _numel(out, n), _stream(stream, out)))
    return out


def qm_sample_fused(target: int, key: int, ctr0: int, out=None, out_is_f64: bool = False,
                    n=None, moments4=None, nu=None, stream=None):
    ref = out if out is not None else moments4
    if n is None:
        n = out.numel()
    _check(load().qm_sample_fused(target, _params(nu), key, ctr0, _ptr(out), int(out_is_f64), n,
                                  _ptr(moments4), _stream(stream, ref)))
    return out


def qm_sample_moments_noalloc(key: int, ctr0: int, n: int, moments4, stream=None):
    _check(load().qm_sample_moments_noalloc(key, ctr0, n, _ptr(moments4), _stream(stream, moments4)))
    return moments4


def qm_recycle(src: int, dst: int, inp, out, nu=None, n=None, stream=None):
    _check(load().qm_recycle(src, dst, _params(nu), _ptr(inp), _ptr(out), _numel(inp, n),
                             _stream(stream, inp)))
    return out


QM_T_NSEG, QM_T_TAIL_TERMS, QM_T_NU_MIN, QM_T_NU_MAX = 280, 30, 0.75, 100.0


def qm_t_table_build(nu: float):
    """Host-built normal -> Student t tables for nu (no GPU): (seg, tail) with
    seg[j, k] the coefficient of s^k about the centre of segment j and tail =
    (nu, log kappa, degree, R_0..R_degree)."""
    import numpy as np
    seg = np.zeros((QM_T_NSEG, 10), dtype=np.float64)
    tail = np.zeros(3 + QM_T_TAIL_TERMS, dtype=np.float64)
    _check(load().qm_t_table_build(float(nu), seg.ctypes.data, tail.ctypes.data))
    return seg, tail


QM_FX_ROW_BYTES = 64
QM_T_NROW = 1120


def qm_t_rows_build(nu: float):
    """The Student-t rows as the device holds them (no GPU): (A, C), A a
    (QM_T_NROW, 4) uint64 array (a0 bits, B0, B1, B2 | e0 << 52) and C a
    (QM_T_NROW, 4) uint32 array (C3, C4, C5, C6 | (32 - c) << 27); row r
    covers r/128 <= |z| < (r + 1)/128."""
    import numpy as np
    buf = np.zeros(QM_T_NROW * 48, dtype=np.uint8)
    _check(load().qm_t_rows_build(float(nu), buf.ctypes.data))
    a = buf[: QM_T_NROW * 32].view(np.uint64).reshape(QM_T_NROW, 4).copy()
    c = buf[QM_T_NROW * 32:].view(np.uint32).reshape(QM_T_NROW, 4).copy()
    return a, c


QM_TC_Z_MAX, QM_TC_HZ_INV, QM_TC_NZ, QM_TC_ROW = 8.5, 16, 272, 11
QM_TC_G_EMIN, QM_TC_G_K, QM_TC_G_NE_MAX = -5, 5, 128


def qm_tcopula_table_build(nu: float):
    """Host-built t-copula tables (no GPU): (chi, g), rows of QM_TC_ROW --
    chi[j, :10] the coefficients of log W(z) about chi[j, 10]; g[0, :10] those
    of G(t) = Phi^{-1}(F_nu(t)) about 0, g[1 + e 2^K + j, :10] those of G in
    r = m / m_c - 1 on |t| = 2^(QM_TC_G_EMIN + e) m, with 1 / m_c in
    g[., 10]."""
    import numpy as np
    chi = np.zeros((QM_TC_NZ, QM_TC_ROW), dtype=np.float64)
    g = np.zeros((1 + QM_TC_G_NE_MAX * (1 << QM_TC_G_K), QM_TC_ROW), dtype=np.float64)
    ne = ctypes.c_int(0)
    _check(load().qm_tcopula_table_build(float(nu), chi.ctypes.data, g.ctypes.data, ctypes.byref(ne)))
    return chi, g[: 1 + ne.value * (1 << QM_TC_G_K)]


QM_HYP_E_MIN, QM_HYP_MAX_BINADES = -30, 64


def qm_hyp_table_build(alpha: float, beta: float, delta: float):
    """Host-built exponential -> hyperbolic tables (no GPU): (right, left,
    e_max, info) -- right/left[i, k] coefficient k of entry i (entry 0 the
    series about 0, entry 1 + 32 (E - E_MIN) + j the expansion about
    2^E (1 + (2j+1)/64)), e_max the last binade per side, info = (p_+, p_-,
    Q'(0+), Q'(0-), log Z)."""
    import numpy as np
    per = 1 + 32 * QM_HYP_MAX_BINADES
    right = np.zeros((per, 10), dtype=np.float64)
    left = np.zeros((per, 10), dtype=np.float64)
    e_max = np.zeros(2, dtype=np.int32)
    info = np.zeros(5, dtype=np.float64)
    _check(load().qm_hyp_table_build(float(alpha), float(beta), float(delta), right.ctypes.data,
                                     left.ctypes.data, e_max.ctypes.data, info.ctypes.data))
    return right, left, e_max, info


def qm_hyp_rows_build(alpha: float, beta: float, delta: float):
    """The biased fixed-point rows the device evaluates (no GPU): (right,
    left, e_max), each side a (32 QM_HYP_MAX_BINADES, 8) uint64 array, row
    32 (E - QM_HYP_E_MIN) + j for segment j of binade E up to e_max."""
    import numpy as np
    per = 32 * QM_HYP_MAX_BINADES
    right = np.zeros((per, QM_FX_ROW_BYTES // 8), dtype=np.uint64)
    left = np.zeros((per, QM_FX_ROW_BYTES // 8), dtype=np.uint64)
    e_max = np.zeros(2, dtype=np.int32)
    _check(load().qm_hyp_rows_build(float(alpha), float(beta), float(delta), right.ctypes.data,
                                    left.ctypes.data, e_max.ctypes.data))
    return right, left, e_max


class Hyperbolic:
    """Exponential -> hyperbolic recycling map for one parameter set
    (qm_hyp_*): x = Q(v) for two-sided exponential samples v."""

    def __init__(self, alpha: float, beta: float, delta: float):
        h = ctypes.c_void_p()
        _check(load().qm_hyp_create(float(alpha), float(beta), float(delta), ctypes.byref(h)))
        self._h = h

    def recycle(self, v, x, n=None, stream=None):
        _check(load().qm_hyp_recycle(self._h, _ptr(v), _ptr(x), _numel(v, n), _stream(stream, v)))
        return x

    def info(self):
        out = (ctypes.c_double * 5)()
        _check(load().qm_hyp_info(self._h, out))
        return {"p_plus": out[0], "p_minus": out[1], "slope_plus": out[2], "slope_minus": out[3],
                "log_z": out[4]}

    def close(self):
        if self._h:
            load().qm_hyp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


QM_COPULA_MAX_DIM = 16


class qm_margin(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("nu", ctypes.c_double)]


class Copula:
    """Gaussian copula (qm_copula_create) or, with nu, t copula
    (qm_tcopula_create) with recycled marginals: chol is a d x d
    lower-triangular Cholesky factor (host array), margins a list of
    (kind, nu) with kind QM_DIST_NORMAL or QM_DIST_STUDENT_T."""

    def __init__(self, chol, margins, nu=None):
        import numpy as np
        L = np.ascontiguousarray(np.asarray(chol, dtype=np.float64))
        d = L.shape[0]
        arr = (qm_margin * d)(*[qm_margin(int(k), float(m_nu or 0.0)) for k, m_nu in margins])
        h = ctypes.c_void_p()
        if nu is None:
            _check(load().qm_copula_create(d, L.ctypes.data, arr, ctypes.byref(h)))
        else:
            _check(load().qm_tcopula_create(d, float(nu), L.ctypes.data, arr, ctypes.byref(h)))
        self._h, self.d, self.nu = h, d, nu

    def sample(self, key: int, ctr0: int, out, n: int, stream=None):
        _check(load().qm_copula_sample(self._h, key, ctr0, _ptr(out), n, _stream(stream, out)))
        return out

    def close(self):
        if self._h:
            load().qm_copula_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """A ragged batch (qm_batch_*): segments are (src, dst, nu, in, out)
    with torch CUDA tensors of doubles."""

    def __init__(self, segments, tuning=None):
        L = load()
        arr = (qm_segment * len(segments))()
        self._keep = []
        for k, (src, dst, nu, inp, out) in enumerate(segments):
            arr[k] = qm_segment(src, dst, float(nu or 0.0), _ptr(inp), _ptr(out), inp.numel())
            self._keep += [inp, out]
        h = ctypes.c_void_p()
        t = None if tuning is None else ctypes.byref(qm_tuning(*tuning))
        _check(L.qm_batch_create(arr, len(segments), t, ctypes.byref(h)))
        self.h = h

    def run(self, stream=None):
        _check(load().qm_batch_run(self.h, _stream(stream)))

    def run_separate(self, stream=None):
        _check(load().qm_batch_run_separate(self.h, _stream(stream)))

    def tuning(self):
        t = qm_tuning()
        _check(load().qm_batch_get_tuning(self.h, ctypes.byref(t)))
        return (t.block, t.ept, t.estrin)

    def set_tuning(self, tuning):
        _check(load().qm_batch_set_tuning(self.h, ctypes.byref(qm_tuning(*tuning))))

    def tune(self, reps=3, stream=None):
        t = qm_tuning()
        _check(load().qm_batch_tune(self.h, reps, _stream(stream), ctypes.byref(t)))
        return (t.block, t.ept, t.estrin)

    def close(self):
        if self.h:
            load().qm_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """The continuous-batching server (qm_server_*)."""

    def __init__(self, mem_budget, max_batch=256, streams=2, release_on_done=False, device=0):
        cfg = qm_server_config(int(mem_budget), int(max_batch), int(streams), int(release_on_done),
                               int(device))
        h = ctypes.c_void_p()
        _check(load().qm_server_create(ctypes.byref(cfg), ctypes.byref(h)))
        self.h = h

    @staticmethod
    def requests(trace):
        arr = (qm_request * len(trace))()
        for k, r in enumerate(trace):
            arr[k] = qm_request(r.get("id", k), r["n"], r["kind"], float(r.get("nu", 0.0)),
                                r["key"], float(r.get("t_arrival", 0.0)))
        return arr

    def replay(self, trace, timeout_s=120.0):
        arr = self.requests(trace)
        out = (qm_completion * len(trace))()
        _check(load().qm_server_replay(self.h, arr, len(trace), float(timeout_s), out))
        return list(out)

    def submit(self, req):
        _check(load().qm_server_submit(self.h, ctypes.byref(self.requests([req])[0])))

    def poll(self, max_items=1024):
        out = (qm_completion * max_items)()
        got = ctypes.c_int()
        _check(load().qm_server_poll(self.h, out, max_items, ctypes.byref(got)))
        return list(out[: got.value])

    def release(self, rid):
        _check(load().qm_server_release(self.h, rid))

    def stats(self):
        st = qm_server_stats_t()
        _check(load().qm_server_stats(self.h, ctypes.byref(st)))
        return {"launches": st.launches, "arena_used": st.arena_used, "arena_capacity": st.arena_capacity}

    def now(self):
        return load().qm_server_now(self.h)

    def close(self):
        if self.h:
            load().qm_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def qm_last_error() -> str:
    return load().qm_last_error().decode()


def qm_version() -> str:
    return load().qm_version().decode()
