"""ctypes binding of ``libgpfagp.so`` (the C ABI declared in ``include/gpfagp.h``).

Argument marshalling only: every step of fit and predict runs in the
library's CUDA kernels. Arrays may be numpy float64 (host pointers; the
library copies) or torch float64 CUDA tensors (device pointers; the call
runs on torch's current stream). Loading fails loudly if the library has
not been built; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import re
from typing import List, Optional, Sequence, Tuple

import numpy as np

from . import build as _build

GP_OK, GP_EINVAL, GP_ENOMEM, GP_ENOTPD, GP_ECUDA, GP_ETIMEOUT, GP_ENODEV = 0, -1, -2, -3, -4, -5, -6
PREC = {"fp64": 0, "mixed": 3}
FIELD = {"L": 1, "c": 2, "b": 3, "d": 4}

HEADER = os.path.join(_build.ROOT, "include", "gpfagp.h")

_lib: Optional[C.CDLL] = None


class GPError(RuntimeError):
    def __init__(self, status: int, detail: int, where: str):
        self.status = status
        self.detail = detail
        super().__init__(f"{where}: {strerror(status)} (status {status}, detail {detail})")


class ServerReport(C.Structure):
    _fields_ = [("predicts_done", C.c_int64), ("refits_done", C.c_int64), ("points", C.c_int64),
                ("p50_ms", C.c_double), ("p99_ms", C.c_double), ("max_ms", C.c_double),
                ("wall_s", C.c_double), ("points_per_s", C.c_double), ("peak_inflight", C.c_int),
                ("peak_batch", C.c_int), ("batches", C.c_int64)]


class FitArgs(C.Structure):
    _fields_ = [("X", C.c_void_p), ("y", C.c_void_p), ("N", C.c_int64), ("p", C.c_int),
                ("n", C.c_int), ("eps", C.c_double), ("alpha", C.c_double), ("sigma2", C.c_double)]


class PredictArgs(C.Structure):
    _fields_ = [("model", C.c_void_p), ("Xs", C.c_void_p), ("Ns", C.c_int64),
                ("mean", C.c_void_p), ("var", C.c_void_p)]


def declared_symbols() -> List[str]:
    """Names of the entry points declared in include/gpfagp.h."""
    txt = open(HEADER).read()
    return re.findall(r"GPFAGP_API\s+[\w\s\*]+?\b(gp_\w+)\s*\(", txt)


def lib(build: bool = True) -> C.CDLL:
    """Load (building first if stale and ``build``) the shared library."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build() if build else _build.LIB
    if not os.path.exists(path):
        raise ImportError(f"libgpfagp.so not found at {path}: build it with "
                          "python -m paper_2403_12797_gb300.build")
    L = C.CDLL(path)
    vp, i64, d, i = C.c_void_p, C.c_int64, C.c_double, C.c_int
    sig = {
        "gp_fit": (vp, [vp, vp, i64, i, i, d, d, d]),
        "gp_predict": (i, [vp, vp, i64, vp, vp]),
        "gp_free": (None, [vp]),
        "gp_last_error": (i, []),
        "gp_last_error_detail": (i64, []),
        "gp_last_error_where": (C.c_char_p, []),
        "gp_strerror": (C.c_char_p, [i]),
        "gp_fit_ex": (i, [vp, vp, i64, i, i, d, d, d, i, vp, i, C.POINTER(vp)]),
        "gp_fit_ard_ex": (i, [vp, vp, i64, i, i, vp, vp, d, i, vp, i, C.POINTER(vp)]),
        "gp_predict_ex": (i, [vp, vp, i64, vp, vp, vp, i]),
        "gp_predict_cov_ex": (i, [vp, vp, i64, vp, vp, i, vp, i]),
        "gp_fit_predict_ex": (i, [vp, vp, i64, i, i, d, d, d, i, vp, i64, vp, vp, vp, i, C.POINTER(vp)]),
        "gp_model_info": (i, [vp, C.POINTER(i64), C.POINTER(i), C.POINTER(i), C.POINTER(i)]),
        "gp_model_read": (i, [vp, i, vp]),
        "gp_model_log_marginal": (i, [vp, vp, i64, C.POINTER(d), vp, i]),
        "gp_model_log_marginal_grad": (i, [vp, vp, i64, C.POINTER(d), C.POINTER(d), vp, i]),
        "gp_gram_ex": (i, [vp, vp, i64, i, i, d, d, i, vp, vp, vp, i]),
        "gp_gram_static": (i, [vp, vp, i64, i, i, d, d, vp, vp, vp]),
        "gp_fit_batch": (i, [i, C.POINTER(FitArgs), i, vp, i, C.POINTER(vp)]),
        "gp_predict_batch": (i, [i, C.POINTER(PredictArgs), vp]),
        "gp_batch_info": (i, [C.POINTER(i), C.POINTER(i)]),
        "gp_batch_plan": (i, [C.POINTER(i), C.POINTER(i), C.POINTER(i), C.POINTER(i), C.POINTER(d)]),
        "gp_fit_gram_ex": (i, [vp, vp, i64, i, i, d, d, d, i, vp, i, C.POINTER(vp)]),
        "gp_gram_packed_ex": (i, [vp, vp, i64, i, i, d, d, i, vp, vp, i]),
        "gp_fit_gram_packed_ex": (i, [vp, i64, i, i, d, d, d, i, vp, i, C.POINTER(vp)]),
        "gp_server_create": (i, [i, i64, C.POINTER(vp)]),
        "gp_server_add_model": (i, [vp, vp, C.POINTER(i)]),
        "gp_server_model": (vp, [vp, i]),
        "gp_server_submit_predict": (i, [vp, i, vp, i64, vp, vp, C.POINTER(i64)]),
        "gp_server_submit_refit": (i, [vp, i, vp, vp, i64, C.POINTER(i64)]),
        "gp_server_wait": (i, [vp, i64, d]),
        "gp_server_stats": (i, [vp, C.POINTER(ServerReport)]),
        "gp_server_destroy": (None, [vp]),
        "gp_server_reset_stats": (i, [vp]),
        "gp_debug_fail_alloc_after": (None, [i]),
        "gp_debug_force_escalation": (None, [i]),
        "gp_debug_barrier_timeout": (None, [d, i]),
        "gp_debug_gram_kernel": (None, [i]),
        "gp_debug_gram_splits": (i, [i, i64, i, C.POINTER(i64)]),
        "gp_debug_column_exponents": (i, [vp, i64, i, i, d, d, vp, vp, vp]),
        "gp_model_flags": (i, [vp]),
        "gp_version": (C.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def strerror(status: int) -> str:
    return lib().gp_strerror(int(status)).decode()


def _check(rc: int, where: str):
    if rc != GP_OK:
        w = lib().gp_last_error_where().decode()
        raise GPError(rc, int(lib().gp_last_error_detail()), where + (f" [{w}]" if w else ""))


# ------------------------------------------------------------------ array marshalling

def _is_torch(a) -> bool:
    return type(a).__module__.startswith("torch")


def _host(a, shape=None) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def _ptr(a) -> int:
    if _is_torch(a):
        return a.data_ptr()
    return a.ctypes.data


def _stream_of(a, stream) -> Optional[int]:
    if stream is not None:
        return int(stream)
    if _is_torch(a):
        import torch
        raw = getattr(torch._C, "_cuda_getCurrentRawStream", None)
        if raw is not None:  # the raw handle, without building a Stream object
            return int(raw(a.device.index if a.device.index is not None else torch.cuda.current_device()))
        return torch.cuda.current_stream(a.device).cuda_stream
    return None


def _prep_xy(X, y):
    """Returns (X, y, N, p, dev) with X (N,p) and y (N,) float64, host or device."""
    if _is_torch(X):
        import torch
        if X.dtype != torch.float64 or not X.is_cuda or not X.is_contiguous():
            raise TypeError("device inputs must be contiguous float64 CUDA tensors")
        if X.dim() == 1:
            X = X.reshape(-1, 1)
        if y is not None and (y.dtype != torch.float64 or not y.is_cuda or not y.is_contiguous()):
            raise TypeError("device inputs must be contiguous float64 CUDA tensors")
        return X, y, int(X.shape[0]), int(X.shape[1]), 1
    X = np.asarray(X, dtype=np.float64)
    if X.ndim == 1:
        X = X.reshape(-1, 1)
    X = np.ascontiguousarray(X)
    yy = None if y is None else _host(y).reshape(-1)
    return X, yy, int(X.shape[0]), int(X.shape[1]), 0


# ------------------------------------------------------------------ public API

class Model:
    """A fitted decomposed-kernel GP (owns a gp_model handle)."""

    def __init__(self, handle: int, shape=None):
        """shape: (M, p, n, prec) when the caller knows them, else read from the model."""
        self._h = C.c_void_p(handle)
        if shape is not None:
            self.M, self.p, self.n, self.prec = (int(v) for v in shape)
            return
        M, p, n, prec = C.c_int64(), C.c_int(), C.c_int(), C.c_int()
        _check(lib().gp_model_info(self._h, C.byref(M), C.byref(p), C.byref(n), C.byref(prec)),
               "gp_model_info")
        self.M, self.p, self.n, self.prec = int(M.value), int(p.value), int(n.value), int(prec.value)

    @property
    def handle(self) -> int:
        return self._h.value or 0

    def predict(self, Xs, var: bool = True, mean_out=None, var_out=None, stream=None):
        """Predictive mean (and variance) at Xs; returns (mean, var or None)."""
        Xs, _, Ns, p, dev = _prep_xy(Xs, None)
        if p != self.p:
            raise ValueError(f"Xs has {p} columns, model has p={self.p}")
        if dev:
            import torch
            mean = mean_out if mean_out is not None else torch.empty(Ns, dtype=torch.float64, device=Xs.device)
            vv = (var_out if var_out is not None else torch.empty(Ns, dtype=torch.float64, device=Xs.device)) if var else None
        else:
            mean = mean_out if mean_out is not None else np.empty(Ns)
            vv = (var_out if var_out is not None else np.empty(Ns)) if var else None
        rc = lib().gp_predict_ex(self._h, C.c_void_p(_ptr(Xs)), Ns, C.c_void_p(_ptr(mean)),
                                 C.c_void_p(_ptr(vv)) if vv is not None else None,
                                 _stream_of(Xs, stream), dev)
        _check(rc, "gp_predict_ex")
        return mean, vv

    def predict_cov(self, Xs, noisy: bool = False, stream=None):
        """Predictive mean and full covariance block (Ns x Ns) at Xs; with
        noisy, sigma^2 is added on the diagonal (covariance of y*)."""
        Xs, _, Ns, p, dev = _prep_xy(Xs, None)
        if p != self.p:
            raise ValueError(f"Xs has {p} columns, model has p={self.p}")
        if dev:
            import torch
            mean = torch.empty(Ns, dtype=torch.float64, device=Xs.device)
            cov = torch.empty((Ns, Ns), dtype=torch.float64, device=Xs.device)
        else:
            mean, cov = np.empty(Ns), np.empty((Ns, Ns))
        rc = lib().gp_predict_cov_ex(self._h, C.c_void_p(_ptr(Xs)), Ns, C.c_void_p(_ptr(mean)),
                                     C.c_void_p(_ptr(cov)), 1 if noisy else 0, _stream_of(Xs, stream), dev)
        _check(rc, "gp_predict_cov_ex")
        return mean, cov

    def log_marginal(self, y, stream=None) -> float:
        """log p(y) of the fitted truncated-kernel GP (y: the training
        targets of the fit, host array or device tensor)."""
        if _is_torch(y):
            import torch
            if y.dtype != torch.float64 or not y.is_cuda or not y.is_contiguous():
                raise TypeError("device inputs must be contiguous float64 CUDA tensors")
            dev = 1
        else:
            y = _host(y).reshape(-1)
            dev = 0
        out = C.c_double()
        _check(lib().gp_model_log_marginal(self._h, C.c_void_p(_ptr(y)), int(y.shape[0]), C.byref(out),
                                           _stream_of(y, stream), dev), "gp_model_log_marginal")
        return float(out.value)

    def log_marginal_grad(self, y, stream=None):
        """(log p(y), d log p(y) / d sigma^2) of the fitted model (y as in log_marginal)."""
        if _is_torch(y):
            import torch
            if y.dtype != torch.float64 or not y.is_cuda or not y.is_contiguous():
                raise TypeError("device inputs must be contiguous float64 CUDA tensors")
            dev = 1
        else:
            y = _host(y).reshape(-1)
            dev = 0
        v, g = C.c_double(), C.c_double()
        _check(lib().gp_model_log_marginal_grad(self._h, C.c_void_p(_ptr(y)), int(y.shape[0]), C.byref(v),
                                                C.byref(g), _stream_of(y, stream), dev),
               "gp_model_log_marginal_grad")
        return float(v.value), float(g.value)

    def read(self, field: str) -> np.ndarray:
        """Host copy of a fitted quantity: 'L' (M x M), 'c', 'b' or 'd' (M)."""
        out = np.empty((self.M, self.M) if field == "L" else self.M)
        _check(lib().gp_model_read(self._h, FIELD[field], out.ctypes.data), "gp_model_read")
        return out

    @property
    def gram_fp64(self) -> bool:
        """True if this mixed-precision fit recomputed its Gram in float64."""
        return bool(lib().gp_model_flags(self._h) & 1)

    def disown(self) -> int:
        """Give up the handle without freeing it (its new owner frees it)."""
        h = self.handle
        self._h = C.c_void_p(0)
        return h

    def free(self):
        if self._h is not None and self._h.value:
            lib().gp_free(self._h)
            self._h = C.c_void_p(0)

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def fit_predict(X, y, n: int, eps: float, alpha: float, sigma2: float, Xs, prec: str = "mixed",
                var: bool = True, mean_out=None, var_out=None, stream=None):
    """fit(X, y, ...) then Model.predict(Xs) in one library call: the
    prediction is enqueued behind the fit with one status read at the end.
    Returns (model, mean, var or None); all arrays host or all device."""
    X, y, N, p, dev = _prep_xy(X, y)
    Xs, _, Ns, ps, devs = _prep_xy(Xs, None)
    if ps != p:
        raise ValueError(f"Xs has {ps} columns, X has {p}")
    if devs != dev:
        raise TypeError("X and Xs must both be host arrays or both device tensors")
    if dev:
        import torch
        mean = mean_out if mean_out is not None else torch.empty(Ns, dtype=torch.float64, device=Xs.device)
        vv = (var_out if var_out is not None else torch.empty(Ns, dtype=torch.float64, device=Xs.device)) if var else None
    else:
        mean = mean_out if mean_out is not None else np.empty(Ns)
        vv = (var_out if var_out is not None else np.empty(Ns)) if var else None
    out = C.c_void_p()
    rc = lib().gp_fit_predict_ex(C.c_void_p(_ptr(X)), C.c_void_p(_ptr(y)), N, p, int(n), float(eps),
                                 float(alpha), float(sigma2), PREC[prec], C.c_void_p(_ptr(Xs)), Ns,
                                 C.c_void_p(_ptr(mean)), C.c_void_p(_ptr(vv)) if vv is not None else None,
                                 _stream_of(X, stream), dev, C.byref(out))
    _check(rc, "gp_fit_predict_ex")
    return Model(out.value, (int(n) ** p, p, int(n), PREC[prec])), mean, vv


def fit(X, y, n: int, eps: float, alpha: float, sigma2: float, prec: str = "mixed",
        stream=None) -> Model:
    """Fit (Sec. 2.2, M x M form) on host numpy arrays or device tensors."""
    X, y, N, p, dev = _prep_xy(X, y)
    out = C.c_void_p()
    rc = lib().gp_fit_ex(C.c_void_p(_ptr(X)), C.c_void_p(_ptr(y)), N, p, int(n), float(eps),
                         float(alpha), float(sigma2), PREC[prec], _stream_of(X, stream), dev,
                         C.byref(out))
    _check(rc, "gp_fit_ex")
    return Model(out.value)


def fit_ard(X, y, n: int, eps, alpha, sigma2: float, prec: str = "mixed", stream=None) -> Model:
    """Fit the ARD kernel (Eq. 17): eps and alpha are sequences of p values, one
    per input dimension (host arrays, copied)."""
    X, y, N, p, dev = _prep_xy(X, y)
    e = np.ascontiguousarray(np.asarray(eps, dtype=np.float64).reshape(-1))
    a = np.ascontiguousarray(np.asarray(alpha, dtype=np.float64).reshape(-1))
    if e.shape != (p,) or a.shape != (p,):
        raise ValueError(f"eps and alpha need {p} values each")
    out = C.c_void_p()
    rc = lib().gp_fit_ard_ex(C.c_void_p(_ptr(X)), C.c_void_p(_ptr(y)), N, p, int(n), e.ctypes.data,
                             a.ctypes.data, float(sigma2), PREC[prec], _stream_of(X, stream), dev, C.byref(out))
    _check(rc, "gp_fit_ard_ex")
    return Model(out.value)


def fit_gram(G, b, N: int, p: int, n: int, eps: float, alpha: float, sigma2: float,
             prec: str = "mixed") -> Model:
    """Fit from a given float64 Gram G = Phi^T Phi (M x M) and b = Phi^T y of N rows (host arrays)."""
    G = np.ascontiguousarray(np.asarray(G, dtype=np.float64))
    b = np.ascontiguousarray(np.asarray(b, dtype=np.float64))
    out = C.c_void_p()
    rc = lib().gp_fit_gram_ex(G.ctypes.data, b.ctypes.data, int(N), int(p), int(n), float(eps), float(alpha),
                              float(sigma2), PREC[prec], None, 0, C.byref(out))
    _check(rc, "gp_fit_gram_ex")
    return Model(out.value)


def packed_size(p: int, n: int) -> int:
    """Length of the packed Gram exchange buffer: M (M + 1) / 2 + M."""
    M = int(n) ** int(p)
    return M * (M + 1) // 2 + M


def gram_packed(X, y, n: int, eps: float, alpha: float, prec: str = "mixed", out=None, stream=None):
    """Lower triangle of G = Phi^T Phi (row by row) then b = Phi^T y, as one
    float64 vector (a device tensor for device inputs, else a host array)."""
    X, y, N, p, dev = _prep_xy(X, y)
    size = packed_size(p, n)
    if out is None:
        if dev:
            import torch
            out = torch.empty(size, dtype=torch.float64, device=X.device)
        else:
            out = np.empty(size)
    rc = lib().gp_gram_packed_ex(C.c_void_p(_ptr(X)), C.c_void_p(_ptr(y)), N, p, int(n), float(eps),
                                 float(alpha), PREC[prec], C.c_void_p(_ptr(out)), _stream_of(X, stream), dev)
    _check(rc, "gp_gram_packed_ex")
    return out


def fit_gram_packed(buf, N: int, p: int, n: int, eps: float, alpha: float, sigma2: float,
                    prec: str = "mixed", stream=None) -> Model:
    """Fit from a packed Gram exchange buffer (gram_packed, summed over the
    row blocks of N training rows); device tensor or host array."""
    if _is_torch(buf):
        import torch
        if buf.dtype != torch.float64 or not buf.is_cuda or not buf.is_contiguous():
            raise TypeError("device inputs must be contiguous float64 CUDA tensors")
        dev = 1
    else:
        buf = np.ascontiguousarray(np.asarray(buf, dtype=np.float64))
        dev = 0
    if buf.shape[0] != packed_size(p, n):
        raise ValueError("packed buffer has the wrong length")
    out = C.c_void_p()
    rc = lib().gp_fit_gram_packed_ex(C.c_void_p(_ptr(buf)), int(N), int(p), int(n), float(eps), float(alpha),
                                     float(sigma2), PREC[prec], _stream_of(buf, stream), dev, C.byref(out))
    _check(rc, "gp_fit_gram_packed_ex")
    return Model(out.value)


def fit_plain(X, y, n, eps, alpha, sigma2) -> Model:
    """The plain ``gp_fit`` entry point (host arrays, mixed precision, default stream)."""
    X, y, N, p, _ = _prep_xy(X, y)
    h = lib().gp_fit(C.c_void_p(_ptr(X)), C.c_void_p(_ptr(y)), N, p, int(n), float(eps),
                     float(alpha), float(sigma2))
    if not h:
        _check(int(lib().gp_last_error()), "gp_fit")
    return Model(h)


def gram(X, y, n: int, eps: float, alpha: float, prec: str = "fp64", stream=None):
    """G = Phi^T Phi (M x M) and b = Phi^T y as float64 (host arrays in, host arrays out)."""
    X, y, N, p, dev = _prep_xy(X, y)
    M = int(n) ** p
    if dev:
        import torch
        G = torch.empty((M, M), dtype=torch.float64, device=X.device)
        b = torch.empty(M, dtype=torch.float64, device=X.device)
    else:
        G = np.empty((M, M))
        b = np.empty(M)
    rc = lib().gp_gram_ex(C.c_void_p(_ptr(X)), C.c_void_p(_ptr(y)), N, p, int(n), float(eps),
                          float(alpha), PREC[prec], C.c_void_p(_ptr(G)), C.c_void_p(_ptr(b)),
                          _stream_of(X, stream), dev)
    _check(rc, "gp_gram_ex")
    return G, b


def fit_batch(problems: Sequence[Tuple], prec: str = "mixed", stream=None) -> List[Model]:
    """Fit many independent problems; each item is (X, y, n, eps, alpha, sigma2)."""
    cnt = len(problems)
    args = (FitArgs * cnt)()
    keep = []
    dev = 0
    for i, (X, y, n, eps, alpha, sigma2) in enumerate(problems):
        X, y, N, p, dev = _prep_xy(X, y)
        keep.append((X, y))
        args[i] = FitArgs(_ptr(X), _ptr(y), N, p, int(n), float(eps), float(alpha), float(sigma2))
    outs = (C.c_void_p * cnt)()
    st = _stream_of(keep[0][0], stream) if cnt else None
    rc = lib().gp_fit_batch(cnt, args, PREC[prec], st, dev, outs)
    models = [Model(o) if o else None for o in outs]
    if rc != GP_OK:
        for m in models:
            if m is not None:
                m.free()
        _check(rc, "gp_fit_batch")
    return models


def batch_plan() -> dict:
    """The plan of this thread's last fit_batch: streams, k, factor_ctas, from_cache, tuned_ms."""
    st, k, fcta, fc, ms = C.c_int(), C.c_int(), C.c_int(), C.c_int(), C.c_double()
    lib().gp_batch_plan(C.byref(st), C.byref(k), C.byref(fcta), C.byref(fc), C.byref(ms))
    return {"streams": st.value, "k": k.value, "factor_ctas": fcta.value, "from_cache": bool(fc.value),
            "tuned_ms": ms.value}


def batch_info() -> Tuple[int, int]:
    """(used_graph, tuned_k) of this thread's last fit_batch."""
    g, k = C.c_int(), C.c_int()
    lib().gp_batch_info(C.byref(g), C.byref(k))
    return g.value, k.value


def predict_batch(reqs: Sequence[Tuple], stream=None):
    """Batched predict on device tensors; each item is (model, Xs, mean_out, var_out or None)."""
    cnt = len(reqs)
    args = (PredictArgs * cnt)()
    for i, (m, Xs, mo, vo) in enumerate(reqs):
        args[i] = PredictArgs(m.handle, _ptr(Xs), int(Xs.shape[0]), _ptr(mo),
                              _ptr(vo) if vo is not None else None)
    st = stream
    if st is None and cnt:
        import torch
        st = torch.cuda.current_stream().cuda_stream
    _check(lib().gp_predict_batch(cnt, args, st), "gp_predict_batch")


def debug_gram_splits(T: int, Npad: int, target_ctas: int):
    """The mixed Gram's row-split plan (host only): ([splits per pair class],
    [rows per split per class], CTAs)."""
    out = (C.c_int64 * 7)()
    _check(lib().gp_debug_gram_splits(int(T), int(Npad), int(target_ctas), out), "gp_debug_gram_splits")
    return list(out[0:3]), list(out[3:6]), int(out[6])


def debug_column_exponents(X, n: int, eps: float, alpha: float):
    """The mixed Gram's column exponents for host rows X (N x p): (E per
    1024-row block [blocks, M], the largest per 4096-row block [blocks4, M],
    the largest overall [M]), int arrays."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    if X.ndim == 1:
        X = X[:, None]
    N, p = X.shape
    M = int(n) ** p
    npad = -(-N // 128) * 128
    ebx = np.empty((-(-npad // 1024), M), dtype=np.int8)
    ebx4 = np.empty((-(-npad // 4096), M), dtype=np.int8)
    ce = np.empty(M, dtype=np.int32)
    _check(lib().gp_debug_column_exponents(X.ctypes.data, N, p, int(n), float(eps), float(alpha),
                                           ebx.ctypes.data, ebx4.ctypes.data, ce.ctypes.data),
           "gp_debug_column_exponents")
    return ebx.astype(np.int64), ebx4.astype(np.int64), ce.astype(np.int64)


def debug_force_escalation(k: int):
    lib().gp_debug_force_escalation(int(k))


def debug_gram_kernel(kind: int):
    """0: automatic, 1: one CTA per 128 x 128 tile pair, 2: CTA pairs where they apply."""
    lib().gp_debug_gram_kernel(int(kind))


def debug_barrier_timeout(limit_s: float, skip_cta: int = -1):
    """Shorten the Cholesky's bounded waits to limit_s (<= 0: the default) and
    make CTA skip_cta of the next Cholesky leave before its first barrier."""
    lib().gp_debug_barrier_timeout(float(limit_s), int(skip_cta))


def debug_fail_alloc_after(k: int):
    lib().gp_debug_fail_alloc_after(int(k))


def version() -> str:
    return lib().gp_version().decode()


# ------------------------------------------------------------------ request server

class Server:
    """Resident models behind a request server (gp_server_* in the C ABI).

    ``add_model`` hands a fitted Model to the server (the Model object is
    emptied); ``submit_predict`` / ``submit_refit`` return a ticket for
    ``wait``. Inputs are host (numpy) arrays kept alive by the ticket.
    """

    def __init__(self, slots: int = 8, mem_budget: int = 0):
        h = C.c_void_p()
        _check(lib().gp_server_create(int(slots), int(mem_budget), C.byref(h)), "gp_server_create")
        self.handle = h.value
        self._p = {}

    def add_model(self, model: "Model") -> int:
        mid = C.c_int()
        _check(lib().gp_server_add_model(self.handle, C.c_void_p(model.handle), C.byref(mid)),
               "gp_server_add_model")
        self._p[mid.value] = model.p
        model.disown()  # the server frees it
        return mid.value

    def submit_predict(self, model_id: int, Xs, var: bool = True):
        Xs = np.ascontiguousarray(np.asarray(Xs, dtype=np.float64))
        if Xs.ndim == 1:
            Xs = Xs[:, None]
        ns = Xs.shape[0]
        mean = np.empty(ns)
        v = np.empty(ns) if var else None
        rid = C.c_int64()
        _check(lib().gp_server_submit_predict(self.handle, int(model_id), Xs.ctypes.data, ns, mean.ctypes.data,
                                              v.ctypes.data if v is not None else None, C.byref(rid)),
               "gp_server_submit_predict")
        return {"id": rid.value, "kind": "predict", "keep": (Xs,), "out": (mean, v)}

    def submit_refit(self, model_id: int, X, y):
        X = np.ascontiguousarray(np.asarray(X, dtype=np.float64))
        if X.ndim == 1:
            X = X[:, None]
        y = np.ascontiguousarray(np.asarray(y, dtype=np.float64))
        rid = C.c_int64()
        _check(lib().gp_server_submit_refit(self.handle, int(model_id), X.ctypes.data, y.ctypes.data,
                                            X.shape[0], C.byref(rid)), "gp_server_submit_refit")
        return {"id": rid.value, "kind": "refit", "keep": (X, y), "out": None}

    def wait(self, ticket, timeout: float = 0.0):
        _check(lib().gp_server_wait(self.handle, ticket["id"], float(timeout)), "gp_server_wait")
        return ticket["out"]

    def stats(self) -> dict:
        r = ServerReport()
        _check(lib().gp_server_stats(self.handle, C.byref(r)), "gp_server_stats")
        return {k: getattr(r, k) for k, _ in ServerReport._fields_}

    def reset_stats(self):
        _check(lib().gp_server_reset_stats(self.handle), "gp_server_reset_stats")

    def model_handle(self, model_id: int):
        return lib().gp_server_model(self.handle, int(model_id))

    def close(self):
        if self.handle:
            lib().gp_server_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
