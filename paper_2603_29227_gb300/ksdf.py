"""Thin Python binding of libksdf.so (C ABI in include/ksdf.h) with the same function names.

Only argument marshalling happens here: every step of the fit, query and adjoint runs in the CUDA
library.  Arrays may be torch tensors (CUDA or CPU) or numpy arrays; the library stages host arrays
itself.  ``KernelSDF`` wraps one context; ``SDFQuery`` is the ``torch.autograd.Function`` for the
differentiation path (gradients with respect to the query points and the sample positions).

If the library has not been built this module raises on first use; it never falls back to CPU code.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libksdf.so")

KSDF_OK, KSDF_ERR_ARG, KSDF_ERR_CUDA, KSDF_ERR_NOT_PD, KSDF_ERR_CAPACITY, KSDF_ERR_NOT_FITTED, \
    KSDF_ERR_NONFINITE, KSDF_ERR_TIMEOUT = range(8)
STATUS_NAMES = {0: "OK", 1: "ERR_ARG", 2: "ERR_CUDA", 3: "ERR_NOT_PD", 4: "ERR_CAPACITY", 5: "ERR_NOT_FITTED",
                6: "ERR_NONFINITE", 7: "ERR_TIMEOUT"}
OUT_SDF, OUT_GRAD, OUT_VAR_SDF, OUT_VAR_F, OUT_WINNER, OUT_FLAGS, OUT_ALL = 1, 2, 4, 8, 16, 32, 63
OUT_VAR_GRAD = 64  # optional: the SDF-gradient variance (Q x dim)
FLAG_FALLBACK, FLAG_NO_GP, FLAG_NEAR_TIE, FLAG_ZERO_GRAD, FLAG_CLAMPED, FLAG_INVALID = 1, 2, 4, 8, 16, 32
CELL_OK, CELL_EMPTY, CELL_NOT_PD = 0, 1, 2
KERNEL_RBF, KERNEL_MATERN32 = 0, 1  # kernel table of Sec. IV-B.2
KERNELS = {"rbf": KERNEL_RBF, "matern32": KERNEL_MATERN32}

# every entry point declared in include/ksdf.h
ABI_FUNCTIONS = ("ksdf_create", "ksdf_destroy", "ksdf_set_stream", "ksdf_reserve", "ksdf_fit", "ksdf_update",
                 "ksdf_update_replace", "ksdf_model_samples", "ksdf_query",
                 "ksdf_query_f64", "ksdf_query_backward", "ksdf_sync_status", "ksdf_last_error", "ksdf_model_size",
                 "ksdf_get_cells", "ksdf_get_fit", "ksdf_bin", "ksdf_candidates", "ksdf_profile", "ksdf_profile_read",
                 "ksdf_fit_gp_noalloc", "ksdf_autotune", "ksdf_autotune_tables", "ksdf_device_math",
                 "ksdf_save", "ksdf_load", "ksdf_wait_diagnostic", "ksdf_set_schedule", "ksdf_get_schedule",
                 "ksdf_autotune_query", "ksdf_autotune_query_configs")


class KsdfError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


class ksdf_params(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("origin", ctypes.c_double * 3), ("cell", ctypes.c_double),
                ("margin", ctypes.c_double), ("n_max", ctypes.c_int), ("k_cand", ctypes.c_int),
                ("lambda_", ctypes.c_double), ("softmin_alpha", ctypes.c_double), ("sign_mode", ctypes.c_int),
                ("kernel", ctypes.c_int)]


_lib = None


def load(path: str = LIB_PATH):
    """Open libksdf.so (raises if it is missing: build it with paper_2603_29227_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libksdf.so is not built (%s); run paper_2603_29227_gb300/build.py" % path)
    lib = ctypes.CDLL(path)
    P, I64, U32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint32
    sig = {
        "ksdf_create": [ctypes.POINTER(ksdf_params), P, ctypes.POINTER(P)],
        "ksdf_destroy": [P],
        "ksdf_set_stream": [P, P],
        "ksdf_reserve": [P, I64, I64],
        "ksdf_fit": [P, P, P, P, I64],
        "ksdf_update": [P, P, P, P, I64, ctypes.POINTER(I64)],
        "ksdf_update_replace": [P, P, P, P, P, I64, ctypes.POINTER(I64)],
        "ksdf_model_samples": [P, ctypes.POINTER(I64)],
        "ksdf_query": [P, P, I64, P, U32, P, P, P, P, P, P, P],
        "ksdf_query_f64": [P, P, I64, P, U32, P, P, P, P, P, P, P],
        "ksdf_query_backward": [P, P, I64, P, P, P, P, P, P],
        "ksdf_sync_status": [P],
        "ksdf_last_error": [P],
        "ksdf_model_size": [P, ctypes.POINTER(I64), ctypes.POINTER(I64)],
        "ksdf_get_cells": [P, P, P, P, P],
        "ksdf_get_fit": [P, P, P, P],
        "ksdf_bin": [P, P, I64, P],
        "ksdf_candidates": [P, P, I64, P, P],
        "ksdf_profile": [P, ctypes.c_int],
        "ksdf_profile_read": [P, ctypes.c_int, P, P, P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(I64)],
        "ksdf_fit_gp_noalloc": [ctypes.POINTER(ksdf_params), P, P, I64, P, P, P, P],
        "ksdf_autotune": [P, ctypes.POINTER(ctypes.c_int), P],
        "ksdf_autotune_tables": [],
        "ksdf_device_math": [P, ctypes.c_int, P, I64, P],
        "ksdf_save": [P, ctypes.c_char_p],
        "ksdf_wait_diagnostic": [P, U32],
        "ksdf_set_schedule": [P, I64, ctypes.c_double],
        "ksdf_autotune_query": [P, P, I64, P, ctypes.POINTER(ctypes.c_int), P],
        "ksdf_autotune_query_configs": [],
        "ksdf_get_schedule": [P, P, P, P],
        "ksdf_load": [P, ctypes.c_char_p],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_char_p if name == "ksdf_last_error" else ctypes.c_int
    _lib = lib
    return lib


def _ptr(a, dtype=None):
    """Raw pointer of a tensor / ndarray (None -> NULL), checking dtype and contiguity."""
    if a is None:
        return None
    if isinstance(a, int):
        return a
    if isinstance(a, np.ndarray):
        if dtype is not None and a.dtype != np.dtype(dtype):
            raise TypeError("expected %s array, got %s" % (np.dtype(dtype), a.dtype))
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    import torch

    if isinstance(a, torch.Tensor):
        if dtype is not None:
            want = {np.float32: torch.float32, np.float64: torch.float64, np.int8: torch.int8,
                    np.int32: torch.int32, np.uint32: torch.uint32 if hasattr(torch, "uint32") else torch.int32,
                    np.uint64: torch.uint64 if hasattr(torch, "uint64") else torch.int64,
                    np.int64: torch.int64}[dtype]
            if a.dtype != want and not (dtype in (np.uint32, np.uint64) and a.dtype in (torch.int32, torch.int64)):
                raise TypeError("expected %s tensor, got %s" % (want, a.dtype))
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    raise TypeError("unsupported array type %r" % type(a))


def _check(h, rc, what):
    if rc != KSDF_OK:
        msg = load().ksdf_last_error(h) if h else b""
        raise KsdfError(rc, "%s: %s" % (what, (msg or b"").decode()))


# ---- the C ABI, one Python function per entry point ----

def make_params(p: dict) -> ksdf_params:
    q = ksdf_params()
    q.dim = int(p["dim"])
    o = list(p.get("origin", (0.0, 0.0, 0.0))) + [0.0, 0.0, 0.0]
    for j in range(3):
        q.origin[j] = float(o[j])
    q.cell = float(p["cell"])
    q.margin = float(p["margin"])
    q.n_max = int(p["n_max"])
    q.k_cand = int(p["k_cand"])
    q.lambda_ = float(p["lambda"])
    q.softmin_alpha = float(p.get("softmin_alpha", 0.0))
    q.sign_mode = int(p.get("sign_mode", 0))
    k = p.get("kernel", KERNEL_RBF)
    q.kernel = KERNELS[k] if isinstance(k, str) else int(k)
    return q


def ksdf_create(params: dict, stream: int | None = None):
    lib = load()
    h = ctypes.c_void_p()
    pr = make_params(params)
    rc = lib.ksdf_create(ctypes.byref(pr), stream, ctypes.byref(h))
    _check(None, rc, "ksdf_create")
    return h


def ksdf_destroy(h):
    _check(None, load().ksdf_destroy(h), "ksdf_destroy")


def ksdf_set_stream(h, stream):
    _check(h, load().ksdf_set_stream(h, stream), "ksdf_set_stream")


def ksdf_reserve(h, max_samples, max_queries):
    _check(h, load().ksdf_reserve(h, int(max_samples), int(max_queries)), "ksdf_reserve")


def ksdf_fit(h, x, var, normals, S, allow_not_pd=True):
    rc = load().ksdf_fit(h, _ptr(x, np.float64), _ptr(var, np.float32), _ptr(normals, np.float32), int(S))
    if rc == KSDF_ERR_NOT_PD and allow_not_pd:
        return rc
    _check(h, rc, "ksdf_fit")
    return rc


def ksdf_autotune(h):
    """Time the fit's candidate size-class tables on the fitted model; returns (chosen index, times in ms)."""
    n = load().ksdf_autotune_tables()
    ms = np.zeros(n)
    t = ctypes.c_int(-1)
    _check(h, load().ksdf_autotune(h, ctypes.byref(t), _ptr(ms)), "ksdf_autotune")
    return int(t.value), ms


def ksdf_autotune_query(h, xq, Q, sign=None):
    """Time the query tile-shape pairs on this batch; returns (chosen index, times in ms)."""
    n = load().ksdf_autotune_query_configs()
    ms = np.zeros(n)
    t = ctypes.c_int(-1)
    _check(h, load().ksdf_autotune_query(h, _ptr(xq, np.float32), int(Q), _ptr(sign, np.int8), ctypes.byref(t),
                                         _ptr(ms)), "ksdf_autotune_query")
    return int(t.value), ms


def ksdf_device_math(h, fn, x):
    """The fit's scalar device routines on float64 inputs x (fn 0: 2^(-x/2^16) from binary64, 1: the same from
    floor(x 2^40) in fixed point, 2: 1/sqrt(x)); returns a float64 array."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.empty_like(x)
    _check(h, load().ksdf_device_math(h, int(fn), _ptr(x), x.size, _ptr(y)), "ksdf_device_math")
    return y


def ksdf_wait_diagnostic(h, spins):
    """Launch the bounded-wait diagnostic (a wait that nothing completes gives up after `spins` polls); the next
    ksdf_sync_status reports KSDF_ERR_TIMEOUT."""
    _check(h, load().ksdf_wait_diagnostic(h, int(spins)), "ksdf_wait_diagnostic")


def ksdf_set_schedule(h, max_refit, eta=1e-3):
    """Refit budget of ksdf_update (cells per update, 0 = all changed cells) and the query-counter weight."""
    _check(h, load().ksdf_set_schedule(h, int(max_refit), float(eta)), "ksdf_set_schedule")


def ksdf_get_schedule(h):
    """(c0, c2, refit) int32 arrays of the model's cells: query counters, training marks, fitted-last flags."""
    G, _ = ksdf_model_size(h)
    out = [np.empty(G, dtype=np.int32) for _ in range(3)]
    _check(h, load().ksdf_get_schedule(h, *[_ptr(a) for a in out]), "ksdf_get_schedule")
    return tuple(out)


def ksdf_save(h, path):
    """Write the model's parameters and samples to `path` (a map file; see include/ksdf.h)."""
    _check(h, load().ksdf_save(h, os.fsencode(path)), "ksdf_save")


def ksdf_load(h, path):
    """Read a map file into the context (same parameters) and fit it; returns the number of samples."""
    rc = load().ksdf_load(h, os.fsencode(path))
    if rc != KSDF_ERR_NOT_PD:
        _check(h, rc, "ksdf_load")
    with open(path, "rb") as f:  # S sits after the magic, four int32 and the 72-byte parameter block
        f.seek(8 + 16 + 72)
        return int(np.frombuffer(f.read(8), dtype=np.int64)[0])


def ksdf_update(h, x_new, var_new, normals_new, S_new, allow_not_pd=True):
    """Append S_new samples and refit the touched cells; returns (status, number of cells refitted)."""
    n = ctypes.c_int64(0)
    rc = load().ksdf_update(h, _ptr(x_new, np.float64), _ptr(var_new, np.float32), _ptr(normals_new, np.float32),
                            int(S_new), ctypes.byref(n))
    if not (rc == KSDF_ERR_NOT_PD and allow_not_pd):
        _check(h, rc, "ksdf_update")
    return rc, int(n.value)


def ksdf_update_replace(h, drop, x_new, var_new, normals_new, S_new, allow_not_pd=True):
    """Remove the samples flagged in drop (S uint8), append S_new samples, refit the changed cells; returns
    (status, number of cells refitted)."""
    n = ctypes.c_int64(0)
    rc = load().ksdf_update_replace(h, _ptr(drop), _ptr(x_new, np.float64), _ptr(var_new, np.float32),
                                    _ptr(normals_new, np.float32), int(S_new), ctypes.byref(n))
    if not (rc == KSDF_ERR_NOT_PD and allow_not_pd):
        _check(h, rc, "ksdf_update_replace")
    return rc, int(n.value)


def ksdf_query(h, xq, Q, sign, out_mask, sdf, grad, var_sdf, var_f, winner, flags, var_grad=None):
    rc = load().ksdf_query(h, _ptr(xq, np.float32), int(Q), _ptr(sign, np.int8), int(out_mask), _ptr(sdf, np.float32),
                           _ptr(grad, np.float32), _ptr(var_sdf, np.float32), _ptr(var_f, np.float32),
                           _ptr(var_grad, np.float32), _ptr(winner, np.int32), _ptr(flags, np.uint32))
    _check(h, rc, "ksdf_query")


def ksdf_query_f64(h, xq, Q, sign, out_mask, sdf, grad, var_sdf, var_f, winner, flags, var_grad=None):
    rc = load().ksdf_query_f64(h, _ptr(xq, np.float64), int(Q), _ptr(sign, np.int8), int(out_mask),
                               _ptr(sdf, np.float64), _ptr(grad, np.float64), _ptr(var_sdf, np.float64),
                               _ptr(var_f, np.float64), _ptr(var_grad, np.float64), _ptr(winner, np.int32),
                               _ptr(flags, np.uint32))
    _check(h, rc, "ksdf_query_f64")


def ksdf_query_backward(h, xq, Q, sign, winner, d_sdf, d_grad, d_xq, d_x):
    rc = load().ksdf_query_backward(h, _ptr(xq, np.float32), int(Q), _ptr(sign, np.int8), _ptr(winner, np.int32),
                                    _ptr(d_sdf, np.float32), _ptr(d_grad, np.float32), _ptr(d_xq, np.float32),
                                    _ptr(d_x, np.float32))
    _check(h, rc, "ksdf_query_backward")


def ksdf_sync_status(h):
    return load().ksdf_sync_status(h)


def ksdf_last_error(h):
    return (load().ksdf_last_error(h) or b"").decode()


def ksdf_model_size(h):
    G, M = ctypes.c_int64(), ctypes.c_int64()
    _check(h, load().ksdf_model_size(h, ctypes.byref(G), ctypes.byref(M)), "ksdf_model_size")
    return G.value, M.value


def ksdf_get_cells(h):
    G, M = ksdf_model_size(h)
    keys = np.empty(G, np.uint64)
    status = np.empty(G, np.int32)
    off = np.empty(G + 1, np.int64)
    mem = np.empty(max(M, 1), np.int64)
    _check(h, load().ksdf_get_cells(h, _ptr(keys), _ptr(status), _ptr(off), _ptr(mem)), "ksdf_get_cells")
    return keys, status, off, mem[:M]


def ksdf_get_fit(h):
    """(alpha float64 [M], chol float64 packed L per cell, linv float32 8-row-blocked L^-1 per cell)"""
    keys, status, off, mem = ksdf_get_cells(h)
    n = np.diff(off)
    alpha = np.empty(max(int(off[-1]), 1), np.float64)
    ntri = int(np.sum(n * (n + 1) // 2))
    nb = (n + 7) // 8
    nlb = int(np.sum(32 * nb * (nb + 1)))
    chol = np.empty(max(ntri, 1), np.float64)
    linv = np.empty(max(nlb, 1), np.float32)
    _check(h, load().ksdf_get_fit(h, _ptr(alpha), _ptr(chol), _ptr(linv)), "ksdf_get_fit")
    return alpha[: int(off[-1])], chol[:ntri], linv[:nlb]


def unpack_linv_blocked(linv_cell, n):
    """Dense n x n L^-1 of one cell from its 8-row-blocked FP32 layout (host helper for tests)."""
    out = np.zeros((n, n), np.float64)
    nb = (n + 7) // 8
    for R in range(nb):
        base = 32 * R * (R + 1)
        cols = 8 * R + 8
        blk = np.asarray(linv_cell[base:base + cols * 8], np.float64).reshape(cols, 8)
        for r in range(8):
            i = 8 * R + r
            if i < n:
                out[i, : min(cols, n)] = blk[: min(cols, n), r]
    return out


def ksdf_bin(h, x, n, keys):
    _check(h, load().ksdf_bin(h, _ptr(x, np.float64), int(n), _ptr(keys, np.uint64)), "ksdf_bin")


def ksdf_candidates(h, keys, n, cand, count):
    _check(h, load().ksdf_candidates(h, _ptr(keys, np.uint64), int(n), _ptr(cand, np.int32), _ptr(count, np.int32)),
           "ksdf_candidates")


def ksdf_profile(h, enable):
    _check(h, load().ksdf_profile(h, int(bool(enable))), "ksdf_profile")


def ksdf_profile_read(h, max_stages=64):
    """{stage: (total_ms, calls)}, launches"""
    names = ctypes.create_string_buffer(32 * max_stages)
    ms = np.zeros(max_stages)
    calls = np.zeros(max_stages, np.int64)
    n = ctypes.c_int()
    launches = ctypes.c_int64()
    _check(h, load().ksdf_profile_read(h, max_stages, ctypes.addressof(names), _ptr(ms), _ptr(calls),
                                       ctypes.byref(n), ctypes.byref(launches)), "ksdf_profile_read")
    raw = names.raw
    out = {}
    for i in range(min(n.value, max_stages)):
        name = raw[32 * i:32 * (i + 1)].split(b"\0", 1)[0].decode()
        out[name] = (float(ms[i]), int(calls[i]))
    return out, launches.value


def ksdf_fit_gp_noalloc(params: dict, x, var, N, alpha, linv, status, stream=None):
    """Fit of one training set with no device allocation (device arrays only); asynchronous on `stream`."""
    pr = make_params(params)
    rc = load().ksdf_fit_gp_noalloc(ctypes.byref(pr), _ptr(x, np.float64), _ptr(var, np.float32), int(N),
                                    _ptr(alpha, np.float64), _ptr(linv, np.float64), _ptr(status, np.int32), stream)
    _check(None, rc, "ksdf_fit_gp_noalloc")


# ---- convenience wrapper over one context (torch tensors) ----

class KernelSDF:
    """One library context bound to the current CUDA device; calls run on torch's current stream."""

    def __init__(self, params: dict):
        import torch

        self.params = dict(params)
        self.dim = int(params["dim"])
        self._torch = torch
        self.h = ksdf_create(self.params, torch.cuda.current_stream().cuda_stream)
        self.S = 0
        self.fit_status = None

    def __del__(self):
        h = getattr(self, "h", None)
        if h is not None and _lib is not None:
            try:
                _lib.ksdf_destroy(h)
            except Exception:
                pass
            self.h = None

    def _stream(self):
        ksdf_set_stream(self.h, self._torch.cuda.current_stream().cuda_stream)

    def reserve(self, max_samples, max_queries):
        ksdf_reserve(self.h, max_samples, max_queries)

    def fit(self, x, var=None, normals=None):
        self._stream()
        self.S = int(x.shape[0])
        self.fit_status = ksdf_fit(self.h, x, var, normals, self.S)
        return self.fit_status

    def save(self, path):
        """Serialise the model (parameters and samples) to `path`."""
        self._stream()
        ksdf_save(self.h, path)

    def load(self, path):
        """Load a map saved with the same parameters and fit it (the model equals the saved one bit for bit)."""
        self._stream()
        self.S = ksdf_load(self.h, path)

    def autotune(self):
        """Pick the fit's team-size table by timing the candidates on this model; returns (index, ms)."""
        self._stream()
        return ksdf_autotune(self.h)

    def autotune_query(self, xq, sign=None):
        """Pick the query's tile shapes by timing the candidates on this batch; returns (index, ms)."""
        self._stream()
        return ksdf_autotune_query(self.h, xq, int(xq.shape[0]), sign)

    def update(self, x_new, var=None, normals=None, S_new=None):
        """Append samples (their ids follow the model's) and refit the cells they touch (within the refit budget
        of ksdf_set_schedule); returns the number of cells refitted.  x_new None with S_new = 0 runs a round over
        the deferred cells."""
        self._stream()
        n_new = int(x_new.shape[0]) if x_new is not None else int(S_new or 0)
        self.fit_status, n = ksdf_update(self.h, x_new, var, normals, n_new)
        self.S += n_new
        return n

    def update_replace(self, drop, x_new, var=None, normals=None):
        """Remove the model's samples flagged in `drop` (S uint8: a tensor or array; the kept samples keep their
        order and are renumbered), append x_new after them, and refit the cells whose training set changed;
        returns the number of cells refitted."""
        self._stream()
        n_new = int(x_new.shape[0]) if x_new is not None else 0
        self.fit_status, n = ksdf_update_replace(self.h, drop, x_new, var, normals, n_new)
        S = ctypes.c_int64(0)
        _check(self.h, load().ksdf_model_samples(self.h, ctypes.byref(S)), "ksdf_model_samples")
        self.S = int(S.value)
        return n

    def query(self, xq, sign=None, mask=OUT_ALL, f64=False):
        torch = self._torch
        self._stream()
        Q = int(xq.shape[0])
        dt = torch.float64 if f64 else torch.float32
        dev = xq.device
        out = {}
        out["sdf"] = torch.empty(Q, dtype=dt, device=dev) if mask & OUT_SDF else None
        out["grad"] = torch.empty((Q, self.dim), dtype=dt, device=dev) if mask & OUT_GRAD else None
        out["var_sdf"] = torch.empty(Q, dtype=dt, device=dev) if mask & OUT_VAR_SDF else None
        out["var_f"] = torch.empty(Q, dtype=dt, device=dev) if mask & OUT_VAR_F else None
        out["winner"] = torch.empty(Q, dtype=torch.int32, device=dev) if mask & OUT_WINNER else None
        out["flags"] = torch.empty(Q, dtype=torch.int32, device=dev) if mask & OUT_FLAGS else None
        vg = torch.empty((Q, self.dim), dtype=dt, device=dev) if mask & OUT_VAR_GRAD else None
        if vg is not None:  # the optional output appears in the dict only when requested
            out["var_grad"] = vg
        fn = ksdf_query_f64 if f64 else ksdf_query
        fn(self.h, xq, Q, sign, mask, out["sdf"], out["grad"], out["var_sdf"], out["var_f"], out["winner"],
           out["flags"], vg)
        return out

    def backward(self, xq, winner, d_sdf, d_grad=None, sign=None, d_x=None):
        torch = self._torch
        self._stream()
        Q = int(xq.shape[0])
        d_xq = torch.empty((Q, self.dim), dtype=torch.float32, device=xq.device)
        if d_x is None:
            d_x = torch.zeros((self.S, self.dim), dtype=torch.float32, device=xq.device)
        ksdf_query_backward(self.h, xq, Q, sign, winner, d_sdf, d_grad, d_xq, d_x)
        return d_xq, d_x

    def sync_status(self):
        rc = ksdf_sync_status(self.h)
        _check(self.h, rc, "device status")

    def cells(self):
        return ksdf_get_cells(self.h)

    def fit_arrays(self):
        return ksdf_get_fit(self.h)


def _make_function():
    import torch

    class SDFQuery(torch.autograd.Function):
        """sdf, grad = SDFQuery.apply(model, xq, x_samples, sign).

        ``x_samples`` must be the (S x dim) tensor the model was fitted on; it is not read in the forward
        pass (the fit holds the model) but receives the sample-position gradient in the backward pass.
        The winner cell of every query is saved for the backward; everything else is recomputed there.
        """

        @staticmethod
        def forward(ctx, model, xq, x_samples, sign):
            out = model.query(xq.detach().contiguous(), sign, OUT_SDF | OUT_GRAD | OUT_WINNER)
            ctx.model = model
            ctx.sign = sign
            ctx.save_for_backward(xq, out["winner"])
            ctx.x_dtype = x_samples.dtype
            return out["sdf"], out["grad"]

        @staticmethod
        def backward(ctx, g_sdf, g_grad):
            xq, winner = ctx.saved_tensors
            model = ctx.model
            if g_sdf is None:
                g_sdf = torch.zeros(xq.shape[0], dtype=torch.float32, device=xq.device)
            d_xq, d_x = model.backward(xq.detach().contiguous(), winner, g_sdf.contiguous().float(),
                                       None if g_grad is None else g_grad.contiguous().float(), ctx.sign)
            return None, d_xq.to(xq.dtype), d_x.to(ctx.x_dtype), None

    return SDFQuery


_fn = None


def sdf_query(model: KernelSDF, xq, x_samples, sign=None):
    """Differentiable SDF + gradient query (see SDFQuery)."""
    global _fn
    if _fn is None:
        _fn = _make_function()
    return _fn.apply(model, xq, x_samples, sign)
