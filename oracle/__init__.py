"""CPU FP64 oracle of the Kernel-SDF back-end query (arXiv 2603.29227).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA library in
``paper_2603_29227_gb300/``; the two meet only through the seeded inputs of
``paper_2603_29227_gb300.scenes``.

The arithmetic lives in ``ksdf_oracle.c`` (plain C, binary64, no fused multiply-add); this module
compiles it with gcc and wraps it with ctypes.  See the C file's header for the paper sections each
step follows and for the readings taken where the paper is silent.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ksdf_oracle.c")
_LIB = os.path.join(_HERE, "libksdf_oracle.so")
_lock = threading.Lock()
_lib = None

FLAG_FALLBACK = 1
FLAG_NO_GP = 2
FLAG_NEAR_TIE = 4
FLAG_ZERO_GRAD = 8
FLAG_CLAMPED = 16
CELL_OK, CELL_EMPTY, CELL_NOT_PD = 0, 1, 2
KERNEL_RBF, KERNEL_MATERN32 = 0, 1
KERNELS = {"rbf": KERNEL_RBF, "matern32": KERNEL_MATERN32}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP, -O2, no FP contraction).  Returns the library path."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "ksdf_oracle.h"))
        ):
            tmp = _LIB + ".tmp%d" % os.getpid()
            cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                   "-shared", "-o", tmp, _SRC, "-lm"]
            subprocess.run(cmd, check=True, cwd=_HERE)
            os.replace(tmp, _LIB)
    return _LIB


class _Params(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("origin", ctypes.c_double * 3), ("cell", ctypes.c_double),
                ("margin", ctypes.c_double), ("n_max", ctypes.c_int), ("k_cand", ctypes.c_int),
                ("lambda_", ctypes.c_double), ("softmin_alpha", ctypes.c_double), ("sign_mode", ctypes.c_int),
                ("kernel", ctypes.c_int)]


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        i64 = ctypes.c_int64
        lib.ko_set_threads.argtypes = [ctypes.c_int]
        lib.ko_get_threads.argtypes = []
        lib.ko_bin.argtypes = [ctypes.POINTER(_Params), P, i64, P]
        lib.ko_fit.argtypes = [ctypes.POINTER(_Params), P, P, P, i64, ctypes.POINTER(ctypes.c_void_p)]
        lib.ko_free.argtypes = [P]
        lib.ko_free.restype = None
        lib.ko_num_cells.argtypes = [P]
        lib.ko_num_cells.restype = i64
        lib.ko_cells.argtypes = [P, P, P, P]
        lib.ko_members.argtypes = [P, P]
        lib.ko_cell_alpha.argtypes = [P, i64, P]
        lib.ko_cell_chol.argtypes = [P, i64, P]
        lib.ko_candidates.argtypes = [P, P, i64, P, P]
        lib.ko_query.argtypes = [P, P, i64, P, P, P, P, P, P, P, P, P]
        lib.ko_query_f64.argtypes = [P, P, i64, P, P, P, P, P, P, P]
        lib.ko_eval_cell.argtypes = [P, P, i64, P, P, P, P, P, P, P]
        lib.ko_var_grad.argtypes = [P, P, i64, P, P]
        lib.ko_backward.argtypes = [P, P, i64, P, P, P, P, P, P]
        lib.ko_backward_f64.argtypes = [P, P, i64, P, P, P, P, P, P]
        _lib = lib
    return _lib


def set_threads(n: int) -> int:
    return _load().ko_set_threads(int(n))


def get_threads() -> int:
    return _load().ko_get_threads()


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def make_params(p: dict) -> _Params:
    q = _Params()
    q.dim = int(p["dim"])
    o = list(p.get("origin", (0.0, 0.0, 0.0))) + [0.0] * 3
    for j in range(3):
        q.origin[j] = float(o[j])
    q.cell = float(p["cell"])
    q.margin = float(p["margin"])
    q.n_max = int(p["n_max"])
    q.k_cand = int(p["k_cand"])
    q.lambda_ = float(p["lambda"])
    q.softmin_alpha = float(p.get("softmin_alpha", 0.0))
    q.sign_mode = int(p.get("sign_mode", 0))
    q.kernel = KERNELS[p.get("kernel", "rbf")] if isinstance(p.get("kernel", 0), str) else int(p.get("kernel", 0))
    return q


def bin_keys(params: dict, x: np.ndarray) -> np.ndarray:
    """Packed cell keys of points x (n x dim, float64)."""
    lib = _load()
    x = np.ascontiguousarray(x, dtype=np.float64)
    keys = np.empty(x.shape[0], dtype=np.uint64)
    pr = make_params(params)
    rc = lib.ko_bin(ctypes.byref(pr), _ptr(x), x.shape[0], _ptr(keys))
    if rc:
        raise ValueError("ko_bin failed (%d)" % rc)
    return keys


def unpack_keys(keys: np.ndarray) -> np.ndarray:
    keys = np.asarray(keys, dtype=np.uint64)
    b = np.int64(1 << 20)
    m = np.uint64(0x1FFFFF)
    cx = (keys & m).astype(np.int64) - b
    cy = ((keys >> np.uint64(21)) & m).astype(np.int64) - b
    cz = ((keys >> np.uint64(42)) & m).astype(np.int64) - b
    return np.stack([cx, cy, cz], axis=1)


class Model:
    """A fitted oracle model (all cells fitted in FP64)."""

    def __init__(self, params: dict, x, var=None, normals=None):
        lib = _load()
        self.params = dict(params)
        self.dim = int(params["dim"])
        self.K = int(params["k_cand"])
        self.x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, self.dim)
        self.S = self.x.shape[0]
        self.var = None if var is None else np.ascontiguousarray(var, dtype=np.float64).reshape(-1)
        self.normals = None if normals is None else np.ascontiguousarray(normals, dtype=np.float64).reshape(-1, self.dim)
        self._p = make_params(params)
        h = ctypes.c_void_p()
        rc = lib.ko_fit(ctypes.byref(self._p), _ptr(self.x), _ptr(self.var), _ptr(self.normals), self.S, ctypes.byref(h))
        if rc:
            raise ValueError("ko_fit failed (%d)" % rc)
        self._h = h
        self.G = lib.ko_num_cells(h)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib is not None:
            _lib.ko_free(h)
            self._h = None

    def cells(self):
        """(keys[G] uint64, status[G] int32, ts_off[G+1] int64, members[ts_off[-1]] int64)"""
        lib = _load()
        keys = np.empty(self.G, dtype=np.uint64)
        status = np.empty(self.G, dtype=np.int32)
        off = np.empty(self.G + 1, dtype=np.int64)
        lib.ko_cells(self._h, _ptr(keys), _ptr(status), _ptr(off))
        mem = np.empty(max(int(off[-1]), 1), dtype=np.int64)
        lib.ko_members(self._h, _ptr(mem))
        return keys, status, off, mem[: int(off[-1])]

    def alpha(self, g: int) -> np.ndarray:
        _, _, off, _ = self.cells()
        a = np.empty(int(off[g + 1] - off[g]), dtype=np.float64)
        rc = _load().ko_cell_alpha(self._h, int(g), _ptr(a))
        if rc:
            raise ValueError("cell %d not fitted" % g)
        return a

    def chol(self, g: int) -> np.ndarray:
        _, _, off, _ = self.cells()
        n = int(off[g + 1] - off[g])
        L = np.empty((n, n), dtype=np.float64)
        rc = _load().ko_cell_chol(self._h, int(g), _ptr(L))
        if rc:
            raise ValueError("cell %d not fitted" % g)
        return L

    def candidates(self, bin_keys_: np.ndarray):
        bk = np.ascontiguousarray(bin_keys_, dtype=np.uint64)
        out = np.empty((bk.shape[0], self.K), dtype=np.int32)
        cnt = np.empty(bk.shape[0], dtype=np.int32)
        rc = _load().ko_candidates(self._h, _ptr(bk), bk.shape[0], _ptr(out), _ptr(cnt))
        if rc:
            raise ValueError("ko_candidates failed (%d)" % rc)
        return out, cnt

    def query(self, xq, sign=None, with_cands=False):
        """Forward query at float32 points; returns a dict of float64/int outputs."""
        xq = np.ascontiguousarray(xq, dtype=np.float32).reshape(-1, self.dim)
        Q = xq.shape[0]
        sg = None if sign is None else np.ascontiguousarray(sign, dtype=np.int8)
        out = dict(sdf=np.empty(Q), grad=np.empty((Q, self.dim)), var_sdf=np.empty(Q), var_f=np.empty(Q),
                   winner=np.empty(Q, dtype=np.int32), flags=np.empty(Q, dtype=np.uint32))
        cu = np.empty((Q, self.K)) if with_cands else None
        ci = np.empty((Q, self.K), dtype=np.int32) if with_cands else None
        rc = _load().ko_query(self._h, _ptr(xq), Q, _ptr(sg), _ptr(out["sdf"]), _ptr(out["grad"]),
                              _ptr(out["var_sdf"]), _ptr(out["var_f"]), _ptr(out["winner"]), _ptr(out["flags"]),
                              _ptr(cu), _ptr(ci))
        if rc:
            raise ValueError("ko_query failed (%d)" % rc)
        if with_cands:
            out["cand_u"] = cu
            out["cand_id"] = ci
        return out

    def query_f64(self, xq, sign=None):
        xq = np.ascontiguousarray(xq, dtype=np.float64).reshape(-1, self.dim)
        Q = xq.shape[0]
        sg = None if sign is None else np.ascontiguousarray(sign, dtype=np.int8)
        out = dict(sdf=np.empty(Q), grad=np.empty((Q, self.dim)), var_sdf=np.empty(Q), var_f=np.empty(Q),
                   winner=np.empty(Q, dtype=np.int32), flags=np.empty(Q, dtype=np.uint32))
        rc = _load().ko_query_f64(self._h, _ptr(xq), Q, _ptr(sg), _ptr(out["sdf"]), _ptr(out["grad"]),
                                  _ptr(out["var_sdf"]), _ptr(out["var_f"]), _ptr(out["winner"]), _ptr(out["flags"]))
        if rc:
            raise ValueError("ko_query_f64 failed (%d)" % rc)
        return out

    def var_grad(self, xq, cell):
        """SDF-gradient variance (Sec. IV-B.3, App. C) of float32 points on the given cells: Q x dim float64."""
        xq = np.ascontiguousarray(xq, dtype=np.float32).reshape(-1, self.dim)
        cell = np.ascontiguousarray(cell, dtype=np.int32)
        out = np.empty((xq.shape[0], self.dim))
        rc = _load().ko_var_grad(self._h, _ptr(xq), xq.shape[0], _ptr(cell), _ptr(out))
        if rc:
            raise ValueError("ko_var_grad failed (%d)" % rc)
        return out

    def eval_cell(self, xq, cell, sign=None):
        """Outputs with cell[q] forced as the winner of query q."""
        xq = np.ascontiguousarray(xq, dtype=np.float32).reshape(-1, self.dim)
        Q = xq.shape[0]
        cell = np.ascontiguousarray(cell, dtype=np.int32)
        sg = None if sign is None else np.ascontiguousarray(sign, dtype=np.int8)
        out = dict(sdf=np.empty(Q), grad=np.empty((Q, self.dim)), var_sdf=np.empty(Q), var_f=np.empty(Q),
                   flags=np.empty(Q, dtype=np.uint32))
        rc = _load().ko_eval_cell(self._h, _ptr(xq), Q, _ptr(cell), _ptr(sg), _ptr(out["sdf"]), _ptr(out["grad"]),
                                  _ptr(out["var_sdf"]), _ptr(out["var_f"]), _ptr(out["flags"]))
        if rc:
            raise ValueError("ko_eval_cell failed (%d)" % rc)
        return out

    def backward(self, xq, d_sdf, d_grad=None, sign=None, winner=None, f64=False):
        """Returns (d_xq [Q x dim], d_x [S x dim])."""
        lib = _load()
        dt = np.float64 if f64 else np.float32
        xq = np.ascontiguousarray(xq, dtype=dt).reshape(-1, self.dim)
        Q = xq.shape[0]
        ds = None if d_sdf is None else np.ascontiguousarray(d_sdf, dtype=np.float64).reshape(-1)
        dg = None if d_grad is None else np.ascontiguousarray(d_grad, dtype=np.float64).reshape(-1, self.dim)
        sg = None if sign is None else np.ascontiguousarray(sign, dtype=np.int8)
        wn = None if winner is None else np.ascontiguousarray(winner, dtype=np.int32)
        dxq = np.zeros((Q, self.dim))
        dx = np.zeros((self.S, self.dim))
        fn = lib.ko_backward_f64 if f64 else lib.ko_backward
        rc = fn(self._h, _ptr(xq), Q, _ptr(sg), _ptr(wn), _ptr(ds), _ptr(dg), _ptr(dxq), _ptr(dx))
        if rc:
            raise ValueError("ko_backward failed (%d)" % rc)
        return dxq, dx
