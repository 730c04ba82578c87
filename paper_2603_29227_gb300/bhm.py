"""Thin Python binding of the BHM front-end entry points of libksdf.so (C ABI in include/ksdf_bhm.h), with the
same function names, and ``BHMap``, one map object.

Only argument marshalling happens here: the block hash, the ray samples, the EM rounds, the threshold, the
prediction and the marching all run in the CUDA library.  Raises if the library is missing; there is no CPU path.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import ksdf
from .ksdf import _ptr

BHM_LOGODDS, BHM_SIGN, BHM_GRAD, BHM_PROB = 1, 2, 4, 8

# every entry point declared in include/ksdf_bhm.h
BHM_ABI_FUNCTIONS = ("ksdf_bhm_create", "ksdf_bhm_destroy", "ksdf_bhm_set_stream", "ksdf_bhm_update",
                     "ksdf_bhm_march", "ksdf_bhm_query", "ksdf_bhm_size", "ksdf_bhm_get", "ksdf_bhm_tau",
                     "ksdf_bhm_sync_status", "ksdf_bhm_last_error", "ksdf_bhm_edges_marked")


class ksdf_bhm_params(ctypes.Structure):
    _fields_ = [("origin", ctypes.c_double * 3), ("hinge_spacing", ctypes.c_double), ("block_hinges", ctypes.c_int),
                ("gamma", ctypes.c_double), ("phi_min", ctypes.c_double), ("prior_var", ctypes.c_double),
                ("em_iters", ctypes.c_int), ("xi_init", ctypes.c_double), ("free_step", ctypes.c_double),
                ("free_gap", ctypes.c_double), ("tau_alpha", ctypes.c_double), ("tau_init", ctypes.c_double),
                ("beta", ctypes.c_double), ("march_sub", ctypes.c_int), ("bias_feature", ctypes.c_int)]


DEFAULTS = dict(origin=(0.0, 0.0, 0.0), hinge_spacing=0.175, block_hinges=8, gamma=41.32, phi_min=1e-3,
                prior_var=1.0, em_iters=2, xi_init=0.0, free_step=0.175, free_gap=0.1, tau_alpha=0.1, tau_init=0.0,
                beta=1.0, march_sub=2, bias_feature=1)

_sigs_done = False


def load():
    global _sigs_done
    lib = ksdf.load()
    if not _sigs_done:
        P, I64, U32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint32
        sig = {
            "ksdf_bhm_create": [ctypes.POINTER(ksdf_bhm_params), I64, I64, P, ctypes.POINTER(P)],
            "ksdf_bhm_destroy": [P],
            "ksdf_bhm_set_stream": [P, P],
            "ksdf_bhm_update": [P, P, P, I64],
            "ksdf_bhm_march": [P, I64, P, P, P, P, ctypes.POINTER(I64)],
            "ksdf_bhm_query": [P, P, I64, U32, P, P, P, P],
            "ksdf_bhm_size": [P, ctypes.POINTER(I64), ctypes.POINTER(I64), ctypes.POINTER(I64)],
            "ksdf_bhm_get": [P, P, P, P, P],
            "ksdf_bhm_tau": [P, ctypes.POINTER(ctypes.c_double)],
            "ksdf_bhm_sync_status": [P],
            "ksdf_bhm_edges_marked": [P, P, I64, P],
            "ksdf_bhm_last_error": [P],
        }
        for name, args in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = ctypes.c_char_p if name == "ksdf_bhm_last_error" else ctypes.c_int
        _sigs_done = True
    return lib


def _check(h, rc, what):
    if rc != ksdf.KSDF_OK:
        msg = load().ksdf_bhm_last_error(h) if h else b""
        raise ksdf.KsdfError(rc, "%s: %s" % (what, (msg or b"").decode()))


def make_params(p: dict) -> ksdf_bhm_params:
    p = dict(DEFAULTS, **p)
    q = ksdf_bhm_params()
    for j in range(3):
        q.origin[j] = float(p["origin"][j])
    for k in ("hinge_spacing", "gamma", "phi_min", "prior_var", "xi_init", "free_step", "free_gap", "tau_alpha",
              "tau_init", "beta"):
        setattr(q, k, float(p[k]))
    for k in ("block_hinges", "em_iters", "march_sub", "bias_feature"):
        setattr(q, k, int(p[k]))
    return q


def ksdf_bhm_create(params: dict, max_blocks: int, max_marked: int = 0, stream=None):
    h = ctypes.c_void_p()
    pr = make_params(params)
    rc = load().ksdf_bhm_create(ctypes.byref(pr), int(max_blocks), int(max_marked), stream, ctypes.byref(h))
    _check(None, rc, "ksdf_bhm_create")
    return h


def ksdf_bhm_destroy(h):
    _check(None, load().ksdf_bhm_destroy(h), "ksdf_bhm_destroy")


def ksdf_bhm_set_stream(h, stream):
    _check(h, load().ksdf_bhm_set_stream(h, stream), "ksdf_bhm_set_stream")


def ksdf_bhm_update(h, p, hits, R):
    pa = (ctypes.c_double * 3)(*[float(v) for v in p])
    _check(h, load().ksdf_bhm_update(h, ctypes.cast(pa, ctypes.c_void_p), _ptr(hits, np.float64), int(R)),
           "ksdf_bhm_update")


def ksdf_bhm_march(h, cap, x=None, var=None, normals=None, keys=None):
    n = ctypes.c_int64(0)
    rc = load().ksdf_bhm_march(h, int(cap), _ptr(x, np.float64), _ptr(var, np.float32), _ptr(normals, np.float32),
                               _ptr(keys, np.uint64), ctypes.byref(n))
    if rc == ksdf.KSDF_ERR_CAPACITY:
        return int(n.value), rc
    _check(h, rc, "ksdf_bhm_march")
    return int(n.value), rc


def ksdf_bhm_query(h, xq, Q, out_mask, logodds=None, sign=None, grad=None, prob=None):
    _check(h, load().ksdf_bhm_query(h, _ptr(xq, np.float32), int(Q), int(out_mask), _ptr(logodds, np.float32),
                                    _ptr(sign, np.int8), _ptr(grad, np.float32), _ptr(prob, np.float32)),
           "ksdf_bhm_query")


def ksdf_bhm_edges_marked(h, keys, n, out):
    _check(h, load().ksdf_bhm_edges_marked(h, _ptr(keys, np.uint64), int(n), _ptr(out)), "ksdf_bhm_edges_marked")


def ksdf_bhm_size(h):
    nb, ns, nf = ctypes.c_int64(0), ctypes.c_int64(0), ctypes.c_int64(0)
    _check(h, load().ksdf_bhm_size(h, ctypes.byref(nb), ctypes.byref(ns), ctypes.byref(nf)), "ksdf_bhm_size")
    return int(nb.value), int(ns.value), int(nf.value)


def ksdf_bhm_get(h, nw):
    nb, _, _ = ksdf_bhm_size(h)
    keys = np.empty(nb, dtype=np.uint64)
    act = np.empty(nb, dtype=np.uint8)
    mu = np.empty((nb, nw), dtype=np.float32)
    prec = np.empty((nb, nw), dtype=np.float32)
    _check(h, load().ksdf_bhm_get(h, _ptr(keys), _ptr(act), _ptr(mu), _ptr(prec)), "ksdf_bhm_get")
    return keys, act, mu, prec


def ksdf_bhm_tau(h):
    t = ctypes.c_double(0.0)
    _check(h, load().ksdf_bhm_tau(h, ctypes.byref(t)), "ksdf_bhm_tau")
    return float(t.value)


def ksdf_bhm_sync_status(h):
    return load().ksdf_bhm_sync_status(h)


class BHMap:
    """One BHM front-end map on the current CUDA device (its calls run on the map's stream)."""

    def __init__(self, params: dict, max_blocks: int, max_marked: int = 0, stream=None):
        self.params = dict(DEFAULTS, **params)
        self.nw = int(self.params["block_hinges"]) ** 3 + 1
        self.h = ksdf_bhm_create(self.params, max_blocks, max_marked, stream)

    def close(self):
        if self.h is not None and self.h.value:
            ksdf_bhm_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def update(self, p, hits):
        """One scan: sensor position p (3 floats) and hits (R x 3 float64, torch tensor or numpy array)."""
        ksdf_bhm_update(self.h, p, hits, int(hits.shape[0]))

    def march(self, device=None):
        """Surface points of the last update: (x R x 3 float64, var R float32, normals R x 3 float32, keys R int64
        holding the uint64 edge keys), torch tensors on `device` (a CUDA device) or numpy arrays when device is
        None."""
        cap = getattr(self, "_cap", 1 << 16)
        for _ in range(3):
            if device is None:
                x, v, nr, k = (np.empty((cap, 3)), np.empty(cap, dtype=np.float32),
                               np.empty((cap, 3), dtype=np.float32), np.empty(cap, dtype=np.uint64))
            else:
                import torch

                x = torch.empty((cap, 3), dtype=torch.float64, device=device)
                v = torch.empty(cap, dtype=torch.float32, device=device)
                nr = torch.empty((cap, 3), dtype=torch.float32, device=device)
                k = torch.empty(cap, dtype=torch.int64, device=device)
            n, rc = ksdf_bhm_march(self.h, cap, x, v, nr, k)
            if rc == ksdf.KSDF_OK:
                return x[:n], v[:n], nr[:n], k[:n]
            cap = max(cap, n + n // 4 + 1)
            self._cap = cap
        raise ksdf.KsdfError(ksdf.KSDF_ERR_CAPACITY, "ksdf_bhm_march: point count keeps growing")

    def query(self, xq, out_mask=BHM_LOGODDS | BHM_SIGN | BHM_GRAD | BHM_PROB):
        """Log-odds, sign, gradient, occupancy probability at xq (Q x 3 float32): a dict of torch tensors on xq's
        device (or numpy arrays for a numpy xq)."""
        Q = int(xq.shape[0])
        if isinstance(xq, np.ndarray):
            out = {"logodds": np.empty(Q, dtype=np.float32), "sign": np.empty(Q, dtype=np.int8),
                   "grad": np.empty((Q, 3), dtype=np.float32), "prob": np.empty(Q, dtype=np.float32)}
        else:
            import torch

            out = {"logodds": torch.empty(Q, dtype=torch.float32, device=xq.device),
                   "sign": torch.empty(Q, dtype=torch.int8, device=xq.device),
                   "grad": torch.empty((Q, 3), dtype=torch.float32, device=xq.device),
                   "prob": torch.empty(Q, dtype=torch.float32, device=xq.device)}
        ksdf_bhm_query(self.h, xq, Q, out_mask, out["logodds"] if out_mask & BHM_LOGODDS else None,
                       out["sign"] if out_mask & BHM_SIGN else None, out["grad"] if out_mask & BHM_GRAD else None,
                       out["prob"] if out_mask & BHM_PROB else None)
        return out

    def edges_marked(self, keys):
        """uint8 flags: 1 for each edge key (as march returns them) processed by the last update's marks."""
        n = int(keys.shape[0])
        if isinstance(keys, np.ndarray):
            out = np.empty(n, dtype=np.uint8)
        else:
            import torch

            out = torch.empty(n, dtype=torch.uint8, device=keys.device)
        ksdf_bhm_edges_marked(self.h, keys, n, out)
        return out

    def size(self, features=False):
        """(allocated blocks, samples of the last update[, hinge features of the last update's samples])."""
        nb, ns, nf = ksdf_bhm_size(self.h)
        return (nb, ns, nf) if features else (nb, ns)

    def weights(self):
        """(keys, active, mu, prec) of the allocated blocks, numpy, slot order."""
        return ksdf_bhm_get(self.h, self.nw)

    @property
    def tau(self):
        return ksdf_bhm_tau(self.h)

    def sync_status(self):
        rc = ksdf_bhm_sync_status(self.h)
        _check(self.h, rc, "ksdf_bhm_sync_status")
