"""GPU parity of the Matern 3/2 kernel (kernel table of Sec. IV-B.2, scaling of App. D) against the oracle: the FP64
fit, the mixed-precision and the plain FP64 query, and the adjoint.  lambda = 100 (the kernel scale sqrt(3)/lambda
of the paper's kernel ablation defaults), the same tolerances as the RBF path (tests/_parity.py)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle  # noqa: E402
from _parity import ADJ_REL, MEDIAL_RATIO, cancellation_ratio, check_f64, check_mixed  # noqa: E402
from paper_2603_29227_gb300 import ksdf, scenes  # noqa: E402

DEV = torch.device("cuda:0")


@pytest.fixture(scope="module", autouse=True)
def _build():
    import __graft_entry__

    __graft_entry__.build()


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def matern_workload(name, **kw):
    w = scenes.workload(name, **kw)
    w.params = dict(w.params, kernel="matern32", softmin_alpha=100.0, **{"lambda": 100.0})
    return w


WORKLOADS = {"plane2d": dict(name="plane2d"), "room3d_small": dict(name="room3d", n_samples=20000, n_queries=30011)}


@pytest.fixture(scope="module", params=list(WORKLOADS))
def case(request):
    w = matern_workload(**WORKLOADS[request.param])
    ref = oracle.Model(w.params, w.x, w.var, w.normals)
    gm = ksdf.KernelSDF(w.params)
    gm.fit(_t(w.x), _t(w.var), _t(w.normals))
    return request.param, w, ref, gm


def _query(gm, xq, sign, f64=False):
    out = gm.query(_t(xq), _t(sign), f64=f64)
    torch.cuda.synchronize()
    gm.sync_status()
    res = {k: v.cpu().numpy() for k, v in out.items()}
    res["flags"] = res["flags"].astype(np.uint32)
    return res


def test_fit_matches_oracle(case):
    name, w, ref, gm = case
    keys, status, off, mem = ref.cells()
    k1, s1, o1, m1 = gm.cells()
    assert np.array_equal(keys, k1) and np.array_equal(off, o1) and np.array_equal(mem, m1)
    alpha_gpu, chol, _ = gm.fit_arrays()
    n = np.diff(off)
    tri_off = np.concatenate([[0], np.cumsum(n * (n + 1) // 2)])
    for g in np.nonzero(status == oracle.CELL_OK)[0][::7]:
        a_ref = ref.alpha(int(g))
        a = alpha_gpu[off[g]:off[g + 1]]
        assert np.max(np.abs(a - a_ref)) <= 1e-9 * np.max(np.abs(a_ref)), (name, g)
        L_ref = ref.chol(int(g))[np.tril_indices(n[g])]
        L = chol[tri_off[g]:tri_off[g + 1]]
        assert np.max(np.abs(L - L_ref)) <= 1e-9 * np.max(np.abs(L_ref)), (name, g)


def test_mixed_query(case):
    name, w, ref, gm = case
    res = _query(gm, w.xq, w.sign)
    print(name, check_mixed(ref, w.xq, w.sign, res, name + " matern mixed"))


def test_fp64_query(case):
    name, w, ref, gm = case
    xq64 = w.xq.astype(np.float64)
    res = _query(gm, xq64, w.sign, f64=True)
    print(name, check_f64(ref, xq64, w.sign, res, name + " matern fp64"))


def test_adjoint(case):
    name, w, ref, gm = case
    res = _query(gm, w.xq, w.sign)
    sdf = res["sdf"].astype(np.float64)
    gw = res["winner"]
    fin = np.isfinite(sdf) & (gw >= 0)
    ratio = cancellation_ratio(ref, w.xq, np.where(fin, gw, -1))
    kept = fin & (np.abs(sdf) > 0.02) & ((res["flags"] & ksdf.FLAG_ZERO_GRAD) == 0) & (ratio >= MEDIAL_RATIO)
    kept_g = kept & ((res["flags"] & (ksdf.FLAG_FALLBACK | ksdf.FLAG_CLAMPED)) == 0)
    rng = np.random.default_rng(5)
    d_sdf = np.where(kept, rng.standard_normal(len(sdf)), 0.0).astype(np.float32)
    d_grad = (0.1 * rng.standard_normal((len(sdf), w.params["dim"])) * kept_g[:, None]).astype(np.float32)
    for with_grad in (False, True):
        dg = d_grad if with_grad else None
        kw = kept_g if with_grad else kept
        d_xq, d_x = gm.backward(_t(w.xq), _t(gw), _t(d_sdf), None if dg is None else _t(dg), _t(w.sign))
        torch.cuda.synchronize()
        gm.sync_status()
        rq, rx = ref.backward(w.xq, d_sdf.astype(np.float64), None if dg is None else dg.astype(np.float64),
                              sign=w.sign, winner=gw)
        gq = d_xq.cpu().numpy().astype(np.float64)
        gx = d_x.cpu().numpy().astype(np.float64)
        e = np.linalg.norm(gq - rq, axis=1)[kw] / np.maximum(np.linalg.norm(rq, axis=1)[kw], 1e-12)
        assert e.max() <= ADJ_REL, (name, with_grad, e.max())
        ex = np.max(np.abs(gx - rx)) / np.max(np.abs(rx))
        assert ex <= ADJ_REL, (name, with_grad, ex)
        print(name, "matern adjoint (d grad %s): d xq %.3g over %d, d x %.3g" % (with_grad, e.max(), kw.sum(), ex))
