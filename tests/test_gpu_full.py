"""GPU parity at the full workload sizes, in the launch configuration bench.py times (one fit of all the
samples, one query call over the whole batch), checked on seeded samples of the outputs that the oracle
computes one by one:

  room3d   200,000 samples, 1,000,000 uniform queries (the bench workload): mixed and plain FP64 paths
  traj3d   the room scene, 2,097,152 trajectory queries: forward, and the adjoint of all of them in one call
           (d sdf and d grad cotangents) against the oracle's FP64 adjoint: d xq per query, d x per sample
  scale3d  2,000,000 samples, a 256^3 grid (16,777,216 queries): mixed path
  room3d with the Matern 3/2 kernel (lambda 100): mixed path and the adjoint of all 1M queries
"""
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
SAMPLE = 20000


@pytest.fixture(scope="module", autouse=True)
def _build():
    import __graft_entry__

    __graft_entry__.build()


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _run(w, f64=False):
    m = ksdf.KernelSDF(w.params)
    m.fit(_t(w.x), _t(w.var), _t(w.normals))
    xq = _t(w.xq.astype(np.float64) if f64 else w.xq)
    out = m.query(xq, _t(w.sign), f64=f64)
    torch.cuda.synchronize()
    m.sync_status()
    res = {k: v.cpu().numpy() for k, v in out.items()}
    res["flags"] = res["flags"].astype(np.uint32)
    return m, res


def _sample(n, seed):
    return np.sort(np.random.default_rng(seed).choice(n, size=min(SAMPLE, n), replace=False))


def _sub(res, sel):
    return {k: v[sel] for k, v in res.items()}


def test_room3d_full_mixed_and_fp64():
    w = scenes.workload("room3d")
    ref = oracle.Model(w.params, w.x, w.var, w.normals)
    sel = _sample(len(w.xq), 11)
    m, res = _run(w)
    st = check_mixed(ref, w.xq[sel], w.sign[sel], _sub(res, sel), "room3d full mixed")
    print(st)
    m64, res64 = _run(w, f64=True)
    st = check_f64(ref, w.xq[sel].astype(np.float64), w.sign[sel], _sub(res64, sel), "room3d full fp64")
    print(st)
    # the two GPU paths agree on the winner except at near ties
    diff = res["winner"] != res64["winner"]
    assert np.all((res64["flags"][diff] & ksdf.FLAG_NEAR_TIE) != 0)


def test_traj3d_full_forward_and_adjoint():
    w = scenes.workload("traj3d")
    assert len(w.xq) == 4096 * 64 * 8
    ref = oracle.Model(w.params, w.x, w.var, w.normals)
    sel = _sample(len(w.xq), 12)
    m, res = _run(w)
    st = check_mixed(ref, w.xq[sel], w.sign[sel], _sub(res, sel), "traj3d full mixed")
    print(st)
    # Adjoint over all 2M queries in one call, with the cotangents of the loss sum(softplus(r + 0.1 - sdf))
    # (collision spheres r = 0.15) and a seeded d grad.  Both sides differentiate on the GPU's winner (the
    # oracle is given it), so near ties need no exclusion; queries where the adjoint is ill-conditioned get a
    # zero cotangent on both sides: near the surface (|sdf| <= 0.02 m: d u / d f' carries 1/u), zero gradients
    # and the medial axis (the gradient direction divides by |grad f'|).  Then every query's d xq and the
    # sample gradient d x (summed over all queries) are compared with the oracle's FP64 adjoint.
    Q = len(w.xq)
    gw = res["winner"]
    sdf = res["sdf"].astype(np.float64)
    fin = np.isfinite(sdf) & (gw >= 0)
    zero = (res["flags"] & ksdf.FLAG_ZERO_GRAD) != 0
    ratio = cancellation_ratio(ref, w.xq, np.where(fin, gw, -1))
    kept = fin & (np.abs(sdf) > 0.02) & ~zero & (ratio >= MEDIAL_RATIO)
    assert kept.mean() > 0.8, kept.mean()
    # the gradient output's cotangent also skips queries whose f' <= 0 (u is then the nearest-sample distance
    # and the GP gradient, whose second derivatives this path takes, no longer describes it; there the oracle's
    # own d grad adjoint moves by percents under 1e-7 m shifts of the query) and clamped ones
    kept_g = kept & ((res["flags"] & (ksdf.FLAG_FALLBACK | ksdf.FLAG_CLAMPED)) == 0)
    d_sdf = np.where(kept, -1.0 / (1.0 + np.exp(-(0.15 + 0.1 - sdf))), 0.0).astype(np.float32)
    d_grad = (0.1 * np.random.default_rng(21).standard_normal((Q, 3)) * kept_g[:, None]).astype(np.float32)
    for with_grad in (False, True):
        dg = d_grad if with_grad else None
        kept_w = kept_g if with_grad else kept
        d_xq, d_x = m.backward(_t(w.xq), _t(gw), _t(d_sdf), None if dg is None else _t(dg), _t(w.sign))
        torch.cuda.synchronize()
        m.sync_status()
        gq = d_xq.cpu().numpy().astype(np.float64)
        gx = d_x.cpu().numpy().astype(np.float64)
        assert np.all(np.isfinite(gq)) and np.all(np.isfinite(gx))
        rq, rx = ref.backward(w.xq, d_sdf.astype(np.float64), None if dg is None else dg.astype(np.float64),
                              sign=w.sign, winner=gw)
        nq = np.linalg.norm(rq, axis=1)
        e = np.linalg.norm(gq - rq, axis=1)[kept_w] / np.maximum(nq[kept_w], 1e-12)
        assert e.max() <= ADJ_REL, (with_grad, e.max(), np.nonzero(kept_w)[0][np.argmax(e)])
        assert np.all(gq[~kept] == 0.0)
        ex = np.max(np.abs(gx - rx)) / np.max(np.abs(rx))
        assert ex <= ADJ_REL, (with_grad, ex)
        print("traj3d adjoint (d grad %s): d xq max rel %.3g over %d kept queries, d x %.3g" % (
            with_grad, e.max(), kept_w.sum(), ex))


def test_scale3d_full_mixed():
    w = scenes.workload("scale3d")
    assert len(w.x) == 2_000_000 and len(w.xq) == 256 ** 3
    ref = oracle.Model(w.params, w.x, w.var, w.normals)
    sel = _sample(len(w.xq), 13)
    m, res = _run(w)
    st = check_mixed(ref, w.xq[sel], w.sign[sel], _sub(res, sel), "scale3d full mixed")
    print(st)


def test_room3d_full_matern_mixed_and_adjoint():
    """The Matern 3/2 kernel (kernel table of Sec. IV-B.2, scaling of App. D) at the full room size: every
    size class of the fit, both phase B kernels (cells up to and beyond the tensor-core class split) and both
    adjoint cell launches run; the same bars as the RBF path."""
    w = scenes.workload("room3d")
    w.params = dict(w.params, kernel="matern32", softmin_alpha=100.0, **{"lambda": 100.0})
    ref = oracle.Model(w.params, w.x, w.var, w.normals)
    sel = _sample(len(w.xq), 14)
    m, res = _run(w)
    st = check_mixed(ref, w.xq[sel], w.sign[sel], _sub(res, sel), "room3d full matern mixed")
    print(st)
    # adjoint of every query (d sdf), compared on the sample; the same conditioning exclusions as traj3d
    Q = len(w.xq)
    gw = res["winner"]
    sdf = res["sdf"].astype(np.float64)
    fin = np.isfinite(sdf) & (gw >= 0)
    zero = (res["flags"] & ksdf.FLAG_ZERO_GRAD) != 0
    kept = fin & (np.abs(sdf) > 0.02) & ~zero
    kept[np.setdiff1d(np.arange(Q), sel)] = False  # cotangents only on the sample: the oracle adjoint's cost
    ratio = np.ones(Q)
    ratio[sel] = cancellation_ratio(ref, w.xq[sel], np.where(fin[sel], gw[sel], -1))
    kept &= ratio >= MEDIAL_RATIO
    assert kept.sum() > 0.8 * len(sel), kept.sum()
    d_sdf = np.where(kept, 1.0, 0.0).astype(np.float32)
    d_xq, d_x = m.backward(_t(w.xq), _t(gw), _t(d_sdf), None, _t(w.sign))
    torch.cuda.synchronize()
    m.sync_status()
    gq = d_xq.cpu().numpy().astype(np.float64)
    gx = d_x.cpu().numpy().astype(np.float64)
    assert np.all(np.isfinite(gq)) and np.all(np.isfinite(gx))
    rq, rx = ref.backward(w.xq[sel], d_sdf[sel].astype(np.float64), None, sign=w.sign[sel], winner=gw[sel])
    k = kept[sel]
    nq = np.linalg.norm(rq, axis=1)
    e = np.linalg.norm(gq[sel] - rq, axis=1)[k] / np.maximum(nq[k], 1e-12)
    assert e.max() <= ADJ_REL, (e.max(), sel[k][np.argmax(e)])
    ex = np.max(np.abs(gx - rx)) / np.max(np.abs(rx))
    assert ex <= ADJ_REL, ex
    print("room3d matern adjoint: d xq max rel %.3g over %d kept queries, d x %.3g" % (e.max(), k.sum(), ex))
