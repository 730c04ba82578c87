"""GPU adjoint (ksdf_query_backward, SDFQuery) against the oracle's FP64 adjoint and finite differences.

Queries are taken off the surface (0.02 m < |sdf| < 1.5 m) and away from winner near-ties and the
medial axis, where the adjoint is well conditioned: the derivative of u = sqrt(-log f'/lambda + d^2)
carries a 1/u factor, so near the surface FP32 rounding of u is amplified without bound.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle  # noqa: E402
from _parity import ADJ_REL, MEDIAL_RATIO, cancellation_ratio  # noqa: E402
from paper_2603_29227_gb300 import ksdf, scenes  # noqa: E402

DEV = torch.device("cuda:0")


@pytest.fixture(scope="module", autouse=True)
def _build():
    import __graft_entry__

    __graft_entry__.build()


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


@pytest.fixture(scope="module")
def setup():
    w = scenes.workload("traj3d", n_samples=20000, n_queries=64 * 8 * 16)
    ref = oracle.Model(w.params, w.x, w.var, w.normals)
    gm = ksdf.KernelSDF(w.params)
    gm.fit(_t(w.x), _t(w.var), _t(w.normals))
    out = gm.query(_t(w.xq), _t(w.sign))
    torch.cuda.synchronize()
    o = {k: v.cpu().numpy() for k, v in out.items()}
    sdf = o["sdf"].astype(np.float64)
    ratio = cancellation_ratio(ref, w.xq, o["winner"])
    keep = (np.abs(sdf) > 0.02) & (np.abs(sdf) < 1.5) & ((o["flags"] & 4) == 0) & (ratio > MEDIAL_RATIO)
    sel = np.nonzero(keep)[0][:3000]
    return w, ref, gm, o, sel


def test_backward_matches_oracle(setup):
    w, ref, gm, o, sel = setup
    rng = np.random.default_rng(3)
    xq = w.xq[sel]
    sg = w.sign[sel]
    win = o["winner"][sel]
    d_sdf = rng.standard_normal(len(sel)).astype(np.float32)
    d_grad = (0.1 * rng.standard_normal((len(sel), 3))).astype(np.float32)
    for with_grad in (False, True):
        dg = d_grad if with_grad else None
        d_xq, d_x = gm.backward(_t(xq), _t(win), _t(d_sdf), None if dg is None else _t(dg), _t(sg))
        torch.cuda.synchronize()
        gm.sync_status()
        rq, rx = ref.backward(xq, d_sdf.astype(np.float64), None if dg is None else dg.astype(np.float64), sign=sg,
                              winner=win)
        gq = d_xq.cpu().numpy().astype(np.float64)
        gx = d_x.cpu().numpy().astype(np.float64)
        eq = np.linalg.norm(gq - rq, axis=1) / np.maximum(np.linalg.norm(rq, axis=1), 1e-12)
        assert eq.max() <= ADJ_REL, (with_grad, eq.max(), sel[np.argmax(eq)])
        ex = np.max(np.abs(gx - rx)) / np.max(np.abs(rx))
        assert ex <= ADJ_REL, (with_grad, ex)


def test_backward_finite_differences(setup):
    """Central differences at h = 1e-4 m of the oracle's FP64 forward (at the FP32 points x +- h) against the
    GPU adjoint d sdf / d xq, for every query whose winner stays the same at both points."""
    w, ref, gm, o, sel = setup
    sel = sel[:400]
    xq = w.xq[sel].astype(np.float32)
    sg = w.sign[sel]
    d_xq, _ = gm.backward(_t(xq), _t(o["winner"][sel]), torch.ones(len(sel), device=DEV), None, _t(sg))
    g = d_xq.cpu().numpy().astype(np.float64)
    h = 1e-4
    fd = np.zeros_like(g)
    for j in range(3):
        e = np.zeros_like(xq)
        e[:, j] = h
        sp = ref.query(xq + e, sg)
        sm = ref.query(xq - e, sg)
        same = (sp["winner"] == o["winner"][sel]) & (sm["winner"] == o["winner"][sel])
        xp = (xq + e).astype(np.float64)[:, j]
        xm = (xq - e).astype(np.float64)[:, j]
        fd[:, j] = (sp["sdf"] - sm["sdf"]) / (xp - xm)
        fd[~same, j] = np.nan
    ok = np.all(np.isfinite(fd), axis=1)
    err = np.linalg.norm(g[ok] - fd[ok], axis=1) / np.linalg.norm(fd[ok], axis=1)
    assert ok.sum() > 300 and err.max() <= ADJ_REL, (ok.sum(), err.max())
    # eikonal: the exact derivative of the SDF has unit norm off the surface (Sec. III)
    assert np.median(np.abs(np.linalg.norm(g, axis=1) - 1.0)) < 0.02


def test_autograd_function(setup):
    w, ref, gm, o, sel = setup
    sel = sel[:1000]
    xq = _t(w.xq[sel]).requires_grad_(True)
    xs = _t(w.x).requires_grad_(True)
    sdf, grad = ksdf.sdf_query(gm, xq, xs, _t(w.sign[sel]))
    wv = torch.linspace(-1, 1, len(sel), device=DEV)
    loss = (wv * sdf).sum() + 0.1 * grad.sum()
    loss.backward()
    d_xq, d_x = gm.backward(xq.detach(), _t(o["winner"][sel]), wv.float().contiguous(),
                            torch.full((len(sel), 3), 0.1, device=DEV), _t(w.sign[sel]))
    assert torch.allclose(xq.grad, d_xq, rtol=1e-5, atol=1e-6)
    assert torch.allclose(xs.grad.float(), d_x, rtol=1e-4, atol=1e-5)
