"""Streaming update (ksdf_update): appending samples and refitting the touched cells gives the model a fresh
fit of all samples would give, bit for bit, and refits exactly the cells whose training set changed."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2603_29227_gb300 import ksdf, scenes  # noqa: E402

DEV = torch.device("cuda:0")


@pytest.fixture(scope="module", autouse=True)
def _build():
    import __graft_entry__

    __graft_entry__.build()


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _state(m, xq):
    keys, status, off, mem = m.cells()
    alpha, chol, linv = m.fit_arrays()
    out = m.query(_t(xq))
    torch.cuda.synchronize()
    q = {k: v.cpu().numpy() for k, v in out.items() if v is not None}
    return dict(keys=keys, status=status, off=off, mem=mem, alpha=alpha, chol=chol, linv=linv, **q)


def _changed_cells(before, after):
    """Cells of `after` whose (key, member list) is not a cell of `before` with an OK fit."""
    old = {}
    for g, k in enumerate(before["keys"]):
        old[int(k)] = (before["status"][g], before["mem"][before["off"][g]:before["off"][g + 1]])
    n = 0
    for g, k in enumerate(after["keys"]):
        mem = after["mem"][after["off"][g]:after["off"][g + 1]]
        o = old.get(int(k))
        if o is None or o[0] != ksdf.CELL_OK or len(mem) == 0 or not np.array_equal(o[1], mem):
            n += 1
    return n


@pytest.mark.parametrize("name", ["room3d", "plane2d"])
def test_update_equals_fresh_fit(name):
    w = scenes.workload(name, n_samples=24000 if name == "room3d" else None, n_queries=20011)
    x, var, nrm = w.x, w.var, w.normals
    # the new samples are those of one region (a frame seeing part of the scene), appended after the rest
    in_b = x[:, 0] < np.quantile(x[:, 0], 0.3)
    order = np.concatenate([np.nonzero(~in_b)[0], np.nonzero(in_b)[0]])
    x, var, nrm = x[order], var[order], nrm[order]
    na = int((~in_b).sum())
    # a second batch inside the first region, to update twice
    nb1 = na + (len(x) - na) // 2

    fresh = ksdf.KernelSDF(w.params)
    fresh.fit(_t(x), _t(var), _t(nrm))
    ref = _state(fresh, w.xq)

    m = ksdf.KernelSDF(w.params)
    m.fit(_t(x[:na]), _t(var[:na]), _t(nrm[:na]))
    s0 = _state(m, w.xq)
    n1 = m.update(_t(x[na:nb1]), _t(var[na:nb1]), _t(nrm[na:nb1]))
    s1 = _state(m, w.xq)
    n2 = m.update(_t(x[nb1:]), _t(var[nb1:]), _t(nrm[nb1:]))
    got = _state(m, w.xq)

    for key in ("keys", "status", "off", "mem", "alpha", "chol", "linv", "sdf", "grad", "var_sdf", "var_f", "winner",
                "flags"):
        assert np.array_equal(ref[key], got[key]), (name, key)
    # exactly the cells whose training set changed were refitted, and the update stayed local
    assert n1 == _changed_cells(s0, s1), name
    assert n2 == _changed_cells(s1, got), name
    assert 0 < n2 < len(got["keys"]), (name, n2, len(got["keys"]))


def test_update_arguments():
    w = scenes.workload("plane2d")
    m = ksdf.KernelSDF(w.params)
    with pytest.raises(ksdf.KsdfError):  # no model yet
        ksdf.ksdf_update(m.h, _t(w.x[:10]), _t(w.var[:10]), _t(w.normals[:10]), 10)
    m.fit(_t(w.x[:500]), _t(w.var[:500]), _t(w.normals[:500]))
    with pytest.raises(ksdf.KsdfError):  # normals required exactly when the model has them
        ksdf.ksdf_update(m.h, _t(w.x[500:510]), _t(w.var[500:510]), None, 10)
    assert m.update(_t(w.x[500:500])) == 0  # an empty batch is a no-op
    n = m.update(_t(w.x[500:600]), _t(w.var[500:600]), _t(w.normals[500:600]))
    assert n > 0


def _remapped(before, keep):
    """`before`'s cells with their members renumbered as ksdf_update_replace numbers the kept samples (a dropped
    member makes the cell unusable for reuse)."""
    newid = np.cumsum(keep) - 1
    out = dict(before)
    mem = before["mem"].copy()
    st = before["status"].copy()
    for g in range(len(before["keys"])):
        m = mem[before["off"][g]:before["off"][g + 1]]
        if np.any(~keep[m]):
            st[g] = ksdf.CELL_EMPTY
        mem[before["off"][g]:before["off"][g + 1]] = np.where(keep[m], newid[m], -1)
    out["mem"], out["status"] = mem, st
    return out


@pytest.mark.parametrize("name", ["room3d", "plane2d"])
def test_update_replace_equals_fresh_fit(name):
    """Dropping samples and appending others (the GP buffer update of Sec. IV-C) gives the model a fresh fit of
    the kept samples followed by the new ones would give, bit for bit, and refits exactly the changed cells."""
    w = scenes.workload(name, n_samples=24000 if name == "room3d" else None, n_queries=20011)
    x, var, nrm = w.x, w.var, w.normals
    rng = np.random.default_rng(11)
    # the model first holds 80% of the samples; a region of it is replaced by the rest (a re-marched region)
    base = np.sort(rng.choice(len(x), size=int(0.8 * len(x)), replace=False))
    rest = np.setdiff1d(np.arange(len(x)), base)
    drop = (x[base, 0] > np.quantile(x[:, 0], 0.6)) & (x[base, 0] < np.quantile(x[:, 0], 0.8))
    keep = ~drop
    xk = np.concatenate([x[base][keep], x[rest]])
    vk = np.concatenate([var[base][keep], var[rest]])
    nk = np.concatenate([nrm[base][keep], nrm[rest]])
    fresh = ksdf.KernelSDF(w.params)
    fresh.fit(_t(xk), _t(vk), _t(nk))
    ref = _state(fresh, w.xq)

    m = ksdf.KernelSDF(w.params)
    m.fit(_t(x[base]), _t(var[base]), _t(nrm[base]))
    s0 = _state(m, w.xq)
    n = m.update_replace(_t(drop.astype(np.uint8)), _t(x[rest]), _t(var[rest]), _t(nrm[rest]))
    got = _state(m, w.xq)
    assert m.S == len(xk)
    for key in ("keys", "status", "off", "mem", "alpha", "chol", "linv", "sdf", "grad", "var_sdf", "var_f", "winner",
                "flags"):
        assert np.array_equal(ref[key], got[key]), (name, key)
    assert n == _changed_cells(_remapped(s0, keep), got), name
    assert 0 < n < len(got["keys"]), name  # some cells kept their fit
    # host drop flags, and a drop of nothing, give the same
    m2 = ksdf.KernelSDF(w.params)
    m2.fit(_t(x[base]), _t(var[base]), _t(nrm[base]))
    m2.update_replace(drop.astype(np.uint8), x[rest], var[rest], nrm[rest])
    assert np.array_equal(_state(m2, w.xq)["chol"], ref["chol"])
    n0 = m2.update_replace(np.zeros(m2.S, dtype=np.uint8), None)
    assert n0 == 0 and np.array_equal(_state(m2, w.xq)["sdf"], ref["sdf"])


def test_update_replace_under_a_budget_refits_cells_that_lost_samples():
    """With a refit budget of one cell, every cell that lost a member is still fitted (it cannot keep a training
    set with a removed sample), and the model stays usable."""
    w = scenes.workload("room3d", n_samples=24000, n_queries=20011)
    m = ksdf.KernelSDF(w.params)
    m.fit(_t(w.x), _t(w.var), _t(w.normals))
    ksdf.ksdf_set_schedule(m.h, 1, 1e-3)
    drop = np.zeros(len(w.x), dtype=np.uint8)
    drop[::97] = 1
    s0 = _state(m, w.xq)
    n = m.update_replace(_t(drop), None)
    got = _state(m, w.xq)
    lost = _remapped(s0, drop == 0)
    # cells that lost a member and still exist (a cell whose own samples were all dropped is gone)
    still = np.isin(s0["keys"], got["keys"])
    n_lost = int(np.sum((lost["status"] != s0["status"]) & still))
    assert n >= n_lost > 0
    gone_lost = int(np.sum((lost["status"] != s0["status"]) & ~still))
    assert len(got["keys"]) + gone_lost >= len(s0["keys"]) - np.sum(~still)
    _, _, refit = ksdf.ksdf_get_schedule(m.h)
    assert int(refit.sum()) == n
    assert np.all(np.isfinite(got["sdf"][got["winner"] >= 0]))
    kept = np.nonzero(drop == 0)[0]
    assert np.all(np.isin(got["mem"], np.arange(len(kept))))
