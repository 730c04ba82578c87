"""Model serialisation (ksdf_save / ksdf_load): a model saved and loaded into a fresh context with the same
parameters has the same cells, fit arrays and query outputs bit for bit (the fit is deterministic), with
and without normals, after a streaming update too; wrong parameters, a missing file, a bad header and a
save without a model are rejected."""
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


@pytest.mark.parametrize("name,normals,update", [("room3d", True, False), ("plane2d", False, True)])
def test_round_trip(tmp_path, name, normals, update):
    w = scenes.workload(name, n_samples=20000 if name == "room3d" else None, n_queries=5003)
    m = ksdf.KernelSDF(w.params)
    nrm = _t(w.normals) if normals else None
    if update:
        h = len(w.x) // 2
        m.fit(_t(w.x[:h]), _t(w.var[:h]), None)
        m.update(_t(w.x[h:]), _t(w.var[h:]), None)
    else:
        m.fit(_t(w.x), _t(w.var), nrm)
    ref = _state(m, w.xq)
    path = str(tmp_path / "map.ksdf")
    m.save(path)
    m2 = ksdf.KernelSDF(w.params)
    m2.load(path)
    assert m2.S == len(w.x)
    got = _state(m2, w.xq)
    for k in ref:
        assert np.array_equal(ref[k], got[k]), (name, k)


def test_errors(tmp_path):
    w = scenes.workload("plane2d")
    m = ksdf.KernelSDF(w.params)
    with pytest.raises(ksdf.KsdfError):  # no model yet
        m.save(str(tmp_path / "a.ksdf"))
    m.fit(_t(w.x), _t(w.var), _t(w.normals))
    path = str(tmp_path / "b.ksdf")
    m.save(path)
    other = dict(w.params, cell=0.5)
    with pytest.raises(ksdf.KsdfError):  # different parameters
        ksdf.KernelSDF(other).load(path)
    with pytest.raises(ksdf.KsdfError):  # missing file
        ksdf.KernelSDF(w.params).load(str(tmp_path / "missing.ksdf"))
    bad = tmp_path / "bad.ksdf"
    bad.write_bytes(b"not a map at all, just bytes" * 8)
    with pytest.raises(ksdf.KsdfError):  # bad header
        ksdf.KernelSDF(w.params).load(str(bad))
