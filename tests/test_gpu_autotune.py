"""Autotuning of the fit's size classes: every candidate table gives the same model bit for bit, and the
choice is kept."""
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


def test_autotune_keeps_the_model():
    w = scenes.workload("room3d", n_samples=40000, n_queries=20011)
    m = ksdf.KernelSDF(w.params)
    with pytest.raises(ksdf.KsdfError):  # no model yet
        m.autotune()
    m.fit(_t(w.x), _t(w.var), _t(w.normals))
    before = m.fit_arrays()
    q0 = {k: v.cpu().numpy() for k, v in m.query(_t(w.xq)).items() if v is not None}
    best, ms = m.autotune()
    n = ksdf.load().ksdf_autotune_tables()
    assert 0 <= best < n and len(ms) == n and np.all(ms > 0)
    assert ms[best] == ms.min()
    after = m.fit_arrays()
    for a, b in zip(before, after):
        assert np.array_equal(a, b)
    q1 = {k: v.cpu().numpy() for k, v in m.query(_t(w.xq)).items() if v is not None}
    for k in q0:
        assert np.array_equal(q0[k], q1[k]), k
    # later fits use the chosen table and still give the same model
    m.fit(_t(w.x), _t(w.var), _t(w.normals))
    for a, b in zip(before, m.fit_arrays()):
        assert np.array_equal(a, b)


def test_query_autotune_keeps_the_outputs():
    """The chosen query tile-shape pair gives the same outputs as the default one bit for bit (the per-query
    arithmetic does not depend on the tiling), and the fastest is kept."""
    w = scenes.workload("scale3d", n_samples=200000, grid=48)
    m = ksdf.KernelSDF(w.params)
    m.fit(_t(w.x), _t(w.var), _t(w.normals))
    xq, sg = _t(w.xq), _t(w.sign)
    with pytest.raises(ksdf.KsdfError):
        ksdf.ksdf_autotune_query(m.h, xq, 0)
    q0 = {k: v.cpu().numpy() for k, v in m.query(xq, sg).items() if v is not None}
    best, ms = m.autotune_query(xq, sg)
    n = ksdf.load().ksdf_autotune_query_configs()
    assert 0 <= best < n and len(ms) == n and np.all(ms > 0) and ms[best] == ms.min()
    q1 = {k: v.cpu().numpy() for k, v in m.query(xq, sg).items() if v is not None}
    for k in q0:
        assert np.array_equal(q0[k], q1[k]), k
