"""Failure detection of the bounded device-side waits, without a fault: the diagnostic kernel waits on an
mbarrier that nothing completes, gives up after a short poll limit the way the production kernels' waits do
(status word bit, tensor memory released, kernel returned), and the host reads KSDF_ERR_TIMEOUT from
ksdf_sync_status.  The context then still fits and answers queries."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle  # noqa: E402
from paper_2603_29227_gb300 import ksdf, scenes  # noqa: E402

DEV = torch.device("cuda:0")


@pytest.fixture(scope="module", autouse=True)
def _build():
    import __graft_entry__

    __graft_entry__.build()


def test_wait_that_runs_out_reports_timeout_and_context_survives():
    w = scenes.workload("plane2d", n_samples=400, grid=16)
    m = ksdf.KernelSDF(w.params)
    assert ksdf.ksdf_sync_status(m.h) == ksdf.KSDF_OK
    for spins in (1, 1000):
        ksdf.ksdf_wait_diagnostic(m.h, spins)
        assert ksdf.ksdf_sync_status(m.h) == ksdf.KSDF_ERR_TIMEOUT
        assert ksdf.ksdf_sync_status(m.h) == ksdf.KSDF_OK  # read and cleared
    with pytest.raises(ksdf.KsdfError):
        ksdf.ksdf_wait_diagnostic(m.h, 0)
    # the context (and the GPU) still work: fit, query, compare with the oracle
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(DEV)  # noqa: E731
    m.fit(t(w.x), t(w.var), t(w.normals))
    out = m.query(t(w.xq), t(w.sign))
    torch.cuda.synchronize()
    m.sync_status()
    ref = oracle.Model(w.params, w.x, w.var, w.normals).query(w.xq, w.sign)
    assert np.max(np.abs(out["sdf"].cpu().numpy() - ref["sdf"])) <= 1e-4
