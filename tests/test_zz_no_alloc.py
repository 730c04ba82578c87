"""The allocation-free fit of one local GP (ksdf_fit_gp_noalloc) against the regular fit.

Callers such as real-time control loops, or programs whose device memory belongs to another allocator,
cannot call cudaMalloc; for them the library offers a context-free fit of one training set whose only
scratch is a static device array.  This test calls it twice in a row through the C ABI (the second call
with a smaller training set, on top of the first call's scratch contents) and checks each result against
the regular ksdf_fit of a one-cell model on the same samples (alpha, and L^-1 against the inverse of the
regular fit's FP64 Cholesky factor), within the FP64 tolerance of the other GPU tests (1e-9 relative).
The file name makes pytest collect it last.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2603_29227_gb300 import ksdf  # noqa: E402

DEV = torch.device("cuda:0")
F64_REL = 1e-9
PARAMS = dict(dim=3, origin=(0.0, 0.0, 0.0), cell=0.5, margin=0.1, n_max=256, k_cand=8, softmin_alpha=300.0,
              sign_mode=0, **{"lambda": 300.0})


@pytest.fixture(scope="module", autouse=True)
def _build():
    import __graft_entry__

    __graft_entry__.build()


def regular_fit(x, var):
    """The existing path: ksdf_fit on a one-cell model (one 64 m cell at the origin holds every sample, in
    id order, with no cap), read back with ksdf_get_fit (alpha and the FP64 Cholesky factor)."""
    p = dict(PARAMS, cell=64.0, margin=0.0, n_max=512, k_cand=1)
    m = ksdf.KernelSDF(p)
    m.fit(torch.from_numpy(x).to(DEV), torch.from_numpy(var).to(DEV), None)
    keys, status, off, mem = m.cells()
    assert len(keys) == 1 and status[0] == ksdf.CELL_OK
    assert np.array_equal(mem, np.arange(len(x)))
    return m.fit_arrays()


def test_noalloc_fit_matches_regular_fit_on_two_calls():
    stream = torch.cuda.current_stream().cuda_stream
    for n, seed in ((300, 1), (120, 2)):
        rng = np.random.default_rng(seed)
        x = rng.uniform(0.2, 0.8, size=(n, 3))
        var = rng.uniform(2.5e-5, 4e-4, size=n).astype(np.float32)
        alpha_ref, chol_ref, _ = regular_fit(x, var)
        L = np.zeros((n, n))
        L[np.tril_indices(n)] = chol_ref
        linv_ref = np.linalg.inv(L)[np.tril_indices(n)]  # L^-1 of the regular fit's FP64 factor
        alpha = torch.empty(n, dtype=torch.float64, device=DEV)
        linv = torch.empty(n * (n + 1) // 2, dtype=torch.float64, device=DEV)
        status = torch.full((1,), -1, dtype=torch.int32, device=DEV)
        ksdf.ksdf_fit_gp_noalloc(PARAMS, torch.from_numpy(x).to(DEV), torch.from_numpy(var).to(DEV), n, alpha,
                                 linv, status, stream)
        torch.cuda.synchronize()
        assert status.item() == ksdf.CELL_OK
        a = alpha.cpu().numpy()
        li = linv.cpu().numpy()
        assert np.max(np.abs(a - alpha_ref)) <= F64_REL * np.max(np.abs(alpha_ref)), n
        assert np.max(np.abs(li - linv_ref)) <= F64_REL * np.max(np.abs(linv_ref)), n


def test_noalloc_rejects_sizes_and_host_arrays():
    x = torch.zeros((600, 3), dtype=torch.float64, device=DEV)
    out = torch.empty(600, dtype=torch.float64, device=DEV)
    linv = torch.empty(600 * 601 // 2, dtype=torch.float64, device=DEV)
    st = torch.empty(1, dtype=torch.int32, device=DEV)
    with pytest.raises(ksdf.KsdfError) as e:
        ksdf.ksdf_fit_gp_noalloc(PARAMS, x, None, 600, out, linv, st)
    assert e.value.status == ksdf.KSDF_ERR_CAPACITY
    with pytest.raises(ksdf.KsdfError) as e:
        ksdf.ksdf_fit_gp_noalloc(PARAMS, np.zeros((10, 3)), None, 10, out, linv, st)
    assert e.value.status == ksdf.KSDF_ERR_ARG
