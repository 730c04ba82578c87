"""GPU parity on cells far above the shared-memory limits: the room scene with 1 m cells and a cap of 301
members, so that most training sets have 150-301 members.  This exercises the paths that only large cells
take: the factorisation with its matrix in a per-CTA global slot (N > 218) and an odd largest N (the
kernel-matrix pass sizes its shared memory by it), L^-1 by the two-warp shared-memory kernel (N <= 256) and
by the global-slot kernel (N > 256), and phase B on the SIMT path for N > 256.  Same bars as the other
parity tests: cells bit-exact, FP64 alpha and L within 1e-9, FP32 L^-1 with L^-1 L = I within 1e-4, the
mixed query within its tolerances.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle  # noqa: E402
from _parity import check_mixed  # noqa: E402
from paper_2603_29227_gb300 import ksdf, scenes  # noqa: E402

DEV = torch.device("cuda:0")


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


@pytest.fixture(scope="module")
def case():
    import __graft_entry__

    __graft_entry__.build()
    w = scenes.workload("room3d", n_samples=200_000, n_queries=6007)
    params = dict(w.params, cell=1.0, n_max=301)
    ref = oracle.Model(params, w.x, w.var, w.normals)
    gm = ksdf.KernelSDF(params)
    gm.fit(_t(w.x), _t(w.var), _t(w.normals))
    return w, params, ref, gm


def test_large_cells_present(case):
    w, params, ref, gm = case
    n = np.diff(ref.cells()[2])
    assert np.sum(n > 256) > 50 and np.sum((n > 218) & (n <= 256)) > 20 and n.max() == 301, np.quantile(n, [0.5, 1])


def test_large_cells_bit_exact_and_fit(case):
    w, params, ref, gm = case
    k0, s0, o0, m0 = ref.cells()
    k1, s1, o1, m1 = gm.cells()
    for a, b in ((k0, k1), (s0, s1), (o0, o1), (m0, m1)):
        assert np.array_equal(a, b)
    alpha_gpu, chol, linv = gm.fit_arrays()
    n = np.diff(o0)
    tri_off = np.concatenate([[0], np.cumsum(n * (n + 1) // 2)])
    nb = (n + 7) // 8
    lb_off = np.concatenate([[0], np.cumsum(32 * nb * (nb + 1))])
    rng = np.random.default_rng(3)
    # every size range: small, up to 218 (shared memory), 219-256 (global slot, TC image), above 256
    picks = []
    for lo, hi in ((0, 96), (96, 218), (218, 256), (256, 400)):
        sel = np.nonzero((n > lo) & (n <= hi) & (s0 == oracle.CELL_OK))[0]
        picks += rng.choice(sel, size=min(12, len(sel)), replace=False).tolist()
    worst_a = worst_l = worst_i = 0.0
    for g in picks:
        a = ref.alpha(g)
        worst_a = max(worst_a, float(np.max(np.abs(a - alpha_gpu[o0[g]:o0[g + 1]])) / np.max(np.abs(a))))
        Lr = ref.chol(g)
        Lg = np.zeros_like(Lr)
        Lg[np.tril_indices(n[g])] = chol[tri_off[g]:tri_off[g + 1]]
        worst_l = max(worst_l, float(np.max(np.abs(Lg - Lr)) / np.max(np.abs(Lr))))
        Li = ksdf.unpack_linv_blocked(linv[lb_off[g]:lb_off[g + 1]], int(n[g]))
        worst_i = max(worst_i, float(np.max(np.abs(Li @ Lr - np.eye(n[g])))))
    assert worst_a <= 1e-9, worst_a
    assert worst_l <= 1e-9, worst_l
    assert worst_i <= 1e-4, worst_i


def test_large_cells_query_mixed(case):
    w, params, ref, gm = case
    out = gm.query(_t(w.xq), _t(w.sign))
    torch.cuda.synchronize()
    gm.sync_status()
    res = {k: (v.cpu().numpy() if v is not None else None) for k, v in out.items()}
    res["flags"] = res["flags"].astype(np.uint32)
    check_mixed(ref, w.xq, w.sign, res, "large cells")
