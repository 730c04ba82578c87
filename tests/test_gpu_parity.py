"""GPU parity: the CUDA path through the C ABI against the CPU FP64 oracle on the same seeded inputs.

Integer work (binning, cells, training sets, candidate lists) is compared bit for bit; floating point
within the tolerances stated in tests/_parity.py.  Sizes span several tiles and ragged tails.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle  # noqa: E402
from _parity import check_f64, check_mixed  # noqa: E402
from paper_2603_29227_gb300 import ksdf, scenes  # noqa: E402

DEV = torch.device("cuda:0")


@pytest.fixture(scope="module", autouse=True)
def _build():
    import __graft_entry__

    __graft_entry__.build()


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def gpu_model(w):
    m = ksdf.KernelSDF(w.params)
    m.fit(_t(w.x), _t(w.var), _t(w.normals))
    return m


def gpu_query(m, xq, sign, f64=False):
    out = m.query(_t(xq), None if sign is None else _t(sign), f64=f64)
    torch.cuda.synchronize()
    m.sync_status()
    res = {k: (v.cpu().numpy() if v is not None else None) for k, v in out.items()}
    res["flags"] = res["flags"].astype(np.uint32)
    return res


WORKLOADS = {
    "plane2d": dict(name="plane2d"),
    "room3d_small": dict(name="room3d", n_samples=20000, n_queries=30011),
    # a cell edge that is not a power of two and an origin off the grid: binning by division (a power-of-two
    # edge bins by the equivalent exact multiplication)
    "room3d_cell03": dict(name="room3d", n_samples=20000, n_queries=20011,
                          params=dict(cell=0.3, origin=(-0.1, 0.05, -0.02))),
}


@pytest.fixture(scope="module", params=list(WORKLOADS))
def case(request):
    spec = dict(WORKLOADS[request.param])
    over = spec.pop("params", None)
    w = scenes.workload(**spec)
    if over:
        w.params = dict(w.params, **over)
    ref = oracle.Model(w.params, w.x, w.var, w.normals)
    gm = gpu_model(w)
    return request.param, w, ref, gm


def test_cells_and_training_sets_bit_exact(case):
    name, w, ref, gm = case
    k0, s0, o0, m0 = ref.cells()
    k1, s1, o1, m1 = gm.cells()
    assert np.array_equal(k0, k1), name
    assert np.array_equal(s0, s1), name
    assert np.array_equal(o0, o1), name
    assert np.array_equal(m0, m1), name


def test_fit_alpha_chol_linv(case):
    """FP64 alpha and Cholesky factor against the oracle (1e-9); FP32 L^-1 is the inverse of L to FP32 level."""
    name, w, ref, gm = case
    keys, status, off, mem = ref.cells()
    alpha_gpu, chol, linv = gm.fit_arrays()
    n = np.diff(off)
    tri_off = np.concatenate([[0], np.cumsum(n * (n + 1) // 2)])
    nb = (n + 7) // 8
    lb_off = np.concatenate([[0], np.cumsum(32 * nb * (nb + 1))])
    worst_a = worst_l = worst_i = 0.0
    rng = np.random.default_rng(0)
    check_inv = set(rng.choice(len(keys), size=min(60, len(keys)), replace=False).tolist()) | {int(np.argmax(n))}
    for g in range(len(keys)):
        if status[g] != oracle.CELL_OK:
            continue
        a = ref.alpha(g)
        worst_a = max(worst_a, float(np.max(np.abs(a - alpha_gpu[off[g]:off[g + 1]])) / np.max(np.abs(a))))
        Lr = ref.chol(g)
        Lg = np.zeros_like(Lr)
        Lg[np.tril_indices(n[g])] = chol[tri_off[g]:tri_off[g + 1]]
        worst_l = max(worst_l, float(np.max(np.abs(Lg - Lr)) / np.max(np.abs(Lr))))
        if g in check_inv:
            Li = ksdf.unpack_linv_blocked(linv[lb_off[g]:lb_off[g + 1]], int(n[g]))
            worst_i = max(worst_i, float(np.max(np.abs(Li @ Lr - np.eye(n[g])))))
    assert worst_a <= 1e-9, (name, worst_a)
    assert worst_l <= 1e-9, (name, worst_l)
    assert worst_i <= 1e-4, (name, worst_i)


def test_candidate_lists_bit_exact(case):
    name, w, ref, gm = case
    bins = np.unique(oracle.bin_keys(w.params, w.xq.astype(np.float64)))
    c0, n0 = ref.candidates(bins)
    K = w.params["k_cand"]
    c1 = np.empty((len(bins), K), np.int32)
    n1 = np.empty(len(bins), np.int32)
    ksdf.ksdf_candidates(gm.h, bins, len(bins), c1, n1)
    assert np.array_equal(n0, n1), name
    assert np.array_equal(c0, c1), name
    # GPU binning of the same points is bit-exact too
    keys = np.empty(len(w.xq), np.uint64)
    ksdf.ksdf_bin(gm.h, w.xq.astype(np.float64), len(w.xq), keys)
    assert np.array_equal(keys, oracle.bin_keys(w.params, w.xq.astype(np.float64)))


def test_candidate_lists_far_bins(case):
    """Bins far from every cell: beyond the search's cell shells (its brick level), and far outside the
    cells' box (its pass over all cells); bit-exact against the oracle's exhaustive search."""
    name, w, ref, gm = case
    p = w.params
    dim, h = p["dim"], p["cell"]
    lo, hi = w.x.min(0), w.x.max(0)
    ext = hi - lo
    rng = np.random.default_rng(7)
    xq = np.concatenate([rng.uniform(lo - 0.5 * ext - 12 * h, hi + 0.5 * ext + 12 * h, size=(4000, dim)),
                         rng.uniform(lo - 300 * h, hi + 300 * h, size=(500, dim))])
    bins = np.unique(oracle.bin_keys(p, xq))
    c0, n0 = ref.candidates(bins)
    K = p["k_cand"]
    c1 = np.empty((len(bins), K), np.int32)
    n1 = np.empty(len(bins), np.int32)
    ksdf.ksdf_candidates(gm.h, bins, len(bins), c1, n1)
    assert np.array_equal(n0, n1), name
    assert np.array_equal(c0, c1), name


def test_query_mixed(case):
    name, w, ref, gm = case
    out = gpu_query(gm, w.xq, w.sign)
    st = check_mixed(ref, w.xq, w.sign, out, name)
    print(name, st)


def test_query_fp64(case):
    name, w, ref, gm = case
    xq64 = w.xq.astype(np.float64)
    out = gpu_query(gm, xq64, w.sign, f64=True)
    st = check_f64(ref, xq64, w.sign, out, name)
    print(name, st)


def test_sign_stand_in_matches_oracle():
    w = scenes.workload("plane2d", n_samples=800, grid=40)
    p = dict(w.params, sign_mode=1)
    ref = oracle.Model(p, w.x, w.var, w.normals)
    m = ksdf.KernelSDF(p)
    m.fit(_t(w.x), _t(w.var), _t(w.normals))
    out = gpu_query(m, w.xq, None)
    r = ref.query(w.xq, None)
    clear = (r["flags"] & 4) == 0
    assert np.mean(np.sign(out["sdf"][clear]) == np.sign(r["sdf"][clear])) > 0.999


def test_host_buffers_match_device(case):
    name, w, ref, gm = case
    xq = w.xq[:5000]
    Q = len(xq)
    dim = w.params["dim"]
    outs = [np.empty(Q, np.float32), np.empty((Q, dim), np.float32), np.empty(Q, np.float32),
            np.empty(Q, np.float32), np.empty(Q, np.int32), np.empty(Q, np.uint32)]
    ksdf.ksdf_query(gm.h, xq, Q, w.sign[:5000], ksdf.OUT_ALL, *outs)
    dev = gpu_query(gm, xq, w.sign[:5000])
    assert np.array_equal(outs[0], dev["sdf"]) and np.array_equal(outs[1], dev["grad"])
    assert np.array_equal(outs[3], dev["var_f"]) and np.array_equal(outs[4], dev["winner"])


def test_edge_cases():
    w = scenes.workload("plane2d", n_samples=300, grid=8)
    m = ksdf.KernelSDF(w.params)
    m.fit(_t(w.x), _t(w.var), _t(w.normals))
    ref = oracle.Model(w.params, w.x, w.var, w.normals)
    # empty query batch
    out = m.query(torch.empty((0, 2), dtype=torch.float32, device=DEV))
    assert out["sdf"].numel() == 0
    # far-away queries take the brute-force candidate path (beyond 16 rings)
    far = np.array([[40.0, -30.0], [-25.0, 5.0], [5.0, 60.0]], np.float32)
    o = gpu_query(m, far, None)
    r = ref.query(far, None)
    assert np.array_equal(o["winner"], r["winner"])
    assert np.max(np.abs(o["sdf"] - r["sdf"])) <= 1e-4
    # NaN / out-of-grid query: flagged, NaN outputs, device status reports it
    bad = np.array([[np.nan, 1.0], [1.0, 2.0], [3.0e7, 0.0]], np.float32)
    o = m.query(_t(bad))
    torch.cuda.synchronize()
    assert ksdf.ksdf_sync_status(m.h) == ksdf.KSDF_ERR_NONFINITE
    fl = o["flags"].cpu().numpy()
    assert fl[0] & ksdf.FLAG_INVALID and fl[2] & ksdf.FLAG_INVALID and not fl[1] & ksdf.FLAG_INVALID
    assert np.isnan(o["sdf"][0].item()) and np.isfinite(o["sdf"][1].item())
    # single-sample model: closed form u = sqrt(z^2 + log(1 + s2)/lambda)
    p = dict(w.params)
    m1 = ksdf.KernelSDF(p)
    x1 = np.array([[2.3, 4.1]])
    m1.fit(_t(x1), _t(np.array([2e-4], np.float32)), None)
    q = np.array([[2.5, 4.0], [2.31, 4.1]], np.float32)
    o = gpu_query(m1, q, None, f64=False)
    z2 = np.sum((q.astype(np.float64) - x1) ** 2, axis=1)
    u = np.sqrt(z2 + np.log1p(2e-4) / p["lambda"])
    assert np.max(np.abs(o["sdf"] - u)) <= 1e-6
    # invalid parameters and fit inputs are rejected with the documented codes
    with pytest.raises(ksdf.KsdfError):
        ksdf.KernelSDF(dict(p, n_max=100000))
    with pytest.raises(ksdf.KsdfError) as e:
        m1.fit(_t(np.array([[np.inf, 0.0]])), None, None)
    assert e.value.status == ksdf.KSDF_ERR_NONFINITE


def test_not_pd_cell_reported():
    p = dict(dim=2, origin=(0.0, 0.0, 0.0), cell=1.0, margin=0.0, n_max=64, k_cand=2, softmin_alpha=50.0,
             sign_mode=0, **{"lambda": 50.0})
    x = np.array([[0.2, 0.2], [0.2, 0.2], [1.5, 0.5]])
    m = ksdf.KernelSDF(p)
    st = m.fit(_t(x), _t(np.zeros(3, np.float32)), None)
    assert st == ksdf.KSDF_ERR_NOT_PD
    keys, status, off, mem = m.cells()
    assert status.tolist() == [ksdf.CELL_NOT_PD, ksdf.CELL_OK]
    o = gpu_query(m, np.array([[0.3, 0.3]], np.float32), None)
    assert o["winner"][0] == 1
