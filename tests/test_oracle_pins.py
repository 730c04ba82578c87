"""Pins of the CPU FP64 oracle against facts that do not come from the oracle itself.

Each test names the paper passage or the mathematical fact it checks.  The pins are chosen so that a
plausible mistake anywhere in the oracle (a dropped term, a wrong sign or index, a transposed operand, an
off-by-one in the binning or the candidate order) fails at least one of them:

  binning / keys        exact dyadic arithmetic, boundaries, translation, key order = (cz, cy, cx)
  training sets         exact rational membership (fractions.Fraction), hand-computed rank selection
  fit                   LAPACK dense solve (numpy) and L L^T = A on random cells
  N = 1, N = 2          closed forms of the posterior (Sec. IV-B.1) and of the softmin variance (Sec. IV-B.3)
  limits                weak / strong correlation (App. E), scaling invariance (App. D)
  candidates            brute force by a full sort over (lattice distance, key)
  min-fusion            consistency with one global GP (App. F, footnote of Sec. IV-B.1)
  geometry              sign inside/outside, eikonal |grad u| = 1 (Sec. III), invariants
  adjoint               central finite differences of the oracle's own forward pass
"""
import json
import os
from fractions import Fraction

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def params(dim=3, cell=0.5, margin=0.1, n_max=256, K=8, lam=300.0, alpha=None, origin=(0.0, 0.0, 0.0), sign_mode=0):
    return dict(dim=dim, origin=origin, cell=cell, margin=margin, n_max=n_max, k_cand=K, softmin_alpha=alpha or lam,
                sign_mode=sign_mode, **{"lambda": lam})


def one_cell(dim, lam, alpha=None):
    """A single huge cell holding every sample: one global GP."""
    return params(dim=dim, cell=1024.0, margin=0.0, n_max=1 << 20, K=1, lam=lam, alpha=alpha,
                  origin=(-512.0, -512.0, -512.0))


# ----------------------------------------------------------------------------------------------------
# binning and keys


def test_bin_exact_dyadic_boundaries(oracle_mod):
    p = params(dim=3, cell=0.5)
    # points exactly on cell boundaries belong to the upper cell; just below go to the lower one
    x = np.array([[0.0, 0.5, 1.0], [-0.5, -1.0, 2.5], [np.nextafter(0.5, 0), 0.25, -1e-300]])
    keys = oracle_mod.bin_keys(p, x)
    c = oracle_mod.unpack_keys(keys)
    assert c.tolist() == [[0, 1, 2], [-1, -2, 5], [0, 0, -1]]


def test_bin_translation_and_key_order(oracle_mod):
    rng = np.random.default_rng(0)
    p = params(dim=3, cell=0.25)
    x = rng.uniform(-20, 20, size=(2000, 3)).round(6)
    c0 = oracle_mod.unpack_keys(oracle_mod.bin_keys(p, x))
    shift = np.array([3, -7, 11])
    c1 = oracle_mod.unpack_keys(oracle_mod.bin_keys(p, x + shift * 0.25))  # multiples of h are exact here
    assert np.array_equal(c1, c0 + shift)
    # ascending key order is lexicographic (cz, cy, cx) order
    keys = oracle_mod.bin_keys(p, x)
    order_keys = np.argsort(keys, kind="stable")
    tuples = sorted(range(len(x)), key=lambda i: (c0[i, 2], c0[i, 1], c0[i, 0], i))
    assert [tuple(c0[i]) for i in order_keys] == [tuple(c0[i]) for i in tuples]
    # 2D keys have cz = 0
    p2 = params(dim=2, cell=1.0)
    c2 = oracle_mod.unpack_keys(oracle_mod.bin_keys(p2, np.array([[-0.5, 3.7], [9.99, -10.0]])))
    assert c2.tolist() == [[-1, 3, 0], [9, -10, 0]]


def test_bin_rejects_out_of_range_and_nan(oracle_mod):
    p = params(dim=2, cell=1.0)
    for bad in ([[2.0 ** 21, 0.0]], [[np.nan, 0.0]], [[0.0, -np.inf]]):
        with pytest.raises(ValueError):
            oracle_mod.bin_keys(p, np.array(bad))


# ----------------------------------------------------------------------------------------------------
# cells and training sets


def exact_members(x, keys_cells, p):
    """Exact (rational) collection-box membership, ascending ids, then rank selection."""
    h, mu = Fraction(p["cell"]), Fraction(p["margin"])
    o = [Fraction(v) for v in p["origin"]]
    dim = p["dim"]
    cc = [[int(v) for v in row] for row in keys_cells]
    xf = [[Fraction(float(v)) for v in row] for row in x]
    out = []
    for c in cc:
        mem = [i for i in range(len(x))
               if all(o[j] + c[j] * h - mu <= xf[i][j] < o[j] + (c[j] + 1) * h + mu for j in range(dim))]
        n = len(mem)
        if n > p["n_max"]:
            mem = [mem[(j * n) // p["n_max"]] for j in range(p["n_max"])]
        out.append(mem)
    return out


@pytest.mark.parametrize("dim", [2, 3])
def test_training_sets_exact(oracle_mod, dim):
    rng = np.random.default_rng(dim)
    n = 400
    x = rng.uniform(0, 2.0, size=(n, dim))
    # put some points exactly on box edges (dyadic values are exact in binary64)
    x[:20, 0] = rng.integers(0, 8, size=20) * 0.25 + np.array([0.0, 0.125, -0.125, 0.375])[rng.integers(0, 4, 20)]
    p = params(dim=dim, cell=0.5, margin=0.125, n_max=40)
    m = oracle_mod.Model(p, x, np.full(n, 1e-4))
    keys, status, off, mem = m.cells()
    cells = oracle_mod.unpack_keys(keys)
    # cells are exactly the distinct bins of the samples, ascending key
    bins = np.unique(oracle_mod.bin_keys(p, x))
    assert np.array_equal(bins, keys)
    ref = exact_members(x, cells, p)
    for g in range(len(keys)):
        assert mem[off[g]:off[g + 1]].tolist() == ref[g], g


def test_rank_selection_hand_example(oracle_mod):
    # 10 samples in one 1 m cell (2D), n_max = 4 keeps ranks floor(j*10/4) = 0, 2, 5, 7
    x = np.stack([np.linspace(0.05, 0.95, 10), np.full(10, 0.5)], axis=1)
    perm = np.array([3, 9, 0, 7, 1, 8, 2, 6, 4, 5])  # ids are scrambled positions
    m = oracle_mod.Model(params(dim=2, cell=1.0, margin=0.0, n_max=4, K=1), x[perm], np.full(10, 1e-3))
    _, _, off, mem = m.cells()
    assert off.tolist() == [0, 4]
    assert mem.tolist() == [0, 2, 5, 7]


def test_not_pd_cell_is_excluded(oracle_mod):
    # duplicate samples with sigma^2 = 0 make K + Sigma singular: the cell fails and is not a candidate
    x = np.array([[0.2, 0.2], [0.2, 0.2], [1.5, 0.5]])
    m = oracle_mod.Model(params(dim=2, cell=1.0, margin=0.0, K=2, lam=50.0), x, np.zeros(3))
    keys, status, off, _ = m.cells()
    assert status.tolist() == [oracle_mod.CELL_NOT_PD, oracle_mod.CELL_OK]
    cand, cnt = m.candidates(keys)
    assert cnt.tolist() == [1, 1] and cand[:, 0].tolist() == [1, 1]


# ----------------------------------------------------------------------------------------------------
# fit against LAPACK


def rbf_matrix(x, lam):
    d2 = np.sum((x[:, None, :] - x[None, :, :]) ** 2, axis=2)
    return np.exp(-lam * d2)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_fit_matches_dense_solve(oracle_mod, seed):
    rng = np.random.default_rng(seed)
    n = 60
    x = rng.uniform(0.0, 0.4, size=(n, 3))
    var = rng.uniform(2.5e-5, 4e-4, size=n)
    lam = 300.0
    m = oracle_mod.Model(one_cell(3, lam), x, var)
    A = rbf_matrix(x, lam) + np.diag(var)
    alpha_ref = np.linalg.solve(A, np.ones(n))
    alpha = m.alpha(0)
    cond = np.linalg.cond(A)
    assert np.max(np.abs(alpha - alpha_ref)) <= 1e-13 * cond * np.max(np.abs(alpha_ref))
    L = m.chol(0)
    assert np.allclose(np.triu(L, 1), 0.0)
    assert np.max(np.abs(L @ L.T - A)) <= 1e-13


# ----------------------------------------------------------------------------------------------------
# closed forms


@pytest.mark.parametrize("dim", [2, 3])
def test_single_sample_closed_form(oracle_mod, dim):
    rng = np.random.default_rng(10 + dim)
    lam, s2 = 300.0, 2e-4
    x1 = rng.uniform(-1, 1, size=(1, dim))
    q = (x1 + rng.normal(scale=0.1, size=(50, dim))).astype(np.float32)
    m = oracle_mod.Model(one_cell(dim, lam), x1, np.array([s2]))
    o = m.query(q)
    qd = q.astype(np.float64)
    z = np.linalg.norm(qd - x1, axis=1)
    # alpha = 1/(1+s2); u^2 = -log(alpha e^{-lam z^2})/lam = z^2 + log(1+s2)/lam
    assert np.allclose(m.alpha(0), [1.0 / (1.0 + s2)], rtol=1e-15, atol=0)
    assert np.allclose(o["sdf"], np.sqrt(z * z + np.log1p(s2) / lam), rtol=1e-12, atol=0)
    assert np.allclose(o["grad"], (qd - x1) / z[:, None], rtol=1e-12, atol=1e-13)
    assert np.allclose(o["var_sdf"], s2, rtol=1e-12)
    assert np.allclose(o["var_f"], 1.0 - np.exp(-2 * lam * z * z) / (1.0 + s2), rtol=1e-12, atol=1e-15)


def test_single_sample_noise_free_is_exact_distance(oracle_mod):
    x1 = np.array([[0.3, -0.2, 0.1]])
    q = np.array([[1.0, 1.0, 1.0], [0.3, -0.2, 0.35]], dtype=np.float32)
    m = oracle_mod.Model(one_cell(3, 500.0), x1, np.zeros(1))
    o = m.query(q)
    assert np.allclose(o["sdf"], np.linalg.norm(q.astype(np.float64) - x1, axis=1), rtol=1e-14)


def test_two_samples_closed_form(oracle_mod):
    lam, s2 = 200.0, 1e-3
    x = np.array([[0.0, 0.0], [0.08, 0.03]])
    rng = np.random.default_rng(3)
    q = rng.uniform(-0.2, 0.3, size=(40, 2)).astype(np.float32)
    m = oracle_mod.Model(one_cell(2, lam), x, np.full(2, s2))
    o = m.query(q)
    qd = q.astype(np.float64)
    k12 = np.exp(-lam * np.sum((x[0] - x[1]) ** 2))
    k1 = np.exp(-lam * np.sum((qd - x[0]) ** 2, axis=1))
    k2 = np.exp(-lam * np.sum((qd - x[1]) ** 2, axis=1))
    a = 1.0 + s2
    # 2x2 inverse: alpha_1 = alpha_2 = 1/(a + k12)
    assert np.allclose(m.alpha(0), 1.0 / (a + k12), rtol=1e-14)
    f = (k1 + k2) / (a + k12)
    assert np.allclose(o["sdf"], np.sqrt(-np.log(f) / lam), rtol=1e-10)
    gvec = (k1[:, None] * (qd - x[0]) + k2[:, None] * (qd - x[1]))
    assert np.allclose(o["grad"], gvec / np.linalg.norm(gvec, axis=1, keepdims=True), rtol=1e-9, atol=1e-12)
    vf = 1.0 - (a * (k1 ** 2 + k2 ** 2) - 2 * k12 * k1 * k2) / (a * a - k12 * k12)
    assert np.allclose(o["var_f"], np.maximum(vf, 0.0), rtol=1e-9, atol=1e-13)
    # softmin variance with two samples (Sec. IV-B.3), alpha_softmin = lambda
    z1 = np.linalg.norm(qd - x[0], axis=1)
    z2 = np.linalg.norm(qd - x[1], axis=1)
    w1, w2 = np.exp(-lam * z1), np.exp(-lam * z2)
    s1, s2w = w1 / (w1 + w2), w2 / (w1 + w2)
    h = s1 * z1 + s2w * z2
    vs = s2 * (s1 ** 2 * (lam * (h - z1) + 1) ** 2 + s2w ** 2 * (lam * (h - z2) + 1) ** 2)
    assert np.allclose(o["var_sdf"], vs, rtol=1e-9)


# ----------------------------------------------------------------------------------------------------
# limits of App. E and the scaling of App. D


def test_weak_correlation_noise_free_underestimate(oracle_mod):
    """App. E, weak regime, sigma = 0: log f = log max k + log S with S >= 1, so u <= distance to the
    nearest sample, and the gap shrinks as lambda grows."""
    rng = np.random.default_rng(5)
    gaps = []
    for lam in (100.0, 300.0, 1000.0):
        delta = np.sqrt(25.0 / lam)  # K_ij <= e^{-25}
        xs = np.stack([np.arange(20) * delta, np.zeros(20)], axis=1)
        m = oracle_mod.Model(one_cell(2, lam), xs, None)
        q = np.stack([rng.uniform(0, 19 * delta, 3000), rng.uniform(-0.3, 0.3, 3000)], axis=1).astype(np.float32)
        zmin = np.min(np.linalg.norm(q.astype(np.float64)[:, None, :] - xs[None], axis=2), axis=1)
        u = m.query(q)["sdf"]
        assert np.all(u <= zmin + 1e-12)
        gaps.append(np.mean(zmin - u))
    assert gaps[0] > gaps[1] > gaps[2] > 0


def test_weak_correlation_limit_formula(oracle_mod):
    """App. E weak limit: f ~ sum_i k_i / (1 + sigma^2) when samples are far apart relative to l."""
    lam, s2 = 300.0, 3e-4
    delta = np.sqrt(40.0 / lam)
    g = np.arange(5) * delta
    xs = np.stack(np.meshgrid(g, g), axis=-1).reshape(-1, 2)
    m = oracle_mod.Model(one_cell(2, lam), xs, np.full(len(xs), s2))
    rng = np.random.default_rng(6)
    q = rng.uniform(0, 4 * delta, size=(500, 2)).astype(np.float32)
    qd = q.astype(np.float64)
    d2 = np.sum((qd[:, None, :] - xs[None]) ** 2, axis=2)
    dmin = d2.min(axis=1)
    logf = np.log(np.sum(np.exp(-lam * (d2 - dmin[:, None])), axis=1)) - lam * dmin - np.log1p(s2)
    u = m.query(q)["sdf"]
    assert np.allclose(u * u, -logf / lam, rtol=0, atol=1e-15 * 1e3)


def test_strong_correlation_limit_formula(oracle_mod):
    """App. E strong limit: a tight cluster of N samples gives f ~ N k(z) / (sigma^2 + N)."""
    lam, s2, N = 300.0, 1e-3, 12
    rng = np.random.default_rng(7)
    c = np.array([0.1, -0.2, 0.05])
    xs = c + rng.normal(scale=1e-7, size=(N, 3))
    m = oracle_mod.Model(one_cell(3, lam), xs, np.full(N, s2))
    q = (c + rng.normal(scale=0.1, size=(100, 3))).astype(np.float32)
    z = np.linalg.norm(q.astype(np.float64) - c, axis=1)
    u = m.query(q)["sdf"]
    expect = np.sqrt(z * z + np.log((s2 + N) / N) / lam)
    assert np.allclose(u, expect, rtol=2e-5)


def test_scaling_is_exact_far_from_samples(oracle_mod):
    """App. D: with the adaptive scaling the UDF is recovered where exp(-lambda r^2) underflows binary64."""
    lam = 300.0
    x1 = np.array([[0.0, 0.0, 0.0]])
    q = np.array([[2.0, 0.0, 0.0], [0.0, 3.0, 4.0]], dtype=np.float32)  # lambda r^2 = 1200, 7500
    m = oracle_mod.Model(one_cell(3, lam), x1, np.zeros(1))
    assert np.allclose(m.query(q)["sdf"], [2.0, 5.0], rtol=1e-14)


# ----------------------------------------------------------------------------------------------------
# candidates


def test_candidates_brute_force(oracle_mod):
    rng = np.random.default_rng(11)
    x = rng.uniform(-3, 3, size=(600, 3))
    x = x[rng.random(600) < 0.5]
    p = params(dim=3, cell=0.5, K=8)
    m = oracle_mod.Model(p, x, np.full(len(x), 1e-4))
    keys, status, _, _ = m.cells()
    cc = oracle_mod.unpack_keys(keys)
    qb = rng.integers(-10, 10, size=(300, 3))
    bkeys = oracle_mod.bin_keys(p, (qb + 0.5) * 0.5)
    cand, cnt = m.candidates(bkeys)
    for b, row, n in zip(qb, cand, cnt):
        order = sorted(range(len(keys)), key=lambda g: (int(np.sum((b - cc[g]) ** 2)), int(keys[g])))
        assert n == min(8, len(keys))
        assert row[:n].tolist() == order[:8]


# ----------------------------------------------------------------------------------------------------
# App. F: min-fused local GPs agree with one global GP


def test_min_fusion_matches_global_gp(oracle_mod):
    golden = json.load(open(os.path.join(GOLDEN, "min_fusion_circle.json")))
    lam, N, m_ov = golden["lambda"], golden["n_samples"], golden["overlap_m"]
    rng = np.random.default_rng(0)
    th = np.arange(N) * 2 * np.pi / N + 0.01
    xs = np.stack([np.cos(th), np.sin(th)], axis=1)
    var = np.full(N, 1e-4)
    # two local GPs split at x = 0 with overlap m: cells [-2,0) and [0,2) in x, one row [-1,1) in y
    local = params(dim=2, cell=2.0, margin=m_ov, n_max=4096, K=2, lam=lam, origin=(-2.0, -3.0, 0.0))
    ml = oracle_mod.Model(local, xs, var)
    mg = oracle_mod.Model(one_cell(2, lam), xs, var)
    assert ml.G == 2
    # queries in a band around the circle, outside the switching ambiguity of points equidistant from
    # both halves (the circle's centre)
    r = rng.uniform(0.8, 1.4, 4000)
    t = rng.uniform(0, 2 * np.pi, 4000)
    q = np.stack([r * np.cos(t), r * np.sin(t)], axis=1).astype(np.float32)
    ol, og = ml.query(q), mg.query(q)
    du = np.abs(ol["sdf"] - og["sdf"])
    ang = np.arccos(np.clip(np.sum(ol["grad"] * og["grad"], axis=1), -1, 1))
    assert np.median(du) <= golden["udf_diff_level_m"]
    assert np.median(ang) <= golden["angle_bound_rad"]
    # away from the two overlap edges (|x| > 0.45) the agreement holds pointwise
    away = np.abs(q[:, 0]) > 0.45
    assert np.quantile(du[away], 0.99) <= 1e3 * golden["udf_diff_level_m"]


# ----------------------------------------------------------------------------------------------------
# geometry: sign, eikonal, invariants


def test_sphere_sign_and_accuracy(oracle_mod):
    rng = np.random.default_rng(12)
    N, R = 3000, 0.8
    v = rng.standard_normal((N, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    xs = R * v
    p = params(dim=3, cell=0.5, margin=0.1, n_max=512, K=8, lam=300.0, sign_mode=1)
    m = oracle_mod.Model(p, xs, np.full(N, 1e-6), normals=v)
    d = rng.uniform(-0.3, 0.3, 2000)
    w = rng.standard_normal((2000, 3))
    w /= np.linalg.norm(w, axis=1, keepdims=True)
    q = (w * (R + d)[:, None]).astype(np.float32)
    o = m.query(q)  # sign from the nearest-normal stand-in
    true = np.linalg.norm(q.astype(np.float64), axis=1) - R
    far = np.abs(true) > 0.02
    assert np.all(np.sign(o["sdf"][far]) == np.sign(true[far]))
    assert np.max(np.abs(o["sdf"] - true)) < 0.05
    # gradient of the SDF points along the radius
    radial = q.astype(np.float64) / np.linalg.norm(q.astype(np.float64), axis=1, keepdims=True)
    cosang = np.sum(o["grad"][far] * radial[far], axis=1)
    assert np.median(cosang) > 0.999 and np.quantile(cosang, 0.02) > 0.95


def test_eikonal_through_adjoint(oracle_mod):
    """Sec. III: |grad d| = 1.  The exact derivative of the returned u (adjoint) has unit norm away from
    the surface when the samples are dense on a plane."""
    g = np.arange(-40, 41) * 0.01
    xs = np.stack(np.meshgrid(g, g), axis=-1).reshape(-1, 2)
    xs = np.concatenate([xs, np.zeros((len(xs), 1))], axis=1)
    lam = 300.0
    m = oracle_mod.Model(one_cell(3, lam), xs, np.full(len(xs), 1e-4))
    rng = np.random.default_rng(13)
    q = np.stack([rng.uniform(-0.1, 0.1, 50), rng.uniform(-0.1, 0.1, 50), rng.uniform(0.05, 0.2, 50)], axis=1)
    dq, _ = m.backward(q, np.ones(50), f64=True)
    assert np.allclose(np.linalg.norm(dq, axis=1), 1.0, atol=2e-3)
    assert np.allclose(m.query_f64(q)["sdf"], q[:, 2], atol=2e-3)


def test_permutation_invariance(oracle_mod):
    w = __import__("paper_2603_29227_gb300.scenes", fromlist=["workload"]).workload("plane2d", n_samples=600, grid=24)
    perm = np.random.default_rng(3).permutation(len(w.x))
    m2 = oracle_mod.Model(dict(w.params, n_max=10 ** 6), w.x[perm], w.var[perm])
    m1 = oracle_mod.Model(dict(w.params, n_max=10 ** 6), w.x, w.var)
    o1, o2 = m1.query(w.xq), m2.query(w.xq)
    ok = (o1["flags"] & 4) == 0
    assert np.allclose(o1["sdf"], o2["sdf"], rtol=1e-12, atol=1e-14)
    assert np.allclose(o1["grad"][ok], o2["grad"][ok], rtol=1e-9, atol=1e-11)
    assert np.allclose(o1["var_f"][ok], o2["var_f"][ok], rtol=1e-8, atol=1e-12)


def test_translation_invariance(oracle_mod):
    rng = np.random.default_rng(14)
    xs = rng.uniform(0, 2, size=(300, 3))
    q = rng.uniform(0, 2, size=(200, 3)).astype(np.float32).astype(np.float64)
    p = params(dim=3, cell=0.5)
    shift = np.array([1.5, -2.0, 0.5])  # multiples of h, exact on these magnitudes
    m1 = oracle_mod.Model(p, xs, np.full(300, 1e-4))
    m2 = oracle_mod.Model(p, xs + shift, np.full(300, 1e-4))
    o1 = m1.query_f64(q)
    o2 = m2.query_f64(q + shift)
    assert np.array_equal(m1.cells()[3], m2.cells()[3])  # same training sets
    assert np.allclose(o1["sdf"], o2["sdf"], rtol=1e-9)
    assert np.allclose(o1["grad"], o2["grad"], rtol=1e-6, atol=1e-8)


def test_mirror_symmetry(oracle_mod):
    rng = np.random.default_rng(15)
    xs = rng.uniform(-1, 1, size=(200, 2))
    q = rng.uniform(-1, 1, size=(100, 2))
    p = params(dim=2, cell=0.5, margin=0.1, K=64, lam=300.0)  # K covers every cell: no tie-break effects
    m1 = oracle_mod.Model(p, xs, np.full(200, 1e-4))
    mir = np.array([-1.0, 1.0])
    m2 = oracle_mod.Model(p, xs * mir, np.full(200, 1e-4))
    o1, o2 = m1.query_f64(q), m2.query_f64(q * mir)
    ok = (o1["flags"] & 4) == 0
    assert np.allclose(o1["sdf"], o2["sdf"], rtol=1e-12)
    assert np.allclose(o1["grad"][ok] * mir, o2["grad"][ok], rtol=1e-8, atol=1e-10)


# ----------------------------------------------------------------------------------------------------
# adjoint vs central finite differences of the oracle itself


@pytest.mark.parametrize("with_grad", [False, True])
def test_adjoint_finite_differences(oracle_mod, with_grad):
    rng = np.random.default_rng(21)
    g = np.arange(-6, 7) * 0.05
    xs = np.stack(np.meshgrid(g, g), axis=-1).reshape(-1, 2)
    xs = np.concatenate([xs, 0.02 * np.sin(7 * xs[:, :1])], axis=1) + rng.normal(scale=0.005, size=(len(xs), 3))
    var = rng.uniform(2.5e-5, 4e-4, len(xs))
    lam = 300.0
    p = one_cell(3, lam)
    m = oracle_mod.Model(p, xs, var)
    q = np.stack([rng.uniform(-0.15, 0.15, 6), rng.uniform(-0.15, 0.15, 6), rng.uniform(0.04, 0.12, 6)], axis=1)
    wsdf = rng.normal(size=6)
    wgrad = rng.normal(size=(6, 3)) if with_grad else None

    def loss(model, qq):
        o = model.query_f64(qq)
        val = np.sum(wsdf * o["sdf"])
        if with_grad:
            val += np.sum(wgrad * o["grad"])
        return val

    dq, dx = m.backward(q, wsdf, wgrad, f64=True)
    h = 1e-5
    for i in range(6):
        for j in range(3):
            e = np.zeros_like(q)
            e[i, j] = h
            fd = (loss(m, q + e) - loss(m, q - e)) / (2 * h)
            assert abs(fd - dq[i, j]) <= 1e-5 * max(1.0, abs(fd)), (i, j, fd, dq[i, j])
    for s in rng.choice(len(xs), size=8, replace=False):
        for j in range(3):
            e = np.zeros_like(xs)
            e[s, j] = h
            fp = loss(oracle_mod.Model(p, xs + e, var), q)
            fm = loss(oracle_mod.Model(p, xs - e, var), q)
            fd = (fp - fm) / (2 * h)
            assert abs(fd - dx[s, j]) <= 1e-5 * max(1.0, abs(fd)), (s, j, fd, dx[s, j])
