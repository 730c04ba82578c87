"""Pins of the oracle's Matern 3/2 kernel (kernel table of Sec. IV-B.2, scaling of App. D) against facts that
do not come from the oracle itself.

With lambda the scale of f = exp(-lambda u) (the kernel scale sqrt(3)/lambda of Sec. IV-B.1, i.e. lambda = sqrt3/l):
  k(r) = (1 + lambda r) exp(-lambda r),   u(f) = -log f / lambda,
  scaled by gamma = exp(lambda d):        k'_i = (1 + lambda r_i) exp(-lambda (r_i - d)),  u = -log f'/lambda + d.

  N = 1            closed forms of u, grad u, V[f] and the softmin variance
  N = 2            closed form through the 2 x 2 inverse
  dense GP         numpy solve of (K + Sigma) alpha = 1 and the unscaled posterior at moderate lambda
  App. D           u recovered where exp(-lambda r) underflows binary64
  App. E (weak)    f' ~ sum_i k'_i / (1 + sigma^2) for samples far apart relative to 1/lambda
  adjoint          central finite differences of the oracle's own forward (query points, sample positions)
"""
import numpy as np
import pytest


def one_cell(dim, lam, kernel="matern32"):
    return dict(dim=dim, origin=(-512.0, -512.0, -512.0), cell=1024.0, margin=0.0, n_max=1 << 20, k_cand=1,
                softmin_alpha=lam, sign_mode=0, kernel=kernel, **{"lambda": lam})


def matern(r, lam):
    return (1.0 + lam * r) * np.exp(-lam * r)


@pytest.mark.parametrize("dim", [2, 3])
def test_single_sample_closed_form(oracle_mod, dim):
    rng = np.random.default_rng(40 + dim)
    lam, s2 = 30.0, 2e-4
    x1 = rng.uniform(-1, 1, size=(1, dim))
    d = rng.normal(size=(50, dim))
    d *= (rng.uniform(0.1, 0.6, size=50) / np.linalg.norm(d, axis=1))[:, None]
    q = (x1 + d).astype(np.float32)
    m = oracle_mod.Model(one_cell(dim, lam), x1, np.array([s2]))
    o = m.query(q)
    qd = q.astype(np.float64)
    z = np.linalg.norm(qd - x1, axis=1)
    # alpha = 1/(1+s2); f' = alpha (1 + lambda z); u = -log f'/lambda + z
    assert np.allclose(m.alpha(0), [1.0 / (1.0 + s2)], rtol=1e-15, atol=0)
    assert np.allclose(o["sdf"], z - np.log((1.0 + lam * z) / (1.0 + s2)) / lam, rtol=1e-12, atol=1e-15)
    assert np.allclose(o["grad"], (qd - x1) / z[:, None], rtol=1e-12, atol=1e-13)
    assert np.allclose(o["var_sdf"], s2, rtol=1e-12)
    assert np.allclose(o["var_f"], 1.0 - matern(z, lam) ** 2 / (1.0 + s2), rtol=1e-12, atol=1e-15)


def test_two_samples_closed_form(oracle_mod):
    lam, s2 = 40.0, 1e-3
    x = np.array([[0.0, 0.0], [0.08, 0.03]])
    rng = np.random.default_rng(13)
    q = rng.uniform(-0.3, 0.4, size=(40, 2)).astype(np.float32)
    m = oracle_mod.Model(one_cell(2, lam), x, np.full(2, s2))
    o = m.query(q)
    qd = q.astype(np.float64)
    k12 = matern(np.linalg.norm(x[0] - x[1]), lam)
    r1 = np.linalg.norm(qd - x[0], axis=1)
    r2 = np.linalg.norm(qd - x[1], axis=1)
    k1, k2 = matern(r1, lam), matern(r2, lam)
    a = 1.0 + s2
    assert np.allclose(m.alpha(0), 1.0 / (a + k12), rtol=1e-14)
    f = (k1 + k2) / (a + k12)
    u = np.maximum(-np.log(f) / lam, 0.0)
    assert np.allclose(o["sdf"], u, rtol=1e-10, atol=1e-14)
    # grad k(r) = -lambda^2 exp(-lambda r) (x - x_i); grad u = -grad f / |grad f|
    gvec = np.exp(-lam * r1)[:, None] * (qd - x[0]) + np.exp(-lam * r2)[:, None] * (qd - x[1])
    assert np.allclose(o["grad"], gvec / np.linalg.norm(gvec, axis=1, keepdims=True), rtol=1e-9, atol=1e-12)
    vf = 1.0 - (a * (k1 ** 2 + k2 ** 2) - 2 * k12 * k1 * k2) / (a * a - k12 * k12)
    assert np.allclose(o["var_f"], np.maximum(vf, 0.0), rtol=1e-9, atol=1e-13)


@pytest.mark.parametrize("seed", [0, 1])
def test_dense_gp(oracle_mod, seed):
    """Unscaled posterior with a dense numpy solve at a lambda where nothing underflows."""
    rng = np.random.default_rng(seed)
    n, lam = 40, 12.0
    x = rng.uniform(0.0, 0.5, size=(n, 3))
    var = rng.uniform(2.5e-5, 4e-4, size=n)
    m = oracle_mod.Model(one_cell(3, lam), x, var)
    R = np.linalg.norm(x[:, None, :] - x[None, :, :], axis=2)
    A = matern(R, lam) + np.diag(var)
    alpha = np.linalg.solve(A, np.ones(n))
    assert np.max(np.abs(m.alpha(0) - alpha)) <= 1e-12 * np.linalg.cond(A) * np.max(np.abs(alpha))
    L = m.chol(0)
    assert np.max(np.abs(L @ L.T - A)) <= 1e-13
    q = rng.uniform(-0.3, 0.8, size=(60, 3)).astype(np.float32)
    qd = q.astype(np.float64)
    r = np.linalg.norm(qd[:, None, :] - x[None], axis=2)
    k = matern(r, lam)
    f = k @ alpha
    ok = f > 0
    o = m.query(q)
    assert np.allclose(o["sdf"][ok], np.maximum(-np.log(f[ok]) / lam, 0.0), rtol=1e-9, atol=1e-12)
    gf = -(lam ** 2) * np.einsum("qi,i,qij->qj", np.exp(-lam * r), alpha, qd[:, None, :] - x[None])
    gu = -gf / np.linalg.norm(gf, axis=1, keepdims=True)
    assert np.allclose(o["grad"][ok], gu[ok], rtol=1e-8, atol=1e-10)
    vf = 1.0 - np.einsum("qi,qi->q", k, np.linalg.solve(A, k.T).T)
    assert np.allclose(o["var_f"], np.maximum(vf, 0.0), rtol=1e-9, atol=1e-12)


def test_scaling_is_exact_far_from_samples(oracle_mod):
    """App. D: gamma = exp(lambda d) recovers u where exp(-lambda r) underflows binary64 (lambda r = 1500, 2500)."""
    lam, s2 = 300.0, 1e-4
    x1 = np.array([[0.0, 0.0, 0.0]])
    q = np.array([[5.0, 0.0, 0.0], [0.0, 6.0, 8.0]], dtype=np.float32)
    m = oracle_mod.Model(one_cell(3, lam), x1, np.array([s2]))
    z = np.array([5.0, 10.0])
    assert np.exp(-lam * z[0]) == 0.0
    assert np.allclose(m.query(q)["sdf"], z - np.log((1.0 + lam * z) / (1.0 + s2)) / lam, rtol=1e-14)


def test_weak_correlation_limit_formula(oracle_mod):
    """App. E weak limit for the Matern kernel: f' ~ sum_i k'_i / (1 + sigma^2) when K ~ I."""
    lam, s2 = 300.0, 3e-4
    delta = 60.0 / lam  # K_ij <= (1 + 60) e^{-60}
    g = np.arange(5) * delta
    xs = np.stack(np.meshgrid(g, g), axis=-1).reshape(-1, 2)
    m = oracle_mod.Model(one_cell(2, lam), xs, np.full(len(xs), s2))
    rng = np.random.default_rng(16)
    q = rng.uniform(0, 4 * delta, size=(400, 2)).astype(np.float32)
    qd = q.astype(np.float64)
    r = np.linalg.norm(qd[:, None, :] - xs[None], axis=2)
    d = r.min(axis=1)
    fp = np.sum((1.0 + lam * r) * np.exp(-lam * (r - d[:, None])), axis=1) / (1.0 + s2)
    u = np.maximum(-np.log(fp) / lam + d, 0.0)
    assert np.allclose(m.query(q)["sdf"], u, rtol=0, atol=1e-12)


@pytest.mark.parametrize("with_grad", [False, True])
def test_adjoint_finite_differences(oracle_mod, with_grad):
    rng = np.random.default_rng(23)
    g = np.arange(-6, 7) * 0.05
    xs = np.stack(np.meshgrid(g, g), axis=-1).reshape(-1, 2)
    xs = np.concatenate([xs, 0.02 * np.sin(7 * xs[:, :1])], axis=1) + rng.normal(scale=0.005, size=(len(xs), 3))
    var = rng.uniform(2.5e-5, 4e-4, len(xs))
    p = one_cell(3, 60.0)
    m = oracle_mod.Model(p, xs, var)
    q = np.stack([rng.uniform(-0.15, 0.15, 6), rng.uniform(-0.15, 0.15, 6), rng.uniform(0.04, 0.12, 6)], axis=1)
    wsdf = rng.normal(size=6)
    wgrad = rng.normal(size=(6, 3)) if with_grad else None
    assert np.all((m.query_f64(q)["flags"] & 17) == 0)  # neither fallback nor clamped

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


def test_kernels_differ_and_rbf_is_default(oracle_mod):
    """The kernel field selects the kernel (a planted swap of the two would fail the closed forms above); the
    default is the RBF kernel."""
    x1 = np.array([[0.0, 0.0, 0.0]])
    q = np.array([[0.2, 0.0, 0.0]], dtype=np.float32)
    p = one_cell(3, 30.0)
    u_m = oracle_mod.Model(p, x1, np.zeros(1)).query(q)["sdf"][0]
    p_rbf = dict(p)
    del p_rbf["kernel"]
    u_r = oracle_mod.Model(p_rbf, x1, np.zeros(1)).query(q)["sdf"][0]
    z = float(q[0, 0])  # the FP32 query point, exactly
    assert abs(u_r - z) < 1e-12  # noise-free RBF single sample: exact distance
    assert abs(u_m - (z - np.log(1.0 + 30.0 * z) / 30.0)) < 1e-12
