"""Pins of the oracle's SDF-gradient variance (Sec. IV-B.3 gradient-variance approximation, App. C) against
what the mathematics fixes, independently of the printed Jacobian:

  * one sample: g = v = (x - x_1)/z is the gradient of the distance, so d g_k / d x_1 = -(e_k - v_k v)/z and
    V[grad_k u] = sigma^2 (1 - v_k^2) / z^2;
  * any N: grad_{x_i} g_k by numerical differentiation of g = grad_x h, where h = s^T z is the softmin
    (g itself by complex-step differentiation of h, exact to rounding; its derivative in x_i by central
    differences), summed as sum_i sigma_i^2 |grad_{x_i} g_k|^2 -- this also fixes which index of the
    printed matrix is k (a transposed matrix gives different norms);
  * permutation invariance and the +inf of a query on a sample.
"""
import numpy as np
import pytest


def one_cell(dim, lam, alpha):
    return dict(dim=dim, origin=(-512.0, -512.0, -512.0), cell=1024.0, margin=0.0, n_max=1 << 20, k_cand=1,
                softmin_alpha=alpha, sign_mode=0, **{"lambda": lam})


def softmin_h(x, X, a):
    """h = s^T z with s the softmin of z = |x - x_i| (complex-safe for the complex step)."""
    d = x[None, :] - X
    z = np.sqrt(np.sum(d * d, axis=1))
    zr = np.min(z.real)
    e = np.exp(-a * (z - zr))
    return np.sum(e * z) / np.sum(e)


def g_of(x, X, a, hstep=1e-20):
    """grad_x h by the complex step (no subtractive cancellation)."""
    out = np.empty(x.shape[0])
    for k in range(x.shape[0]):
        xc = x.astype(complex)
        xc[k] += 1j * hstep
        out[k] = softmin_h(xc, X.astype(complex), a).imag / hstep
    return out


def var_grad_numeric(x, X, s2, a, step=1e-6):
    dim = x.shape[0]
    out = np.zeros(dim)
    for i in range(X.shape[0]):
        J = np.empty((dim, dim))  # J[k, b] = d g_k / d x_{i,b}
        for b in range(dim):
            Xp, Xm = X.copy(), X.copy()
            Xp[i, b] += step
            Xm[i, b] -= step
            J[:, b] = (g_of(x, Xp, a) - g_of(x, Xm, a)) / (2 * step)
        out += s2[i] * np.sum(J * J, axis=1)
    return out


@pytest.mark.parametrize("dim", [2, 3])
def test_single_sample_closed_form(oracle_mod, dim):
    rng = np.random.default_rng(40 + dim)
    s2 = 3e-4
    x1 = rng.uniform(-1, 1, size=(1, dim))
    q = (x1 + rng.normal(scale=0.2, size=(40, dim))).astype(np.float32)
    m = oracle_mod.Model(one_cell(dim, 300.0, 250.0), x1, np.array([s2]))
    vg = m.var_grad(q, np.zeros(len(q), np.int32))
    d = q.astype(np.float64) - x1
    z2 = np.sum(d * d, axis=1)
    v2 = d * d / z2[:, None]
    assert np.allclose(vg, s2 * (1.0 - v2) / z2[:, None], rtol=1e-12, atol=0)


@pytest.mark.parametrize("dim,a", [(3, 300.0), (3, 20.0), (2, 120.0)])
def test_numerical_differentiation(oracle_mod, dim, a):
    rng = np.random.default_rng(int(a) + dim)
    N = 7
    X = rng.uniform(0.0, 0.3, size=(N, dim))
    s2 = rng.uniform(0.5, 2.0, size=N) * 1e-4
    m = oracle_mod.Model(one_cell(dim, 300.0, a), X, s2)
    q = rng.uniform(-0.1, 0.4, size=(6, dim)).astype(np.float32)
    ids = m.cells()[3]  # the training set order (ascending sample id = X's order here)
    assert np.array_equal(ids, np.arange(N))
    vg = m.var_grad(q, np.zeros(len(q), np.int32))
    for j in range(len(q)):
        ref = var_grad_numeric(q[j].astype(np.float64), X, s2, a)
        assert np.allclose(vg[j], ref, rtol=2e-6, atol=0), (j, vg[j], ref)


def test_permutation_invariance_and_on_sample(oracle_mod):
    rng = np.random.default_rng(5)
    X = rng.uniform(0, 0.5, size=(20, 3))
    s2 = rng.uniform(0.5, 2.0, size=20) * 1e-4
    q = rng.uniform(-0.1, 0.6, size=(30, 3)).astype(np.float32)
    m1 = oracle_mod.Model(one_cell(3, 300.0, 300.0), X, s2)
    perm = rng.permutation(20)
    m2 = oracle_mod.Model(one_cell(3, 300.0, 300.0), X[perm], s2[perm])
    c = np.zeros(len(q), np.int32)
    assert np.allclose(m1.var_grad(q, c), m2.var_grad(q, c), rtol=1e-12, atol=0)
    on = X[3:4].astype(np.float32)
    m3 = oracle_mod.Model(one_cell(3, 300.0, 300.0), on.astype(np.float64), s2[:1])
    assert np.all(np.isinf(m3.var_grad(on, np.zeros(1, np.int32))))
