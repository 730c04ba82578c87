"""Pins of the BHM front-end oracle (oracle/bhm.py) against facts that do not come from the oracle itself:
the Jaakkola-Jordan bound, closed forms of the diagonal EM, stationarity of the variational bound of App. A at
the EM fixed point, Monte Carlo expectations, exact sequential/batch equivalence, brute-force feature and edge
enumerations, finite differences, and the geometry of a scanned plane."""
import math

import numpy as np
import pytest

from oracle import bhm

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _log_sigmoid(v):
    return -np.logaddexp(0.0, -v)


def _lam(xi):
    # lambda(xi) = (1/2 - sigmoid(xi)) / (2 xi) written through tanh: sigmoid(xi) - 1/2 = tanh(xi / 2) / 2
    return -np.tanh(xi / 2.0) / (4.0 * xi)


def test_jj_coefficient_is_the_tangent_bound():
    """c(xi) / 2 is the curvature of the Jaakkola-Jordan bound: log sigmoid(r) >= log sigmoid(xi) + (r - xi)/2
    - c/2 (r^2 - xi^2) for every r, with equality at r = +-xi.  A factor error in c breaks one of the two."""
    r = np.linspace(-12.0, 12.0, 4001)
    for xi in (0.05, 0.3, 1.0, 2.5, 6.0, 11.0):
        c = float(bhm.jj_coef(xi))
        lower = _log_sigmoid(xi) + (r - xi) / 2.0 - 0.5 * c * (r * r - xi * xi)
        assert np.all(_log_sigmoid(r) - lower >= -1e-12), xi
        for rr in (xi, -xi):
            gap = _log_sigmoid(rr) - (_log_sigmoid(xi) + (rr - xi) / 2.0 - 0.5 * c * (rr * rr - xi * xi))
            assert abs(gap) < 1e-12, (xi, rr)
        assert abs(c - 2.0 * abs(_lam(xi))) < 1e-14
    assert float(bhm.jj_coef(0.0)) == 0.25
    assert abs(float(bhm.jj_coef(1e-6)) - 0.25) < 1e-9


def test_em_one_weight_closed_form():
    """One weight, one occupied sample at phi = 1, prior N(0, 1), xi_0 = 0: P = 1 + 1/4, mu = (1/2) / P; a
    second round uses xi^2 = 1/P + mu^2 and c = tanh(xi/2) / (2 xi)."""
    rows = [(np.array([0]), np.array([1.0]))]
    mu, P, _ = bhm.em_diag(rows, [1], [0.0], [1.0], 0.0, 1)
    assert P[0] == 1.25 and abs(mu[0] - 0.4) < 1e-15
    xi = math.sqrt(1.0 / 1.25 + 0.4 * 0.4)
    c = math.tanh(xi / 2.0) / (2.0 * xi)
    mu2, P2, xi2 = bhm.em_diag(rows, [1], [0.0], [1.0], 0.0, 2)
    assert abs(xi2[0] - xi) < 1e-15
    assert abs(P2[0] - (1.0 + c)) < 1e-15 and abs(mu2[0] - 0.5 / (1.0 + c)) < 1e-15
    # a free sample (t = 0) pulls the mean the other way by the same amount
    mu3, _, _ = bhm.em_diag(rows, [0], [0.0], [1.0], 0.0, 1)
    assert abs(mu3[0] + 0.4) < 1e-15


def _elbo_one_weight(mu, s2, xi, phi, t, mu0, P0):
    """Variational lower bound of App. A for one weight w ~ N(mu, s2) with prior N(mu0, 1/P0): the JJ bound of
    each likelihood term in expectation, minus KL(N(mu, s2) || N(mu0, 1/P0))."""
    r_mean = (2.0 * t - 1.0) * mu * phi
    r2 = phi * phi * (s2 + mu * mu)
    lik = np.sum(_log_sigmoid(xi) + (r_mean - xi) / 2.0 + _lam(xi) * (r2 - xi * xi))
    kl = 0.5 * (P0 * s2 + P0 * (mu - mu0) ** 2 - 1.0 - math.log(P0 * s2))
    return lik - kl


def test_em_fixed_point_is_stationary_point_of_the_bound():
    """With a single weight the diagonal EM is exact coordinate ascent on the bound, so its fixed point zeroes
    every partial derivative of the bound (mean, variance, each xi), computed here by central differences."""
    rng = np.random.default_rng(5)
    K = 7
    phi = rng.uniform(0.05, 1.0, K)
    t = rng.integers(0, 2, K).astype(np.float64)
    mu0, P0 = 0.3, 2.0
    rows = [(np.array([0]), np.array([phi[k]])) for k in range(K)]
    mu, P, _ = bhm.em_diag(rows, t, [mu0], [P0], 0.0, 300)
    mu, s2 = float(mu[0]), 1.0 / float(P[0])
    xi = np.sqrt(phi * phi * (s2 + mu * mu))  # the M-step's xi for the converged posterior
    f = lambda a, b, c: _elbo_one_weight(a, b, c, phi, t, mu0, P0)
    e = 1e-6
    assert abs((f(mu + e, s2, xi) - f(mu - e, s2, xi)) / (2 * e)) < 1e-7
    assert abs((f(mu, s2 + e, xi) - f(mu, s2 - e, xi)) / (2 * e)) < 1e-6
    for k in range(K):
        d = np.zeros(K)
        d[k] = e
        assert abs((f(mu, s2, xi + d) - f(mu, s2, xi - d)) / (2 * e)) < 1e-7
    # and it is a maximum along the mean
    assert f(mu, s2, xi) >= f(mu + 1e-3, s2, xi) and f(mu, s2, xi) >= f(mu - 1e-3, s2, xi)


def test_em_disjoint_weights_decouple():
    """Samples that each reach one weight: the diagonal EM on the joint design equals independent one-weight
    problems (what a full-covariance EM also gives when the features do not overlap)."""
    rng = np.random.default_rng(6)
    rows, t, per = [], [], {0: ([], []), 1: ([], []), 2: ([], [])}
    for k in range(12):
        w = int(rng.integers(0, 3))
        ph = float(rng.uniform(0.1, 1.0))
        lab = int(rng.integers(0, 2))
        rows.append((np.array([w]), np.array([ph])))
        t.append(lab)
        per[w][0].append((np.array([0]), np.array([ph])))
        per[w][1].append(lab)
    mu0, P0 = np.array([0.1, -0.2, 0.0]), np.array([1.0, 3.0, 0.5])
    mu, P, _ = bhm.em_diag(rows, t, mu0, P0, 1.0, 3)
    for w in range(3):
        if per[w][0]:
            m1, p1, _ = bhm.em_diag(per[w][0], per[w][1], [mu0[w]], [P0[w]], 1.0, 3)
            assert abs(m1[0] - mu[w]) < 1e-14 and abs(p1[0] - P[w]) < 1e-13


def test_m_step_is_the_posterior_second_moment():
    """xi_k^2 of the M-step equals E_Q[(w^T phi_k)^2] under w ~ N(mu, diag(1/P)) (Monte Carlo, 4e5 draws)."""
    rng = np.random.default_rng(7)
    M, K = 6, 5
    rows = []
    for k in range(K):
        idx = np.sort(rng.choice(M, size=3, replace=False))
        rows.append((idx, rng.uniform(0.1, 1.0, 3)))
    t = rng.integers(0, 2, K)
    mu0, P0 = rng.normal(0, 0.5, M), rng.uniform(0.5, 2.0, M)
    mu1, P1, _ = bhm.em_diag(rows, t, mu0, P0, 0.0, 1)
    _, _, xi2 = bhm.em_diag(rows, t, mu0, P0, 0.0, 2)
    w = mu1[None, :] + rng.standard_normal((400_000, M)) / np.sqrt(P1)[None, :]
    for k, (idx, ph) in enumerate(rows):
        r = w[:, idx] @ ph
        est, se = np.mean(r * r), np.std(r * r) / math.sqrt(len(r))
        assert abs(xi2[k] ** 2 - est) < 4 * se + 1e-12, (k, xi2[k] ** 2, est)


def test_sequential_updates_equal_one_batch_at_fixed_xi():
    """With one E-step round at a fixed xi the update is conjugate: D1 then D2 equals D1 u D2 at once."""
    rng = np.random.default_rng(8)
    M = 5

    def make(K):
        rows = [(np.sort(rng.choice(M, size=2, replace=False)), rng.uniform(0.1, 1.0, 2)) for _ in range(K)]
        return rows, rng.integers(0, 2, K)

    r1, t1 = make(6)
    r2, t2 = make(9)
    mu0, P0 = rng.normal(0, 1, M), rng.uniform(0.5, 2.0, M)
    m1, p1, _ = bhm.em_diag(r1, t1, mu0, P0, 0.7, 1)
    m2, p2, _ = bhm.em_diag(r2, t2, m1, p1, 0.7, 1)
    mb, pb, _ = bhm.em_diag(r1 + r2, np.concatenate([t1, t2]), mu0, P0, 0.7, 1)
    assert np.allclose(p2, pb, rtol=1e-14, atol=0) and np.allclose(m2, mb, rtol=1e-12, atol=1e-14)


def test_diagonal_precision_is_the_diagonal_of_the_full_update():
    """P_t = diag(P_{t-1} + Phi^T diag(c) Phi) (App. A's precision update restricted to its diagonal), the full
    matrix formed here by a dense product."""
    rng = np.random.default_rng(9)
    M, K = 7, 11
    Phi = np.zeros((K, M))
    rows = []
    for k in range(K):
        idx = np.sort(rng.choice(M, size=3, replace=False))
        ph = rng.uniform(0.05, 1.0, 3)
        Phi[k, idx] = ph
        rows.append((idx, ph))
    t = rng.integers(0, 2, K)
    P0 = rng.uniform(0.5, 2.0, M)
    _, P, _ = bhm.em_diag(rows, t, np.zeros(M), P0, 0.0, 1)
    full = np.diag(P0) + Phi.T @ np.diag(np.full(K, 0.25)) @ Phi
    assert np.allclose(P, np.diag(full), rtol=1e-14, atol=0)
    # and the mean is the diagonal solve of the natural parameter
    mu, _, _ = bhm.em_diag(rows, t, np.zeros(M), P0, 0.0, 1)
    assert np.allclose(mu * P, Phi.T @ (t - 0.5), rtol=1e-13, atol=1e-15)


def _tiny_map(P=None, seed=3, n=60):
    P = P or bhm.BHMParams()
    o = bhm.BHMOracle(P)
    rng = np.random.default_rng(seed)
    p = np.array([0.3, 0.2, 1.8])
    ang = rng.uniform(0, 2 * np.pi, n)
    r = np.sqrt(rng.uniform(1.0, 4.0, n))
    hits = np.stack([p[0] + r * np.cos(ang), p[1] + r * np.sin(ang), rng.normal(0, 0.02, n)], 1)
    o.update(p, hits)
    return o, p, hits


def test_features_match_brute_force_threshold():
    """The kept hinges are those with exp(-gamma |x - x~|^2) >= phi_min (brute force over a wide window), and
    each value is that exponential."""
    o, _, _ = _tiny_map()
    P = o.P
    rng = np.random.default_rng(11)
    keys = list(o.slot)
    for _ in range(40):
        b = keys[int(rng.integers(len(keys)))]
        x = tuple((b[a] + rng.uniform(0, 1)) * P.block_hinges * P.hinge_spacing + P.origin[a] for a in range(3))
        u = o.lattice(x)
        got = {g: phi for _, phi, g in o.features_u(u, x) if g is not None}
        g0 = [math.floor(u[a]) for a in range(3)]
        want = {}
        for dz in range(-6, 7):
            for dy in range(-6, 7):
                for dx in range(-6, 7):
                    g = (g0[0] + dx, g0[1] + dy, g0[2] + dz)
                    if o.weight_of_hinge(g) is None:
                        continue
                    r2 = sum((x[a] - (P.origin[a] + g[a] * P.hinge_spacing)) ** 2 for a in range(3))
                    v = math.exp(-P.gamma * r2)
                    if abs(v / P.phi_min - 1.0) < 1e-6:
                        got.pop(g, None)  # on the threshold: either decision is right
                        continue
                    if v >= P.phi_min:
                        want[g] = v
        assert set(got) == set(want)
        for g, v in want.items():
            assert abs(got[g] - v) <= 1e-15 * max(1.0, v)


def test_samples_lie_on_the_ray_at_the_free_step():
    """With every block active, ray j has floor((L - gap) / step) free samples at distance j step from the
    sensor on the segment, then its hit; samples in inactive blocks are dropped and no others."""
    P = bhm.BHMParams()
    o = bhm.BHMOracle(P)
    p = (0.31, 0.22, 1.8)
    hits = np.array([[3.1, 0.4, 0.01], [0.2, -2.7, 0.3], [1.0, 1.0, -0.4]])
    for xh in hits:  # make every block along the rays active
        for s in np.linspace(0.0, 1.0, 400):
            x = np.asarray(p) + s * (xh - np.asarray(p))
            b = o.block_of_u(o.lattice(x))
            o._alloc(b)
            o.active[o.slot[b]] = True
    smp = o.samples(p, hits)
    k = 0
    for xh in hits:
        L = float(np.linalg.norm(xh - np.asarray(p)))
        n = int(math.floor((L - P.free_gap) / P.free_step))
        d = (xh - np.asarray(p)) / L
        for j in range(1, n + 1):
            u, x, t = smp[k]
            assert t == 0
            want = np.asarray(p) + j * P.free_step * d
            assert np.max(np.abs(np.asarray(x) - want)) < 1e-8  # fixed-point stepping: 2^-32 j hinge spacings
            k += 1
        assert smp[k][2] == 1 and np.array_equal(np.asarray(smp[k][1]), xh)
        k += 1
    assert k == len(smp)
    # deactivate one block: exactly the samples inside it disappear
    drop = o.block_of_u(smp[3][0])
    o.active[o.slot[drop]] = False
    smp2 = o.samples(p, hits)
    kept = [s for s in smp if s[2] == 1 or o.block_of_u(s[0]) != drop]
    assert len(smp2) == len(kept)
    assert all(np.array_equal(a[0], b[0]) for a, b in zip(smp2, kept))


def test_gradient_matches_finite_differences():
    o, _, hits = _tiny_map()
    rng = np.random.default_rng(12)
    P = o.P
    bsz = P.block_hinges * P.hinge_spacing
    n_ok = 0
    for k in range(40):
        x = hits[k % len(hits)] + rng.normal(0, 0.1, 3)
        if np.any(np.abs((x / bsz) - np.round(x / bsz)) * bsz < 1e-3):
            continue  # a block face: the bias jumps there
        l, g, _ = o.eval_u(o.lattice(x), tuple(x))
        e = 1e-6
        fd = np.zeros(3)
        for a in range(3):
            xp, xm = x.copy(), x.copy()
            xp[a] += e
            xm[a] -= e
            fd[a] = (o.eval_u(o.lattice(xp), tuple(xp))[0] - o.eval_u(o.lattice(xm), tuple(xm))[0]) / (2 * e)
        assert np.max(np.abs(fd - g)) <= 1e-5 * max(1.0, np.max(np.abs(g))), (k, fd, g)
        n_ok += 1
    assert n_ok > 30


def test_probit_occupancy_matches_monte_carlo():
    """P(occupied) ~ sigmoid(l / sqrt(1 + pi/8 phi^T Sigma phi)) (App. B) is within 0.02 of E[sigmoid(w^T phi)]
    under the posterior (Monte Carlo over the weights); with no posterior variance it is sigmoid(l)."""
    o, _, hits = _tiny_map(bhm.BHMParams(prior_var=4.0))
    rng = np.random.default_rng(13)
    xq = hits[:12] + rng.normal(0, 0.05, (12, 3))
    L, S, G, Pr = o.query(xq)
    for k in range(len(xq)):
        f = o.features_u(o.lattice(xq[k]), tuple(xq[k]))
        mu = np.array([o.mu[s][i] for (s, i), _, _ in f])
        sd = np.array([1.0 / math.sqrt(o.prec[s][i]) for (s, i), _, _ in f])
        ph = np.array([phi for _, phi, _ in f])
        w = mu[None, :] + rng.standard_normal((100_000, len(mu))) * sd[None, :]
        mc = np.mean(bhm.sigmoid(w @ ph))
        assert abs(Pr[k] - mc) < 0.02, (k, Pr[k], mc)
        assert abs(L[k] - mu @ ph) < 1e-12
        assert S[k] == (1 if L[k] < o.tau else -1)


def test_tau_moving_average():
    """alpha = 1: tau is the mean log-odds of the update's hits after the update; alpha = 1/2 over two updates:
    tau_2 = (tau_1 + mean_2) / 2."""
    o, p, hits = _tiny_map(bhm.BHMParams(tau_alpha=1.0))
    L, _, _, _ = o.query(hits)
    assert abs(o.tau - np.mean(L)) < 1e-12
    o2, p, hits = _tiny_map(bhm.BHMParams(tau_alpha=0.5, tau_init=0.3))
    L1, _, _, _ = o2.query(hits)
    assert abs(o2.tau - (0.5 * 0.3 + 0.5 * np.mean(L1))) < 1e-12
    t1 = o2.tau
    h2 = hits[::-1] + 0.01
    o2.update(p, h2)
    L2, _, _, _ = o2.query(h2)
    assert abs(o2.tau - (0.5 * t1 + 0.5 * np.mean(L2))) < 1e-12


def test_marked_edges_brute_force():
    """The edge set is every (node, axis) edge one of whose four adjacent cells is marked, each once; marked
    cells are the hit cells dilated by one."""
    o, _, hits = _tiny_map(n=20)
    m = o.P.march_sub
    cells = set()
    for xh in hits:
        u = o.lattice(xh)
        c = [math.floor(u[a] * m) for a in range(3)]
        for d in np.ndindex(3, 3, 3):
            cells.add(tuple(c[a] + d[a] - 1 for a in range(3)))
    assert cells == o.marked
    lo = np.min(np.array(list(cells)), axis=0)
    hi = np.max(np.array(list(cells)), axis=0) + 1
    want = set()
    for nu in np.ndindex(*(hi - lo + 1)):
        nu = tuple(int(nu[a] + lo[a]) for a in range(3))
        for a in range(3):
            b, c = [x for x in range(3) if x != a]
            for ib in (0, 1):
                for ic in (0, 1):
                    cell = list(nu)
                    cell[b] -= ib
                    cell[c] -= ic
                    if tuple(cell) in cells:
                        want.add((nu, a))
    assert want == o.marked_edges()


def test_march_points_cross_the_level_set():
    """Each point lies on its edge, between two nodes on opposite sides of tau, at the linear interpolation;
    every crossing edge gives a point; the normal is -grad l / |grad l|; keys ascend."""
    o, _, _ = _tiny_map(n=25)
    X, V, N, K = o.march()
    assert len(X) > 10
    assert K == sorted(K)
    m, h = o.P.march_sub, o.P.hinge_spacing
    crossing = 0
    for nu, a in o.marked_edges():
        nv = list(nu)
        nv[a] += 1
        la = o.eval_u(o.node_u(nu))[0]
        lb = o.eval_u(o.node_u(tuple(nv)))[0]
        crossing += (la >= o.tau) != (lb >= o.tau)
    assert crossing == len(X)
    for k in range(len(X)):
        nz, ny, nx, a = K[k]
        nu = (nx, ny, nz)
        x0 = np.array([o.P.origin[i] + nu[i] * h / m for i in range(3)])
        d = X[k] - x0
        other = [i for i in range(3) if i != a]
        assert np.all(np.abs(d[other]) < 1e-12) and -1e-12 <= d[a] <= h / m + 1e-12
        nv = list(nu)
        nv[a] += 1
        la = o.eval_u(o.node_u(nu))[0]
        lb = o.eval_u(o.node_u(tuple(nv)))[0]
        assert abs(d[a] / (h / m) - (o.tau - la) / (lb - la)) < 1e-9
        l, g, _ = o.eval_u(o.lattice(X[k]), tuple(X[k]))
        assert np.allclose(N[k], -g / np.linalg.norm(g), atol=1e-9)
        assert abs(V[k] - o.P.beta * (o.tau - l) ** 2 / (g @ g)) <= 1e-9 * max(V[k], 1e-12)


def test_scanned_plane_gives_an_upward_surface_at_the_ground():
    """A sensor 1.8 m above the plane z = 0: points above the ground are free (sign +1), points below occupied
    (-1); the extracted surface lies within a few centimetres of z = 0 with normals pointing up."""
    P = bhm.BHMParams(tau_alpha=1.0)
    o = bhm.BHMOracle(P)
    rng = np.random.default_rng(21)
    p = np.array([0.3, 0.2, 1.8])
    n = 700
    ang = rng.uniform(0, 2 * np.pi, n)
    r = np.sqrt(rng.uniform(4.0, 9.0, n))
    hits = np.stack([p[0] + r * np.cos(ang), p[1] + r * np.sin(ang), rng.normal(0, 0.02, n)], 1)
    o.update(p, hits)
    q = np.array([[p[0] + 2.5 * math.cos(a), p[1] + 2.5 * math.sin(a), z] for a in (0.3, 2.0, 4.0)
                  for z in (0.3, 0.5, -0.3, -0.5)])
    _, S, _, _ = o.query(q)
    assert list(S) == [1, 1, -1, -1] * 3
    X, V, N, _ = o.march()
    core = np.hypot(X[:, 0] - p[0], X[:, 1] - p[1])
    sel = (core > 2.2) & (core < 2.8)
    assert sel.sum() > 50
    assert abs(np.median(X[sel, 2])) < 0.08
    assert np.median(N[sel, 2]) > 0.9


def test_surface_variance_is_the_first_order_distance_to_the_level_set():
    """Eq. surface_point_uncertainty comes from a first-order Taylor step: sqrt(sigma^2 / beta) = |tau - l(x_i)| /
    |grad l(x_i)| is the distance from x_i to the tau level set along the gradient.  Found here by bisection on the
    field itself (bias off, so the field has no jumps at block faces); the rest is the field's curvature, second
    order in sigma."""
    P = bhm.BHMParams(tau_alpha=1.0, bias_feature=0, beta=2.0)
    o = bhm.BHMOracle(P)
    rng = np.random.default_rng(21)
    p = np.array([0.3, 0.2, 1.8])
    n = 400
    ang = rng.uniform(0, 2 * np.pi, n)
    r = np.sqrt(rng.uniform(4.0, 9.0, n))
    hits = np.stack([p[0] + r * np.cos(ang), p[1] + r * np.sin(ang), rng.normal(0, 0.02, n)], 1)
    o.update(p, hits)
    X, V, _, _ = o.march()
    rel = []
    for k in range(0, len(X), 9):
        x = X[k]
        _, g, _ = o.eval_u(o.lattice(x), tuple(x))
        d = g / np.linalg.norm(g)
        sig = math.sqrt(V[k] / P.beta)
        if not 1e-5 < sig < 0.02:
            continue
        f = lambda t: o.eval_u(o.lattice(x + t * d), tuple(x + t * d))[0] - o.tau  # noqa: E731
        lo, hi = -3 * sig - 1e-4, 3 * sig + 1e-4
        assert f(lo) * f(hi) <= 0
        for _ in range(40):
            mid = 0.5 * (lo + hi)
            if f(lo) * f(mid) <= 0:
                hi = mid
            else:
                lo = mid
        rel.append(abs(abs(0.5 * (lo + hi)) - sig) / sig)
    assert len(rel) > 40
    assert np.median(rel) < 0.02 and np.quantile(rel, 0.9) < 0.1, (np.median(rel), np.quantile(rel, 0.9))
