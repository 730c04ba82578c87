"""GPU parity of the BHM front-end (include/ksdf_bhm.h) with the binary64 oracle (oracle/bhm.py) on frames of the
city scan: blocks, active flags and the sample count exactly; weights, threshold, log-odds, gradient and occupancy
within the binary32 bound below; the sign and the marched edge set exactly wherever the oracle's values are
farther from tau than that bound; the surface points within the bound propagated through the interpolation.

Tolerance.  The GPU forms each feature as a product of three binary32 exponentials of binary32 arguments
(relative error a few 2^-24 each) and sums and accumulates in binary32 (sums of up to ~10^3 terms, atomics in
no fixed order).  A quantity that is a sum of terms t_i is therefore within c * sum |t_i| of the binary64 value
with c of order 10^3 2^-24 ~ 6e-5 at worst; the tests use c = 2e-4 on the magnitude sums the oracle reports."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

C_REL = 2e-4


@pytest.fixture(scope="module")
def dev():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2603_29227_gb300 import build

    build.build()
    return torch.device("cuda:0")


def _oracle(params):
    from oracle import bhm as ob

    return ob.BHMOracle(ob.BHMParams(**params))


def _unpack_block(k):
    k = int(k)
    b = 1 << 20
    return ((k & 0x1FFFFF) - b, ((k >> 21) & 0x1FFFFF) - b, ((k >> 42) & 0x1FFFFF) - b)


def _mags(o, x):
    """(sum |mu phi| + |bias|, 2 gamma sum |mu phi| |x - x~|) of the oracle at point x: magnitude sums that bound
    the binary32 error of l and grad l."""
    P = o.P
    f = o.features_u(o.lattice(x), tuple(x))
    sl, sg = 0.0, 0.0
    for (s, i), phi, g in f:
        t = abs(o.mu[s][i] * phi)
        sl += t
        if g is not None:
            d = math.sqrt(sum((x[a] - (P.origin[a] + g[a] * P.hinge_spacing)) ** 2 for a in range(3)))
            sg += 2.0 * P.gamma * t * d
    return sl, sg


def _compare_maps(o, m):
    keys, act, mu, prec = m.weights()
    blocks = {_unpack_block(k): s for s, k in enumerate(keys)}
    assert set(blocks) == set(o.slot), "allocated block sets differ"
    for b, s in blocks.items():
        so = o.slot[b]
        assert bool(act[s]) == o.active[so], b
        Po, mo = o.prec[so], o.mu[so]
        assert np.all(np.abs(prec[s] - Po) <= C_REL * Po), b
        # mu = (P0 mu0 + B) / P: bounded by the magnitude of its numerator over P, and by mu's own rounding
        tol = C_REL * (o.mag[so] + np.abs(mo)) + 1e-7
        assert np.all(np.abs(mu[s] - mo) <= tol), (b, np.max(np.abs(mu[s] - mo) - tol))


def _frame(n_hits, f=0, radius=10.0, seed=0):
    from paper_2603_29227_gb300 import scenes

    city = scenes.make_city()
    return scenes.city_bhm_frame(city, f, radius=radius, max_hits=n_hits, seed=seed)


def _params(**kw):
    from paper_2603_29227_gb300 import scenes

    return dict(scenes.CITY_BHM, **kw)


@pytest.fixture(scope="module")
def two_frames(dev):
    """Two frames (poses 0 and 1) through the oracle and the GPU map, with snapshots after each."""
    import torch
    from paper_2603_29227_gb300 import bhm

    P = _params()
    o = _oracle(P)
    m = bhm.BHMap(P, max_blocks=20000)
    snaps = []
    for f in (0, 1):
        p, hits = _frame(1200, f=f)
        o.update(p, hits)
        m.update(p, torch.from_numpy(hits).to(dev))
        m.sync_status()
        nb, ns, nf = m.size(features=True)
        assert nf == o.last_features  # the kept-feature decisions are exact
        snaps.append((p, hits, ns, o.last_samples, m.tau, o.tau))
        if f == 0:
            _compare_maps(o, m)  # after the first frame
    return o, m, snaps


def test_update_blocks_samples_weights_tau(two_frames):
    o, m, snaps = two_frames
    sl_max = 0.0
    for p, hits, ns_gpu, ns_oracle, tau_gpu, tau_oracle in snaps:
        assert ns_gpu == ns_oracle
        # tau is a moving average of hit log-odds: within the largest of their bounds
        sl_max = max(sl_max, max(_mags(o, h)[0] for h in hits[::5]))
        assert abs(tau_gpu - tau_oracle) <= 2 * C_REL * sl_max + 1e-7, (tau_gpu, tau_oracle)
    _compare_maps(o, m)


def test_query_logodds_sign_grad_prob(two_frames, dev):
    import torch

    o, m, snaps = two_frames
    p, hits, *_ = snaps[-1]
    rng = np.random.default_rng(3)
    xq = np.concatenate([hits[::7] + rng.normal(0, 0.15, (len(hits[::7]), 3)),
                         p + rng.uniform(-8, 8, (200, 3)) * np.array([1, 1, 0.2])]).astype(np.float32)
    out = m.query(torch.from_numpy(xq).to(dev))
    got = {k: v.cpu().numpy() for k, v in out.items()}
    L, S, G, Pr = o.query(xq.astype(np.float64))
    tau = o.tau
    dtau = abs(m.tau - tau)
    n_sign = 0
    for k in range(len(xq)):
        sl, sg = _mags(o, xq[k].astype(np.float64))
        tl = C_REL * sl + 1e-6
        assert abs(got["logodds"][k] - L[k]) <= tl, (k, got["logodds"][k], L[k])
        assert np.max(np.abs(got["grad"][k] - G[k])) <= C_REL * sg + 1e-5, (k, got["grad"][k], G[k])
        assert abs(got["prob"][k] - Pr[k]) <= (tl + C_REL * abs(L[k])) / 4 + 1e-6, (k, got["prob"][k], Pr[k])
        if abs(L[k] - tau) > tl + dtau:
            assert got["sign"][k] == S[k], k
            n_sign += 1
        else:
            assert got["sign"][k] == (1 if got["logodds"][k] < m.tau else -1)
    assert n_sign > 0.95 * len(xq)


@pytest.mark.parametrize("march_sub", [2, 4])
def test_march_parity(dev, march_sub):
    import torch
    from paper_2603_29227_gb300 import bhm

    P = _params(march_sub=march_sub)
    p, hits = _frame(300 if march_sub == 2 else 120, f=2, radius=9.0, seed=1)
    o = _oracle(P)
    o.update(p, hits)
    m = bhm.BHMap(P, max_blocks=20000)
    m.update(p, torch.from_numpy(hits).to(dev))
    x, var, nrm, keys = m.march(device=dev)
    m.sync_status()
    x, var, nrm = x.cpu().numpy(), var.cpu().numpy(), nrm.cpu().numpy()
    keys = keys.cpu().numpy().view(np.uint64)
    assert np.all(keys[1:] > keys[:-1])  # ascending, unique
    X, V, N, K = o.march()
    B = 1 << 19
    ko = np.array([((k[0] + B) << 42) | ((k[1] + B) << 22) | ((k[2] + B) << 2) | k[3] for k in K], dtype=np.uint64)
    gi = {int(k): i for i, k in enumerate(keys)}
    oi = {int(k): i for i, k in enumerate(ko)}
    tau = o.tau
    dtau = abs(m.tau - tau)
    m_ = o.P.march_sub
    h = o.P.hinge_spacing
    decided, matched = 0, 0
    for nu, a in o.marked_edges():
        nv = list(nu)
        nv[a] += 1
        ua, ub = o.node_u(nu), o.node_u(tuple(nv))
        la, lb = o.eval_u(ua)[0], o.eval_u(ub)[0]
        xa = tuple(o.P.origin[i] + ua[i] * h for i in range(3))
        xb = tuple(o.P.origin[i] + ub[i] * h for i in range(3))
        ta = C_REL * _mags(o, np.array(xa))[0] + 1e-6 + dtau
        tb = C_REL * _mags(o, np.array(xb))[0] + 1e-6 + dtau
        key = int(((nu[2] + B) << 42) | ((nu[1] + B) << 22) | ((nu[0] + B) << 2) | a)
        if abs(la - tau) <= ta or abs(lb - tau) <= tb:
            continue  # the binary32 side may decide this edge either way
        decided += 1
        assert (key in gi) == (key in oi), (nu, a, la, lb, tau)
        if key not in oi:
            continue
        i, j = oi[key], gi[key]
        matched += 1
        # position along the edge: t = (tau - la) / (lb - la), each l within its bound
        dt = (ta + tb) / abs(lb - la) * (1.0 + 1e-3)
        assert np.max(np.abs(x[j] - X[i])) <= dt * h / m_ + 1e-9, (key, x[j], X[i])
        sl, sg = _mags(o, X[i])
        l, g, _ = o.eval_u(o.lattice(X[i]), tuple(X[i]))
        gnorm = float(np.linalg.norm(g))
        # the gradient moves with the point (second derivatives ~ 2 gamma |grad l|) and by its own rounding
        dxp = dt * h / m_
        tg = C_REL * sg + 1e-5 + 2.0 * o.P.gamma * (sl + gnorm) * dxp
        dl = C_REL * sl + 1e-6 + gnorm * dxp + tg * dxp
        sig_o = math.sqrt(V[i])
        sig_g = math.sqrt(float(var[j]))
        bound = (dl + abs(tau - l) * tg / gnorm) / max(gnorm - tg, 1e-3 * gnorm) * math.sqrt(o.P.beta) + 1e-7
        assert abs(sig_g - sig_o) <= bound, (key, sig_g, sig_o, bound)
        assert np.max(np.abs(nrm[j] - N[i])) <= 2.0 * tg / gnorm + 1e-6, (key, nrm[j], N[i])
    assert decided > 100 and matched > 50
    assert abs(len(keys) - len(ko)) <= max(5, 0.02 * len(ko))


def test_edge_cases(dev):
    """R = 0, NaN hits, a capacity overflow, queries far from every block, and EM rounds 1 and 3 with xi_0 = 1."""
    import torch
    from paper_2603_29227_gb300 import bhm, ksdf

    P = _params()
    m = bhm.BHMap(P, max_blocks=20000)
    p, hits = _frame(200, f=3, radius=8.0)
    # no hits: nothing happens, tau unchanged
    m.update(p, torch.zeros((0, 3), dtype=torch.float64, device=dev))
    m.sync_status()
    assert m.size() == (0, 0) and m.tau == P["tau_init"]
    x, _, _, _ = m.march()
    assert len(x) == 0
    # a NaN hit is reported and skipped; the rest matches an oracle run without it
    bad = hits.copy()
    bad[5] = np.nan
    m.update(p, torch.from_numpy(bad).to(dev))
    with pytest.raises(ksdf.KsdfError) as e:
        m.sync_status()
    assert e.value.status == ksdf.KSDF_ERR_NONFINITE
    o = _oracle(P)
    o.update(p, np.delete(hits, 5, axis=0))
    keys, act, _, _ = m.weights()
    assert {_unpack_block(k) for k in keys} == set(o.slot)
    # far from any block: log-odds 0, probability 1/2, gradient 0
    q = m.query(torch.tensor([[p[0] + 500.0, p[1], 0.5]], dtype=torch.float32, device=dev))
    assert float(q["logodds"][0]) == 0.0 and abs(float(q["prob"][0]) - 0.5) < 1e-7
    assert torch.all(q["grad"] == 0)
    # capacity: too few blocks
    small = bhm.BHMap(P, max_blocks=10)
    small.update(p, torch.from_numpy(hits).to(dev))
    with pytest.raises(ksdf.KsdfError) as e:
        small.sync_status()
    assert e.value.status == ksdf.KSDF_ERR_CAPACITY
    assert small.size()[0] == 10
    # other EM schedules, and no bias feature, against the oracle
    for iters, xi0, bias in ((1, 0.0, 1), (3, 1.0, 1), (2, 0.0, 0)):
        Pq = _params(em_iters=iters, xi_init=xi0, bias_feature=bias)
        o = _oracle(Pq)
        o.update(p, hits)
        mm = bhm.BHMap(Pq, max_blocks=20000)
        mm.update(p, torch.from_numpy(hits).to(dev))
        mm.sync_status()
        _compare_maps(o, mm)
        assert abs(mm.tau - o.tau) <= C_REL * (1.0 + abs(o.tau)) * 10


def test_invalid_query_point(dev):
    import torch
    from paper_2603_29227_gb300 import bhm, ksdf

    m = bhm.BHMap(_params(), max_blocks=100)
    q = m.query(torch.tensor([[float("nan"), 0.0, 0.0], [1e9, 0.0, 0.0]], dtype=torch.float32, device=dev))
    assert torch.all(torch.isnan(q["logodds"])) and torch.all(q["sign"] == 1)
    with pytest.raises(ksdf.KsdfError) as e:
        m.sync_status()
    assert e.value.status == ksdf.KSDF_ERR_NONFINITE


def test_front_end_feeds_the_back_end(dev):
    """The paper's pipeline on three city frames: BHM update, surface points with their variance, the GP fit on
    those points, and the SDF query signed by the BHM.  Points the scans saw to be free -- on a ray at least half
    a metre before its hit, above the ground, in an active block -- are free for the BHM sign and have a positive
    SDF."""
    import torch
    from paper_2603_29227_gb300 import bhm, ksdf, scenes

    city = scenes.make_city()
    P = _params()
    m = bhm.BHMap(P, max_blocks=200000)
    pts, vs = [], []
    for f in range(3):
        p, hits = scenes.city_bhm_frame(city, f, radius=15.0)
        m.update(p, torch.from_numpy(hits).to(dev))
        x, var, _, _ = m.march(device=dev)
        pts.append(x)
        vs.append(var)
    m.sync_status()
    x = torch.cat(pts)
    var = torch.cat(vs)
    assert len(x) > 10000 and torch.all(var >= 0)
    gp = ksdf.KernelSDF(dict(city.params, sign_mode=0))
    gp.fit(x, var, None)
    rng = np.random.default_rng(4)
    sel = rng.choice(len(hits), size=20000, replace=False)
    s = rng.uniform(0.2, 0.9, len(sel))[:, None]
    xf = p + s * (hits[sel] - p)
    keep = (np.linalg.norm(hits[sel] - xf, axis=1) > 0.5) & (xf[:, 2] > 0.3)
    keys, act, _, _ = m.weights()
    active = {_unpack_block(k) for k, a in zip(keys, act) if a}
    nh, h = P["block_hinges"], P["hinge_spacing"]
    blk = np.floor(np.floor(xf / h) / nh).astype(np.int64)
    keep &= np.array([tuple(b) in active for b in blk])
    xq = torch.from_numpy(xf[keep].astype(np.float32)).to(dev)
    assert len(xq) > 1000
    sgn = m.query(xq, bhm.BHM_SIGN)["sign"]
    free_bhm = float((sgn == 1).float().mean())
    o = gp.query(xq, sgn)
    pos = float((o["sdf"] > 0).float().mean())
    assert free_bhm > 0.97 and pos > 0.97, (free_bhm, pos)


def test_full_frame_properties(dev):
    """A whole city frame (~125k hits, ~2.3M samples), checked by properties that hold at any size: tau is the
    moving average of the hits' log-odds (queried back from the map), the sign is l < tau, and every surface point
    sits on its edge between nodes on opposite sides of tau, with the variance and normal of the field there."""
    import torch
    from paper_2603_29227_gb300 import bhm, scenes

    city = scenes.make_city()
    P = _params()
    p, hits = scenes.city_bhm_frame(city, 0)
    assert len(hits) > 100000
    m = bhm.BHMap(P, max_blocks=60000)
    m.update(p, torch.from_numpy(hits).to(dev))
    x, var, nrm, keys = m.march(device=dev)
    m.sync_status()
    nb, ns, nf = m.size(features=True)
    assert ns > 2_000_000 and nf > 40 * ns
    tau = m.tau
    # tau = (1 - alpha) tau0 + alpha mean l(hits): the query's binary32 log-odds at the binary32-rounded hits
    q = m.query(torch.from_numpy(hits.astype(np.float32)).to(dev), bhm.BHM_LOGODDS | bhm.BHM_SIGN)
    lh = q["logodds"].double().cpu().numpy()
    want = (1 - P["tau_alpha"]) * P["tau_init"] + P["tau_alpha"] * lh.mean()
    assert abs(tau - want) <= 1e-3 * (1.0 + np.abs(lh).mean()), (tau, want)
    sg = q["sign"].cpu().numpy()
    far = np.abs(lh - tau) > 1e-4 * (1 + np.abs(lh))
    assert np.all(sg[far] == np.where(lh[far] < tau, 1, -1))
    # surface points
    n = len(x)
    assert n > 50000
    rng = np.random.default_rng(5)
    sel = torch.from_numpy(rng.choice(n, size=4000, replace=False)).to(dev)
    xs = x[sel].cpu().numpy()
    ks = keys[sel].cpu().numpy().view(np.uint64).astype(np.uint64)
    vs = var[sel].double().cpu().numpy()
    ns_ = nrm[sel].double().cpu().numpy()
    B = np.uint64(1 << 19)
    M20 = np.uint64((1 << 20) - 1)
    axis = (ks & np.uint64(3)).astype(np.int64)
    nu = np.stack([((ks >> np.uint64(2)) & M20), ((ks >> np.uint64(22)) & M20), ((ks >> np.uint64(42)) & M20)], 1)
    nu = nu.astype(np.int64) - int(B)
    step = P["hinge_spacing"] / P["march_sub"]
    x0 = nu * step
    d = xs - x0
    onax = d[np.arange(len(d)), axis]
    d[np.arange(len(d)), axis] = 0.0
    assert np.all(np.abs(d) < 1e-9) and np.all(onax >= -1e-9) and np.all(onax <= step + 1e-9)
    x1 = x0.copy()
    x1[np.arange(len(x1)), axis] += step
    la = m.query(torch.from_numpy(x0.astype(np.float32)).to(dev), bhm.BHM_LOGODDS)["logodds"].double().cpu().numpy()
    lb = m.query(torch.from_numpy(x1.astype(np.float32)).to(dev), bhm.BHM_LOGODDS)["logodds"].double().cpu().numpy()
    # binary32 query points can fall across a block face (another bias) or a feature threshold (a jump of about
    # 1e-3 |mu|): leave out points on block faces and values within a margin of tau
    C = P["block_hinges"] * P["march_sub"]
    face = np.any(nu % C == 0, axis=1) | ((nu[np.arange(len(nu)), axis] + 1) % C == 0)
    sure = ~face & (np.abs(la - tau) > 0.05 + 1e-3 * np.abs(la)) & (np.abs(lb - tau) > 0.05 + 1e-3 * np.abs(lb))
    assert sure.sum() > 1000
    assert np.all((la[sure] >= tau) != (lb[sure] >= tau))
    qi = m.query(torch.from_numpy(xs.astype(np.float32)).to(dev), bhm.BHM_LOGODDS | bhm.BHM_GRAD)
    li = qi["logodds"].double().cpu().numpy()
    gi = qi["grad"].double().cpu().numpy()
    gn = np.linalg.norm(gi, axis=1)
    ok = (gn > 1e-2 * np.median(gn)) & ~face
    # binary32 positions move the field by about |grad l| 1e-5 m (and, rarely, across a feature threshold);
    # sigma = sqrt(beta) |tau - l| / |grad l|, the normal -grad l / |grad l|
    sig_q = np.sqrt(P["beta"]) * np.abs(tau - li) / gn
    good = np.abs(np.sqrt(vs[ok]) - sig_q[ok]) <= 1e-3 * (1 + sig_q[ok]) + 2e-5
    assert good.mean() > 0.99, good.mean()
    goodn = np.max(np.abs(ns_[ok] + gi[ok] / gn[ok, None]), axis=1) < 1e-3
    assert goodn.mean() > 0.99, goodn.mean()


def test_edges_marked_and_persistent_surface_map(dev):
    """ksdf_bhm_edges_marked flags exactly the oracle's processed edges; and a GP buffer kept across frames by
    dropping the re-marched edges' points and appending the new march (ksdf_update_replace) holds one point per
    edge and equals a fresh fit of those points."""
    import torch
    from paper_2603_29227_gb300 import bhm, ksdf, scenes

    P = _params()
    p, hits = _frame(150, f=4, radius=8.0, seed=3)
    o = _oracle(P)
    o.update(p, hits)
    m = bhm.BHMap(P, max_blocks=20000)
    m.update(p, torch.from_numpy(hits).to(dev))
    B = 1 << 19
    edges = sorted(o.marked_edges())
    kin = np.array([((nu[2] + B) << 42) | ((nu[1] + B) << 22) | ((nu[0] + B) << 2) | a for nu, a in edges],
                   dtype=np.uint64)
    rng = np.random.default_rng(2)
    # other edges near them: shifted by a few cells
    sh = np.array([((nu[2] + 3 + B) << 42) | ((nu[1] - 2 + B) << 22) | ((nu[0] + 5 + B) << 2) | a
                   for nu, a in [edges[i] for i in rng.choice(len(edges), 500)]], dtype=np.uint64)
    marked = {int(k) for k in kin}
    keys = np.concatenate([kin, sh])
    got = m.edges_marked(keys)
    want = np.array([int(k) in marked for k in keys], dtype=np.uint8)
    assert np.array_equal(got, want)
    got_dev = m.edges_marked(torch.from_numpy(keys.view(np.int64)).to(dev)).cpu().numpy()
    assert np.array_equal(got_dev, want)

    # a persistent buffer over three city frames
    city = scenes.make_city()
    fm = bhm.BHMap(P, max_blocks=200000)
    gp = None
    gkeys = None
    for f in range(3):
        p, hits = scenes.city_bhm_frame(city, f, radius=12.0)
        fm.update(p, torch.from_numpy(hits).to(dev))
        x, var, _, k = fm.march(device=dev)
        if gp is None:
            gp = ksdf.KernelSDF(dict(city.params, sign_mode=0))
            gp.fit(x, var, None)
            gkeys, gx, gv = k.clone(), x.clone(), var.clone()
        else:
            drop = fm.edges_marked(gkeys)
            gp.update_replace(drop, x, var)
            kept = drop == 0
            gkeys = torch.cat([gkeys[kept], k])
            gx = torch.cat([gx[kept], x])
            gv = torch.cat([gv[kept], var])
    fm.sync_status()
    assert len(torch.unique(gkeys)) == len(gkeys)  # one point per edge
    assert gp.S == len(gx)
    fresh = ksdf.KernelSDF(dict(city.params, sign_mode=0))
    fresh.fit(gx.contiguous(), gv.contiguous(), None)
    a1, c1, _ = gp.fit_arrays()
    a2, c2, _ = fresh.fit_arrays()
    assert np.array_equal(a1, a2) and np.array_equal(c1, c2)
