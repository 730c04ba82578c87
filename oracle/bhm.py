"""CPU FP64 oracle of the Kernel-SDF front-end: the Bayesian Hilbert map (BHM) occupancy field with a diagonal
weight covariance, its sign and threshold, and the surface points it hands to the back-end (Sec. IV-A, App. A,
App. B of arXiv 2603.29227).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
may import this module.  It shares no code with the CUDA library; plain Python and numpy in binary64.

What it computes, in the paper's order and notation:

  Features (Sec. IV-A.1).  Hinge points x~_g = o + g h on the integer lattice g in Z^3 (spacing h), the RBF kernel
  k(x, x~) = exp(-gamma |x - x~|^2), and phi(x) = [k(x, x~_1), ..., k(x, x~_M), 1].  A feature is dropped when it is
  below the threshold phi_min (App. A, "practical optimization"; 1e-3 in the paper).

  Map layout (replaces the octree of local BHMs, Sec. IV-A.2).  The lattice is cut into blocks of n_h^3 hinges
  (block B owns the hinges g with floor(g / n_h) = B).  A block is *active* once a hit has fallen in it, and the
  26 blocks around an active block are *allocated* as well, so every hinge within reach of a sample in an active
  block has a weight.  Each block carries its own bias weight (the trailing 1 of phi): a point's bias is the one of
  the block it lies in.  One weight per hinge, shared by every sample that reaches it, so the weight sync of
  Sec. IV-A.2 has nothing left to do.  A new weight has the prior N(0, prior_var).

  Samples (Sec. IV-A.1, IV-A.2).  For a sensor position p and a hit x, the ray has length L = |x - p|; the free
  samples are x_j = p + s_j (x - p) for j = 1 .. floor((L - free_gap) / free_step), s_j = j free_step / L,
  labelled y = -1 (free) and kept when their block is active (the ray pruning of Sec. IV-A.2); the hit itself is
  an occupied sample, y = +1.  Rays are taken in input order, each ray's free samples before its hit.

  Update (App. A).  Sequential variational EM with the Jaakkola-Jordan bound, the weights' covariance kept
  diagonal (independent weights, Sec. IV-A.2), the label mapped to t = (y + 1) / 2 in {0, 1} for the E-step:
    E-step:  P_t = P_{t-1} + sum_k c(xi_k) phi_k^2,   mu_t = (P_{t-1} mu_{t-1} + sum_k (t_k - 1/2) phi_k) / P_t,
             with P = diag(Sigma)^{-1} and c(xi) = |(1/2 - sigmoid(xi)) / xi| (1/4 at xi = 0);
    M-step:  xi_k^2 = phi_k^T (Sigma_t + mu_t mu_t^T) phi_k = sum_m phi_km^2 / P_t,m + (mu_t^T phi_k)^2.
  em_iters rounds of E-step (with the current xi) then M-step, xi starting at xi_init; the last round's M-step is
  not needed.  (P_{t-1}, mu_{t-1}) is the map before this update, in every round.

  Threshold (eq. online_surf_logodds).  After the update, tau <- (1 - alpha) tau + (alpha / K) sum_k l(x_k) over
  the K hits of the update, where l(x) = mu^T phi(x).

  Sign (eq. sign_prediction).  s(x) = +1 when l(x) < tau, else -1.

  Occupancy and gradient (App. B).  P(occupied | x) ~ sigmoid(l / sqrt(1 + pi/8 phi^T Sigma phi)); the gradient of
  the log-odds grad l = sum_m mu_m phi_m(x) (-2 gamma) (x - x~_m); the normal n = -grad l / |grad l|.

  Surface points (Sec. IV-A.4).  Marching grid of spacing h / m (m = march_sub in {1, 2, 4, 8}): node nu at
  o + nu h / m, cell nu covering [nu, nu + 1) h / m.  The cells holding a hit of the last update, and their 26
  neighbours, are marked; every edge of a marked cell whose two nodes lie on different sides of the level set
  (one with l >= tau, the other with l < tau) gives one point, at the linear interpolation of l along the edge,
  with sigma^2 = beta (tau - l(x_i))^2 / |grad l(x_i)|^2 (eq. surface_point_uncertainty) and the normal above.
  Points where grad l = 0 are not emitted.  Points come out in ascending edge key (nu_z, nu_y, nu_x, axis).

Readings where the paper is silent or garbled:
  - The E-step writes y_k - 1/2 with y in {0, 1} while the samples carry y in {-1, 1}: read t = (y + 1) / 2.  The
    absolute value in the precision update is kept; it changes nothing, since (sigmoid(xi) - 1/2) / xi >= 0.
  - "Drop phi_m below 1e-3" is decided on the squared lattice distance d^2 = |u - g|^2 (u = (x - o) / h):
    phi_m is kept when floor-quantised d^2 <= ln(1 / phi_min) / (gamma h^2), both sides in units of 2^-40 (each
    coordinate's fraction u - floor(u) first truncated to 2^-20).  It equals phi_m >= phi_min up to that
    quantisation, and the GPU takes the same integer decision.
  - Lattice coordinates: u = (x - o) / h per axis in binary64 (subtraction, then division), g0 = floor(u),
    block = floor(g0 / n_h).  A free sample's lattice coordinates are stepped in 2^-32 fixed point, exactly, in
    integers: U_p = rint(2^32 u_p), U_x = rint(2^32 u_x), D = rint((U_x - U_p) (free_step / L)) per axis (binary64
    product, round half to even), U_j = U_p + j D and u_j = U_j / 2^32 -- within 2^-32 j hinge spacings of
    u_p + s_j (u_x - u_p).  The positions x_j = o + u_j h are only used for the kernel distances.
  - Marching cells: nu = floor(m u) per axis (m a power of two, so m u is exact).
  - The paper does not fix the prior, the free-sample spacing, the gap before the hit, alpha, beta or the
    marching resolution: they are parameters here.  The per-block bias can be switched off (bias_feature = 0):
    with it, a block whose samples are mostly free drags the log-odds of its unobserved interior down.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

Q20 = 1 << 20  # fixed-point scale of the lattice fraction


@dataclass
class BHMParams:
    origin: tuple = (0.0, 0.0, 0.0)
    hinge_spacing: float = 0.175   # h
    block_hinges: int = 8          # n_h: a block owns n_h^3 hinges
    gamma: float = 41.32           # k(r) = exp(-gamma r^2), gamma = 1 / (2 l^2)
    phi_min: float = 1e-3
    prior_var: float = 1.0
    em_iters: int = 2
    xi_init: float = 0.0
    free_step: float = 0.175
    free_gap: float = 0.1
    tau_alpha: float = 0.1
    tau_init: float = 0.0
    beta: float = 1.0
    march_sub: int = 2
    bias_feature: int = 1          # 1: the trailing 1 of phi, one bias weight per block; 0: no bias feature


def sigmoid(v):
    v = np.asarray(v, dtype=np.float64)
    return np.where(v >= 0, 1.0 / (1.0 + np.exp(-np.abs(v))), np.exp(-np.abs(v)) / (1.0 + np.exp(-np.abs(v))))


def jj_coef(xi):
    """c(xi) = |(1/2 - sigmoid(xi)) / xi| of the E-step precision update (App. A), its limit 1/4 at xi = 0."""
    xi = np.asarray(xi, dtype=np.float64)
    safe = np.where(xi == 0.0, 1.0, xi)
    return np.where(xi == 0.0, 0.25, np.abs((0.5 - sigmoid(safe)) / safe))


def r2_quantised(P: BHMParams) -> int:
    """Largest kept squared lattice distance, in units of 2^-40: floor(ln(1 / phi_min) / (gamma h^2) 2^40)."""
    return int(math.floor(math.log(1.0 / P.phi_min) / (P.gamma * P.hinge_spacing * P.hinge_spacing) * 2.0 ** 40))


def em_diag(rows, t, mu0, P0, xi0, iters):
    """Diagonal-covariance sequential EM of App. A on an explicit sparse design.

    rows: list of (idx int array, phi float array), the kept features of each sample (indices into the weight
    vector); t: labels in {0, 1}; (mu0, P0): prior mean and precision of every weight; xi0: initial xi; iters >= 1
    rounds.  Returns (mu, P, xi) with xi the one used by the last E-step."""
    mu0 = np.asarray(mu0, dtype=np.float64)
    P0 = np.asarray(P0, dtype=np.float64)
    K = len(rows)
    xi = np.full(K, float(xi0))
    idx = np.concatenate([r[0] for r in rows]) if K else np.zeros(0, dtype=np.int64)
    phi = np.concatenate([r[1] for r in rows]) if K else np.zeros(0)
    owner = np.repeat(np.arange(K), [len(r[0]) for r in rows]) if K else np.zeros(0, dtype=np.int64)
    tk = np.asarray(t, dtype=np.float64)
    B = np.zeros_like(mu0)
    np.add.at(B, idx, (tk[owner] - 0.5) * phi)
    for it in range(iters):
        if it > 0:  # M-step with the previous round's posterior
            var_term = np.zeros(K)
            np.add.at(var_term, owner, phi * phi / P[idx])
            mean_term = np.zeros(K)
            np.add.at(mean_term, owner, mu[idx] * phi)
            xi = np.sqrt(var_term + mean_term * mean_term)
        c = jj_coef(xi)
        P = P0.copy()
        np.add.at(P, idx, c[owner] * phi * phi)
        mu = (P0 * mu0 + B) / P
    return mu, P, xi


def _floor_div(a, b):
    return a // b  # Python integer floor division (rounds towards -inf)


@dataclass
class BHMOracle:
    P: BHMParams
    slot: dict = field(default_factory=dict)       # block key (bx, by, bz) -> slot
    keys: list = field(default_factory=list)       # slot -> block key
    active: list = field(default_factory=list)     # slot -> bool
    mu: list = field(default_factory=list)         # slot -> float64[n_h^3 + 1] (last = bias)
    prec: list = field(default_factory=list)       # slot -> float64[n_h^3 + 1]
    mag: list = field(default_factory=list)        # slot -> float64[n_h^3 + 1], see update()
    tau: float = 0.0
    marked: set = field(default_factory=set)       # marked cells of the last update
    last_samples: int = 0
    last_features: int = 0                          # kept hinge features (no bias) over the last update's samples

    def __post_init__(self):
        self.tau = float(self.P.tau_init)
        self.nw = self.P.block_hinges ** 3 + 1
        self.r2q = r2_quantised(self.P)
        self.rwin = int(math.isqrt(self.r2q) // Q20) + 1  # offsets tried: -rwin .. rwin + 1 (a superset)
        r = np.arange(-self.rwin, self.rwin + 2)
        dz, dy, dx = np.meshgrid(r, r, r, indexing="ij")
        self._offsets = np.stack([dx.ravel(), dy.ravel(), dz.ravel()], axis=1).astype(np.int64)

    # ---- lattice --------------------------------------------------------------------------------------
    def lattice(self, x):
        o, h = self.P.origin, self.P.hinge_spacing
        return tuple((float(x[a]) - o[a]) / h for a in range(3))

    def block_of_u(self, u):
        n = self.P.block_hinges
        return tuple(_floor_div(int(math.floor(u[a])), n) for a in range(3))

    def _alloc(self, key):
        if key not in self.slot:
            self.slot[key] = len(self.keys)
            self.keys.append(key)
            self.active.append(False)
            self.mu.append(np.zeros(self.nw))
            self.prec.append(np.full(self.nw, 1.0 / self.P.prior_var))
            self.mag.append(np.zeros(self.nw))
        return self.slot[key]

    def weight_of_hinge(self, g):
        """(slot, local index) of hinge g, or None when its block is not allocated."""
        n = self.P.block_hinges
        b = tuple(_floor_div(g[a], n) for a in range(3))
        s = self.slot.get(b)
        if s is None:
            return None
        lx, ly, lz = (g[a] - n * b[a] for a in range(3))
        return s, (lz * n + ly) * n + lx

    def features_u(self, u, x=None):
        """Kept features at lattice coordinates u (x = o + u h unless given): list of ((slot, local), phi, g), the
        bias of the point's block last (phi = 1, g = None) when that block is allocated."""
        o, h, gam = self.P.origin, self.P.hinge_spacing, self.P.gamma
        if x is None:
            x = tuple(o[a] + u[a] * h for a in range(3))
        g0 = np.array([math.floor(u[a]) for a in range(3)], dtype=np.int64)
        q = np.array([math.floor((u[a] - g0[a]) * Q20) for a in range(3)], dtype=np.int64)
        d = self._offsets
        D = ((q[None, :] - d * Q20) ** 2).sum(axis=1)
        g = g0[None, :] + d[D <= self.r2q]
        hx = np.asarray(o, dtype=np.float64)[None, :] + g.astype(np.float64) * h
        r2 = ((np.asarray(x, dtype=np.float64)[None, :] - hx) ** 2).sum(axis=1)
        phi = np.exp(-gam * r2)
        out = []
        for k in range(len(g)):
            gk = (int(g[k, 0]), int(g[k, 1]), int(g[k, 2]))
            w = self.weight_of_hinge(gk)
            if w is not None:
                out.append((w, float(phi[k]), gk))
        b = self.block_of_u(u)
        s = self.slot.get(b)
        if s is not None and self.P.bias_feature:
            out.append(((s, self.nw - 1), 1.0, None))
        return out

    # ---- prediction (Sec. IV-A.3, App. B) -------------------------------------------------------------
    def eval_u(self, u, x=None):
        """(l, grad l, phi^T Sigma phi) at lattice coordinates u."""
        o, h, gam = self.P.origin, self.P.hinge_spacing, self.P.gamma
        if x is None:
            x = tuple(o[a] + u[a] * h for a in range(3))
        l, v = 0.0, 0.0
        g = np.zeros(3)
        for (s, i), phi, hinge in self.features_u(u, x):
            m = self.mu[s][i]
            l += m * phi
            v += phi * phi / self.prec[s][i]
            if hinge is not None:
                for a in range(3):
                    g[a] += m * phi * (-2.0 * gam) * (x[a] - (o[a] + hinge[a] * h))
        return l, g, v

    def query(self, xq):
        """Log-odds, sign, gradient and occupancy probability at points xq (n x 3)."""
        xq = np.asarray(xq, dtype=np.float64).reshape(-1, 3)
        n = len(xq)
        L, S, G, Pr = np.zeros(n), np.zeros(n, dtype=np.int8), np.zeros((n, 3)), np.zeros(n)
        for k in range(n):
            u = self.lattice(xq[k])
            l, g, v = self.eval_u(u, tuple(float(c) for c in xq[k]))
            L[k], G[k] = l, g
            S[k] = 1 if l < self.tau else -1
            Pr[k] = float(sigmoid(l / math.sqrt(1.0 + math.pi / 8.0 * v)))
        return L, S, G, Pr

    # ---- update (Sec. IV-A.1 to IV-A.3, App. A) -------------------------------------------------------
    def samples(self, p, hits):
        """The update's samples: list of (u, x, t) with t in {0 (free), 1 (hit)}."""
        P = self.P
        o, h = P.origin, P.hinge_spacing
        up = self.lattice(p)
        Up = [int(np.rint(up[a] * 2.0 ** 32)) for a in range(3)]
        out = []
        for xh in hits:
            xh = tuple(float(c) for c in xh)
            ux = self.lattice(xh)
            dx, dy, dz = xh[0] - p[0], xh[1] - p[1], xh[2] - p[2]
            L = math.sqrt(dx * dx + dy * dy + dz * dz)
            jmax = int(math.floor((L - P.free_gap) / P.free_step)) if L > 0 else 0
            if jmax > 0:
                sig = P.free_step / L
                Ux = [int(np.rint(ux[a] * 2.0 ** 32)) for a in range(3)]
                D = [int(np.rint(float(Ux[a] - Up[a]) * sig)) for a in range(3)]
            for j in range(1, jmax + 1):
                U = [Up[a] + j * D[a] for a in range(3)]
                u = tuple(U[a] / 2.0 ** 32 for a in range(3))
                b = tuple(_floor_div(U[a] >> 32, P.block_hinges) for a in range(3))
                sl = self.slot.get(b)
                if sl is None or not self.active[sl]:
                    continue
                out.append((u, tuple(o[a] + u[a] * h for a in range(3)), 0))
            out.append((ux, xh, 1))
        return out

    def update(self, p, hits):
        P = self.P
        p = tuple(float(c) for c in p)
        hits = np.asarray(hits, dtype=np.float64).reshape(-1, 3)
        # 1. blocks: a hit's block becomes active, its 26 neighbours are allocated
        for xh in hits:
            b = self.block_of_u(self.lattice(xh))
            for dz in (-1, 0, 1):
                for dy in (-1, 0, 1):
                    for dx in (-1, 0, 1):
                        self._alloc((b[0] + dx, b[1] + dy, b[2] + dz))
            self.active[self.slot[b]] = True
        # 2. samples
        smp = self.samples(p, hits)
        self.last_samples = len(smp)
        # 3. EM on the flattened weight vector
        nw = self.nw
        rows, t = [], []
        self.last_features = 0
        for u, x, tk in smp:
            f = self.features_u(u, x)
            self.last_features += sum(1 for _, _, g in f if g is not None)
            rows.append((np.array([s * nw + i for (s, i), _, _ in f], dtype=np.int64),
                         np.array([phi for _, phi, _ in f])))
            t.append(tk)
        mu0 = np.concatenate(self.mu) if self.mu else np.zeros(0)
        P0 = np.concatenate(self.prec) if self.prec else np.zeros(0)
        if rows:
            mu, Pn, _ = em_diag(rows, t, mu0, P0, P.xi_init, P.em_iters)
            # magnitude of the mean's numerator over the precision, (P0 |mu0| + sum |t - 1/2| phi) / P: a scale
            # for comparing a lower-precision evaluation with this one (not used by the method)
            absB = np.zeros_like(mu0)
            np.add.at(absB, np.concatenate([r[0] for r in rows]), 0.5 * np.concatenate([r[1] for r in rows]))
            mag = (P0 * np.abs(mu0) + absB) / Pn
            for s in range(len(self.keys)):
                self.mu[s] = mu[s * nw:(s + 1) * nw].copy()
                self.prec[s] = Pn[s * nw:(s + 1) * nw].copy()
                self.mag[s] = mag[s * nw:(s + 1) * nw].copy()
        # 4. threshold
        if len(hits):
            lsum = sum(self.eval_u(self.lattice(xh), tuple(xh))[0] for xh in hits)
            self.tau = (1.0 - P.tau_alpha) * self.tau + P.tau_alpha / len(hits) * lsum
        # 5. marching cells of this update
        m = P.march_sub
        self.marked = set()
        for xh in hits:
            u = self.lattice(xh)
            c = tuple(int(math.floor(u[a] * m)) for a in range(3))
            for dz in (-1, 0, 1):
                for dy in (-1, 0, 1):
                    for dx in (-1, 0, 1):
                        self.marked.add((c[0] + dx, c[1] + dy, c[2] + dz))

    # ---- surface points (Sec. IV-A.4) -----------------------------------------------------------------
    def marked_edges(self):
        """Every edge (node, axis) of a marked cell, each once."""
        edges = set()
        for c in self.marked:
            for a in range(3):
                b, cc = [ax for ax in range(3) if ax != a]
                for ib in (0, 1):
                    for ic in (0, 1):
                        nu = list(c)
                        nu[b] += ib
                        nu[cc] += ic
                        edges.add((tuple(nu), a))
        return edges

    def node_u(self, nu):
        m = self.P.march_sub
        return tuple(nu[a] / m for a in range(3))

    def march(self):
        """Surface points of the last update's marked cells: (x n x 3, var n, normals n x 3, keys list of
        (nu_z, nu_y, nu_x, axis)), ascending key."""
        P = self.P
        m = P.march_sub
        o, h = P.origin, P.hinge_spacing
        cache = {}

        def lnode(nu):
            if nu not in cache:
                cache[nu] = self.eval_u(self.node_u(nu))[0]
            return cache[nu]

        pts = []
        for nu, a in sorted(self.marked_edges(), key=lambda e: (e[0][2], e[0][1], e[0][0], e[1])):
            nv = list(nu)
            nv[a] += 1
            la, lb = lnode(nu), lnode(tuple(nv))
            if (la >= self.tau) == (lb >= self.tau):
                continue
            t = (self.tau - la) / (lb - la)
            u = list(self.node_u(nu))
            u[a] = (nu[a] + t) / m
            x = tuple(o[k] + u[k] * h for k in range(3))
            l, g, _ = self.eval_u(tuple(u), x)
            g2 = float(g @ g)
            if not g2 > 0.0:
                continue
            var = P.beta * (self.tau - l) ** 2 / g2
            pts.append((x, var, -g / math.sqrt(g2), (nu[2], nu[1], nu[0], a)))
        X = np.array([p[0] for p in pts]).reshape(-1, 3)
        V = np.array([p[1] for p in pts])
        N = np.array([p[2] for p in pts]).reshape(-1, 3)
        return X, V, N, [p[3] for p in pts]

    # ---- introspection --------------------------------------------------------------------------------
    def weights(self):
        """dict block key -> (active, mu, prec)."""
        return {k: (self.active[s], self.mu[s], self.prec[s]) for k, s in self.slot.items()}
