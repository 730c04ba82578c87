"""Seeded synthetic inputs for the Kernel-SDF back-end query.

This module only makes inputs: analytic scenes, noisy surface samples with per-sample variances and
outward normals, query points and their true signs.  It holds none of the method's arithmetic, and it
is the only module that both the CUDA path's tests and the CPU oracle's tests draw inputs from.

The paper's datasets (Replica, Cow&Lady, Newer College) are not available; these scenes stand in for
them with the paper's setting: surface samples a few centimetres apart on planar and curved surfaces,
noise of about a centimetre, lambda of 300-500 and cells of tens to hundreds of samples.

Recipes (numpy PCG64, one seed per workload):
  plane2d   "2D plain FP64": a 10 x 10 m box border (free inside) and 20 circles (centres U[0,10]^2,
            radius U[0.2,1]); 2,000 samples uniform in arc length over all visible boundaries, isotropic
            N(0, 0.01^2) noise; 1 m cells, n_max 64, lambda 500; queries at the centres of a 128 x 128
            grid over the box.
  room3d    "3D": a 20 x 20 x 5 m room (walls, floor, ceiling) with 50 primitives (spheres and axis-
            aligned boxes, 50/50, sizes U[0.2,2] m) inside it; 200,000 samples uniform in area,
            N(0, 0.01^2) noise; 0.5 m cells, n_max 256, lambda 300; 1,000,000 queries uniform in the room.
  scale3d   "mixed-precision scale": a 50 x 50 x 10 m scene with 1,000 primitives and 2,000,000 samples;
            0.5 m cells, n_max 512; queries on a 256^3 grid over the bounding box.
  traj3d    "differentiation": the room3d scene; 4,096 cubic Bezier trajectories x 64 waypoints x 8
            collision-sphere centres (corners of a 0.3 m cube around each waypoint) = 2,097,152 queries.
  city      "streaming": a 100 x 100 m ground with 200 boxes (footprints U[4,20] m, heights U[3,30] m), a
            64 x 2048 LiDAR-like scanner (elevation -25..+15 deg, 100 m range, range noise 0.02 m, sigma_i =
            0.02 m) at 1.8 m on a smooth closed 100-pose path; per frame 1,000,000 queries in the 40 x 40 m
            square around the pose, 0..6 m high; normals from the analytic scene (sign stand-in).
Per-sample variance fed to the GP: sigma_i^2 = (sigma_noise * U[0.5, 2])^2, standing in for the
front-end's per-point uncertainty.  Normals point from the obstacle into free space.  Samples that fall
inside another obstacle (or outside the room) are rejected and redrawn.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

__all__ = ["Scene", "make_plane2d", "make_room3d", "make_scale3d", "Workload", "workload", "WORKLOADS", "City",
           "make_city"]


@dataclass
class Scene:
    """Analytic scene: a free box (room) minus solid spheres/circles and axis-aligned boxes."""

    dim: int
    room_lo: np.ndarray
    room_hi: np.ndarray
    centres: np.ndarray = field(default_factory=lambda: np.zeros((0, 3)))
    radii: np.ndarray = field(default_factory=lambda: np.zeros(0))
    box_lo: np.ndarray = field(default_factory=lambda: np.zeros((0, 3)))
    box_hi: np.ndarray = field(default_factory=lambda: np.zeros((0, 3)))

    # ---- ground truth (used by tests for sanity checks and by the generators for rejection) ----
    def _in_primitives(self, x: np.ndarray, tol: float) -> np.ndarray:
        """Points strictly inside some sphere/circle (radius - tol) or box (shrunk by tol).  With many
        primitives, each one is tested only against the points of the 1 m grid cells its bounding box
        touches (same result as testing every point)."""
        n = x.shape[0]
        out = np.zeros(n, dtype=bool)
        nprim = len(self.radii) + len(self.box_lo)
        if nprim <= 64 or n < 4096:
            for c, r in zip(self.centres, self.radii):
                out |= np.sum((x - c) ** 2, axis=1) < (r - tol) ** 2
            for lo, hi in zip(self.box_lo, self.box_hi):
                out |= np.all((x > lo + tol) & (x < hi - tol), axis=1)
            return out
        g0 = self.room_lo - 1.0
        dims = (np.ceil((self.room_hi - g0) / 1.0).astype(np.int64) + 2)
        cell = np.clip(np.floor(x - g0).astype(np.int64), 0, dims - 1)
        lin = cell[:, 0]
        for j in range(1, self.dim):
            lin = lin * dims[j] + cell[:, j]
        order = np.argsort(lin, kind="stable")
        starts = np.searchsorted(lin[order], np.arange(int(np.prod(dims)) + 1))

        def candidates(lo, hi):
            a = np.clip(np.floor(lo - g0).astype(np.int64), 0, dims - 1)
            b = np.clip(np.floor(hi - g0).astype(np.int64), 0, dims - 1)
            rng = [np.arange(a[j], b[j] + 1) for j in range(self.dim)]
            mesh = np.meshgrid(*rng, indexing="ij")
            l = mesh[0].ravel()
            for j in range(1, self.dim):
                l = l * dims[j] + mesh[j].ravel()
            parts = [order[starts[v]:starts[v + 1]] for v in l]
            return np.concatenate(parts) if parts else np.zeros(0, np.int64)

        for c, r in zip(self.centres, self.radii):
            idx = candidates(c - r, c + r)
            if idx.size:
                out[idx] |= np.sum((x[idx] - c) ** 2, axis=1) < (r - tol) ** 2
        for lo, hi in zip(self.box_lo, self.box_hi):
            idx = candidates(lo, hi)
            if idx.size:
                out[idx] |= np.all((x[idx] > lo + tol) & (x[idx] < hi - tol), axis=1)
        return out

    def occupied(self, x: np.ndarray) -> np.ndarray:
        x = np.asarray(x, dtype=np.float64)
        occ = np.any((x < self.room_lo) | (x > self.room_hi), axis=1)
        return occ | self._in_primitives(x, 0.0)

    def sign(self, x: np.ndarray) -> np.ndarray:
        """+1 in free space, -1 inside an obstacle (int8)."""
        return np.where(self.occupied(x), -1, 1).astype(np.int8)

    def dist_free(self, x: np.ndarray) -> np.ndarray:
        """Exact distance to the occupied set for points in free space (Sec. III definition)."""
        x = np.asarray(x, dtype=np.float64)
        d = np.min(np.minimum(x - self.room_lo, self.room_hi - x), axis=1)
        for c, r in zip(self.centres, self.radii):
            d = np.minimum(d, np.sqrt(np.sum((x - c) ** 2, axis=1)) - r)
        for lo, hi in zip(self.box_lo, self.box_hi):
            e = np.maximum(np.maximum(lo - x, 0.0), x - hi)
            d = np.minimum(d, np.sqrt(np.sum(e * e, axis=1)))
        return d

    # ---- surface sampling ----
    def _pieces(self):
        """(kind, index, area-or-length) for every boundary piece."""
        out = []
        L = self.room_hi - self.room_lo
        for ax in range(self.dim):
            other = np.prod(np.delete(L, ax)) if self.dim == 3 else np.delete(L, ax)[0]
            out.append(("room_lo", ax, other))
            out.append(("room_hi", ax, other))
        for i, r in enumerate(self.radii):
            out.append(("ball", i, 4 * np.pi * r * r if self.dim == 3 else 2 * np.pi * r))
        for i, (lo, hi) in enumerate(zip(self.box_lo, self.box_hi)):
            e = hi - lo
            for ax in range(self.dim):
                other = np.prod(np.delete(e, ax)) if self.dim == 3 else np.delete(e, ax)[0]
                out.append(("box_lo", (i, ax), other))
                out.append(("box_hi", (i, ax), other))
        return out

    def _draw(self, rng: np.random.Generator, n: int):
        pieces = self._pieces()
        w = np.array([p[2] for p in pieces], dtype=np.float64)
        pick = rng.choice(len(pieces), size=n, p=w / w.sum())
        x = np.empty((n, self.dim))
        nrm = np.zeros((n, self.dim))
        order = np.argsort(pick, kind="stable")
        bounds = np.searchsorted(pick[order], np.arange(len(pieces) + 1))
        for k, (kind, idx, _) in enumerate(pieces):
            sel = order[bounds[k]:bounds[k + 1]]
            m = sel.size
            if m == 0:
                continue
            if kind in ("room_lo", "room_hi", "box_lo", "box_hi"):
                if kind.startswith("room"):
                    lo, hi, ax = self.room_lo, self.room_hi, idx
                    inward = 1.0  # free space is inside the room
                else:
                    i, ax = idx
                    lo, hi = self.box_lo[i], self.box_hi[i]
                    inward = -1.0  # free space is outside the box
                p = lo + rng.random((m, self.dim)) * (hi - lo)
                if kind.endswith("lo"):
                    p[:, ax] = lo[ax]
                    nrm[sel, ax] = 1.0 * inward
                else:
                    p[:, ax] = hi[ax]
                    nrm[sel, ax] = -1.0 * inward
                x[sel] = p
            else:  # ball / circle
                v = rng.standard_normal((m, self.dim))
                v /= np.linalg.norm(v, axis=1, keepdims=True)
                x[sel] = self.centres[idx] + self.radii[idx] * v
                nrm[sel] = v
        return x, nrm

    def sample_surface(self, rng: np.random.Generator, n: int, noise: float):
        """n accepted samples: (x float64, var float32, normals float32)."""
        xs, ns = [], []
        have = 0
        while have < n:
            batch = max(1024, int(1.3 * (n - have)))
            x, nrm = self._draw(rng, batch)
            # reject points strictly inside another obstacle or outside the room (tolerance 1e-9 m keeps
            # the point's own surface)
            keep = ~self._inside_other(x, 1e-9)
            xs.append(x[keep])
            ns.append(nrm[keep])
            have += int(keep.sum())
        x = np.concatenate(xs)[:n]
        nrm = np.concatenate(ns)[:n]
        x = x + noise * rng.standard_normal(x.shape)
        var = (noise * rng.uniform(0.5, 2.0, size=n)) ** 2
        return x, var.astype(np.float32), nrm.astype(np.float32)

    def _inside_other(self, x: np.ndarray, tol: float) -> np.ndarray:
        bad = np.any((x < self.room_lo - tol) | (x > self.room_hi + tol), axis=1)
        return bad | self._in_primitives(x, tol)


def make_plane2d(rng: np.random.Generator, n_circles: int = 20, size: float = 10.0) -> Scene:
    c = rng.uniform(0.0, size, size=(n_circles, 2))
    r = rng.uniform(0.2, 1.0, size=n_circles)
    return Scene(dim=2, room_lo=np.zeros(2), room_hi=np.full(2, size), centres=c, radii=r,
                 box_lo=np.zeros((0, 2)), box_hi=np.zeros((0, 2)))


def _primitives3d(rng, n, room_hi):
    is_ball = rng.random(n) < 0.5
    cen, rad, blo, bhi = [], [], [], []
    for b in is_ball:
        if b:
            r = 0.5 * rng.uniform(0.2, 2.0)
            c = rng.uniform(r, room_hi - r)
            cen.append(c)
            rad.append(r)
        else:
            e = rng.uniform(0.2, 2.0, size=3)
            lo = rng.uniform(0.0, room_hi - e)
            blo.append(lo)
            bhi.append(lo + e)
    z3 = np.zeros((0, 3))
    return (np.array(cen) if cen else z3, np.array(rad), np.array(blo) if blo else z3, np.array(bhi) if bhi else z3)


def make_room3d(rng: np.random.Generator, room=(20.0, 20.0, 5.0), n_prims: int = 50) -> Scene:
    hi = np.array(room, dtype=np.float64)
    c, r, lo, bh = _primitives3d(rng, n_prims, hi)
    return Scene(dim=3, room_lo=np.zeros(3), room_hi=hi, centres=c, radii=r, box_lo=lo, box_hi=bh)


def make_scale3d(rng: np.random.Generator) -> Scene:
    return make_room3d(rng, room=(50.0, 50.0, 10.0), n_prims=1000)


@dataclass
class Workload:
    name: str
    params: dict
    scene: Scene
    x: np.ndarray        # S x dim float64 sample positions
    var: np.ndarray      # S float32 per-sample variance sigma_i^2
    normals: np.ndarray  # S x dim float32 outward normals
    xq: np.ndarray       # Q x dim float32 query points
    sign: np.ndarray     # Q int8 true sign (+1 free, -1 occupied)


def _grid_queries(lo, hi, n, dim):
    axes = [lo[j] + (np.arange(n) + 0.5) * (hi[j] - lo[j]) / n for j in range(dim)]
    mesh = np.meshgrid(*axes, indexing="ij")
    # x fastest in memory order (row = z, y, x in 3D)
    pts = np.stack([m.ravel(order="F") for m in mesh], axis=1)
    return pts


def _bezier_queries(rng, scene: Scene, n_traj: int, n_way: int):
    lo, hi = scene.room_lo + 0.3, scene.room_hi - 0.3
    P = lo + rng.random((n_traj, 4, 3)) * (hi - lo)
    t = (np.arange(n_way) + 0.5) / n_way
    B = np.stack([(1 - t) ** 3, 3 * (1 - t) ** 2 * t, 3 * (1 - t) * t ** 2, t ** 3], axis=1)  # n_way x 4
    way = np.einsum("wk,tkj->twj", B, P).reshape(-1, 3)
    off = np.array([[sx, sy, sz] for sz in (-1, 1) for sy in (-1, 1) for sx in (-1, 1)], dtype=np.float64) * 0.15
    return (way[:, None, :] + off[None, :, :]).reshape(-1, 3)


def workload(name: str, seed: int | None = None, n_samples: int | None = None, n_queries: int | None = None,
             grid: int | None = None) -> Workload:
    """Build a named workload.  Optional overrides shrink it for tests (same recipe, smaller sizes)."""
    if name == "plane2d":
        rng = np.random.default_rng(1 if seed is None else seed)
        sc = make_plane2d(rng)
        S = 2000 if n_samples is None else n_samples
        x, var, nrm = sc.sample_surface(rng, S, 0.01)
        n = 128 if grid is None else grid
        xq = _grid_queries(sc.room_lo, sc.room_hi, n, 2)
        params = dict(dim=2, origin=(0.0, 0.0, 0.0), cell=1.0, margin=0.1, n_max=64, k_cand=4, **{"lambda": 500.0},
                      softmin_alpha=500.0, sign_mode=0)
    elif name in ("room3d", "traj3d"):
        rng = np.random.default_rng((2 if name == "room3d" else 4) if seed is None else seed)
        sc = make_room3d(np.random.default_rng(2 if seed is None else seed))
        S = 200_000 if n_samples is None else n_samples
        x, var, nrm = sc.sample_surface(np.random.default_rng(rng.integers(1 << 62)), S, 0.01)
        if name == "room3d":
            Q = 1_000_000 if n_queries is None else n_queries
            xq = sc.room_lo + rng.random((Q, 3)) * (sc.room_hi - sc.room_lo)
        else:
            nt = 4096 if n_queries is None else max(1, n_queries // (64 * 8))
            xq = _bezier_queries(rng, sc, nt, 64)
        params = dict(dim=3, origin=(0.0, 0.0, 0.0), cell=0.5, margin=0.1, n_max=256, k_cand=8,
                      **{"lambda": 300.0}, softmin_alpha=300.0, sign_mode=0)
    elif name == "scale3d":
        rng = np.random.default_rng(5 if seed is None else seed)
        sc = make_scale3d(rng)
        S = 2_000_000 if n_samples is None else n_samples
        x, var, nrm = sc.sample_surface(rng, S, 0.01)
        n = 256 if grid is None else grid
        xq = _grid_queries(sc.room_lo, sc.room_hi, n, 3)
        params = dict(dim=3, origin=(0.0, 0.0, 0.0), cell=0.5, margin=0.1, n_max=512, k_cand=8,
                      **{"lambda": 300.0}, softmin_alpha=300.0, sign_mode=0)
    else:
        raise KeyError(name)
    perm = np.random.default_rng(12345).permutation(x.shape[0])  # stream order, not surface order
    x, var, nrm = x[perm], var[perm], nrm[perm]
    xq = np.ascontiguousarray(xq, dtype=np.float32)
    return Workload(name=name, params=params, scene=sc, x=np.ascontiguousarray(x), var=var,
                    normals=np.ascontiguousarray(nrm), xq=xq, sign=sc.sign(xq.astype(np.float64)))


WORKLOADS = ("plane2d", "room3d", "traj3d", "scale3d")


# ---------------------------------------------------------------------------------------------------------
# streaming: a city block scanned by a LiDAR-like sensor along a closed path

@dataclass
class City:
    """A 100 x 100 m ground plane with axis-aligned boxes (buildings), a smooth closed sensor path at 1.8 m and
    a 64-beam (elevation -25..+15 deg) x 2048-azimuth range scanner (max range 100 m, range noise 0.02 m)."""

    box_lo: np.ndarray
    box_hi: np.ndarray
    poses: np.ndarray   # F x 3 sensor positions
    params: dict
    seed: int
    sigma: float = 0.02
    max_range: float = 100.0
    n_beams: int = 64
    n_az: int = 2048

    def scan(self, f: int):
        """Hits of frame f: (x S x 3 float64, var S float32, normals S x 3 float32), nearest surface per ray
        (ground z = 0 or a box face), range noise along the ray; rays without a hit are dropped."""
        rng = np.random.default_rng(self.seed * 1000 + 17 + f)
        el = np.radians(np.linspace(-25.0, 15.0, self.n_beams))
        az = np.arange(self.n_az) * (2.0 * np.pi / self.n_az) + rng.uniform(0.0, 2.0 * np.pi / self.n_az)
        ce, se = np.cos(el)[:, None], np.sin(el)[:, None]
        d = np.stack([(ce * np.cos(az)).ravel(), (ce * np.sin(az)).ravel(), np.repeat(se, self.n_az, axis=1).ravel()],
                     axis=1)
        o = self.poses[f]
        R = d.shape[0]
        t_hit = np.full(R, np.inf)
        nrm = np.zeros((R, 3))
        down = d[:, 2] < 0
        tg = np.where(down, -o[2] / np.where(down, d[:, 2], -1.0), np.inf)
        t_hit = np.minimum(t_hit, tg)
        nrm[np.isfinite(tg)] = (0.0, 0.0, 1.0)
        inv = 1.0 / np.where(np.abs(d) < 1e-12, 1e-12, d)
        for b0 in range(0, len(self.box_lo), 16):
            lo, hi = self.box_lo[b0:b0 + 16], self.box_hi[b0:b0 + 16]  # B x 3
            t1 = (lo[None, :, :] - o) * inv[:, None, :]
            t2 = (hi[None, :, :] - o) * inv[:, None, :]
            tn3 = np.minimum(t1, t2)
            tnear = tn3.max(axis=2)
            tfar = np.maximum(t1, t2).min(axis=2)
            hit = (tnear <= tfar) & (tnear > 1e-6)
            tnear = np.where(hit, tnear, np.inf)
            j = np.argmin(tnear, axis=1)
            tb = tnear[np.arange(R), j]
            better = tb < t_hit
            if np.any(better):
                ax = np.argmax(tn3[np.arange(R), j], axis=1)  # entry face
                nb = np.zeros((R, 3))
                nb[np.arange(R), ax] = -np.sign(d[np.arange(R), ax])
                t_hit = np.where(better, tb, t_hit)
                nrm[better] = nb[better]
        ok = t_hit < self.max_range
        t = t_hit[ok] + rng.normal(0.0, self.sigma, size=int(ok.sum()))
        x = o + t[:, None] * d[ok]
        var = np.full(x.shape[0], self.sigma ** 2, dtype=np.float32)
        return np.ascontiguousarray(x), var, np.ascontiguousarray(nrm[ok], dtype=np.float32)

    def queries(self, f: int, Q: int):
        """Q points uniform in the 40 x 40 m square around the pose, 0..6 m above the ground."""
        rng = np.random.default_rng(self.seed * 1000 + 911 + f)
        o = self.poses[f]
        lo = np.array([o[0] - 20.0, o[1] - 20.0, 0.0])
        hi = np.array([o[0] + 20.0, o[1] + 20.0, 6.0])
        return np.ascontiguousarray(lo + rng.random((Q, 3)) * (hi - lo), dtype=np.float32)


def make_city(seed: int = 3, n_boxes: int = 200, n_poses: int = 100, size: float = 100.0) -> City:
    """Boxes with footprints U[4, 20] m and heights U[3, 30] m; the path is a seeded smooth closed curve around
    the block centre (radius 30 m with low-frequency wobble); boxes within 4 m of the path are removed."""
    rng = np.random.default_rng(seed)
    s = np.linspace(0.0, 2.0 * np.pi, n_poses, endpoint=False)
    a = rng.normal(0.0, 3.0, size=(3, 2))
    r = 30.0 + a[0, 0] * np.sin(s) + a[0, 1] * np.cos(2 * s) + a[1, 0] * np.sin(3 * s)
    poses = np.stack([size / 2 + r * np.cos(s), size / 2 + r * np.sin(s), np.full(n_poses, 1.8)], axis=1)
    fp = rng.uniform(4.0, 20.0, size=(n_boxes, 2))
    h = rng.uniform(3.0, 30.0, size=n_boxes)
    lo_xy = rng.uniform(0.0, 1.0, size=(n_boxes, 2)) * (size - fp)
    lo = np.concatenate([lo_xy, np.zeros((n_boxes, 1))], axis=1)
    hi = np.concatenate([lo_xy + fp, h[:, None]], axis=1)
    # distance from each pose to each box footprint; keep boxes at least 4 m from the path
    dx = np.maximum(np.maximum(lo[None, :, 0] - poses[:, None, 0], poses[:, None, 0] - hi[None, :, 0]), 0.0)
    dy = np.maximum(np.maximum(lo[None, :, 1] - poses[:, None, 1], poses[:, None, 1] - hi[None, :, 1]), 0.0)
    keep = np.min(np.hypot(dx, dy), axis=0) > 4.0
    params = dict(dim=3, origin=(0.0, 0.0, 0.0), cell=0.5, margin=0.1, n_max=256, k_cand=8, **{"lambda": 300.0},
                  softmin_alpha=300.0, sign_mode=1)
    return City(box_lo=lo[keep], box_hi=hi[keep], poses=poses, params=params, seed=seed)


# ---------------------------------------------------------------------------------------------------------
# front-end (BHM) inputs from the same city scans

# BHM parameters of the city stream, read from App. I's outdoor LiDAR setting (0.7 m octree voxels, local BHM boxes
# of two voxels with 9 hinges per axis, so a hinge spacing of 0.175 m and 8 owned hinges per block axis; kernel
# scale l = 0.11 m, gamma = 1 / (2 l^2)).  Free samples one hinge spacing apart, none within 0.1 m of the hit;
# marching cells of half a hinge spacing.
CITY_BHM = dict(origin=(0.0, 0.0, 0.0), hinge_spacing=0.175, block_hinges=8, gamma=1.0 / (2.0 * 0.11 ** 2),
                phi_min=1e-3, prior_var=1.0, em_iters=2, xi_init=0.0, free_step=0.175, free_gap=0.1, tau_alpha=0.1,
                tau_init=0.0, beta=1.0, march_sub=2, bias_feature=1)


def city_bhm_frame(city: City, f: int, radius: float | None = None, max_hits: int | None = None, seed: int = 0):
    """Sensor position and hits (R x 3 float64) of frame f: every hit, or those within `radius` of the sensor,
    subsampled (seeded, order kept) to at most max_hits."""
    x, _, _ = city.scan(f)
    p = city.poses[f]
    if radius is not None:
        x = x[np.linalg.norm(x - p, axis=1) <= radius]
    if max_hits is not None and len(x) > max_hits:
        rng = np.random.default_rng(seed * 7919 + f)
        x = x[np.sort(rng.choice(len(x), size=max_hits, replace=False))]
    return np.asarray(p, dtype=np.float64), np.ascontiguousarray(x, dtype=np.float64)
