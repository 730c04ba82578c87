"""Refit scheduling of the streaming update (Sec. IV-C, App. G) on the GPU against the reference in
oracle/schedule.py: query counters from the candidate lists, the per-update choice of the cells to fit under a
budget (score c2 (1 + eta c0), cells without a fit first), deferred cells keeping their previous training set and
fit, and the counters afterwards; then rounds with no new samples drain the deferred cells until the model equals a
fresh fit of all samples bit for bit."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle  # noqa: E402
from oracle import schedule  # noqa: E402
from paper_2603_29227_gb300 import ksdf, scenes  # noqa: E402

DEV = torch.device("cuda:0")


@pytest.fixture(scope="module", autouse=True)
def _build():
    import __graft_entry__

    __graft_entry__.build()


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def gpu_cells(m):
    keys, status, off, mem = ksdf.ksdf_get_cells(m.h)
    sets = {int(k): tuple(mem[off[g]:off[g + 1]].tolist()) for g, k in enumerate(keys)}
    return keys, status, off, sets


def oracle_sets(params, x, var):
    om = oracle.Model(params, x, var)
    keys, status, off, mem = om.cells()
    return ({int(k): tuple(mem[off[g]:off[g + 1]].tolist()) for g, k in enumerate(keys)},
            {int(k): status[g] == oracle.CELL_OK for g, k in enumerate(keys)}, om)


def test_scheduled_updates_follow_the_reference():
    w = scenes.workload("room3d", n_samples=12000, n_queries=40000)
    p = w.params
    rng = np.random.default_rng(3)
    order = rng.permutation(len(w.x))
    parts = [order[:6000], order[6000:8000], order[8000:10000], order[10000:]]
    budget, eta = 150, 1e-3
    m = ksdf.KernelSDF(p)
    ksdf.ksdf_set_schedule(m.h, budget, eta)
    xs, vs = w.x[parts[0]], w.var[parts[0]]
    m.fit(_t(xs), _t(vs), None)
    sets, ok, om = oracle_sets(p, xs, vs)
    state = schedule.initial(sets, ok)
    qrng = np.random.default_rng(4)
    rounds = [(part, budget) for part in parts[1:]] + [(None, budget), (None, 1 << 30)]
    for step, (part, bud) in enumerate(rounds):
        ksdf.ksdf_set_schedule(m.h, bud, eta)
        # queries concentrated in a corner of the room raise those cells' priority
        xq = (w.scene.room_lo + qrng.random((20000, 3)) * (w.scene.room_hi - w.scene.room_lo) * 0.4).astype(np.float32)
        m.query(_t(xq))
        torch.cuda.synchronize()
        schedule.add_requests(state, schedule.requests(om, xq, p, oracle.bin_keys))
        c0, c2, _ = ksdf.ksdf_get_schedule(m.h)
        keys, _, _, gsets = gpu_cells(m)
        assert [state[int(k)]["c0"] for k in keys] == c0.tolist(), step
        prev_alpha = {int(k): a for k, a in zip(keys, np.split(m.fit_arrays()[0], np.cumsum(
            [len(gsets[int(k)]) for k in keys])[:-1]))}
        if part is not None:
            xs, vs = np.concatenate([xs, w.x[part]]), np.concatenate([vs, w.var[part]])
            m.update(_t(w.x[part]), _t(w.var[part]), None)
        else:
            m.update(None, None, None, S_new=0)
        sets, ok, om = oracle_sets(p, xs, vs)
        state, refit, deferred = schedule.update(state, sets, ok, bud, eta)
        keys, status, off, gsets = gpu_cells(m)
        c0, c2, rf = ksdf.ksdf_get_schedule(m.h)
        assert [int(k) for k in keys] == sorted(state), step
        for g, k in enumerate(keys):
            k = int(k)
            assert gsets[k] == state[k]["members"], (step, k)
            assert (c0[g], c2[g], rf[g]) == (state[k]["c0"], state[k]["c2"], int(k in refit)), (step, k)
        # deferred cells kept their fit bit for bit
        alpha = m.fit_arrays()[0]
        for g, k in enumerate(keys):
            if int(k) in deferred:
                assert np.array_equal(alpha[off[g]:off[g + 1]], prev_alpha[int(k)]), (step, int(k))
        print("step %d: refit %d, deferred %d" % (step, len(refit), len(deferred)))
    assert not deferred, "the deferred cells did not drain"
    # drained: the model equals a fresh fit of all samples bit for bit
    fresh = ksdf.KernelSDF(p)
    fresh.fit(_t(xs), _t(vs), None)
    a1, l1, _ = m.fit_arrays()
    a2, l2, _ = fresh.fit_arrays()
    assert np.array_equal(a1, a2) and np.array_equal(l1, l2)


def test_schedule_arguments():
    w = scenes.workload("plane2d", n_samples=300, grid=8)
    m = ksdf.KernelSDF(w.params)
    with pytest.raises(ksdf.KsdfError):
        ksdf.ksdf_set_schedule(m.h, -1)
    with pytest.raises(ksdf.KsdfError):
        ksdf.ksdf_set_schedule(m.h, 10, float("nan"))
    with pytest.raises(ksdf.KsdfError):
        ksdf.ksdf_get_schedule(m.h)  # no model yet
