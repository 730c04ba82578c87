"""Pins of the refit-scheduling reference (oracle/schedule.py; training queue of Sec. IV-C and App. G) on
hand-worked cases: the score c2 (1 + eta c0) and its order, cells without a fit first, the budget, deferral,
counter reset and halving, and the cap of the query counter."""
import numpy as np

from oracle import schedule


def st(members, fitted=True, c0=0, c2=0):
    return dict(members=tuple(members), fitted=fitted, c0=c0, c2=c2)


def test_update_hand_example():
    state = {10: st([1, 2], c0=100, c2=0),   # changes: c2 -> 1, score 1 * (1 + 0.01 * 100) = 2
             20: st([3], c0=0, c2=2),        # changes: c2 -> 3, score 3
             30: st([4, 5], c0=7, c2=0),     # unchanged
             40: st([6], c0=300, c2=0)}      # changes: c2 -> 1, score 1 * (1 + 3) = 4
    new_sets = {10: (1, 2, 9), 20: (3, 8), 30: (4, 5), 40: (6, 7), 50: (11,)}  # 50 is new: must be fitted
    ok = {k: True for k in new_sets}
    s2, refit, deferred = schedule.update(state, new_sets, ok, budget=2, eta=0.01)
    # order: 50 (must fit), 40 (4), 20 (3), 10 (2); budget 2 -> 50 and 40
    assert refit == {50, 40} and deferred == {20, 10}
    assert s2[40] == dict(members=(6, 7), fitted=True, c0=150, c2=0)      # fitted: c2 = 0, c0 halved
    assert s2[50] == dict(members=(11,), fitted=True, c0=0, c2=0)
    assert s2[20] == dict(members=(3,), fitted=True, c0=0, c2=3)          # deferred: old set, marks kept
    assert s2[10] == dict(members=(1, 2), fitted=True, c0=100, c2=1)
    assert s2[30] == dict(members=(4, 5), fitted=True, c0=7, c2=0)        # unchanged
    # no budget: every changed cell is fitted
    _, refit0, deferred0 = schedule.update(state, new_sets, ok, budget=0, eta=0.01)
    assert refit0 == {10, 20, 40, 50} and not deferred0


def test_ties_go_in_key_order_and_failed_fits_must_refit():
    state = {5: st([1], c2=0), 3: st([2], c2=0), 8: st([3], fitted=False)}
    new_sets = {5: (1, 4), 3: (2, 4), 8: (3,)}
    s2, refit, deferred = schedule.update(state, new_sets, {5: True, 3: True, 8: False}, budget=2, eta=0.5)
    # 8 had no usable fit: fitted first (even with an unchanged set); 3 and 5 tie at score 1: key 3 first
    assert refit == {8, 3} and deferred == {5}
    assert s2[8]["fitted"] is False  # the fit failed again


def test_score_is_binary32_and_monotone():
    k1 = schedule.score_key(1, 0, 1e-3)
    k2 = schedule.score_key(2, 0, 1e-3)
    k3 = schedule.score_key(2, 10000, 1e-3)
    assert k3 < k2 < k1 < (1 << 40)
    # 2 (1 + 1e-3 * 10000) = 22 in binary32
    assert k3 == 1 + 0xFFFFFFFF - int(np.float32(22.0).view(np.uint32))


def test_request_cap():
    state = {1: st([0], c0=9990)}
    schedule.add_requests(state, {1: 25, 2: 5})
    assert state[1]["c0"] == schedule.CAP == 10000
