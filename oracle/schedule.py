"""Reference of the refit scheduling of the streaming update (training queue of Sec. IV-C and App. G).

TEST INFRASTRUCTURE ONLY, like the rest of this package: the GPU tests replay an update sequence here and compare
the library's per-cell state with it.  Plain Python over dictionaries keyed by the packed cell key; it shares no
code with the CUDA library.

State per cell: its training set (global sample ids, ascending), whether it holds a usable fit, the query counter
c0 and the training marks c2.
  - A query adds one request to each cell fused for it (the K candidates of its bin); c0 is capped at 10000.
  - An update recomputes every cell's training set from all samples.  A cell changed when it had no usable fit or
    its new set differs from the one it was fitted on; a changed cell gains one training mark.  Cells without a
    usable fit must be fitted; the other changed cells are ranked by the score c2 (1 + eta c0) (binary32, each
    operation rounded), ties in ascending key order, and the first ones fill the budget (cells that must be
    fitted count towards it and are always fitted).  Changed cells beyond it keep their previous training set.
  - A fitted cell resets c2 to 0 and halves c0 (integer).
"""
from __future__ import annotations

import numpy as np

CAP = 10000


def requests(model, xq, params, bin_keys_fn):
    """Requests per cell key added by one query batch: for every occupied bin, its query count on each of its
    candidate cells (the oracle's candidate lists)."""
    keys = bin_keys_fn(params, np.asarray(xq, dtype=np.float64))
    ub, cnt = np.unique(keys, return_counts=True)
    cand, ncand = model.candidates(ub)
    cell_keys, _, _, _ = model.cells()
    out = {}
    for b in range(len(ub)):
        add = int(min(cnt[b], CAP))
        for k in range(int(ncand[b])):
            ck = int(cell_keys[cand[b, k]])
            out[ck] = out.get(ck, 0) + add
    return out


def add_requests(state, req):
    for k, add in req.items():
        if k in state:
            state[k]["c0"] = min(state[k]["c0"] + add, CAP)


def score_key(c2, c0, eta):
    s = np.float32(c2) * (np.float32(1.0) + np.float32(eta) * np.float32(c0))
    return 1 + (0xFFFFFFFF - int(np.float32(s).view(np.uint32)))


def update(state, new_sets, new_ok, budget, eta):
    """One scheduled update.  state: key -> dict(members, fitted, c0, c2) (the model before the update);
    new_sets: key -> tuple of member ids recomputed from all samples; new_ok: key -> whether a fit of that new
    set succeeds.  Returns (new state, set of refitted keys, set of deferred keys)."""
    keys = sorted(new_sets)
    rank = []
    info = {}
    for i, k in enumerate(keys):
        o = state.get(k)
        fitted_before = o is not None and o["fitted"]
        same = fitted_before and tuple(o["members"]) == tuple(new_sets[k]) and len(new_sets[k]) > 0
        c0 = o["c0"] if o is not None else 0
        c2 = (o["c2"] if o is not None else 0) + (0 if same else 1)
        if not fitted_before:
            key = 0
        elif not same:
            key = score_key(c2, c0, eta)
        else:
            key = 1 << 40
        info[k] = dict(same=same, c0=c0, c2=c2, fitted_before=fitted_before)
        rank.append((key, i, k))
    rank.sort()
    selected = set()
    for r, (key, _, k) in enumerate(rank):
        if key == 0 or (key < (1 << 40) and (budget <= 0 or r < budget)):
            selected.add(k)
    new_state, refit, deferred = {}, set(), set()
    for k in keys:
        it = info[k]
        if not it["same"] and k not in selected:
            deferred.add(k)
            o = state[k]
            new_state[k] = dict(members=tuple(o["members"]), fitted=True, c0=it["c0"], c2=it["c2"])
            continue
        if it["same"]:
            new_state[k] = dict(members=tuple(new_sets[k]), fitted=True, c0=it["c0"], c2=it["c2"])
            continue
        refit.add(k)
        new_state[k] = dict(members=tuple(new_sets[k]), fitted=bool(new_ok[k]), c0=it["c0"] >> 1, c2=0)
    return new_state, refit, deferred


def initial(sets, ok):
    """The state after a fresh fit: every cell fitted, counters zero."""
    return {k: dict(members=tuple(v), fitted=bool(ok[k]), c0=0, c2=0) for k, v in sets.items()}
