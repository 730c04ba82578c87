"""One or more steps of the Kernel-SDF path (fit, query of all outputs, adjoint) on a named synthetic workload,
for an external profiler:

    python -m paper_2603_29227_gb300.profile_step <workload> [steps] [--autotune]

The library must have been built (``__graft_entry__.build()``).  Each step runs ksdf_fit, ksdf_query and
ksdf_query_backward once, eagerly, on the library's stream; the first step doubles as the warm-up.  The script
prints, per step, how many kernels the library launched, so that a profiler can skip the first step's launches.
With --autotune the fit tables and the query tile shapes are tuned before the first step (as the benchmark
does); their launches come before the first step's and are printed separately.
"""
from __future__ import annotations

import sys

import numpy as np


def main(argv):
    import torch

    from paper_2603_29227_gb300 import ksdf, scenes

    args = [a for a in argv if not a.startswith("--")]
    name = args[0] if args else "scale3d"
    steps = int(args[1]) if len(args) > 1 else 2
    tune = "--autotune" in argv
    w = scenes.workload(name)
    dev = torch.device("cuda:0")

    def t(a):
        return torch.from_numpy(np.ascontiguousarray(a)).to(dev)

    x, var, nrm, xq, sg = t(w.x), t(w.var), t(w.normals), t(w.xq), t(w.sign)
    Q = len(w.xq)
    d_sdf = torch.ones(Q, device=dev)
    d_grad = torch.full((Q, 3), 0.1, device=dev)
    m = ksdf.KernelSDF(w.params)
    _, base = ksdf.ksdf_profile_read(m.h)  # the library's count of its own kernel launches
    if tune:
        m.fit(x, var, nrm)
        m.autotune()
        m.autotune_query(xq, sg)
        torch.cuda.synchronize()
        _, n = ksdf.ksdf_profile_read(m.h)
        print(f"autotune launches {n - base}")
        base = n
    for s in range(steps):
        m.fit(x, var, nrm)
        o = m.query(xq, sg)
        m.backward(xq, o["winner"], d_sdf, d_grad, sg)
        torch.cuda.synchronize()
        _, n = ksdf.ksdf_profile_read(m.h)
        print(f"step {s} launches {n - base}")
        base = n
    m.sync_status()
    print("ok", name, Q)


if __name__ == "__main__":
    main(sys.argv[1:])
