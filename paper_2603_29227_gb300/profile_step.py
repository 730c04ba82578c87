"""One or more steps of the Kernel-SDF path (fit, query of all outputs, adjoint) on a named synthetic workload,
for an external profiler:

    python -m paper_2603_29227_gb300.profile_step <workload> [steps] [--autotune]
    python -m paper_2603_29227_gb300.profile_step city_frontend [frames]
    python -m paper_2603_29227_gb300.profile_step --summarize <ncu launch list .csv>

The second form turns an ncu CSV launch list of such a run (gpu__time_duration.sum, optionally
dram__bytes_read.sum and dram__bytes_write.sum) into a per-kernel table of its last step, each kernel assigned to
the stage that launched it (fit, query, adjoint), with the DRAM bytes of the query and adjoint kernels and a digest
of their sources.

city_frontend runs the BHM front-end (include/ksdf_bhm.h) on the first frames of the city stream -- per frame the
update, the surface points and the sign of the frame's 1M queries -- on a map sized for a profiler (40,000 blocks,
about 0.4 GB).

The library must have been built (``__graft_entry__.build()``).  Each step runs ksdf_fit, ksdf_query and
ksdf_query_backward once, eagerly, on the library's stream; the first step doubles as the warm-up.  The script
prints, per step, how many kernels the library launched, so that a profiler can skip the first step's launches.
With --autotune the fit tables and the query tile shapes are tuned before the first step (as the benchmark
does); their launches come before the first step's and are printed separately.
"""
from __future__ import annotations

import sys

import numpy as np


def frontend(frames):
    import torch

    from paper_2603_29227_gb300 import bhm, scenes

    city = scenes.make_city()
    dev = torch.device("cuda:0")
    m = bhm.BHMap(scenes.CITY_BHM, max_blocks=40000, max_marked=20000)
    for f in range(frames):
        x, _, _ = city.scan(f)
        hits = torch.from_numpy(x).to(dev)
        xq = torch.from_numpy(city.queries(f, 1_000_000)).to(dev)
        m.update(city.poses[f], hits)
        pts = m.march(device=dev)
        m.query(xq, bhm.BHM_SIGN)
        torch.cuda.synchronize()
        nb, ns, nf = m.size(features=True)
        print("frame %d hits %d samples %d features %d points %d blocks %d" % (f, len(x), ns, nf, len(pts[0]), nb))
    m.sync_status()
    print("ok city_frontend", frames)


def main(argv):
    import torch

    from paper_2603_29227_gb300 import ksdf, scenes

    args = [a for a in argv if not a.startswith("--")]
    name = args[0] if args else "scale3d"
    if name == "city_frontend":
        return frontend(int(args[1]) if len(args) > 1 else 2)
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


def source_digest():
    """Digest of the query and adjoint kernel sources (the same one bench.py checks before it reports traffic)."""
    import hashlib
    import os

    here = os.path.join(os.path.dirname(os.path.abspath(__file__)), "csrc")
    hs = hashlib.sha256()
    for f in ("ksdf_query.cu", "ksdf_backward.cu", "ksdf_internal.cuh"):
        with open(os.path.join(here, f), "rb") as fh:
            hs.update(fh.read())
    return hs.hexdigest()[:16]


def summarize(path):
    import csv
    from collections import OrderedDict

    rows, hdr = [], None
    with open(path) as fh:
        for r in csv.reader(fh):
            if r and r[0] == "ID":
                hdr = r
                continue
            if hdr and len(r) == len(hdr):
                rows.append(dict(zip(hdr, r)))
    launches = OrderedDict()
    for r in rows:
        d = launches.setdefault(int(r["ID"]), {"name": r["Kernel Name"].split("(")[0].replace("void ", "")})
        d[r["Metric Name"]] = float(r["Metric Value"].replace(",", ""))
    seq = [launches[i] for i in sorted(launches)]
    for d in seq:
        d["name"] = d["name"].replace("ksdf::<unnamed>::", "").replace("ksdf::", "")
    starts = [k for k, d in enumerate(seq) if d["name"] == "k_bin_samples"]
    if not starts:
        raise SystemExit("no fit launch (k_bin_samples) in %s" % path)
    step = seq[starts[-1]:]
    stage, per = "fit", OrderedDict()
    for d in step:
        n = d["name"]
        if n.startswith("k_q_bin"):
            stage = "query"
        elif n.startswith("k_bw_count"):
            stage = "adjoint"
        st = stage if n.startswith("k_") else "other (PyTorch)"
        a = per.setdefault((st, n), {"n": 0, "ns": 0.0, "rd": 0.0, "wr": 0.0})
        a["n"] += 1
        a["ns"] += d.get("gpu__time_duration.sum", 0.0)
        a["rd"] += d.get("dram__bytes_read.sum", 0.0)
        a["wr"] += d.get("dram__bytes_write.sum", 0.0)
    tot = sum(a["ns"] for a in per.values())
    print("| stage | kernel | launches | ms (serialised) | share | DRAM read GB | DRAM write GB |")
    print("|---|---|---|---|---|---|---|")
    for (st, n), a in sorted(per.items(), key=lambda kv: -kv[1]["ns"]):
        print("| %s | %s | %d | %.3f | %.1f%% | %.3f | %.3f |" % (st, n, a["n"], a["ns"] / 1e6, 100 * a["ns"] / tot,
                                                            a["rd"] / 1e9, a["wr"] / 1e9))
    for st in ("fit", "query", "adjoint"):
        sel = [a for (s2, _), a in per.items() if s2 == st]
        print("\n%s: %d launches, %.3f ms, DRAM %.3f GB" % (st, sum(a["n"] for a in sel), sum(a["ns"] for a in sel) / 1e6,
                                                          sum(a["rd"] + a["wr"] for a in sel) / 1e9))
    qa = sum(a["rd"] + a["wr"] for (s2, _), a in per.items() if s2 in ("query", "adjoint"))
    print("\nstep total %.3f ms over %d launches" % (tot / 1e6, sum(a["n"] for a in per.values())))
    print("source_digest %s" % source_digest())
    print("query_adjoint_dram_bytes %d" % int(qa))


if __name__ == "__main__":
    if len(sys.argv) > 2 and sys.argv[1] == "--summarize":
        summarize(sys.argv[2])
    else:
        main(sys.argv[1:])
