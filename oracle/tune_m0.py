"""Seeded bisection of the bare mass m0 for a workload (oracle only).

The workload recipe asks for m0 such that the plain FP64 BiCGStab solve of
K x = b to relative residual 1e-10 takes a target number of iterations.  This
script measures that count with the oracle's full-operator BiCGStab (plain C
loops, oracle/c/oracle_dirac.c) on a Gaussian source seeded with 99, scanning
m0 on successively finer grids (8 values per pass, one process each), and
writes the result to oracle/m0_tuned.json.  The count falls monotonically as
m0 grows away from the critical mass.

    python -m oracle.tune_m0 tiny_4x8 medium_16x32
    python -m oracle.tune_m0 --bisect paper_24x128 -0.03 0.02 6 7
"""
import json
import multiprocessing as mp
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

import synth  # noqa: E402


def _count(args):
    u, m0, wl_name = args
    from oracle.dirac import WilsonClover
    from oracle.fast import FastK
    wl = synth.WORKLOADS[wl_name]
    b = synth.random_spinor(wl.ns, wl.nt, seed=99)
    fk = FastK(WilsonClover(u, m0, wl.csw, wl.xi))
    x, it, rr = fk.solve(b, tol=1e-10, maxiter=4 * wl.target_iters, nthreads=1)
    return m0, it, rr


def tune(name, lo=-0.16, hi=0.04, passes=3, width=8):
    from oracle import gauge
    wl = synth.WORKLOADS[name]
    u, _ = gauge.prepare_links(wl.gauge(), wl.rho_stout, wl.n_stout4d, 0)
    ctx = mp.get_context("spawn")
    history = []
    with ctx.Pool(width) as pool:
        for _ in range(passes):
            grid = np.linspace(lo, hi, width)
            res = pool.map(_count, [(u, float(m), name) for m in grid])
            history.extend(res)
            print(name, [(round(m, 5), it) for m, it, _ in res], flush=True)
            above = [m for m, it, _ in res if it >= wl.target_iters]
            below = [m for m, it, _ in res if it < wl.target_iters]
            if not above or not below:
                break
            lo, hi = max(above), min(below)
    best = min(history, key=lambda r: abs(r[1] - wl.target_iters))
    return {"m0": best[0], "iters": best[1], "relres": best[2], "target": wl.target_iters,
            "scan": [[m, it] for m, it, _ in sorted(history)]}


def bisect(name, lo, hi, probes, nthreads, cap_factor=2):
    """For lattices where one probe takes long: a plain bisection of m0 between lo (count above
    the target) and hi (below it), one probe at a time, each application of K split over
    nthreads threads; probes stop at cap_factor times the target iteration count."""
    from oracle import gauge
    from oracle.dirac import WilsonClover
    from oracle.fast import FastK
    wl = synth.WORKLOADS[name]
    u, _ = gauge.prepare_links(wl.gauge(), wl.rho_stout, wl.n_stout4d, 0)
    b = synth.random_spinor(wl.ns, wl.nt, seed=99)
    history = []
    for _ in range(probes):
        m = 0.5 * (lo + hi)
        fk = FastK(WilsonClover(u, m, wl.csw, wl.xi))
        _, it, rr = fk.solve_split(b, tol=1e-10, maxiter=cap_factor * wl.target_iters, nthreads=nthreads)
        history.append((m, it, rr))
        print(name, round(m, 6), it, rr, flush=True)
        if it >= wl.target_iters:
            lo = m
        else:
            hi = m
    best = min(history, key=lambda r: abs(r[1] - wl.target_iters))
    return {"m0": best[0], "iters": best[1], "relres": best[2], "target": wl.target_iters,
            "scan": [[m, it] for m, it, _ in sorted(history)], "method": "bisection"}


if __name__ == "__main__":
    out_path = os.path.join(HERE, "m0_tuned.json")
    data = json.load(open(out_path)) if os.path.exists(out_path) else {}
    if sys.argv[1:2] == ["--bisect"]:
        # python -m oracle.tune_m0 --bisect <workload> <lo> <hi> <probes> <threads>
        name, lo, hi, probes, nth = sys.argv[2], float(sys.argv[3]), float(sys.argv[4]), int(sys.argv[5]), int(sys.argv[6])
        data[name] = bisect(name, lo, hi, probes, nth)
        with open(out_path, "w") as f:
            json.dump(data, f, indent=1)
        print(name, data[name]["m0"], data[name]["iters"], flush=True)
        sys.exit(0)
    for name in sys.argv[1:]:
        data[name] = tune(name)
        with open(out_path, "w") as f:
            json.dump(data, f, indent=1)
        print(name, data[name]["m0"], data[name]["iters"], flush=True)
