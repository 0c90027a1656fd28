#!/usr/bin/env python
"""Benchmark of the stochastic-LapH quark-line path on GB300.

Default workload: the paper-shaped lattice 24^3 x 128, xi = 3.5, N_v = 64, dilution
(TI16, SF, LI8): 16 time-interlace groups x 4 spins x 8 LapH projectors = 512 diluted
sources per noise, four noises (two pion lines and the four lines of the I = 2 pi pi
correlator).  Per gauge configuration the Laplacian eigenvectors of all 128 slices are
computed once (a1, reported separately, as are gauge smearing and the sources).  One step =
one block of B diluted sources of one noise (default B = 32: one time-interlace group):
Z4 sources (a2), one batched mixed-precision solve of the block to FP64 true residual 1e-10
(a3), sink coefficients (a4); after the last noise of a group, the pion and I = 2 pi pi
correlators of that group's eight source times (a5).  Steps cycle through noises and groups.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--block B]

Prints one JSON line (rank 0).  Under torchrun every rank runs an independent replica (its
own noises); value = sources of all ranks / max rank time.  `--workload medium_16x32` runs
the 16^3 x 32 pipelined whole-path step instead (eigenvectors in every step).

    python bench.py --dslash-sweep [--dslash-nr 1,8,16,32,64] [--dslash-iters 50]

prints the Dslash half of the metric instead: the even-odd hop's algorithmic HBM GB/s
at several right-hand-side counts, FP32 (inner solver) and FP64, timed with CUDA events
around every hop launch inside solver iterations on the workload's lattice.
"""
import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "diluted LapH sources solved/s at resid 1e-10, learned vs plain; Dslash HBM GB/s"
UNIT = "sources/s"


def parse_args(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--workload", default="paper_24x128")
    p.add_argument("--mode", choices=["mixed", "bf16", "plain"], default="mixed",
                   help="mixed: FP32 inner solver; bf16: BF16-stored inner solver; plain: FP64 BiCGStab")
    p.add_argument("--block", type=int, default=32, help="diluted sources per step (paper-shaped workload; 8, 16 "
                                                           "or 32: a time-interlace group is 32)")
    p.add_argument("--variants", action="store_true",
                   help="also time the single-change ablations (paper-shaped workload; minutes)")
    p.add_argument("--plain-sample", type=int, default=1, help="sources solved by the plain FP64 comparison")
    p.add_argument("--e2e-steps", type=int, default=2)
    p.add_argument("--rhs-block", type=int, default=0, help="right-hand sides per solver launch (0: autotuned)")
    p.add_argument("--no-overlap", action="store_true",
                   help="run each step's stages one after another (default: the next batch's eigenvectors "
                        "overlap this batch's solves)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-clock-sampler", action="store_true",
                   help="do not run nvidia-smi beside the timed steps (for runs under a profiler)")
    p.add_argument("--inner-tol", type=float, default=None,
                   help="relative reduction each FP32 inner solve of the defect correction asks for (default: "
                        "3e-3 on the paper-shaped workload, where it measured fastest, else the library's 3e-4)")
    p.add_argument("--learned-sample", type=int, default=64, help="sources solved with the learned preconditioner")
    p.add_argument("--learned-pairs", type=int, default=64, help="(rho, phi) training pairs")
    p.add_argument("--learned-epochs", type=int, default=8)
    p.add_argument("--learned-batch", type=int, default=8)
    p.add_argument("--learned-lr", type=float, default=2e-3)
    p.add_argument("--learned-study", action="store_true",
                   help="print the held-out-field study of the learned preconditioner instead of the path step")
    p.add_argument("--study-fields", type=int, default=20, help="seeded fields (the last 4 held out)")
    p.add_argument("--study-workload", default="medium_16x32", help="lattice, smearing recipe and mass of the study")
    p.add_argument("--study-pairs", type=int, default=16, help="training pairs per training field")
    p.add_argument("--study-epochs", type=int, default=4, help="passes over all training fields")
    p.add_argument("--study-rhs", type=int, default=16, help="sources solved per held-out field")
    p.add_argument("--nn-sweep", action="store_true",
                   help="time one learned-network application (FP32 layers and tensor-core layers) against one "
                        "application of K on the medium lattice instead of the path step")
    p.add_argument("--nn-nr", type=int, default=64, help="right-hand sides of the network sweep")
    p.add_argument("--nn-reps", type=int, default=3, help="timed repetitions of the network sweep")
    p.add_argument("--dslash-sweep", action="store_true", help="print the Dslash GB/s sweep instead of the path step")
    p.add_argument("--dslash-nr", default="1,8,16,32,64", help="right-hand-side counts of the Dslash sweep")
    p.add_argument("--dslash-iters", type=int, default=50, help="solver iterations per sweep point")
    p.add_argument("--dslash-prec", default="fp32,fp64", help="precisions of the Dslash sweep")
    p.add_argument("--dslash-direct", action="store_true",
                   help="time laph_dslash_eo launches alone (clover-inverse mode) instead of inside solver iterations")
    p.add_argument("--dslash-nt", type=int, default=0,
                   help="time extent of the Dslash sweep's lattice (0: the workload's); the spatial extent stays the "
                        "workload's, so a short slab keeps an ncu capture to a few GB on the device")
    return p.parse_args(argv)


# ----------------------------------------------------------------------------- distribution
def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def aggregate_max(value, world, device=None):
    """Max of a float over ranks (barrier included); identity for one rank."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def whole_job_rate(units_per_rank, world, max_seconds):
    return units_per_rank * world / max_seconds


def replica_noise_ids(rank, nnoise):
    """Noise ids of one replica: rank r draws noises r*nnoise .. r*nnoise + nnoise - 1, so no
    two ranks solve the same diluted source (Z4 noise is a pure function of the id)."""
    return [rank * nnoise + k for k in range(nnoise)]


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.proc = None
        self.out = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(gpu_index)], stdout=self.out,
                                         stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.out.flush()
        self.out.seek(0)
        rows = [r.split(",") for r in self.out.read().strip().splitlines() if r.strip()]
        os.unlink(self.out.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except (ValueError, IndexError):
                continue
            for name, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------- CPU oracle sample
def oracle_sample(wl, seconds=15.0, threads=None, _cache={}):
    """Times the oracle's plain-C BiCGStab (oracle/c/oracle_dirac.c, one single-thread solve per
    host core, run concurrently) for a bounded number of iterations and scales to sources/s
    with the iteration count a full solve to 1e-10 takes at this m0 (oracle/m0_tuned.json).
    The loops' work does not depend on the link or clover values, so the seeded unsmeared links
    are used and, on lattices too large for the numpy clover (more than 2e5 sites), the site
    matrix without its clover term (the C loops still multiply by the full 12x12 matrix)."""
    from oracle.dirac import WilsonClover
    from oracle.fast import FastK
    import synth
    cores = threads or os.cpu_count() or 1
    big = wl.volume > 200_000
    key = (wl.name, cores)
    if key not in _cache:
        fk = FastK(WilsonClover(wl.gauge(), wl.m0, 0.0 if big else wl.csw, wl.xi))
        one = synth.random_spinor(wl.ns, wl.nt, seed=7)
        _cache[key] = (fk, np.ascontiguousarray(np.broadcast_to(one, (cores,) + one.shape)))
    fk, b = _cache[key]
    tuned = os.path.join(ROOT, "oracle", "m0_tuned.json")
    need = wl.target_iters
    if os.path.exists(tuned):
        rec = json.load(open(tuned)).get(wl.name.split("_nv")[0])   # the mass, not N_v, sets the count
        if rec:
            need = rec["iters"]
    if big:
        iters = 1 if seconds < 10 else 2
    else:
        t = time.perf_counter()
        fk.solve(b[:1], tol=1e-30, maxiter=4, nthreads=1)
        per_iter = (time.perf_counter() - t) / 4.0
        # stay below the length of a full solve so every thread runs exactly `iters` iterations
        iters = max(4, min(int(seconds / max(per_iter, 1e-6)), need // 2))
    t = time.perf_counter()
    _, its, _ = fk.solve(b, tol=1e-30, maxiter=iters, nthreads=cores)
    wall = time.perf_counter() - t
    iters = int(np.mean(its))
    rate = cores / (wall * need / iters)
    return {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{cores} concurrent single-thread oracle BiCGStab solves (plain C, full operator"
                      f"{', site term without clover' if big else ''}) on {wl.ns}^3x{wl.nt} run for {iters} "
                      f"iterations in {wall:.1f} s, scaled to the {need} iterations a solve to 1e-10 takes at "
                      f"this m0; eigenvectors, sources, sinks and contractions not included"}


# ----------------------------------------------------------------------------- ncu traffic record
HOP_KERNEL_VERSION = "hop3_tma_ns2_zblock8_pair_cj"


def measured_traffic_ratio(workload, family="dslash_fp32"):
    """DRAM bytes over algorithmic bytes of one captured hop launch (hop3_kernel) from the
    committed ncu summary profiles/hop3_kernel_<precision>_<workload>.md, line
    'traffic_bytes_per_launch: N version V nr R algorithmic A'; None when absent or taken on
    another kernel version.  The capture runs a smaller lattice than the bench (the device
    memory rule for ncu captures); traffic scales with the sites x RHS processed, so the bench
    reports ratio x its own algorithmic bytes per launch."""
    prec = family.split("_")[-1]
    workload = workload.split("_nv")[0]   # the stencil does not depend on N_v
    path = os.path.join(ROOT, "profiles", f"hop3_kernel_{prec}_{workload}.md")
    if not os.path.exists(path):
        return None
    for line in open(path):
        parts = line.split()
        if len(parts) >= 8 and parts[0] == "traffic_bytes_per_launch:" and parts[2] == "version":
            if parts[3] == HOP_KERNEL_VERSION and parts[6] == "algorithmic":
                return float(parts[1]) / float(parts[7])
    return None


def learned_leg(L, torch, path, wl, u, rhs, args):
    """The learned right preconditioner in FGCR(16) on a sample of the step's diluted sources.
    Training pairs (rho, phi = K^-1 rho): seeded Gaussian rho on the same gauge field, solved by
    the library to 1e-10; training runs on the GPU with the library's kernels and is reported
    separately, not in the solve rate.  The sample is then solved with the trained network and
    with the seeded start network, which shows what training gains."""
    ctx, lat = path.ctx, path.lat
    npairs = args.learned_pairs
    gen = torch.Generator(device="cuda")
    gen.manual_seed(4242)
    shape = (npairs, wl.nt, wl.ns, wl.ns, wl.ns, 4, 3)
    rho = torch.complex(torch.randn(shape, dtype=torch.float64, device="cuda", generator=gen),
                        torch.randn(shape, dtype=torch.float64, device="cuda", generator=gen))
    phi = torch.empty_like(rho)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    L.dirac_solve_batch(ctx, lat, u, wl.m0, wl.csw, rho, phi, npairs, L.solver_params(mode=L.MIXED_FP32))
    torch.cuda.synchronize()
    pairs_s = time.perf_counter() - t0
    nw = L.laph_precond_size()
    w0 = np.zeros(nw, dtype=np.float32)
    L.laph_precond_init(7, wl.m0 + 1.0 + 3.0 / wl.xi, w0)
    w = w0.copy()
    adam = np.zeros(2 * nw, dtype=np.float32)
    grad = torch.empty(nw // 2, dtype=torch.complex128, device="cuda")
    nb = min(npairs, 16)
    loss0 = L.laph_precond_grad(ctx, lat, u, wl.m0, wl.csw, w0, rho[:nb], phi[:nb], nb, grad)
    t0 = time.perf_counter()
    L.laph_precond_train(ctx, lat, u, wl.m0, wl.csw, rho, phi, npairs, args.learned_epochs, args.learned_batch,
                         args.learned_lr, 0, w, adam)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    loss1 = L.laph_precond_grad(ctx, lat, u, wl.m0, wl.csw, w, rho[:nb], phi[:nb], nb, grad)
    del rho, phi
    n = min(args.learned_sample, rhs.shape[0])
    sub = rhs[:n].clone()
    xs = torch.empty_like(sub)
    out = {"sample": n, "train_pairs": npairs, "train_epochs": args.learned_epochs, "train_batch": args.learned_batch,
           "pairs_solve_s": pairs_s, "train_s": train_s, "loss_start": loss0, "loss_trained": loss1, "_weights": w}
    stream = torch.cuda.current_stream()
    # the seeded start network converges ~10x slower: it is timed on the first 8 sources only
    for name, ww, m in (("trained", w, n), ("start", w0, min(n, 8))):
        wdev = torch.from_numpy(ww).cuda()
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        reps = L.dirac_solve_batch(ctx, lat, u, wl.m0, wl.csw, sub[:m], xs[:m], m,
                                   L.solver_params(mode=L.LEARNED, weights=wdev, rhs_block=m))
        ev1.record(stream)
        torch.cuda.synchronize()
        out[name] = {"sources_per_s": m / (ev0.elapsed_time(ev1) / 1000.0), "sample": m,
                     "iters_mean": float(np.mean([r.iters for r in reps])), "iters_max": max(r.iters for r in reps),
                     "fallback_used": int(sum(r.fallback_used for r in reps)),
                     "true_resid_max": max(r.true_resid for r in reps)}
    return out


class PathStep:
    """Buffers and the five stages of one pass: eigenvectors, sources for every source
    time and noise, one batched solve of all diluted sources, sinks, and the
    correlators of every channel and source time."""

    def __init__(self, L, torch, path, spec, wl, rank, mode, rhs_block, projectors_for_time):
        self.L, self.torch, self.path, self.wl = L, torch, path, wl
        self.mode, self.rhs_block = mode, rhs_block
        self.t0s = list(wl.source_times)
        self.bss = [projectors_for_time(spec, t0) for t0 in self.t0s]
        self.nb = len(self.bss[0])
        self.nnoise = wl.n_noise
        self.nsrc = len(self.t0s) * self.nnoise * self.nb
        self.noise_ids = replica_noise_ids(rank, self.nnoise)
        self.rhs = path.field(self.nsrc)
        self.sol = torch.empty_like(self.rhs)
        self.coef = torch.empty((self.nsrc, wl.nt, 4, wl.nv), dtype=torch.complex128, device="cuda")
        self.codes = torch.empty((self.nnoise, wl.nt, 4, wl.nv), dtype=torch.uint8, device="cuda")
        self.evals = torch.empty((wl.nt, wl.nv), dtype=torch.float64, device="cuda")
        self.evecs = torch.empty((wl.nt, wl.nv, wl.ns ** 3, 3), dtype=torch.complex128, device="cuda")
        self.channels = [L.CH_PION, L.CH_SCALAR, L.CH_RHO]
        self.corr = torch.empty((len(self.t0s), len(self.channels), wl.nt), dtype=torch.complex128, device="cuda")
        self.corr_host = torch.empty_like(self.corr, device="cpu").pin_memory()
        self.stats = {}

    def block(self, ti, k):
        o = (ti * self.nnoise + k) * self.nb
        return slice(o, o + self.nb)

    def enable_overlap(self, eig_path):
        """Pipelined steps: the eigenvectors of the next batch are computed by a second library
        context on its own stream (FP64-bound kernels) while this batch's sources, solves (FP32
        and memory bound), sinks and correlators run on the main stream.  Each step still does
        the whole path's work: over K steps, K eigensolves and K solve stages."""
        torch = self.torch
        self.eig_path = eig_path
        # the solves keep the SMs first; the eigensolver's blocks fill what they leave
        self.main_stream = torch.cuda.Stream(priority=-1)
        self.eig_stream = torch.cuda.Stream(priority=0)
        self.evecs_next = torch.empty_like(self.evecs)
        self.evals_next = torch.empty_like(self.evals)
        self.primed = False

    def run_overlapped(self, u_in, ut_in, read_back=False):
        import threading
        torch = self.torch
        if not self.primed:   # the first batch's eigenvectors (outside any timed region)
            with torch.cuda.stream(self.eig_stream):
                self.eig_path.eigvecs(ut_in, self.evals_next, self.evecs_next)
            self.eig_stream.synchronize()
            self.primed = True
        # this batch uses the vectors computed during the previous step
        self.evecs, self.evecs_next = self.evecs_next, self.evecs
        self.evals, self.evals_next = self.evals_next, self.evals
        box = {}

        def eig_lane():
            try:
                with torch.cuda.stream(self.eig_stream):
                    box["rep"] = self.eig_path.eigvecs(ut_in, self.evals_next, self.evecs_next)[2]
            except Exception as e:   # surfaced on the main thread below
                box["err"] = e

        th = threading.Thread(target=eig_lane)
        th.start()
        with torch.cuda.stream(self.main_stream):
            self.run(u_in, ut_in, read_back=read_back, skip_eig=True)
        th.join()
        if "err" in box:
            raise box["err"]
        self.main_stream.wait_stream(self.eig_stream)
        rep = box["rep"]
        self.stats["eig"] = (rep.restarts, rep.matvecs, rep.max_resid)

    def run(self, u_in, ut_in, read_back=False, events=None, skip_eig=False):
        p = self.path
        mark = (lambda i: events[i].record(self.torch.cuda.current_stream())) if events else (lambda i: None)
        mark(0)
        if not skip_eig:
            _, _, rep = p.eigvecs(ut_in, self.evals, self.evecs)
            self.stats["eig"] = (rep.restarts, rep.matvecs, rep.max_resid)
        mark(1)
        for ti, bs in enumerate(self.bss):
            for k in range(self.nnoise):
                p.sources(self.evecs, self.noise_ids[k], self.wl.config_id, bs, out=self.rhs[self.block(ti, k)],
                          codes=self.codes[k])
        mark(2)
        _, reps = p.solve(u_in, self.rhs, mode=self.mode, sol=self.sol, rhs_block=self.rhs_block)
        mark(3)
        p.sinks(self.evecs, self.sol, out=self.coef)
        mark(4)
        for ti, (t0, bs) in enumerate(zip(self.t0s, self.bss)):
            for i, ch in enumerate(self.channels):
                p.correlate(ch, t0, bs, [self.coef[self.block(ti, 0)], self.coef[self.block(ti, 1)]],
                            [self.codes[0], self.codes[1]], out=self.corr[ti, i])
        mark(5)
        if read_back:
            self.corr_host.copy_(self.corr, non_blocking=True)
        self.stats["iters"] = [r.iters for r in reps]
        self.stats["resid"] = max(r.true_resid for r in reps)


def profiled_step(L, torch, st, u, ut):
    """ms per stage (CUDA events on the launching stream) and per kernel family of one step."""
    torch.cuda.synchronize()
    L.laph_profile_reset()
    L.laph_profile_enable(2)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
    st.run(u, ut, events=ev)
    torch.cuda.synchronize()
    L.laph_profile_enable(0)
    names = ["eigvecs", "sources", "solve", "sinks", "correlate"]
    stages = {n: ev[i].elapsed_time(ev[i + 1]) for i, n in enumerate(names)}
    fams = {}
    for f in L.laph_profile_families():
        n, ms, by, fl = L.laph_profile_read(f)
        fams[f] = {"launches": n, "ms": ms, "bytes": by}
    L.laph_profile_reset()
    return {"stage_ms": stages, "family_ms": fams}


class StreamStep:
    """One step of the paper-shaped workload: B diluted sources of one noise (a2), their batched
    mixed solve (a3) and sink coefficients (a4); after the last block of the last noise of a
    time-interlace group, the correlators of the group's source times (a5).  Step i works on
    noise (i // parts) % nnoise and group (i // (parts nnoise)) % nT, part i % parts of its 32
    projectors, so consecutive steps cycle through every source of a configuration."""

    def __init__(self, L, torch, path, spec, wl, rank, mode, block, evecs, inner_tol=0.0):
        from paper_1104_3870_gb300.pipeline import n_projectors
        self.L, self.torch, self.path, self.wl, self.mode = L, torch, path, wl, mode
        self.inner_tol = inner_tol
        (kT, JT), (kS, JS), (kL, JL) = spec.dil
        assert kT == 3, "the streaming step expects time interlacing"
        self.nT = JT
        nS, nL = n_projectors(kS, JS, 4), n_projectors(kL, JL, wl.nv)
        self.groups = [[(g * nS + a) * nL + l for a in range(nS) for l in range(nL)] for g in range(self.nT)]
        self.ng = len(self.groups[0])
        assert self.ng % block == 0, "the block must divide a time-interlace group"
        self.block, self.parts = block, self.ng // block
        self.nnoise = wl.n_noise
        self.noise_ids = replica_noise_ids(rank, self.nnoise)
        self.evecs = evecs
        self.rhs = path.field(block)
        self.sol = torch.empty_like(self.rhs)
        dev = self.rhs.device
        self.coef = torch.empty((self.nnoise, self.ng, wl.nt, 4, wl.nv), dtype=torch.complex128, device=dev)
        self.codes = torch.empty((self.nnoise, wl.nt, 4, wl.nv), dtype=torch.uint8, device=dev)
        self.ntimes = wl.nt // self.nT
        self.corr = torch.zeros((3, self.ntimes, wl.nt), dtype=torch.complex128, device=dev)
        self.coef_host = torch.empty((block, wl.nt, 4, wl.nv), dtype=torch.complex128).pin_memory()
        self.i = 0
        self.stats = {"iters_max": 0, "resid_max": 0.0, "correlator_groups": 0}

    def where(self, i):
        part = i % self.parts
        k = (i // self.parts) % self.nnoise
        g = (i // (self.parts * self.nnoise)) % self.nT
        return k, g, part

    def run(self, u_in, read_back=False, events=None):
        p, L = self.path, self.L
        mark = (lambda j: events[j].record(self.torch.cuda.current_stream())) if events else (lambda j: None)
        k, g, part = self.where(self.i)
        lo = part * self.block
        bs = self.groups[g][lo:lo + self.block]
        mark(0)
        p.sources(self.evecs, self.noise_ids[k], self.wl.config_id, bs, out=self.rhs, codes=self.codes[k])
        mark(1)
        _, reps = p.solve(u_in, self.rhs, mode=self.mode, sol=self.sol, rhs_block=self.block, inner_tol=self.inner_tol)
        mark(2)
        p.sinks(self.evecs, self.sol, out=self.coef[k, lo:lo + self.block])
        mark(3)
        if k == self.nnoise - 1 and part == self.parts - 1:
            bg = self.groups[g]
            c, n = self.coef, self.codes
            for j in range(self.ntimes):
                t0 = g + j * self.nT
                p.correlate(L.CH_PION, t0, bg, [c[0], c[1]], [n[0], n[1]], out=self.corr[0, j])
                if self.nnoise >= 4:
                    p.correlate(L.CH_PION, t0, bg, [c[2], c[3]], [n[2], n[3]], out=self.corr[1, j])
                    p.correlate(L.CH_PIPI_I2, t0, bg, [c[0], c[1], c[2], c[3]], [n[0], n[1], n[2], n[3]],
                                out=self.corr[2, j])
            self.stats["correlator_groups"] += 1
        mark(4)
        if read_back:
            self.coef_host.copy_(self.coef[k, lo:lo + self.block], non_blocking=True)
        self.stats["iters_max"] = max(self.stats["iters_max"], max(r.iters for r in reps))
        self.stats["resid_max"] = max(self.stats["resid_max"], max(r.true_resid for r in reps))
        self.i += 1


def roofline_from(L, fam_name, kernel, n, kms, kbytes, hbm_peak, peaks, ratio):
    achieved = kbytes / (kms / 1000.0) / 1e9 if kms else None
    return {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
            "frac": (achieved / hbm_peak) if achieved else None,
            "traffic": ratio * kbytes / n if (ratio and n) else None,
            "kernel": kernel, "family": fam_name, "launches": n, "avg_launch_us": 1000.0 * kms / n if n else None,
            "algorithmic_bytes_per_launch": kbytes / n if n else None,
            "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)" if peaks else "fallback 6.8 TB/s"}


def nvtx_push(name):
    try:
        import torch
        torch.cuda.nvtx.range_push(name)
    except Exception:   # an NVTX-less build only loses the profiler marker
        pass


def nvtx_pop():
    try:
        import torch
        torch.cuda.nvtx.range_pop()
    except Exception:
        pass


def run_stream(args):
    """The paper-shaped workload (see the module docstring): eigenvectors once, then K timed
    steps of B diluted sources each."""
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    from paper_1104_3870_gb300 import build
    build.build()
    from paper_1104_3870_gb300 import laph as L
    from paper_1104_3870_gb300.pipeline import LapHPath, LatticeSpec
    import synth

    wl = synth.WORKLOADS[args.workload]
    spec = LatticeSpec(wl.ns, wl.nt, wl.xi, wl.m0, wl.csw, wl.nv, (wl.dil_time, wl.dil_spin, wl.dil_laph),
                       wl.rho_stout, wl.n_stout4d, wl.n_stout3d)
    path = LapHPath(spec, local)
    stream = torch.cuda.current_stream()

    def ev_pair():
        return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    setup = {}
    t = time.perf_counter()
    u0 = wl.gauge()
    setup["gauge_host_s"] = time.perf_counter() - t
    a, b = ev_pair()
    a.record(stream)
    u, ut = path.prepare_links(u0)                       # a0: setup
    b.record(stream)
    del u0
    e0, e1 = ev_pair()
    e0.record(stream)
    evals, evecs, erep = path.eigvecs(ut)                # a1: once per configuration
    e1.record(stream)
    torch.cuda.synchronize()
    setup["smear_ms"] = a.elapsed_time(b)
    setup["eigvecs_ms"] = e0.elapsed_time(e1)
    setup["eigvecs"] = {"restarts": erep.restarts, "matvecs_per_slice": erep.matvecs, "nconv": erep.nconv,
                        "max_resid": erep.max_resid, "lambda_C_max": erep.lambda_C}
    del ut
    mode = {"mixed": L.MIXED_FP32, "bf16": L.MIXED_BF16, "plain": L.PLAIN_FP64}[args.mode]
    if args.inner_tol is None:
        # measured on this workload (blocks of 32, one GB300): 3e-4 -> 12.9 s per step, 2e-3 -> 11.9 s,
        # 3e-3 -> 11.5 s; a looser inner goal restarts BiCGStab from the FP64 residual more often
        args.inner_tol = 3e-3
    st = StreamStep(L, torch, path, spec, wl, rank, mode, args.block, evecs, args.inner_tol)

    for _ in range(args.warmup):
        st.run(u)
    torch.cuda.synchronize()
    barrier(world)
    clocks = ClockSampler(local) if rank == 0 and not args.no_clock_sampler else None
    L.laph_profile_enable(0)
    launches0 = L.laph_launch_count()
    t0, t1 = ev_pair()
    torch.cuda.synchronize()
    nvtx_push("timed_steps")   # lets a profiler keep to the timed launches (ncu --nvtx-include timed_steps/)
    t0.record(stream)
    for _ in range(args.steps):
        st.run(u)
    t1.record(stream)
    torch.cuda.synchronize()
    nvtx_pop()
    launches = L.laph_launch_count() - launches0
    clk = clocks.stop() if clocks else None
    ms = t0.elapsed_time(t1) / args.steps
    ms_max = aggregate_max(ms, world, device="cuda")
    barrier(world)
    value = whole_job_rate(args.block, world, ms_max / 1000.0)

    # roofline of the dominant kernel family from a separate pass with per-launch event timing
    peaks_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    peaks = json.load(open(peaks_path)) if os.path.exists(peaks_path) else {}
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    L.laph_profile_reset()
    L.laph_profile_enable(1)
    for _ in range(2):
        st.run(u)
    torch.cuda.synchronize()
    L.laph_profile_enable(0)
    fam = {L.MIXED_FP32: "dslash_fp32", L.MIXED_BF16: "dslash_bf16"}.get(mode, "dslash_fp64")
    n, kms, kbytes, _ = L.laph_profile_read(fam)
    ratio = measured_traffic_ratio(wl.name, fam)
    kernel = {"dslash_fp32": "FP32 even-odd hop (hop3_kernel, TMA-fed, FP32 spinors)",
              "dslash_bf16": "even-odd hop (hop3_kernel, TMA-fed, BF16 spinors, FP32 links/clover/arithmetic)",
              "dslash_fp64": "hop_kernel<double>"}[fam]
    roofline = roofline_from(L, fam, kernel, n, kms, kbytes, hbm_peak, peaks, ratio)
    roofline["note"] = "two untimed steps with every stencil launch timed by CUDA events on its stream"

    # breakdown: one more step with every kernel family timed, and per-stage events
    L.laph_profile_reset()
    L.laph_profile_enable(2)
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
    st.run(u, events=evs)
    torch.cuda.synchronize()
    L.laph_profile_enable(0)
    stages = {nm: evs[j].elapsed_time(evs[j + 1]) for j, nm in enumerate(["sources", "solve", "sinks", "correlate"])}
    fams = {}
    for f in L.laph_profile_families():
        nn, fms, fby, _ = L.laph_profile_read(f)
        fams[f] = {"launches": nn, "ms": fms, "bytes": fby,
                   "GBs": (fby / (fms / 1000.0) / 1e9) if (fms and fby) else None}
    L.laph_profile_reset()

    # e2e through the public API with host buffers: the links sit in pinned host memory and are
    # staged by the library in every solve; the step's coefficients are read back to the host.
    u_h = u.cpu().pin_memory()
    torch.cuda.synchronize()
    t = time.perf_counter()
    for _ in range(args.e2e_steps):
        st.run(u_h, read_back=True)
    torch.cuda.synchronize()
    e2e_s = aggregate_max((time.perf_counter() - t) / max(args.e2e_steps, 1), world, device="cuda")
    e2e = {"value": whole_job_rate(args.block, world, e2e_s), "unit": UNIT,
           "h2d_bytes_per_step": int(u_h.numel() * u_h.element_size()),
           "d2h_bytes_per_step": int(st.coef_host.numel() * st.coef_host.element_size())}
    del u_h

    variants = stream_variants(L, torch, path, wl, u, st, args, mode)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": {L.MIXED_FP32: "f32/f64", L.MIXED_BF16: "bf16-storage/f32/f64"}.get(mode, "f64"),
            "data": "synthetic",
            "config": {"workload": f"{wl.name}: {wl.ns}^3x{wl.nt}, xi={wl.xi}, N_v={wl.nv}, dilution (TI{st.nT}, SF, "
                                   f"LI8), {st.ng * st.nT} diluted sources per noise, {st.nnoise} noises per "
                                   f"replica, m0={wl.m0}",
                       "sources_per_step": args.block, "solver": args.mode, "tol": 1e-10, "rhs_block": args.block,
                       "inner_tol": args.inner_tol,
                       "step": "Z4 sources + one batched solve + sinks of one block (+ the correlators of a "
                               "time-interlace group after its last block); eigenvectors once per configuration "
                               "(setup.eigvecs_ms)",
                       "l2": "inputs larger than L2 (one block's solver fields > 10 GB)",
                       "parallelism": f"replicas{world}"},
            "roofline": roofline, "e2e": e2e, "gpu_launches": launches, "clocks": clk,
            "setup": setup, "breakdown": {"stage_ms": stages, "family_ms": fams}, "variants": variants,
            "path_stats": dict(st.stats)}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = oracle_sample(wl)
    if rank == 0:
        print(json.dumps(line), flush=True)
    path.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def stream_variants(L, torch, path, wl, u, st, args, mode):
    """Comparisons on samples of the workload's own diluted sources, each timed with CUDA events
    on the current stream: the plain FP64 solve one right-hand side per launch (the baseline the
    reshaped solver must beat) and, with --variants, the single-change ablations."""
    stream = torch.cuda.current_stream()
    out = {}
    if mode == L.PLAIN_FP64 or args.plain_sample <= 0:
        return out

    def timed_solve(n, prm):
        sub = st.rhs[:n].clone()
        xs = torch.empty_like(sub)
        torch.cuda.synchronize()
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        reps = L.dirac_solve_batch(path.ctx, path.lat, u, wl.m0, wl.csw, sub, xs, n, prm)
        a1.record(stream)
        torch.cuda.synchronize()
        return {"sources_per_s": n / (a0.elapsed_time(a1) / 1000.0), "sample": n,
                "iters": [r.iters for r in reps], "true_resid_max": max(r.true_resid for r in reps)}

    n = min(args.plain_sample, args.block)
    out["plain_fp64_one_rhs"] = timed_solve(n, L.solver_params(mode=L.PLAIN_FP64, rhs_block=1))
    if args.variants:
        out["ablations"] = {
            "precision_only: mixed FP32/FP64, one RHS per launch":
                timed_solve(min(2, args.block), L.solver_params(mode=L.MIXED_FP32, rhs_block=1)),
            "batching_only: plain FP64, 8 RHS per launch":
                timed_solve(min(8, args.block), L.solver_params(mode=L.PLAIN_FP64, rhs_block=8)),
        }
    return out


def run_ours(args):
    if args.workload.startswith("paper_24x128"):
        run_stream(args)
    else:
        run_path(args)


# ----------------------------------------------------------------------------- our arm
def run_path(args):
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    from paper_1104_3870_gb300 import build
    build.build()
    from paper_1104_3870_gb300 import laph as L
    from paper_1104_3870_gb300.pipeline import LapHPath, LatticeSpec, projectors_for_time
    import synth

    wl = synth.WORKLOADS[args.workload]
    spec = LatticeSpec(wl.ns, wl.nt, wl.xi, wl.m0, wl.csw, wl.nv, (wl.dil_time, wl.dil_spin, wl.dil_laph),
                       wl.rho_stout, wl.n_stout4d, wl.n_stout3d)
    path = LapHPath(spec, local)
    u, ut = path.prepare_links(wl.gauge())          # a0: setup, not timed
    mode = L.MIXED_FP32 if args.mode == "mixed" else L.PLAIN_FP64
    st = PathStep(L, torch, path, spec, wl, rank, mode, args.rhs_block, projectors_for_time)
    nsrc, nb, nnoise = st.nsrc, st.nb, st.nnoise
    rhs, sol, corr_host, stats = st.rhs, st.sol, st.corr_host, st.stats

    overlap = not args.no_overlap
    eig_path = None
    if overlap:
        eig_path = LapHPath(spec, local)
        st.enable_overlap(eig_path)

    def step(u_in, ut_in, read_back=False):
        if overlap:
            st.run_overlapped(u_in, ut_in, read_back=read_back)
        else:
            st.run(u_in, ut_in, read_back=read_back)

    # the first warm-up step runs alone: the solver's block autotuner times its candidates then,
    # on a GPU no other stream is using
    st.run(u, ut)
    for _ in range(max(args.warmup - 1, 0)):
        step(u, ut)
    torch.cuda.synchronize()
    barrier(world)
    clocks = ClockSampler(local) if rank == 0 and not args.no_clock_sampler else None
    L.laph_profile_reset()
    L.laph_profile_enable(1)
    launches0 = L.laph_launch_count()
    stream = st.main_stream if overlap else torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        step(u, ut)
    e1.record(stream)
    torch.cuda.synchronize()
    launches = L.laph_launch_count() - launches0
    L.laph_profile_enable(0)
    clk = clocks.stop() if clocks else None
    ms = e0.elapsed_time(e1) / args.steps
    ms_max = aggregate_max(ms, world, device="cuda")
    barrier(world)
    value = whole_job_rate(nsrc, world, ms_max / 1000.0)
    n32, ms32, by32, fl32 = L.laph_profile_read("dslash_fp32")
    n64, ms64, by64, fl64 = L.laph_profile_read("dslash_fp64")
    peaks_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    peaks = json.load(open(peaks_path)) if os.path.exists(peaks_path) else {}
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    if mode == L.MIXED_FP32 and n32:
        fam, n, kms, kbytes = "dslash_fp32 (hop3_kernel: TMA-fed FP32 hop)", n32, ms32, by32
    else:
        fam, n, kms, kbytes = "dslash_fp64 (hop_kernel<double>)", n64, ms64, by64
    achieved = kbytes / (kms / 1000.0) / 1e9 if kms else None
    ratio = measured_traffic_ratio(wl.name)
    traffic = ratio * kbytes / n if (ratio and n and mode == L.MIXED_FP32) else None
    roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                "frac": (achieved / hbm_peak) if achieved else None, "traffic": traffic,
                "kernel": fam, "launches": n, "avg_launch_us": 1000.0 * kms / n if n else None,
                "algorithmic_bytes_per_launch": kbytes / n if n else None,
                "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)" if peaks else "fallback 6.8 TB/s"}

    # one more (untimed) step with every kernel family timed and per-stage events: the breakdown
    breakdown = profiled_step(L, torch, st, u, ut)
    # the same roofline figure from that sequential step, where the stencil has the GPU to itself
    # (in the timed region the next batch's eigensolver shares the SMs with it)
    iso = breakdown["family_ms"].get("dslash_fp32" if mode == L.MIXED_FP32 else "dslash_fp64")
    if iso and iso["ms"]:
        a_iso = iso["bytes"] / (iso["ms"] / 1000.0) / 1e9
        roofline_isolated = {"achieved": a_iso, "peak": hbm_peak, "unit": "GB/s", "frac": a_iso / hbm_peak,
                             "launches": iso["launches"], "avg_launch_us": 1000.0 * iso["ms"] / iso["launches"],
                             "note": "one untimed step with the stages run one after another"}
    else:
        roofline_isolated = None

    # e2e through the public API with host buffers: links in pinned host memory are staged by the
    # library each call; the correlators are read back to host.
    u_h = u.cpu().pin_memory()
    ut_h = ut.cpu().pin_memory()
    torch.cuda.synchronize()
    t = time.perf_counter()
    for _ in range(args.e2e_steps):
        step(u_h, ut_h, read_back=True)
    torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t) / max(args.e2e_steps, 1)
    e2e_s = aggregate_max(e2e_s, world, device="cuda")
    e2e = {"value": whole_job_rate(nsrc, world, e2e_s), "unit": UNIT,
           "h2d_bytes_per_step": int(u_h.numel() * u_h.element_size() * 2),
           "d2h_bytes_per_step": int(corr_host.numel() * corr_host.element_size())}

    # plain FP64 comparison on a sample of the same sources: one right-hand side per launch.
    # The variants run on this thread's current stream and are timed there.
    stream = torch.cuda.current_stream()
    variants = {}
    if args.plain_sample > 0 and mode == L.MIXED_FP32:
        sub = rhs[:args.plain_sample].clone()
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        _, preps = path.solve(u, sub, mode=L.PLAIN_FP64, rhs_block=1)
        ev1.record(stream)
        torch.cuda.synchronize()
        ms_plain = ev0.elapsed_time(ev1)
        variants["plain_fp64_one_rhs"] = {"sources_per_s": args.plain_sample / (ms_plain / 1000.0),
                                          "iters": [r.iters for r in preps], "sample": args.plain_sample,
                                          "true_resid_max": max(r.true_resid for r in preps)}
    solve_only = None
    if mode == L.MIXED_FP32:
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        _, sreps = path.solve(u, rhs, mode=L.MIXED_FP32, sol=sol)
        ev1.record(stream)
        torch.cuda.synchronize()
        solve_only = nsrc / (ev0.elapsed_time(ev1) / 1000.0)
        vh = wl.ns ** 3 * wl.nt // 2
        tuned = max([L.laph_tuned_block(path.ctx, vh, c) for c in (16, 32, 64, 128)])
        variants["mixed_fp32_batched_solve_only"] = {"sources_per_s": solve_only,
                                                     "rhs_block": (args.rhs_block or tuned),
                                                     "rhs_block_source": "argument" if args.rhs_block else "autotuned",
                                                     "iters_max": max(r.iters for r in sreps)}

    if args.learned_sample > 0 and mode == L.MIXED_FP32:
        variants["learned_fgcr"] = learned_leg(L, torch, path, wl, u, rhs, args)
        w_trained = variants["learned_fgcr"].pop("_weights")
    else:
        w_trained = None

    # single-change ablations on small samples of the same sources: each turns on one of
    # precision (FP32 inner), batching (many RHS per launch) or the learned preconditioner
    if args.plain_sample > 0 and mode == L.MIXED_FP32:
        def timed_solve(n, prm):
            sub = rhs[:n].clone()
            xs = torch.empty_like(sub)
            torch.cuda.synchronize()
            a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            reps = L.dirac_solve_batch(path.ctx, path.lat, u, wl.m0, wl.csw, sub, xs, n, prm)
            a1.record(stream)
            torch.cuda.synchronize()
            return {"sources_per_s": n / (a0.elapsed_time(a1) / 1000.0), "sample": n,
                    "iters_mean": float(np.mean([r.iters for r in reps])),
                    "true_resid_max": max(r.true_resid for r in reps)}
        abl = {"precision_only: mixed FP32/FP64, one RHS per launch":
               timed_solve(2, L.solver_params(mode=L.MIXED_FP32, rhs_block=1)),
               "batching_only: plain FP64, 8 RHS per launch":
               timed_solve(8, L.solver_params(mode=L.PLAIN_FP64, rhs_block=8))}
        if w_trained is not None:
            abl["learned_only: learned FGCR, one RHS per launch"] = timed_solve(
                2, L.solver_params(mode=L.LEARNED, weights=torch.from_numpy(w_trained).cuda(), rhs_block=1))
        variants["ablations"] = abl

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32/f64" if mode == L.MIXED_FP32 else "f64", "data": "synthetic",
            "config": {"workload": f"{wl.name}: {wl.ns}^3x{wl.nt}, xi={wl.xi}, N_v={wl.nv}, dilution "
                                   f"{(wl.dil_time, wl.dil_spin, wl.dil_laph)} at source times {list(wl.source_times)}, "
                                   f"{nnoise} noises x {nb} projectors each per replica",
                       "sources_per_step": nsrc, "solver": args.mode, "tol": 1e-10,
                       "overlap": "next batch's eigenvectors beside this batch's solves" if overlap else "none",
                       "l2": "inputs larger than L2 (solver working set > 1 GB)", "parallelism": f"replicas{world}"},
            "roofline": roofline, "roofline_isolated": roofline_isolated, "e2e": e2e, "gpu_launches": launches,
            "clocks": clk, "breakdown": breakdown,
            "variants": variants,
            "path_stats": {"true_resid_max": stats.get("resid"), "inner_iters_max": max(stats.get("iters", [0])),
                           "eig_restarts_matvecs_resid": stats.get("eig")}}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = oracle_sample(wl)
    if rank == 0:
        print(json.dumps(line), flush=True)
    path.close()
    if eig_path is not None:
        eig_path.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# ----------------------------------------------------------------------------- reference arm (the oracle)
def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return
    import synth
    wl = synth.WORKLOADS[args.workload]
    for _ in range(args.warmup):
        oracle_sample(wl, seconds=4.0)
    vals = []
    t = time.perf_counter()
    for _ in range(args.steps):
        vals.append(oracle_sample(wl, seconds=8.0))
    wall = (time.perf_counter() - t) / args.steps
    v = float(np.mean([x["value"] for x in vals]))
    cb = dict(vals[-1])
    cb["value"] = v
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000.0 * wall, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl.name, "sources_per_step": "bounded sample", "solver": "oracle BiCGStab"},
            "cpu_baseline": cb,
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def dslash_direct_rows(L, torch, path, wl, u, prec, fam, real, hbm, args):
    """One laph_dslash_eo call per repetition (clover-inverse mode, even output parity) on
    random half-lattice fields; the library times the hop launch itself with CUDA events.
    Each call rebuilds the operator first, so the links and clover may still be in L2 when
    the hop starts (an optimistic figure for small right-hand-side counts)."""
    vh = wl.ns ** 3 * wl.nt // 2
    cdt = torch.complex64 if prec == "fp32" else torch.complex128
    rows = []
    for nr in [int(v) for v in args.dslash_nr.split(",")]:
        x = torch.randn((vh, 12, nr), dtype=cdt, device="cuda")
        out = torch.empty_like(x)
        times = []
        by = 0.0
        for rep in range(max(args.dslash_iters, 1)):
            L.laph_profile_reset()
            L.laph_profile_enable(1)
            L.laph_dslash_eo(path.ctx, path.lat, u, wl.m0, wl.csw, 0, L.HOP_CLOVINV,
                             L.PREC_FP32 if prec == "fp32" else L.PREC_FP64, x, None, out, nr)
            torch.cuda.synchronize()
            L.laph_profile_enable(0)
            n, ms, by, fl = L.laph_profile_read(fam)
            times.append(ms / n)
        med = sorted(times)[len(times) // 2]
        gbs = by / n / (med / 1000.0) / 1e9
        rows.append({"precision": prec, "nr": nr, "mode": "clovinv (direct)", "reps": len(times),
                     "median_launch_us": 1000.0 * med, "algorithmic_bytes_per_launch": by / n, "GBs": gbs,
                     "frac": gbs / hbm})
        del x, out
    return rows


def run_dslash_sweep(args):
    """Hop launches inside `--dslash-iters` BiCGStab iterations of a block of nr random
    right-hand sides (the solve stops early, by design, before it converges), averaged
    per launch by the library's event timer.  Algorithmic bytes per launch: 48 reals of
    spinor per site and RHS (read 24, write 24) plus 8 links x 12 reals and 72 clover
    reals per site (FP32 or FP64 reals), as the library's hop_bytes counts them; the XPAY
    launches read z as well.  Rows whose solver working set fits in L2 say so."""
    import torch
    from paper_1104_3870_gb300 import build
    build.build()
    from paper_1104_3870_gb300 import laph as L
    from paper_1104_3870_gb300.pipeline import LapHPath, LatticeSpec
    import synth

    wl = synth.WORKLOADS[args.workload]
    if args.dslash_nt > 0:   # a slab of the workload's slices: same spatial extent, fewer slices
        import dataclasses
        wl = dataclasses.replace(wl, nt=args.dslash_nt)
    spec = LatticeSpec(wl.ns, wl.nt, wl.xi, wl.m0, wl.csw, wl.nv, (wl.dil_time, wl.dil_spin, wl.dil_laph),
                       wl.rho_stout, wl.n_stout4d, wl.n_stout3d)
    path = LapHPath(spec, 0)
    u, _ = path.prepare_links(wl.gauge())
    peaks_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    peaks = json.load(open(peaks_path)) if os.path.exists(peaks_path) else {}
    hbm = peaks.get("hbm_gbs", 6800.0)
    l2_bytes = 129e6
    vh = wl.ns ** 3 * wl.nt // 2
    rows = []
    for prec in args.dslash_prec.split(","):
        mode, fam, real = ((L.MIXED_FP32, "dslash_fp32", 4) if prec == "fp32" else (L.PLAIN_FP64, "dslash_fp64", 8))
        if args.dslash_direct:
            rows += dslash_direct_rows(L, torch, path, wl, u, prec, fam, real, hbm, args)
            continue
        for nr in [int(v) for v in args.dslash_nr.split(",")]:
            b = torch.randn((nr, wl.nt, wl.ns, wl.ns, wl.ns, 4, 3), dtype=torch.complex128, device="cuda")
            x = torch.empty_like(b)
            prm = L.solver_params(tol=1e-14, maxiter=args.dslash_iters, mode=mode, rhs_block=nr,
                                  inner_tol=1e-14)
            L.laph_profile_reset()
            L.laph_profile_enable(1)
            L.dirac_solve_batch(path.ctx, path.lat, u, wl.m0, wl.csw, b, x, nr, prm, allow_not_converged=True)
            torch.cuda.synchronize()
            L.laph_profile_enable(0)
            n, ms, by, fl = L.laph_profile_read(fam)
            gbs = by / (ms / 1000.0) / 1e9 if ms else None
            working = 8 * vh * 12 * nr * 2 * real            # about eight half-lattice solver vectors
            rows.append({"precision": prec, "nr": nr, "launches": n, "avg_launch_us": 1000.0 * ms / n if n else None,
                         "algorithmic_bytes_per_launch": by / n if n else None, "GBs": gbs,
                         "frac": gbs / hbm if gbs else None, "gflops": fl / (ms / 1000.0) / 1e9 if ms else None,
                         "l2_resident": working < l2_bytes,
                         "kernel": ("hop3_kernel (TMA-fed)" if prec == "fp32" and nr % 32 == 0 and nr & (nr - 1) == 0
                                    else "hop2_kernel" if prec == "fp32" else "hop_kernel<double>")})
            del b, x
    print(json.dumps({"metric": "Dslash HBM GB/s (algorithmic bytes / event-timed launch)", "unit": "GB/s",
                      "workload": wl.name, "lattice": f"{wl.ns}^3x{wl.nt}", "peak": hbm, "kernel_version": HOP_KERNEL_VERSION,
                      "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)" if peaks else "fallback 6.8 TB/s",
                      "rows": rows}), flush=True)


def run_nn_sweep(args):
    """One application of the learned network with FP32 layers (laph_precond_apply) and with
    tensor-core layers (laph_precond_apply_tc) on nr random fields of the medium lattice, against
    one application of K in the FP32 stencil (the two even-odd hops of laph_dslash_eo in the
    apply mode).  Each figure is the library's CUDA-event time of the kernels themselves (the
    network's four layer launches, the two hop launches), summed over --nn-reps calls after one
    untimed call, so the calls' operator set-up and layout conversions are not counted."""
    import torch
    from paper_1104_3870_gb300 import build
    build.build()
    from paper_1104_3870_gb300 import laph as L
    from paper_1104_3870_gb300.pipeline import LapHPath, LatticeSpec
    import synth

    wl = synth.WORKLOADS["medium_16x32"]
    spec = LatticeSpec(wl.ns, wl.nt, wl.xi, wl.m0, wl.csw, wl.nv, (wl.dil_time, wl.dil_spin, wl.dil_laph),
                       wl.rho_stout, wl.n_stout4d, wl.n_stout3d)
    path = LapHPath(spec, 0)
    u, _ = path.prepare_links(wl.gauge())
    nr = args.nn_nr
    w = np.zeros(L.laph_precond_size(), dtype=np.float32)
    L.laph_precond_init(7, wl.m0 + 1.0 + 3.0 / wl.xi, w)
    wdev = torch.from_numpy(w).cuda()
    gen = torch.Generator(device="cuda")
    gen.manual_seed(11)
    shape = (nr, wl.nt, wl.ns, wl.ns, wl.ns, 4, 3)
    x = torch.complex(torch.randn(shape, dtype=torch.float64, device="cuda", generator=gen),
                      torch.randn(shape, dtype=torch.float64, device="cuda", generator=gen))
    y = torch.empty_like(x)
    vh = wl.ns ** 3 * wl.nt // 2
    xe = torch.randn((vh, 12, nr), dtype=torch.complex64, device="cuda")
    ye = torch.empty_like(xe)
    lat = path.lat

    def kernel_ms(fn, family):
        fn()
        torch.cuda.synchronize()
        L.laph_profile_reset()
        L.laph_profile_enable(2)
        for _ in range(args.nn_reps):
            fn()
        torch.cuda.synchronize()
        L.laph_profile_enable(0)
        n, ms, _, _ = L.laph_profile_read(family)
        return ms / args.nn_reps, n // args.nn_reps

    k_ms, k_n = kernel_ms(lambda: [L.laph_dslash_eo(path.ctx, lat, u, wl.m0, wl.csw, p, L.HOP_APPLY, L.PREC_FP32, xe,
                                                    xe, ye, nr) for p in (0, 1)], "dslash_fp32")
    fp32_ms, fp32_n = kernel_ms(lambda: L.laph_precond_apply(path.ctx, lat, u, wl.m0, wl.csw, wdev, x, y, nr),
                                "nn_layer")
    tc_ms, tc_n = kernel_ms(lambda: L.laph_precond_apply_tc(path.ctx, lat, u, wl.m0, wl.csw, wdev, x, y, nr),
                            "nn_layer_tc")
    print(json.dumps({"metric": "learned-network application vs K application (library CUDA events per kernel)",
                      "lattice": f"{wl.ns}^3x{wl.nt}", "nr": nr, "reps": args.nn_reps,
                      "K_fp32_ms": k_ms, "K_launches": k_n, "network_fp32_ms": fp32_ms, "network_fp32_launches": fp32_n,
                      "network_tc_ms": tc_ms, "network_tc_launches": tc_n,
                      "fp32_in_K": fp32_ms / k_ms, "tc_in_K": tc_ms / k_ms}), flush=True)
    path.close()


def run_learned_study(args):
    """Learned preconditioner across gauge fields: fields are seeded 2000 + i on the medium
    lattice (the workload's smearing recipe and m0); the network is trained on (rho, phi =
    K^-1 rho) pairs of all but the last four fields (Adam state carried across fields, one
    epoch per field per pass), then on each held-out field the same seeded sources are solved
    with learned FGCR(16) (batched, FP32 inner, FP64 outer) and with plain FP64 BiCGStab (one
    right-hand side per launch) and with the mixed batched BiCGStab; iterations and wall time
    are reported per field."""
    import torch
    from paper_1104_3870_gb300 import build
    build.build()
    from paper_1104_3870_gb300 import laph as L
    from paper_1104_3870_gb300.pipeline import LapHPath, LatticeSpec
    import synth

    wl = synth.WORKLOADS[args.study_workload]
    spec = LatticeSpec(wl.ns, wl.nt, wl.xi, wl.m0, wl.csw, wl.nv, (wl.dil_time, wl.dil_spin, wl.dil_laph),
                       wl.rho_stout, wl.n_stout4d, wl.n_stout3d)
    path = LapHPath(spec, 0)
    ctx, lat = path.ctx, path.lat
    nf, held = args.study_fields, 4
    shape = lambda n: (n, wl.nt, wl.ns, wl.ns, wl.ns, 4, 3)
    gen = torch.Generator(device="cuda")
    nw = L.laph_precond_size()
    w = np.zeros(nw, dtype=np.float32)
    L.laph_precond_init(7, wl.m0 + 1.0 + 3.0 / wl.xi, w)
    adam = np.zeros(2 * nw, dtype=np.float32)
    step = 0
    t_pairs = t_train = 0.0
    train = []
    for f in range(nf - held):
        u, _ = path.prepare_links(synth.random_su3_field(wl.ns, wl.nt, seed=2000 + f))
        gen.manual_seed(7000 + f)
        rho = torch.complex(torch.randn(shape(args.study_pairs), dtype=torch.float64, device="cuda", generator=gen),
                            torch.randn(shape(args.study_pairs), dtype=torch.float64, device="cuda", generator=gen))
        phi = torch.empty_like(rho)
        torch.cuda.synchronize()
        t = time.perf_counter()
        L.dirac_solve_batch(ctx, lat, u, wl.m0, wl.csw, rho, phi, args.study_pairs, L.solver_params(mode=L.MIXED_FP32))
        torch.cuda.synchronize()
        t_pairs += time.perf_counter() - t
        train.append((u, rho, phi))
    batch = min(8, args.study_pairs)
    losses = []
    for ep in range(args.study_epochs):
        tot = 0.0
        for (u, rho, phi) in train:
            t = time.perf_counter()
            tot += L.laph_precond_train(ctx, lat, u, wl.m0, wl.csw, rho, phi, args.study_pairs, 1, batch, 2e-3, step,
                                        w, adam)
            torch.cuda.synchronize()
            t_train += time.perf_counter() - t
            step += args.study_pairs // batch
        losses.append(tot / len(train))
    del train
    wdev = torch.from_numpy(w).cuda()
    stream = torch.cuda.current_stream()

    def timed(fn):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        reps = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1000.0, reps

    fields = []
    n = args.study_rhs
    for f in range(nf - held, nf):
        u, _ = path.prepare_links(synth.random_su3_field(wl.ns, wl.nt, seed=2000 + f))
        gen.manual_seed(9000 + f)
        b = torch.complex(torch.randn(shape(n), dtype=torch.float64, device="cuda", generator=gen),
                          torch.randn(shape(n), dtype=torch.float64, device="cuda", generator=gen))
        x = torch.empty_like(b)
        row = {"seed": 2000 + f}
        for name, prm in (("learned_fgcr", L.solver_params(mode=L.LEARNED, weights=wdev, rhs_block=n)),
                          ("plain_fp64_bicgstab", L.solver_params(mode=L.PLAIN_FP64, rhs_block=1)),
                          ("mixed_bicgstab", L.solver_params(mode=L.MIXED_FP32, rhs_block=n))):
            sec, reps = timed(lambda: L.dirac_solve_batch(ctx, lat, u, wl.m0, wl.csw, b, x, n, prm))
            it = float(np.mean([r.iters for r in reps]))
            # operator applications per source: an FGCR step applies K once and the network once; a
            # BiCGStab iteration applies the even-odd Schur operator twice (four hops, two K's worth)
            learned = name == "learned_fgcr"
            row[name] = {"s": sec, "sources_per_s": n / sec, "iters_mean": it,
                         "K_applications_mean": it if learned else 2.0 * it,
                         "network_applications_mean": it if learned else 0.0,
                         "network_layers": ("tensor cores" if n % 32 == 0 else "FP32") if learned else None,
                         "true_resid_max": max(r.true_resid for r in reps),
                         "fallback_used": int(sum(r.fallback_used for r in reps))}
        fields.append(row)
    agg = {k: {"sources_per_s": float(np.mean([r[k]["sources_per_s"] for r in fields])),
               "iters_mean": float(np.mean([r[k]["iters_mean"] for r in fields])),
               "K_applications_mean": float(np.mean([r[k]["K_applications_mean"] for r in fields])),
               "network_applications_mean": float(np.mean([r[k]["network_applications_mean"] for r in fields]))}
           for k in ("learned_fgcr", "plain_fp64_bicgstab", "mixed_bicgstab")}
    print(json.dumps({"metric": "learned preconditioner on held-out fields (diluted-source solves to 1e-10)",
                      "workload": f"{wl.name} lattice, fields seeded 2000..{2000 + nf - 1}, last {held} held out",
                      "train": {"fields": nf - held, "pairs_per_field": args.study_pairs, "epochs": args.study_epochs,
                                "batch": batch, "lr": 2e-3, "pairs_solve_s": t_pairs, "train_s": t_train,
                                "loss_per_epoch": losses},
                      "held_out": fields, "mean": agg,
                      "iteration_ratio_learned_vs_plain": agg["learned_fgcr"]["iters_mean"] /
                      agg["plain_fp64_bicgstab"]["iters_mean"],
                      "wall_ratio_learned_vs_plain": agg["plain_fp64_bicgstab"]["sources_per_s"] /
                      agg["learned_fgcr"]["sources_per_s"]}), flush=True)
    path.close()


def main(argv=None):
    args = parse_args(argv)
    if args.nn_sweep:
        run_nn_sweep(args)
    elif args.learned_study:
        run_learned_study(args)
    elif args.dslash_sweep:
        run_dslash_sweep(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
