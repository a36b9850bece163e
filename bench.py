#!/usr/bin/env python
"""SupPCG iterations/s on one GB300 (or N independent replicas).

Workload: 512 x 512 image on the unit square, 720 views over [0, pi), 725
bins (ray spacing = pixel size), 20-ellipse phantom, Poisson data with 1e5
incident photons per ray, log-transformed; SupPCG with K=1, gamma=0.5,
a=0.995, mu=1e-5, rho=0.8.  A step is one execution of the while body of
Algorithm 3 (S_TV, forward projection with residual, backprojection,
preconditioner, CG scalars and axpys, forward and back projection of p).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload plain512|batched64|large2048|learned512|sweep243|art512|memory2048|network512]

--impl reference times the FP64 CPU oracle on the host cores on the same
workload (it is the only other implementation of the method here).
--workload batched64: 64 independent problems of uneven sizes (images
256^2-1024^2 with 2^a 3^b 5^c sides, 180-1440 views, ceil(1.42 N) bins,
ellipse phantoms, 1 % Gaussian noise) solved by one batched schedule, timed
against solving them one after another (same iterates, so the time ratio is
the time-to-equal ratio).
--workload learned512: the learned direction.  Training pairs (x_k, tbar,
K-step S_TV displacement) from plain SupPCG runs (Table 1: K=40,
a=1-1e-5, gamma=1e-2, mu=1e-5, rho=0.8) on 400 random 512^2 / 720-view
problems x 50 iterations (20k pairs), network trained on the GPU, then plain
vs learned SupPCG (trained and untrained networks) on the 512^2 / 720-view
Poisson workload: wall time for the learned solve to reach the plain solve's
final residual and TV; and the batched learned solve over 8 held-out
problems against plain SupPCG on them.  The default workload's line carries
the same comparison with a small training set (1024 pairs) in its
time_to_equal object.
--workload sweep243: the paper's parameter selection (Sec. 4.2) for SupPCG as
one batched sweep: 180 grid points (K, a, gamma, mu, rho; rho = 0.4 excluded)
x 15 iterations on a 243^2 / 360-view / 345-bin head stand-in (Poisson 1e5),
scored by the selective error of Eq. (4.1), timed against the same solves one
after another.
--workload art512: ART on the Bayesian criterion and SupART (Sec. 3.4) on the
512^2 / 720-view Poisson workload with Table 1's parameters (ART r = 5,
lambda = 1e-2; SupART K = 10, a = 1 - 1e-5, gamma = 1e-2, r = 5,
lambda = 5e-2): cycles/s on the GPU, and one cycle of the FP64 oracle on the
host cores.
--workload memory2048: the memory-bound kernels (vector, preconditioner, S_TV)
of a 2048^2 / 2880-view SupPCG iteration against the HBM peak.
--workload network512: the network's convolutions (inference, training step)
at 512^2 against the BF16 tensor peak.
--workload large2048: 8 slices of 2048^2, 2880 views, 2900 bins (40 ellipses
on a textured background, Poisson 1e4 photons): FP32- and BF16-stored
projector pair timed on the batch, errors of both against the FP64 oracle on
a 256^2 / 360-view / 364-bin crop geometry.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WL = dict(N=512, V=720, U=725, n_ell=20, seed=2001, I0=1e5, noise_seed=2501, K=1, a=0.995, gamma=0.5,
          mu=1e-5, rho=0.8)
WORKLOAD = "suppcg_512x512_720views_725bins_poisson1e5"
OPS_PER_INTERSECTION = 7   # FP32 ops of one ray-pixel term as written: fma position, sub, sub, mul, max, min, fma
FALLBACK_HBM_GBS = 6800.0


def env_int(k, d):
    try:
        return int(os.environ.get(k, d))
    except ValueError:
        return d


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.3)
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def __exit__(self, *a):
        time.sleep(0.25)
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            return json.load(open(p)), "measured"
        except ValueError:
            pass
    return {"hbm_gbs": FALLBACK_HBM_GBS}, "fallback"


def nnz_per_projection(N, V, U, d_over_ds=1.0):
    """Ray-pixel intersections of one projection: every pixel meets, per view,
    (|cos|+|sin|) d/ds bins on average (all footprints inside the detector
    when U >= sqrt(2) N d/ds)."""
    s = sum(abs(math.cos(v * math.pi / V)) + abs(math.sin(v * math.pi / V)) for v in range(V))
    return N * N * s * d_over_ds


def workload_data(seed=None, noise_seed=None):
    """b of the benchmark workload, the same array for both arms: exact line
    integrals of the continuous 20-ellipse phantom (the paper's simulations
    take line integrals through a continuous phantom), Poisson counts at 1e5
    photons per ray, log-transformed, rounded to FP32."""
    import numpy as np
    from paper_1807_10151_gb300 import synth
    seed = WL["seed"] if seed is None else seed
    noise_seed = WL["noise_seed"] if noise_seed is None else noise_seed
    clean = synth.ellipse_sinogram(WL["n_ell"], seed, WL["V"], WL["U"], 1.0 / WL["N"])
    return synth.poisson_log(clean, WL["I0"], noise_seed).astype(np.float32)


def workload_config(iters):
    """config of the contract line: the workload alone, identical in both arms."""
    return {"workload": WORKLOAD, "image": [WL["N"], WL["N"]], "views": WL["V"], "bins": WL["U"],
            "iterations": iters, "K": WL["K"], "gamma": WL["gamma"], "a": WL["a"], "mu": WL["mu"],
            "rho": WL["rho"], "phantom": f"{WL['n_ell']} ellipses, seed {WL['seed']}",
            "data": f"analytic line integrals, Poisson {WL['I0']:g} photons per ray, seed {WL['noise_seed']}",
            "l2": "flushed (256 MB write) before every timed solve; one 512^2 problem's working set "
                  "(~16 MB) then stays L2-resident across its iterations"}


def make_problem(rank, device):
    import paper_1807_10151_gb300 as S
    from paper_1807_10151_gb300 import replicas
    G = S.Geometry(WL["N"], n_views=WL["V"], n_bins=WL["U"])
    seed, noise_seed = replicas.rank_seeds(rank, WL["seed"], WL["noise_seed"])   # each replica its own problem
    return G, workload_data(seed, noise_seed)


def solve_kw(iters, graph=True):
    return dict(K=WL["K"], a=WL["a"], gamma=WL["gamma"], mu=WL["mu"], rho=WL["rho"], max_iter=iters,
                graph=graph)


def oracle_sample(iters):
    """The FP64 oracle on the same workload: explicit CSR R, then SupPCG."""
    import numpy as np
    from oracle import oracle as O
    og = O.Geometry(WL["N"], V=WL["V"], U=WL["U"])
    t0 = time.perf_counter()
    R = O.CSR(og)
    t_build = time.perf_counter() - t0
    b = workload_data().astype(np.float64)   # the GPU arm's b, bit for bit
    t0 = time.perf_counter()
    out = O.suppcg(R, b, K=WL["K"], a=WL["a"], gamma=WL["gamma"], mu=WL["mu"], rho=WL["rho"], max_iter=iters)
    t_solve = time.perf_counter() - t0
    assert out["status"] == 0
    return {"t_build_s": t_build, "t_solve_s": t_solve, "iters": iters, "cores": O.num_threads(), "nnz": R.nnz}


def smooth_sides(lo=256, hi=1024):
    """Image sides in [lo, hi] of the form 2^a 3^b 5^c."""
    out = []
    for n in range(lo, hi + 1):
        m = n
        for p in (2, 3, 5):
            while m % p == 0:
                m //= p
        if m == 1:
            out.append(n)
    return out


def batched_comparison(steps, warmup, dev, tune=True):
    """64 uneven problems (images 256^2-1024^2 with 2^a 3^b 5^c sides, 180-1440
    views, ceil(1.42 N) bins, 15-ellipse phantoms, 1 % Gaussian noise) solved by
    one batched schedule, then the same problems one after another.  Both give
    the same iterates (bitwise), so the time ratio is the time-to-equal ratio.
    Each geometry's forward tile is chosen by the autotuner first (cached per
    geometry bucket).  Returns a dict with its own clock record."""
    import numpy as np
    import torch
    import paper_1807_10151_gb300 as S
    from paper_1807_10151_gb300 import autotune, synth
    rng = np.random.default_rng(3000)
    sides = smooth_sides()
    geoms, bs = [], []
    nnz = 0.0
    tiles = {}
    for c in range(64):
        N = int(rng.choice(sides))
        V = int(rng.integers(180, 1441))
        U = int(math.ceil(1.42 * N))
        G = S.Geometry(N, n_views=V, n_bins=U)
        if tune:
            t = autotune.tune(G, reps=3)["tile"]
            tiles[t] = tiles.get(t, 0) + 1
        x = synth.ellipse_phantom(N, 15, 3000 + c)
        clean = G.project(torch.tensor(x, dtype=torch.float32, device=dev)).double().cpu().numpy()
        bs.append(torch.tensor(synth.gaussian_noise(clean, 0.01, 3500 + c), dtype=torch.float32, device=dev))
        geoms.append(G)
        nnz += nnz_per_projection(N, V, U)
    kw = dict(K=WL["K"], a=WL["a"], gamma=WL["gamma"], mu=WL["mu"], rho=WL["rho"])
    st = torch.cuda.current_stream()
    xs = [torch.zeros(g.ny, g.nx, device=dev) for g in geoms]
    S.solve_batched(geoms, bs, xs, max_iter=warmup, **kw)
    for g, b in zip(geoms, bs):      # warm each geometry's own workspace for the sequential run
        g.solve(b, max_iter=1, **kw)
    for x in xs:
        x.zero_()
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    l0 = S.supcg_kernel_launches()
    with ClockSampler(dev.index or 0) as clk:
        ev[0].record(st)
        reps = S.solve_batched(geoms, bs, xs, max_iter=steps, **kw)
        ev[1].record(st)
        torch.cuda.synchronize()
        launches = S.supcg_kernel_launches() - l0
        ev[2].record(st)
        for g, b in zip(geoms, bs):
            g.solve(b, max_iter=steps, **kw)
        ev[3].record(st)
        torch.cuda.synchronize()
    assert all(r["status"] == 0 for r in reps), reps
    t_batch = ev[0].elapsed_time(ev[1]) / 1000.0
    t_seq = ev[2].elapsed_time(ev[3]) / 1000.0
    out = {"problems": 64, "iterations": steps, "batched_s": t_batch, "sequential_s": t_seq,
           "time_to_equal_ratio": t_seq / t_batch,
           "problem_iterations_per_s": {"batched": 64 * steps / t_batch, "sequential": 64 * steps / t_seq},
           "intersections_per_s_batched": 4.0 * nnz * steps / t_batch, "gpu_launches_batched": int(launches),
           "sides": [min(g.nx for g in geoms), max(g.nx for g in geoms)],
           "views": [min(g.V for g in geoms), max(g.V for g in geoms)],
           "fwd_tiles": {str(k): v for k, v in sorted(tiles.items())}, "clocks": clk.summary(),
           "equal_by": "identical iterates (the batched schedule runs the same kernels per problem)"}
    for g in geoms:
        g.close()
    return out


def run_batched(args, dev):
    """64 uneven problems in one batched schedule vs one at a time."""
    r = batched_comparison(args.steps, args.warmup, dev)
    line = {
        "metric": "SupPCG problem-iterations/s (batched)", "value": r["problem_iterations_per_s"]["batched"],
        "unit": "problem-iterations/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000.0 * r["batched_s"] / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "suppcg_batched_64_uneven", "problems": 64, "sides": r["sides"], "views": r["views"],
                   "K": WL["K"], "gamma": WL["gamma"], "a": WL["a"], "mu": WL["mu"], "rho": WL["rho"],
                   "l2": "working set of the batch (several GB) exceeds L2"},
        "sequential": {"seconds": r["sequential_s"], "problem_iterations_per_s": r["problem_iterations_per_s"]["sequential"],
                       "time_to_equal_ratio": r["time_to_equal_ratio"]},
        "intersections_per_s": r["intersections_per_s_batched"], "fwd_tiles": r["fwd_tiles"],
        "gpu_launches": r["gpu_launches_batched"], "clocks": r["clocks"],
    }
    print(json.dumps(line), flush=True)
    return 0


SWEEP_GRID = [dict(K=K, a=a, gamma=g, mu=mu, rho=rho)
              for K in (10, 20, 40) for a in (1 - 1e-5, 1 - 1e-4, 1 - 1e-3, 1 - 1e-2, 1 - 1e-1)
              for g in (1e-2, 5e-2) for mu in (1e-5, 1e-4, 1e-3) for rho in (0.6, 0.8)]


def run_sweep(args, dev):
    """Sec. 4.2's parameter selection for SupPCG as one batched sweep: the grid
    K x a x gamma x mu x rho of the paper (rho = 0.4 excluded: h(pi) <= 0), 15
    iterations each, scored by the selective error SE of Eq. (4.1) against the
    phantom; timed against the same 180 solves one after another."""
    import numpy as np
    import torch
    import paper_1807_10151_gb300 as S
    from paper_1807_10151_gb300 import synth
    N, V, U, its = 243, 360, 345, 15
    x = synth.head_standin(N, 6001)
    G = S.Geometry(N, n_views=V, n_bins=U)
    clean = G.project(torch.tensor(x, dtype=torch.float32, device=dev)).double().cpu().numpy()
    b = torch.tensor(synth.poisson_log(clean, 1e5, 6002), dtype=torch.float32, device=dev)
    ref = torch.tensor(x, dtype=torch.float32, device=dev)
    params = [dict(q, max_iter=its) for q in SWEEP_GRID]
    st = torch.cuda.current_stream()
    for _ in range(args.warmup):
        S.solve_sweep(G, b, [dict(q, max_iter=3) for q in SWEEP_GRID], ref=ref)
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    l0 = S.supcg_kernel_launches()
    with ClockSampler(dev.index or 0) as clk:
        ev[0].record(st)
        xs, reps, se = S.solve_sweep(G, b, params, ref=ref)
        ev[1].record(st)
        torch.cuda.synchronize()
    launches = S.supcg_kernel_launches() - l0
    assert all(r["status"] == 0 for r in reps), [r for r in reps if r["status"]]
    t_batch = ev[0].elapsed_time(ev[1]) / 1000.0
    se = se.cpu().numpy()
    best = int(np.argmin(se.min(axis=1)))
    best_it = int(np.argmin(se[best])) + 1
    # the same solves one after another
    G.solve(b, **params[0])
    torch.cuda.synchronize()
    ev[2].record(st)
    for q in params:
        G.solve(b, **q)
    ev[3].record(st)
    torch.cuda.synchronize()
    t_seq = ev[2].elapsed_time(ev[3]) / 1000.0
    n = len(params)
    line = {
        "metric": "SupPCG problem-iterations/s (parameter sweep)", "value": n * its / t_batch,
        "unit": "problem-iterations/s", "n_gpus": 1, "steps": its, "warmup": args.warmup,
        "ms_per_step": 1000.0 * t_batch / its, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": "sweep_243x243_360views_345bins_head_standin_poisson1e5", "solves": n,
                   "grid": {"K": [10, 20, 40], "a": "1 - 1e-5 .. 1 - 1e-1", "gamma": [1e-2, 5e-2],
                            "mu": [1e-5, 1e-4, 1e-3], "rho": [0.6, 0.8]},
                   "se_axes": list(S.SE_AXES), "l2": "180 working sets of ~6 MB: the batch exceeds L2"},
        "sequential": {"seconds": t_seq, "problem_iterations_per_s": n * its / t_seq,
                       "time_to_equal_ratio": t_seq / t_batch},
        "best": {"params": SWEEP_GRID[best], "iteration": best_it, "se": float(se[best, best_it - 1]),
                 "se_plain_first_iteration_median": float(np.median(se[:, 0]))},
        "gpu_launches": int(launches), "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)
    return 0


def run_art(args, dev):
    """ART and SupART (Sec. 3.4) on the 512^2 / 720-view workload: cycles per
    second, each cycle visiting every ray once (V x S grid barriers: the rays
    of one view and residue class run in parallel)."""
    import numpy as np
    import torch
    import paper_1807_10151_gb300 as S
    G, b_host = make_problem(0, dev)
    b = torch.tensor(b_host, device=dev)
    st = torch.cuda.current_stream()
    art_kw = dict(r=5.0, lam=1e-2)
    sup_kw = dict(r=5.0, lam=5e-2, K=10, a=1 - 1e-5, gamma=1e-2)
    cycles = max(2, min(args.steps, 10))
    for _ in range(args.warmup):
        G.art(b, cycles=1, **art_kw)
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    l0 = S.supcg_kernel_launches()
    with ClockSampler(dev.index or 0) as clk:
        ev[0].record(st)
        x, rep = G.art(b, cycles=cycles, **art_kw)
        ev[1].record(st)
        ev[2].record(st)
        xs, reps = G.art(b, cycles=cycles, **sup_kw)
        ev[3].record(st)
        torch.cuda.synchronize()
    assert rep["status"] == 0 and reps["status"] == 0, (rep, reps)
    t_art = ev[0].elapsed_time(ev[1]) / 1000.0
    t_sup = ev[2].elapsed_time(ev[3]) / 1000.0
    cpu = None
    if not args.no_cpu_baseline:
        from oracle import oracle as O
        from paper_1807_10151_gb300 import synth
        og = O.Geometry(WL["N"], V=WL["V"], U=WL["U"])
        R = O.CSR(og)
        t0 = time.perf_counter()
        O.art(R, b_host, cycles=1, **art_kw)
        t_cpu = time.perf_counter() - t0
        cpu = {"value": 1.0 / t_cpu, "unit": "cycles/s", "cores": 1, "kind": "oracle",
               "sample": "one ART cycle of the FP64 oracle (sequential over the 522000 rays of the explicit CSR R, "
                         "built beforehand, not timed)"}
    line = {
        "metric": "ART cycles/s (Bayesian criterion, Sec. 3.4)", "value": cycles / t_art, "unit": "cycles/s",
        "n_gpus": 1, "steps": cycles, "warmup": args.warmup, "ms_per_step": 1000.0 * t_art / cycles,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32 (ray sums f64)",
        "data": "synthetic",
        "config": {"workload": "art_512x512_720views_725bins_poisson1e5", "art": art_kw, "supart": sup_kw,
                   "class_barriers_per_cycle": WL["V"] * 2, "l2": "the 14 MB working set stays L2-resident"},
        "supart": {"value": cycles / t_sup, "unit": "iterations/s (S_TV + one cycle)", "ell": reps["ell"]},
        "gpu_launches": int(S.supcg_kernel_launches() - l0), "clocks": clk.summary(),
    }
    if cpu:
        line["cpu_baseline"] = cpu
    print(json.dumps(line), flush=True)
    return 0


def memory_bound_legs(G, b, N, peak_gbs):
    """Steady-state per-iteration time of the HBM-bound kernels of one SupPCG solve
    on an N x N slice (its working set, images, spectrum and sinograms, exceeds L2):
    the difference of two profiled solves (4 and 12 iterations) removes the one-off
    staging and steps 1-9.  Bytes per iteration (n = N^2; x and g are double-float
    pairs, x + xlo and g + glo; the layouts the forward projector reads, p^T, the
    S_TV displacement d and d^T, and with mirror pairs of views the left-right
    mirrored images, are written by the kernels that produce p and d):
      vector: x update (read x, xlo, p; write x, xlo) 20n + p update (read p, z, g, glo;
           write p, p^T, with mirror pairs also p mirrored and its transpose) 24n (32n);
      fft: rows (read g and glo 8n, write the half spectrum, 16 B per stored complex),
           columns (read and write it, read the quarter table of D, 8 B per entry),
           inverse rows (read it, write z, read h for z^T h);
      stv (K = 1): tbar pass (read x, write tbar) 8n, every trial (read x, tbar) 8n,
           last step (read x, xlo, tbar; write x, xlo, d, d^T, with mirror pairs also d
           mirrored and its transpose) 28n (36n)."""
    n = N * N
    mir = G.mirror_pairs() > 0
    hx = N // 2 + 1
    spec = 16 * hx * N
    fft_bytes = (8 * n + spec) + (2 * spec + 8 * (N // 2 + 1) * hx) + (spec + 8 * n)
    runs = {}
    for it in (4, 12):
        _, rep, kinds = G.solve_profiled(b, **solve_kw(it, graph=False))
        assert rep["status"] == 0 and rep["iters"] == it, rep
        runs[it] = (rep, kinds)
    d_it = 8
    trials = runs[12][0]["ell"] - runs[4][0]["ell"]   # K = 1: l advances once per trial
    out = {}
    vec_bytes = (20 + (32 if mir else 24)) * n
    stv_bytes = (8 + (36 if mir else 28)) * n + 8 * n * trials / d_it
    for kind, launches, nbytes in (("vector", 2, vec_bytes), ("fft", 3, fft_bytes), ("stv", 1, stv_bytes)):
        ms = (runs[12][1][kind][0] - runs[4][1][kind][0]) / d_it
        nl = (runs[12][1][kind][1] - runs[4][1][kind][1]) / d_it
        gbs = nbytes / (ms / 1000.0) / 1e9
        out[kind] = {"ms_per_iteration": ms, "launches_per_iteration": nl, "bytes_per_iteration": nbytes,
                     "achieved_gbs": gbs, "frac_of_hbm": gbs / peak_gbs}
    out["stv"]["trials_per_iteration"] = trials / d_it
    return out


def run_large(args, dev):
    """8 slices of 2048^2: FP32 vs BF16 storage of the projector pair."""
    import numpy as np
    import torch
    import paper_1807_10151_gb300 as S
    from paper_1807_10151_gb300 import synth
    from oracle import oracle as O
    N, V, U, B = 2048, 2880, 2900, 8
    st = torch.cuda.current_stream()
    xs = []
    for c in range(B):
        x = synth.ellipse_phantom(N, 40, 5000 + c) + synth.textured_background(N, 5100 + c)
        xs.append(x)
    X = torch.tensor(np.stack(xs), dtype=torch.float32, device=dev)
    res = {}
    for storage, dt in (("f32", torch.float32), ("bf16", torch.bfloat16)):
        G = S.Geometry(N, n_views=V, n_bins=U, storage=storage)
        Xs = X.to(dt)
        Y = G.project(Xs)
        Z = G.backproject(Y)
        for _ in range(max(3, args.warmup)):
            G.project(Xs, out=Y)
            G.backproject(Y, out=Z)
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        with ClockSampler(dev.index or 0) as clk_p:
            ev[0].record(st)
            for _ in range(args.steps):
                G.project(Xs, out=Y)
            ev[1].record(st)
            for _ in range(args.steps):
                G.backproject(Y, out=Z)
            ev[2].record(st)
            torch.cuda.synchronize()
        res[storage] = {"project_ms": ev[0].elapsed_time(ev[1]) / args.steps,
                        "backproject_ms": ev[1].elapsed_time(ev[2]) / args.steps, "clocks": clk_p.summary()}
        if storage == "f32":
            # one slice as a SupPCG problem: Poisson data with 1e4 incident photons per ray
            rng = np.random.default_rng(5200)
            counts = rng.poisson(1e4 * np.exp(-Y[0].double().cpu().numpy()))
            b0 = torch.tensor(-np.log(np.maximum(counts, 1) / 1e4), dtype=torch.float32, device=dev)
            G1 = S.Geometry(N, n_views=V, n_bins=U)
            peaks, peak_src = measured_peaks()
            with ClockSampler(dev.index or 0) as clk_m:
                mem_legs = memory_bound_legs(G1, b0, N, peaks["hbm_gbs"])
            mem_legs["hbm_peak_gbs"] = peaks["hbm_gbs"]
            mem_legs["peak_source"] = peak_src
            mem_legs["clocks"] = clk_m.summary()
            G1.close()
            del b0
        G.close()
        del Y, Z, Xs
    # errors on the 256^2 crop geometry against the FP64 oracle
    og = O.Geometry(256, V=360, U=364)
    R = O.CSR(og)
    crop = xs[0][N // 2 - 128:N // 2 + 128, N // 2 - 128:N // 2 + 128]
    ref_p = R.project(crop.astype(np.float32).astype(np.float64))
    yr = np.random.default_rng(9).standard_normal((og.V, og.U)).astype(np.float32)
    ref_b = R.backproject(yr.astype(np.float64))
    err = {}
    for storage, dt in (("f32", torch.float32), ("bf16", torch.bfloat16)):
        G = S.Geometry(256, n_views=360, n_bins=364, storage=storage)
        gp = G.project(torch.tensor(crop, dtype=torch.float32, device=dev).to(dt)).double().cpu().numpy()
        gb = G.backproject(torch.tensor(yr, device=dev).to(dt)).double().cpu().numpy()
        # BF16 inputs are themselves rounded: compare with the oracle on the same rounded inputs
        xin = torch.tensor(crop, dtype=torch.float32).to(dt).double().numpy()
        yin = torch.tensor(yr).to(dt).double().numpy()
        e_p = np.linalg.norm(gp - R.project(xin)) / np.linalg.norm(R.project(xin))
        e_b = np.linalg.norm(gb - R.backproject(yin)) / np.linalg.norm(R.backproject(yin))
        e_p0 = np.linalg.norm(gp - ref_p) / np.linalg.norm(ref_p)
        e_b0 = np.linalg.norm(gb - ref_b) / np.linalg.norm(ref_b)
        err[storage] = {"project_rel_l2_same_input": e_p, "backproject_rel_l2_same_input": e_b,
                        "project_rel_l2_vs_fp32_input": e_p0, "backproject_rel_l2_vs_fp32_input": e_b0}
    nnz = nnz_per_projection(N, V, U) * B
    line = {
        "metric": "projector pair intersections/s (2048^2 x 8 slices)",
        "value": 2 * nnz / ((res["f32"]["project_ms"] + res["f32"]["backproject_ms"]) / 1000.0),
        "unit": "intersections/s", "n_gpus": 1, "steps": args.steps, "warmup": max(3, args.warmup),
        "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "projector_2048x2048_2880views_2900bins_x8", "slices": B,
                   "l2": "inputs (8 x 16 MB images, 8 x 33 MB sinograms) exceed L2"},
        "timing_ms": res, "crop_errors_vs_fp64_oracle": err,
        "memory_bound_kernels_2048": mem_legs,
    }
    print(json.dumps(line), flush=True)
    return 0


def learned_comparison(dev, steps, warmup, n_problems, iters_train, epochs, batch_problems=8, timings=False):
    """The learned direction (Table 1's parameters) on the 512^2 / 720-view workload.

    Training pairs (x_k, tbar at x_k, K-step S_TV displacement) come from plain
    SupPCG runs on `n_problems` random 512^2 / 720-view problems x `iters_train`
    iterations (the evaluation's own image size); the network trains on the GPU.
    Then, each with its own clock record:
      - trained and untrained networks (the untrained one proposes tbar itself)
        against plain SupPCG on the benchmark's problem: wall time to reach the
        plain run's final f and TV after `steps` iterations;
      - the batched learned solve over `batch_problems` held-out problems against
        plain SupPCG on them, batched and one after another."""
    import numpy as np
    import torch
    import paper_1807_10151_gb300 as S
    from paper_1807_10151_gb300 import learned as Lr, synth
    N, V = WL["N"], WL["V"]
    t0 = time.perf_counter()
    X, T, D = Lr.make_training_set(n_problems, N=N, V=V, iters=iters_train, seed0=4000, device=dev)
    t_data = time.perf_counter() - t0
    Xh, Th, Dh = Lr.make_training_set(2, N=N, V=V, iters=8, seed0=4900, device=dev)
    bt = min(16, X.shape[0])
    net = S.CNN(N, N, max_batch=max(bt, batch_problems), seed=11)
    _, loss_untrained = net.gradients(Xh[:bt], Th[:bt], Dh[:bt])
    t0 = time.perf_counter()
    hist = Lr.train(net, X, T, D, epochs=epochs, batch=bt, lr=1e-3, log_every=100)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    _, loss_trained = net.gradients(Xh[:bt], Th[:bt], Dh[:bt])
    params = net.get_params()
    del X, T, D, Xh, Th, Dh
    torch.cuda.empty_cache()
    out = {"training": {"pairs": n_problems * iters_train, "images": f"{N}x{N}, {V} views", "data_s": t_data,
                        "train_s": t_train, "epochs": epochs, "batch": bt,
                        "heldout_loss_untrained": loss_untrained, "heldout_loss_trained": loss_trained,
                        "loss_history": hist}}
    G, b_host = make_problem(0, dev)
    b = torch.tensor(b_host, device=dev)
    nets = {}
    for name in ("trained", "untrained"):
        nn = S.CNN(N, N, max_batch=batch_problems, seed=11)
        if name == "trained":
            nn.set_params(params)
        nets[name] = nn
        with ClockSampler(dev.index or 0) as clk:
            r = Lr.time_to_equal(G, b, nn, iters=steps, device=dev, warmup=warmup)
        r["clocks"] = clk.summary()
        out[name] = r
    # the batched learned form over held-out problems of the same acquisition
    geoms, bs = [], []
    for c in range(batch_problems):
        Gc, bc = Lr.make_problem(S, synth, N, V, 4950 + c, dev, noise="poisson")
        geoms.append(Gc)
        bs.append(bc)
    with ClockSampler(dev.index or 0) as clk:
        rb = Lr.batched_time_to_equal(geoms, bs, nets["trained"], iters=steps, device=dev, warmup=warmup)
    rb["clocks"] = clk.summary()
    out["batched_trained"] = rb
    if timings:
        st = torch.cuda.current_stream()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        xi = torch.rand(N, N, device=dev)
        ti = torch.randn(N, N, device=dev)
        nn = nets["trained"]
        for _ in range(3):
            nn.forward(xi, ti)
        ev0.record(st)
        for _ in range(20):
            nn.forward(xi, ti)
        ev1.record(st)
        torch.cuda.synchronize()
        xb = xi.expand(batch_problems, N, N).contiguous()
        tb = ti.expand(batch_problems, N, N).contiguous()
        t1 = ev0.elapsed_time(ev1) / 20
        for _ in range(3):
            nn.forward(xb, tb)
        ev0.record(st)
        for _ in range(20):
            nn.forward(xb, tb)
        ev1.record(st)
        torch.cuda.synchronize()
        tB = ev0.elapsed_time(ev1) / 20
        for _ in range(3):
            nn.train_step(xb, tb, tb, lr=1e-12, want_loss=False)
        ev0.record(st)
        for _ in range(10):
            nn.train_step(xb, tb, tb, lr=1e-12, want_loss=False)
        ev1.record(st)
        torch.cuda.synchronize()
        out["network_ms"] = {"inference_1x512x512": t1, f"inference_{batch_problems}x512x512": tB,
                             f"train_step_{batch_problems}x512x512": ev0.elapsed_time(ev1) / 10,
                             "flop_per_pixel_inference": 57024}
    for g in geoms:
        g.close()
    out["params"] = params
    return out


def run_memory2048(args, dev):
    """The kernels of a SupPCG iteration that are bound by memory rather than by
    instruction issue, on one 2048^2 / 2880-view / 2900-bin slice (Poisson 1e4
    data from the analytic sinogram of a 40-ellipse phantom), whose working set
    exceeds L2: per-iteration time, algorithmic bytes and fraction of the HBM
    peak (memory_bound_legs), with the clock record."""
    import numpy as np
    import torch
    import paper_1807_10151_gb300 as S
    from paper_1807_10151_gb300 import synth
    N, V, U = 2048, 2880, 2900
    clean = synth.ellipse_sinogram(40, 5000, V, U, 1.0 / N)
    b = torch.tensor(synth.poisson_log(clean, 1e4, 5200), dtype=torch.float32, device=dev)
    G = S.Geometry(N, n_views=V, n_bins=U)
    G.solve(b, **solve_kw(2, graph=False))
    peaks, peak_src = measured_peaks()
    with ClockSampler(dev.index or 0) as clk:
        legs = memory_bound_legs(G, b, N, peaks["hbm_gbs"])
    line = {"metric": "memory-bound kernels of a 2048^2 SupPCG iteration, fraction of HBM peak",
            "value": legs["vector"]["frac_of_hbm"], "unit": "fraction (vector kernels)", "n_gpus": 1,
            "steps": 8, "warmup": 2, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": "memory_2048x2048_2880views_2900bins_poisson1e4",
                       "l2": "working set (images, spectrum, sinograms ~0.2 GB) exceeds L2"},
            "kernels": legs, "hbm_peak_gbs": peaks["hbm_gbs"], "peak_source": peak_src, "clocks": clk.summary()}
    print(json.dumps(line), flush=True)
    G.close()
    return 0


def run_network512(args, dev):
    """The learned-direction network's convolutions on the tensor cores at the
    512^2 evaluation size: inference of 1 and 8 images and one training step
    (forward, loss, backward, Adam) of 8 images, CUDA events after warm-up,
    against the measured BF16 peak.  FLOP per pixel of one inference: 2 x 9 x
    (2 x 32 + 3 x 32 x 32 + 32 x 1) = 57 024 (the real channels; layer 0's
    storage pads its 2 input channels to 16)."""
    import torch
    import paper_1807_10151_gb300 as S
    N, B = 512, 8
    net = S.CNN(N, N, max_batch=B, seed=11)
    p = net.get_params()
    rng = __import__("numpy").random.default_rng(3)
    p[:] = 0.05 * rng.standard_normal(p.size).astype(p.dtype)
    net.set_params(p)
    st = torch.cuda.current_stream()
    x = torch.rand(B, N, N, device=dev)
    t = torch.randn(B, N, N, device=dev)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = max(args.steps, 5)

    def timed(fn):
        for _ in range(max(3, args.warmup)):
            fn()
        torch.cuda.synchronize()
        ev0.record(st)
        for _ in range(reps):
            fn()
        ev1.record(st)
        torch.cuda.synchronize()
        return ev0.elapsed_time(ev1) / reps

    with ClockSampler(dev.index or 0) as clk:
        t1 = timed(lambda: net.forward(x[:1], t[:1]))
        tB = timed(lambda: net.forward(x, t))
        tT = timed(lambda: net.train_step(x, t, t, lr=1e-12, want_loss=False))
    flop_px = 57024
    peaks, peak_src = measured_peaks()
    peak = peaks.get("bf16_tflops", 1900.0)
    achieved = B * N * N * flop_px / (tB / 1000.0) / 1e12
    line = {"metric": "learned-direction network inference throughput (512^2, batch 8)", "value": achieved,
            "unit": "TFLOP/s", "n_gpus": 1, "steps": reps, "warmup": max(3, args.warmup), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "bf16 (fp32 accumulate)", "data": "synthetic",
            "config": {"workload": "network_512x512", "layers": "3x3 convs 2->32->32->32->32->1", "batch": B,
                       "l2": "activations of one layer (16 MB per image) stay L2-resident"},
            "ms": {"inference_1x512x512": t1, f"inference_{B}x512x512": tB, f"train_step_{B}x512x512": tT},
            "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "peak_source": peak_src,
                         "basis": f"{flop_px} FLOP per pixel x {B} x {N}^2 pixels per inference"},
            "clocks": clk.summary()}
    print(json.dumps(line), flush=True)
    return 0


def run_learned(args, dev):
    import numpy as np
    warm = max(3, args.warmup)
    r = learned_comparison(dev, args.steps, warm, n_problems=400, iters_train=50, epochs=2, timings=True)
    params = r.pop("params")
    line = {
        "metric": "time-to-equal (residual, TV): learned vs plain SupPCG", "value": r["trained"]["speedup"],
        "unit": "x (plain time / learned time)", "n_gpus": 1, "steps": args.steps, "warmup": warm,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32 (network bf16)",
        "data": "synthetic",
        "config": {"workload": "learned_512x512_720views_725bins_poisson1e5", "K": 40, "a": 1 - 1e-5,
                   "gamma": 1e-2, "mu": 1e-5, "rho": 0.8, "train_pairs": 20000, "train_images": "512x512",
                   "epochs": 2, "batch": 16},
    }
    line.update(r)
    print(json.dumps(line), flush=True)
    if args.save_params:
        np.save(args.save_params, params)
    return 0


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    s = oracle_sample(max(args.steps, 1))
    val = s["iters"] / s["t_solve_s"]
    line = {
        "impl": "reference", "metric": "SupPCG iterations/s", "value": val, "unit": "iterations/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000.0 * s["t_solve_s"] / s["iters"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(s["iters"]),
        "cpu_baseline": {"value": val, "unit": "iterations/s", "cores": s["cores"], "kind": "oracle",
                         "sample": f"FP64 oracle SupPCG on the same b, {s['iters']} iterations (plus steps 1-9) after building "
                                   f"the explicit R ({s['nnz']} nonzeros, {s['t_build_s']:.1f} s, not timed)"},
        "e2e": {"value": val, "unit": "iterations/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-iters", type=int, default=3)
    ap.add_argument("--repeats", type=int, default=5, help="timed solves; the line reports their median")
    ap.add_argument("--no-time-to-equal", action="store_true",
                    help="skip the batched-vs-sequential time-to-equal measurement of the default workload")
    ap.add_argument("--save-params", default=None, help="learned512: write the trained network's parameters here")
    ap.add_argument("--workload", default="plain512",
                    choices=["plain512", "batched64", "large2048", "learned512", "sweep243", "art512", "memory2048",
                             "network512"])
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    world = env_int("WORLD_SIZE", 1)
    rank = env_int("RANK", 0)
    local = env_int("LOCAL_RANK", 0)

    import torch
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if args.impl == "ours" else "gloo")
    if args.impl == "reference":
        rc = run_reference(args, rank, world)
        if dist:
            dist.destroy_process_group()
        return rc

    import numpy as np
    import paper_1807_10151_gb300 as S
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    st = torch.cuda.current_stream()
    if args.workload == "batched64":
        return run_batched(args, dev)
    if args.workload == "large2048":
        return run_large(args, dev)
    if args.workload == "learned512":
        return run_learned(args, dev)
    if args.workload == "sweep243":
        return run_sweep(args, dev)
    if args.workload == "art512":
        return run_art(args, dev)
    if args.workload == "memory2048":
        return run_memory2048(args, dev)
    if args.workload == "network512":
        return run_network512(args, dev)
    G, b_host = make_problem(rank, dev)
    b = torch.tensor(b_host, device=dev)
    from paper_1807_10151_gb300 import autotune, replicas
    tiling = autotune.tune(G)          # forward-projector tile for this geometry (cached per bucket)

    def barrier():
        torch.cuda.synchronize()
        if dist:
            dist.barrier()

    # warm-up: graph capture and W iterations
    x, rep, _ = G.solve(b, **solve_kw(args.warmup))
    assert rep["status"] == 0, rep
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)   # 256 MB > L2
    repeats = max(1, args.repeats)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(repeats)]
    launches0 = S.supcg_kernel_launches()
    with ClockSampler(local) as clk:
        for r in range(repeats):     # one timed solve of `steps` iterations per repeat, L2 flushed before each
            flush.fill_(float(r))
            barrier()
            ev[r][0].record(st)
            x, rep, _ = G.solve(b, **solve_kw(args.steps))
            ev[r][1].record(st)
            barrier()
            assert rep["status"] == 0 and rep["iters"] == args.steps, rep
    launches = (S.supcg_kernel_launches() - launches0) // repeats
    solve_s = [e0.elapsed_time(e1) / 1000.0 for e0, e1 in ev]
    t_med = statistics.median(solve_s)
    ms_max = 1000.0 * replicas.slowest(t_med, dist, dev)   # slowest rank
    value = replicas.job_rate(args.steps, world, ms_max / 1000.0)

    # end to end through the host-buffer entry point (copies in the timed region), median of the repeats
    b_pin = torch.tensor(b_host).pin_memory()
    x_pin = torch.zeros(WL["N"], WL["N"], dtype=torch.float32).pin_memory()
    e2e_s = []
    for r in range(repeats):
        flush.fill_(float(r))
        barrier()
        t0 = time.perf_counter()
        rep_h = G.solve_host(b_pin.numpy(), x_pin.numpy(), **solve_kw(args.steps))
        e2e_s.append(time.perf_counter() - t0)
        assert rep_h["status"] == 0, rep_h
    e2e_value = replicas.job_rate(args.steps, world, replicas.slowest(statistics.median(e2e_s), dist, dev))

    # per-kernel breakdown of the same solve (events around every launch)
    _, rep_p, kinds = G.solve_profiled(b, **solve_kw(args.steps, graph=False))
    fwd_ms, fwd_n = kinds["forward"]
    tot_ms = sum(v[0] for v in kinds.values())
    clocks = clk.summary()

    peaks, peak_src = measured_peaks()
    nnz = nnz_per_projection(WL["N"], WL["V"], WL["U"])
    fwd_avg_s = fwd_ms / max(fwd_n, 1) / 1000.0
    achieved = nnz * OPS_PER_INTERSECTION / fwd_avg_s / 1e12
    sm_max = clocks["sm_max_mhz"] or 2070.0
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    peak_alu = nsm * 128 * sm_max * 1e6 / 1e12
    traffic = None
    tf = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tf):
        try:
            import hashlib
            rec = json.load(open(tf)).get("k_forward", {})
            # the kernel's sources: the projector and the shared header it inlines
            h = hashlib.sha1()
            for f in ("projector.cu", "internal.cuh"):
                h.update(open(os.path.join(ROOT, "paper_1807_10151_gb300", "csrc", f), "rb").read())
            if rec.get("sources_sha1") == h.hexdigest():
                traffic = rec.get("bytes_per_launch")
        except (ValueError, OSError):
            traffic = None

    tte = None
    if rank == 0 and world == 1 and not args.no_time_to_equal:
        tte = {"batched_vs_sequential": batched_comparison(args.steps, args.warmup, dev)}
        lc = learned_comparison(dev, args.steps, args.warmup, n_problems=64, iters_train=16, epochs=1)
        lc.pop("params")
        tte["learned_vs_plain"] = lc

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        s = oracle_sample(args.cpu_iters)
        cpu = {"value": s["iters"] / s["t_solve_s"], "unit": "iterations/s", "cores": s["cores"], "kind": "oracle",
               "sample": f"same workload and b, {s['iters']} SupPCG iterations (plus steps 1-9) of the FP64 oracle "
                         f"after building its explicit R ({s['nnz']} nonzeros, {s['t_build_s']:.1f} s, not timed)"}

    if rank == 0:
        line = {
            "metric": "SupPCG iterations/s", "value": value, "unit": "iterations/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": workload_config(args.steps),
            "timing": {"repeats": repeats, "statistic": "median", "solve_s": solve_s,
                       "timed_region": "one supcg_solve of `steps` iterations (staging and steps 1-9 included) "
                                       "per repeat, CUDA events on the launching stream"},
            "impl": {"graph": True, "parallelism": f"replicas{world}", "fwd_tile": tiling["tile"]},
            "roofline": {"bound": "alu", "kernel": "k_forward", "achieved": achieved, "peak": peak_alu,
                         "unit": "TOP/s", "frac": achieved / peak_alu, "traffic": traffic,
                         "basis": f"{nnz:.4g} intersections x {OPS_PER_INTERSECTION} FP32 ops per launch; peak = "
                                  f"{nsm} SMs x 128 FP32 lanes x {sm_max:.0f} MHz"},
            "kernels": {k: {"ms_total": v[0], "launches": v[1], "share": v[0] / tot_ms if tot_ms else None}
                        for k, v in kinds.items()},
            "hbm_peak_gbs": peaks.get("hbm_gbs"), "peak_source": peak_src,
            "e2e": {"value": e2e_value, "unit": "iterations/s",
                    "h2d_bytes_per_step": 4.0 * (WL["V"] * WL["U"] + WL["N"] ** 2) / args.steps,
                    "d2h_bytes_per_step": 4.0 * WL["N"] ** 2 / args.steps,
                    "note": "median of the repeats of one supcg_solve_host call of `steps` iterations; b and x_0 "
                            "copied in, x copied out"},
            "gpu_launches": int(launches),
            "clocks": clocks,
            "report": {"f_last": rep["f_last"], "tv_last": rep["tv_last"], "ell": rep["ell"]},
        }
        if tte:
            line["time_to_equal"] = tte
        if cpu:
            line["cpu_baseline"] = cpu
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
