"""Training and evaluation driver of the learned perturbation direction.

The network (supcg_cnn_*) learns, from pairs the method itself produces, the
direction of the whole K-step superiorization of Algorithm 1: its input is
the iterate x_k and tbar at x_k (the first step's direction, Sec. 3.1), its
target the total S_TV displacement s_k (Algorithm 1 returns y - x).  In
SupPCG (supcg_solve_learned) one accepted step along the proposal replaces
the K sequential steps.

Every computation runs in the library's kernels: trace solves record x_k,
supcg_tv_tbar gives tbar, supcg_superiorize gives s_k, supcg_cnn_train_step
trains.  This module only orders the calls and keeps the tensors.
"""
from __future__ import annotations

import math
import time

import numpy as np

TABLE1 = dict(K=40, a=1 - 1e-5, gamma=1e-2, mu=1e-5, rho=0.8)   # SupPCG row of Table 1


def make_problem(S, synth, N, V, seed, device, noise="gaussian", level=0.01, I0=1e5, n_ell=15, G=None):
    """Geometry (a new one unless G is given) and data b of one random-ellipse
    problem (the projector gives the clean data)."""
    import torch
    if G is None:
        G = S.Geometry(N, n_views=V, n_bins=int(math.ceil(1.42 * N)))
    x = synth.ellipse_phantom(N, n_ell, seed)
    clean = G.project(torch.tensor(x, dtype=torch.float32, device=device)).double().cpu().numpy()
    if noise == "poisson":
        b = synth.poisson_log(clean, I0, seed + 500)
    else:
        b = synth.gaussian_noise(clean, level, seed + 500)
    return G, torch.tensor(b, dtype=torch.float32, device=device)


def make_training_set(n_problems, N=128, V=180, iters=50, seed0=4000, device="cuda", params=TABLE1):
    """(X, T, S): iterates x_k, tbar at x_k and K-step displacements s_k of plain SupPCG runs."""
    import torch
    import paper_1807_10151_gb300 as S
    from paper_1807_10151_gb300 import synth
    kw = dict(params)
    n_pairs = n_problems * iters
    X = torch.empty(n_pairs, N, N, device=device)
    T = torch.empty_like(X)
    D = torch.empty_like(X)
    q = 0
    G = S.Geometry(N, n_views=V, n_bins=int(math.ceil(1.42 * N)))   # one acquisition, many phantoms
    for c in range(n_problems):
        G, b = make_problem(S, synth, N, V, seed0 + c, device, G=G)
        _, rep, log, trace = G.solve_trace(b, max_iter=iters, **kw)
        assert rep["status"] == 0, rep
        ell_in = [0] + [int(v) for v in log[:-1, 3].cpu().numpy()]
        for k in range(iters):
            xk = trace[k].contiguous()
            _, _, tb = G.tv_tbar(xk)
            y = xk.clone()
            rc, _, _ = G.superiorize(y, ell_in[k], kw["a"], kw["gamma"], kw["K"])
            assert rc == 0
            X[q].copy_(xk)
            T[q].copy_(tb)
            D[q].copy_(y).sub_(xk)
            q += 1
    G.close()
    return X, T, D


def train(net, X, T, D, epochs=3, batch=32, lr=1e-3, seed=0, log_every=0):
    """Adam on shuffled minibatches; returns the list of (step, loss) it logged."""
    import torch
    n = X.shape[0]
    g = torch.Generator(device="cpu").manual_seed(seed)
    hist = []
    step = 0
    for ep in range(epochs):
        perm = torch.randperm(n, generator=g)
        for s0 in range(0, n - batch + 1, batch):
            idx = perm[s0:s0 + batch].to(X.device)
            xb, tb, db = X.index_select(0, idx), T.index_select(0, idx), D.index_select(0, idx)
            want = log_every and (step % log_every == 0)
            loss = net.train_step(xb, tb, db, lr=lr, want_loss=bool(want))
            if want:
                hist.append((step, loss))
            step += 1
    return hist


def time_to_equal(G, b, net, iters=100, params=TABLE1, device="cuda", warmup=3):
    """Plain SupPCG for `iters` iterations sets the target (f*, TV*); the learned
    variant's wall time to reach f <= f* and TV <= TV* (and the 1 %-relaxed
    f <= 1.01 f*, TV <= 1.01 TV*) is compared with the plain run's (both after
    untimed `warmup`-iteration solves).  Returns a dict of the measurements."""
    import torch
    import paper_1807_10151_gb300 as S
    kw = dict(params)
    st = torch.cuda.current_stream()
    # each timed solve follows an untimed one of the same kind: a solve keeps one captured
    # graph, re-captured when the kind (plain / learned, logged or not) changes
    G.solve(b, max_iter=warmup, **kw)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    xp, rp, _ = G.solve(b, max_iter=iters, **kw)
    e1.record(st)
    torch.cuda.synchronize()
    t_plain = e0.elapsed_time(e1) / 1000.0
    f_star, tv_star = rp["f_last"], rp["tv_last"]
    # learned: iterate until both targets are met (at most 4x the plain budget)
    lim = 4 * iters
    _, rl_all, ll = G.solve_learned(net, b, max_iter=lim, log=True, **kw)
    ll = ll.cpu().numpy()

    def timed_hit(relax):
        """Learned iterations and wall time to f <= relax f* and TV <= relax TV*."""
        hit = np.nonzero((ll[:, 0] <= relax * f_star) & (ll[:, 2] <= relax * tv_star))[0]
        k_hit = int(hit[0]) + 1 if hit.size else None
        if k_hit is None:
            return None, None
        G.solve_learned(net, b, max_iter=warmup, **kw)
        torch.cuda.synchronize()
        e0.record(st)
        G.solve_learned(net, b, max_iter=k_hit, **kw)
        e1.record(st)
        torch.cuda.synchronize()
        return k_hit, e0.elapsed_time(e1) / 1000.0

    k_hit, t_learned = timed_hit(1.0)
    k_hit1, t_learned1 = timed_hit(1.01)
    return {"plain_iters": iters, "plain_s": t_plain, "f_star": f_star, "tv_star": tv_star,
            "learned_iters": k_hit, "learned_s": t_learned,
            "speedup": (t_plain / t_learned) if t_learned else None,
            "learned_iters_1pct": k_hit1, "learned_s_1pct": t_learned1,
            "speedup_1pct": (t_plain / t_learned1) if t_learned1 else None,
            "learned_accepted": rl_all["n_learned"], "learned_fallbacks": rl_all["n_fallback"],
            "learned_f_last": rl_all["f_last"], "learned_tv_last": rl_all["tv_last"]}


def batched_time_to_equal(geoms, bs, net, iters=100, params=TABLE1, device="cuda", warmup=3):
    """The learned direction in the batched schedule against plain SupPCG on the
    same problems.  Plain SupPCG (batched; the same iterates as one at a time)
    for `iters` iterations sets every problem's target (f*, TV*); each
    problem's first iteration with f <= f* and TV <= TV* under the learned
    direction comes from its single learned solve's log (the batched learned
    solve gives the same iterates bit for bit); the batched learned solve is
    then timed for the largest of those iterations, so that every problem of
    the batch has reached its target.  Returns a dict of the measurements."""
    import torch
    import paper_1807_10151_gb300 as S
    kw = dict(params)
    st = torch.cuda.current_stream()
    xs = [torch.zeros(g.ny, g.nx, device=device) for g in geoms]
    for g, b in zip(geoms, bs):
        g.solve(b, max_iter=warmup, **kw)
    S.solve_batched(geoms, bs, xs, max_iter=warmup, **kw)   # (each timed solve follows one of its kind)
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
    for x in xs:
        x.zero_()
    ev[0].record(st)
    reps = S.solve_batched(geoms, bs, xs, max_iter=iters, **kw)
    ev[1].record(st)
    ev[2].record(st)
    for g, b in zip(geoms, bs):
        g.solve(b, max_iter=iters, **kw)
    ev[3].record(st)
    torch.cuda.synchronize()
    t_batched, t_seq = ev[0].elapsed_time(ev[1]) / 1000.0, ev[2].elapsed_time(ev[3]) / 1000.0
    hits, accepted = [], []
    for g, b, r in zip(geoms, bs, reps):
        _, rl, ll = g.solve_learned(net, b, max_iter=4 * iters, log=True, **kw)
        ll = ll.cpu().numpy()
        hit = np.nonzero((ll[:, 0] <= r["f_last"]) & (ll[:, 2] <= r["tv_last"]))[0]
        hits.append(int(hit[0]) + 1 if hit.size else None)
        accepted.append(rl["n_learned"])
    if any(h is None for h in hits):
        return {"problems": len(geoms), "plain_iters": iters, "learned_hits": hits, "reached": False}
    k_hit = max(hits)
    S.solve_batched_learned(geoms, net, bs, xs, max_iter=warmup, **kw)
    for x in xs:
        x.zero_()
    torch.cuda.synchronize()
    ev[4].record(st)
    lrep = S.solve_batched_learned(geoms, net, bs, xs, max_iter=k_hit, **kw)
    ev[5].record(st)
    torch.cuda.synchronize()
    t_learned = ev[4].elapsed_time(ev[5]) / 1000.0
    assert all(r["status"] == 0 for r in lrep), lrep
    # (a problem's f and TV need not stay below its target after its first hit: TV grows as
    # CG fits the data, so the batch's last iterate is not the criterion, the first hit is)
    return {"problems": len(geoms), "plain_iters": iters, "learned_iters": k_hit, "learned_hits": hits,
            "plain_batched_s": t_batched, "plain_sequential_s": t_seq, "learned_batched_s": t_learned,
            "speedup_vs_plain_batched": t_batched / t_learned, "speedup_vs_plain_sequential": t_seq / t_learned,
            "accepted_proposals": accepted}
