"""SupPCG with the learned direction (supcg_solve_learned).

The learned step is an addition to the paper: a proposal t is used only if it
is nonascending for TV at x_k (the one-sided directional derivative of the
Sec. 3.1 definition is negative), with one step of length
2^-j gamma sum_{i<K} a^(l+i); otherwise Algorithm 1's K plain steps run."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1807_10151_gb300 import synth

from gpu_cases import config1_problem, gpu_geometry, rel_l2, to_dev

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def test_untrained_proposal_step_matches_its_definition():
    """Untrained network: the proposal is tbar itself.  One learned body from x_1
    reproduced with the oracle's TV, direction and directional derivative."""
    import paper_1807_10151_gb300 as S
    og, R, x_true, b = config1_problem(seed=1101)
    G = gpu_geometry(og)
    net = S.CNN(og.ny, og.nx, max_batch=1, seed=1)
    b32 = f32(b)
    K, a, gamma = 5, 0.99, 0.05
    kw = dict(K=K, a=a, gamma=gamma, mu=1e-5, rho=0.8)
    xg, rep, _ = G.solve_learned(net, to_dev(b32), max_iter=1, **kw)
    assert rep["status"] == 0 and rep["n_learned"] == 1 and rep["n_fallback"] == 0
    x1 = O.suppcg(R, b32, max_iter=0, **kw)["x_last"]       # x_1 of Algorithm 3
    t = O.tv_direction(x1)
    assert O.tv_dirderiv(x1, t) < 0
    L0 = gamma * (1 - a ** K) / (1 - a)
    tv0 = O.tv(x1)
    j = 0
    while O.tv(x1 + L0 * 2.0 ** -j * t) > tv0:
        j += 1
    assert rep["ell"] == K + j
    ref = x1 + L0 * 2.0 ** -j * t
    assert rel_l2(xg.double().cpu().numpy(), ref) <= 1e-5


def test_ascending_proposal_falls_back_to_plain_superiorization():
    """A network that proposes -tbar (ascending) is rejected every iteration and the
    solve is bitwise the plain SupPCG solve."""
    import paper_1807_10151_gb300 as S
    og, R, x_true, b = config1_problem(seed=1102, N=48, V=60, U=70)
    G = gpu_geometry(og)
    net = S.CNN(og.ny, og.nx, max_batch=1, seed=1)
    p = np.zeros(net.nparam, dtype=np.float32)
    layers = S.CNN.unflatten(p)          # views into p
    layers[0][0][0, 1, 1, 1] = 1.0       # a1_0 = relu(t~)
    layers[0][0][1, 1, 1, 1] = -1.0      # a1_1 = relu(-t~)
    for li in (1, 2, 3):
        layers[li][0][0, 0, 1, 1] = 1.0
        layers[li][0][1, 1, 1, 1] = 1.0
    layers[4][0][0, 0, 1, 1] = -2.0      # out = t~ - 2 relu(t~) + 2 relu(-t~) = -t~
    layers[4][0][0, 1, 1, 1] = 2.0
    net.set_params(p)
    kw = dict(K=3, a=0.9, gamma=0.1, mu=1e-5, rho=0.8, max_iter=12)
    b32 = to_dev(f32(b))
    xl, rl, _ = G.solve_learned(net, b32, **kw)
    xp, rp, _ = G.solve(b32, **kw)
    assert rl["n_fallback"] == 12 and rl["n_learned"] == 0
    np.testing.assert_array_equal(xl.cpu().numpy(), xp.cpu().numpy())
    assert rl["ell"] == rp["ell"]


def test_learned_solve_keeps_theorem1_and_nonascent():
    import paper_1807_10151_gb300 as S
    og, R, x_true, b = config1_problem(seed=1103)
    G = gpu_geometry(og)
    net = S.CNN(og.ny, og.nx, max_batch=1, seed=1)
    K, a, gamma = 4, 0.95, 0.1
    x, rep, lg = G.solve_learned(net, to_dev(f32(b)), log=True, max_iter=20, K=K, a=a, gamma=gamma)
    lg = lg.cpu().numpy()
    assert rep["status"] == 0 and rep["n_learned"] + rep["n_fallback"] == 20
    for k in range(1, 21):
        assert lg[k - 1, 2] <= lg[k - 1, 1] * (1 + 1e-7)                       # TV(x_{k+1/2}) <= TV(x_k)
        assert math.sqrt(lg[k - 1, 6]) <= K * gamma * a ** ((k - 1) * K) * (1 + 1e-5)
        assert lg[k - 1, 3] >= k * K


def test_training_on_method_pairs_beats_the_untrained_direction():
    """Pairs from plain SupPCG runs (x_k, tbar, K-step displacement) with steps long
    enough for the K-step path to bend (gamma = 0.5): after training, the held-out
    error of the proposed direction is below that of the untrained network, which
    proposes tbar itself.  (With Table 1's short steps the path is nearly straight
    and tbar is already within about 1 % of the K-step direction.)"""
    import paper_1807_10151_gb300 as S
    from paper_1807_10151_gb300 import learned as Lr
    params = dict(K=10, a=0.99, gamma=0.5, mu=1e-5, rho=0.8)
    X, T, D = Lr.make_training_set(10, N=64, V=90, iters=12, seed0=4100, params=params)
    Xh, Th, Dh = Lr.make_training_set(2, N=64, V=90, iters=12, seed0=4900, params=params)
    net = S.CNN(64, 64, max_batch=24, seed=3)
    _, base_loss = net.gradients(Xh, Th, Dh)
    Lr.train(net, X, T, D, epochs=30, batch=24, lr=1e-3)
    _, trained_loss = net.gradients(Xh, Th, Dh)
    assert base_loss > 1e-3                     # the path bends: tbar alone is not the answer
    assert trained_loss < 0.8 * base_loss, (base_loss, trained_loss)


def test_batched_learned_solve_equals_the_single_learned_solves():
    """Three problems of one image size with different views and bins, the network
    run once per iteration over all three (supcg_solve_batched_learned): each
    problem's image, l and counts of accepted and rejected proposals equal those
    of supcg_solve_learned on it alone, bit for bit.  The network's last layer is
    seeded away from zero, so its proposals differ from tbar."""
    import paper_1807_10151_gb300 as S
    net = S.CNN(64, 64, max_batch=4, seed=5)
    p = net.get_params()
    layers = S.CNN.unflatten(p)
    layers[4][0][...] = 0.05 * np.random.default_rng(6).standard_normal(layers[4][0].shape)
    net.set_params(p)
    kw = dict(K=6, a=0.97, gamma=0.3, mu=1e-5, rho=0.8, max_iter=12)
    geoms, bs = [], []
    for c, (V, U) in enumerate(((90, 95), (61, 92), (45, 101))):
        og, R, x_true, b = config1_problem(seed=1200 + c, N=64, V=V, U=U)
        geoms.append(gpu_geometry(og))
        bs.append(to_dev(f32(b)))
    singles = [g.solve_learned(net, b, **kw) for g, b in zip(geoms, bs)]
    xs = [torch.zeros(64, 64, device="cuda") for _ in geoms]
    reps = S.solve_batched_learned(geoms, net, bs, xs, **kw)
    for (xs1, r1, _), xb, rb in zip(singles, xs, reps):
        assert r1["status"] == 0 and rb["status"] == 0
        assert rb["iters"] == r1["iters"] == 12 and rb["ell"] == r1["ell"]
        assert rb["n_learned"] == r1["n_learned"] and rb["n_fallback"] == r1["n_fallback"]
        np.testing.assert_array_equal(xb.cpu().numpy(), xs1.cpu().numpy())
    assert sum(r["n_learned"] for r in reps) > 0


def test_batched_learned_solve_rejects_other_image_sizes():
    import paper_1807_10151_gb300 as S
    net = S.CNN(64, 64, max_batch=2, seed=5)
    og1, _, _, b1 = config1_problem(seed=1210, N=64, V=30, U=95)
    og2, _, _, b2 = config1_problem(seed=1211, N=48, V=30, U=70)
    geoms = [gpu_geometry(og1), gpu_geometry(og2)]
    xs = [torch.zeros(g.ny, g.nx, device="cuda") for g in geoms]
    with pytest.raises(S.SupcgError) as e:
        S.solve_batched_learned(geoms, net, [to_dev(f32(b1)), to_dev(f32(b2))], xs, max_iter=2)
    assert e.value.code == -8
    with pytest.raises(S.SupcgError) as e:   # more problems than the network's batch
        S.solve_batched_learned([geoms[0]] * 3, net, [to_dev(f32(b1))] * 3, [xs[0]] * 3, max_iter=2)
    assert e.value.code == -1
