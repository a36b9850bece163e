"""Batched solve (problems of different geometries in one schedule of
launches): every problem gets the same iterates as its own solve, and the
oracle's."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1807_10151_gb300 import synth

from gpu_cases import gpu_geometry, rel_l2, to_dev

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

SHAPES = [(48, 48, 60, 70), (64, 40, 50, 92), (37, 37, 41, 53), (96, 96, 72, 137), (30, 50, 33, 72)]


def problems():
    out = []
    for c, (nx, ny, V, U) in enumerate(SHAPES):
        og = O.Geometry(nx, ny=ny, V=V, U=U)
        R = O.CSR(og)
        x = synth.ellipse_phantom(max(nx, ny), 8, 3000 + c)[:ny, :nx]
        b = np.asarray(synth.gaussian_noise(R.project(x), 0.01, 3500 + c), np.float32).astype(np.float64)
        out.append((og, R, b))
    return out


def test_batched_equals_single_solves_and_oracle():
    import paper_1807_10151_gb300 as S
    probs = problems()
    kw = dict(K=2, a=0.99, gamma=0.3, mu=1e-4, rho=0.8, max_iter=12)
    geoms = [gpu_geometry(og) for og, _, _ in probs]
    bs = [to_dev(b) for _, _, b in probs]
    xs = [torch.zeros(og.ny, og.nx, device="cuda") for og, _, _ in probs]
    reps = S.solve_batched(geoms, bs, xs, **kw)
    for (og, R, b), G, bd, xb, rep in zip(probs, geoms, bs, xs, reps):
        assert rep["status"] == 0 and rep["iters"] == 12
        xs1, rep1, _ = G.solve(bd, **kw)
        np.testing.assert_array_equal(xb.cpu().numpy(), xs1.cpu().numpy())
        assert rep["ell"] == rep1["ell"] and rep["f_last"] == rep1["f_last"]
        ref = O.suppcg(R, b, **kw)
        assert rep["ell"] == ref["ell"]
        assert rel_l2(xb.double().cpu().numpy(), ref["x_half"]) <= 1e-4


def test_batched_epsilon_mode_stops_each_problem_on_its_own():
    import paper_1807_10151_gb300 as S
    probs = problems()[:3]
    kw = dict(K=1, a=0.995, gamma=0.5, mu=1e-5, rho=0.8)
    geoms = [gpu_geometry(og) for og, _, _ in probs]
    eps = []
    for og, R, b in probs:
        ref = O.suppcg(R, b, max_iter=20, **kw)
        eps.append(float(ref["f"][4 + len(eps) * 3]) * 1.2)
    # one eps for all problems: each stops when its own f drops below it
    e = float(np.median(eps))
    bs = [to_dev(b) for _, _, b in probs]
    xs = [torch.zeros(og.ny, og.nx, device="cuda") for og, _, _ in probs]
    reps = S.solve_batched(geoms, bs, xs, eps=e, max_iter=200, **kw)
    for (og, R, b), rep in zip(probs, reps):
        ref = O.suppcg(R, b, eps=e, max_iter=200, **kw)
        assert rep["iters"] == ref["iters"]
        assert rep["f_last"] <= e
