"""Iterate parity of whole SupPCG solves (Algorithm 3) against the FP64 oracle
on the benchmark's own workload and on Table 1's long-backtracking parameters.

Bar (the same for both): after 50 while-body executions the returned image
x_{k-1/2} is within 1e-4 relative L2 of the oracle's, the l sequence is
identical, the logged f(x_{k+1/2}) and TV(x_{k+1/2}) of every iteration are
within 1e-4, and the reported final f is the residual of the returned image
(1e-5) and near the oracle's final f (gpu_cases.F_LAST_REL).  Inputs come from
the seeded generators and are fed identically to both sides: the benchmark's
own b (analytic line integrals) for its workload, the oracle's explicit R for
Table 1's case.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1807_10151_gb300 import synth

from gpu_cases import F_LAST_REL, F_OF_IMAGE_REL, gpu_geometry, rel_l2, residual_energy, to_dev

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def _compare(G, R, b, kw, label):
    ref = O.suppcg(R, b, **kw)
    assert ref["status"] == 0
    x, rep, lg = G.solve(to_dev(b), log=True, **kw)
    lg = lg.cpu().numpy()
    xg = x.double().cpu().numpy()
    err = rel_l2(xg, ref["x_half"])
    e_f = rel_l2(lg[:, 0], ref["f"])
    e_tv = rel_l2(lg[:, 2], ref["tv_half"])
    print(f"\n{label}: x {err:.3e}  f-log {e_f:.3e}  tv-log {e_tv:.3e}  "
          f"f_last {rep['f_last']:.9e} vs {ref['f'][-1]:.9e}  l {rep['ell']} vs {ref['ell']}")
    assert rep["status"] == 0 and rep["iters"] == kw["max_iter"]
    np.testing.assert_array_equal(lg[:, 3].astype(np.int64), ref["ell_log"])
    assert rep["ell"] == ref["ell"]
    assert err <= 1e-4, err
    assert e_f <= 1e-4, e_f
    assert e_tv <= 1e-4, e_tv
    assert rep["f_last"] == pytest.approx(residual_energy(R, xg, b), rel=F_OF_IMAGE_REL)
    assert rep["f_last"] == pytest.approx(ref["f"][-1], rel=F_LAST_REL)
    return ref, lg


def test_benchmark_workload_50_iterations_match_oracle():
    """512 x 512 unit square, 720 views over [0, pi), 725 bins, the benchmark's own
    b (analytic line integrals of the 20-ellipse phantom, seed 2001, Poisson
    counts at 1e5 photons per ray, seed 2501, log data); K = 1, gamma = 0.5,
    a = 0.995, mu = 1e-5, rho = 0.8: the configuration the benchmark times,
    50 iterations."""
    import bench
    og = O.Geometry(512, V=720, U=725)
    R = O.CSR(og)
    b = f32(bench.workload_data())
    G = gpu_geometry(og)
    kw = dict(K=1, a=0.995, gamma=0.5, mu=1e-5, rho=0.8, max_iter=50)
    _compare(G, R, b, kw, "512^2/720/725 Poisson 1e5")


@pytest.mark.parametrize("seed", [7001, 7002])
def test_table1_long_backtracking_50_iterations_match_oracle(seed):
    """Table 1's SupPCG parameters (K = 40, a = 1 - 1e-5, gamma = 1e-2,
    mu = 1e-5, rho = 0.8) on a 128 x 128 / 180-view / 182-bin Poisson problem:
    every iteration runs 40 S_TV steps, so l grows by at least 40 per
    iteration and Algorithm 1's trial loop is exercised 2000 times."""
    og = O.Geometry(128, V=180, U=182)
    R = O.CSR(og)
    x_true = synth.ellipse_phantom(128, 12, seed)
    b = f32(synth.poisson_log(R.project(x_true), 1e5, seed + 500))
    G = gpu_geometry(og)
    kw = dict(K=40, a=1 - 1e-5, gamma=1e-2, mu=1e-5, rho=0.8, max_iter=50)
    ref, lg = _compare(G, R, b, kw, f"128^2 Table 1 seed {seed}")
    assert ref["ell"] >= 50 * 40
