"""SupPCG on the Bayesian primary criterion of Eq. (2.3) (GPU, C ABI) vs the oracle.

f(x) = r^2 ||R x - b||^2 + ||x - mu_X||^2: the CG operator is A = r^2 R^T R + I and
the right-hand side r^2 R^T b + mu_X; every reported f (eps test, log, report) is
this criterion.  mu_X is given, or estimated on the device from b (Sec. 2)."""
import numpy as np
import pytest

from oracle import oracle as O

from gpu_cases import config1_problem, gpu_geometry, rel_l2, to_dev

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


@pytest.mark.parametrize("bayes_mu", [0.3, None])
def test_bayesian_suppcg_matches_oracle(bayes_mu):
    og, R, x_true, b = config1_problem(seed=1201)
    G = gpu_geometry(og)
    b32 = f32(b)
    kw = dict(K=1, a=0.995, gamma=0.5, mu=1e-5, rho=0.8, max_iter=30, bayes_r=5.0, bayes_mu=bayes_mu)
    ref = O.suppcg(R, b32, **kw)
    x, rep, lg = G.solve(to_dev(b32), log=True, **kw)
    assert rep["status"] == 0 and rep["iters"] == 30 and rep["ell"] == ref["ell"]
    lg = lg.cpu().numpy()
    np.testing.assert_array_equal(lg[:, 3].astype(np.int64), ref["ell_log"])
    assert rel_l2(lg[:, 0], ref["f"]) <= 1e-4                 # the Bayesian f of every iteration
    assert rep["f0"] == pytest.approx(ref["f0"], rel=1e-5)
    assert rel_l2(x.double().cpu().numpy(), ref["x_half"]) <= 1e-4


def test_gray_level_estimated_on_the_device():
    """f(x_0 = 0) = r^2 ||b||^2 + n mu_X^2 exposes the device's estimate of mu_X."""
    og, R, x_true, b = config1_problem(seed=1202)
    G = gpu_geometry(og)
    b32 = f32(b)
    r = 5.0
    _, rep, _ = G.solve(to_dev(b32), max_iter=0, bayes_r=r, bayes_mu=None)
    mu_dev = np.sqrt((rep["f0"] - r * r * np.sum(b32 ** 2)) / og.n)
    mu_ref = O.gray_level(og, b32)
    assert mu_dev == pytest.approx(mu_ref, rel=1e-4)
    assert mu_ref == pytest.approx(float(np.mean(x_true)), rel=3e-2)   # close to the phantom's mean


@pytest.mark.parametrize("precond", [True, False])
def test_bayesian_unperturbed_matches_oracle(precond):
    """PCG / CG on the Bayesian criterion: iterates over 6 iterations (FP32 CG parts
    from FP64 CG as its residual falls, the loss of conjugacy seen for least squares
    too), then 30 iterations by property: f never increases."""
    og, R, x_true, b = config1_problem(seed=1203, N=48, V=60, U=70)
    G = gpu_geometry(og)
    b32 = f32(b)
    kw = dict(mu=1e-3, rho=0.6, max_iter=6, bayes_r=10.0, bayes_mu=0.2)
    D = None if precond else np.ones((og.ny, og.nx))
    ref = O.suppcg(R, b32, perturb=False, D=D, **kw)
    x, rep, lg = G.solve(to_dev(b32), log=True, perturb=False, precondition=precond, **kw)
    assert rep["status"] == 0
    assert rel_l2(x.double().cpu().numpy(), ref["x_half"]) <= 1e-4
    assert rel_l2(lg.cpu().numpy()[:, 0], ref["f"]) <= 1e-5
    kw["max_iter"] = 30
    _, rep, lg = G.solve(to_dev(b32), log=True, perturb=False, precondition=precond, **kw)
    f = lg.cpu().numpy()[:, 0]
    assert rep["status"] == 0 and np.all(np.diff(f) <= 1e-6 * f[:-1])
    fmin = O.suppcg(R, b32, perturb=False, D=D, **kw)["f"][-1]
    assert f[-1] <= fmin * (1 + 1e-3)
