"""Oracle pins for the Bayesian primary criterion of Eq. (2.3),
f(x) = r^2 ||R x - b||^2 + ||x - mu_X||^2 (normal equations (r^2 R^T R + I) x =
r^2 R^T b + mu_X), and for the gray level mu_X estimated from the data (Sec. 2)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1807_10151_gb300 import synth


def small_problem(seed=3, N=8, V=12, U=13):
    og = O.Geometry(N, V=V, U=U)
    R = O.CSR(og)
    x = synth.ellipse_phantom(N, 3, seed)
    b = R.project(x) + 0.01 * np.random.default_rng(seed).standard_normal((og.V, og.U))
    return og, R, x, b


@pytest.mark.parametrize("precond", [False, True])
def test_cg_on_the_bayesian_criterion_reaches_the_dense_solution(precond):
    """Unperturbed (P)CG on A = r^2 R^T R + I converges to the direct solve of the
    normal equations (an independent method: LU of the dense A)."""
    og, R, x, b = small_problem()
    r, mu = 3.0, 0.25
    A = r * r * (R.dense().T @ R.dense()) + np.eye(og.n)
    y = r * r * (R.dense().T @ b.ravel()) + mu
    ref = np.linalg.solve(A, y)
    kw = dict(perturb=False, max_iter=3 * og.n, eps=-1.0, bayes_r=r, bayes_mu=mu)
    if not precond:
        kw["D"] = np.ones((og.ny, og.nx))       # M = I: plain CG
    out = O.suppcg(R, b, **kw)
    assert out["status"] == 0
    err = np.linalg.norm(out["x_half"].ravel() - ref) / np.linalg.norm(ref)
    assert err <= 1e-8, err
    # f at the minimiser is the criterion's value there
    fmin = r * r * np.sum((R.dense() @ ref - b.ravel()) ** 2) + np.sum((ref - mu) ** 2)
    assert out["f"][-1] == pytest.approx(fmin, rel=1e-8)


def test_bayesian_f_at_x0_is_its_closed_form():
    og, R, x, b = small_problem(seed=4)
    r, mu = 2.0, 0.3
    out = O.suppcg(R, b, perturb=False, max_iter=1, bayes_r=r, bayes_mu=mu)
    assert out["f0"] == pytest.approx(r * r * np.sum(b ** 2) + og.n * mu * mu, rel=1e-12)


def test_large_r_approaches_least_squares():
    """As r grows the criterion's minimiser tends to the least-squares one (the
    regularising term's weight 1/r^2 vanishes)."""
    og, R, x, b = small_problem(seed=5)
    ls = O.suppcg(R, b, perturb=False, max_iter=3 * og.n, D=np.ones((og.ny, og.nx)))["x_half"]
    prev = None
    for r in (10.0, 100.0, 1000.0, 10000.0):
        xb = O.suppcg(R, b, perturb=False, max_iter=3 * og.n, D=np.ones((og.ny, og.nx)),
                      bayes_r=r, bayes_mu=0.0)["x_half"]
        d = np.linalg.norm(xb - ls) / np.linalg.norm(ls)
        if prev is not None:
            assert d < prev
        prev = d
    assert prev < 1e-3


def test_gray_level_recovers_the_mean_of_a_constant_image():
    """For x = c everywhere, each view's b sums to the image integral c n d^2 (up to
    the sampling of the footprints), so the estimate is c."""
    og = O.Geometry(48, V=60, U=70)
    R = O.CSR(og)
    c = 0.37
    b = R.project(np.full((og.ny, og.nx), c))
    assert O.gray_level(og, b) == pytest.approx(c, rel=2e-3)
    # and the mean of a phantom, from its own projections
    x = synth.ellipse_phantom(48, 8, 6)
    assert O.gray_level(og, R.project(x)) == pytest.approx(float(np.mean(x)), rel=2e-3)
