"""Oracle pins for ART on the Bayesian criterion of Eq. (2.3) (Sec. 3.4: the
row-action method of Herman, Hurwitz and Lent) and for SupART.

What fixes the oracle here is not its own update formula: ART's fixed point is
the minimiser of r^2 ||R x - b||^2 + ||x - mu_X||^2, obtained independently by
a dense direct solve; one relaxed step with lambda = 1 lands exactly on its
hyperplane; rays of one view S bins apart share no pixel (read off the explicit
matrix), so their order inside a class cannot matter; and S_TV with gamma = 0
leaves every iterate unchanged."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1807_10151_gb300 import synth


def small_problem(seed=3, N=8, V=12, U=13, **geo):
    og = O.Geometry(N, V=V, U=U, **geo)
    R = O.CSR(og)
    x = synth.ellipse_phantom(N, 3, seed)
    b = R.project(x) + 0.01 * np.random.default_rng(seed).standard_normal((og.V, og.U))
    return og, R, x, b


@pytest.mark.parametrize("geo", [dict(N=64, V=90, U=95), dict(N=24, V=30, U=40, ds=0.6 / 24),
                                 dict(N=24, V=17, U=21, ds=1.4 / 24), dict(N=20, V=16, U=29, off=0.013)])
def test_rays_one_class_apart_share_no_pixel(geo):
    N = geo.pop("N")
    og = O.Geometry(N, **geo)
    R = O.CSR(og)
    S = O.art_spacing(og)
    assert S >= 1
    for v in range(og.V):
        pix = [set(R.ci[R.rp[v * og.U + u]:R.rp[v * og.U + u + 1]]) for u in range(og.U)]
        for u in range(og.U - S):
            assert not (pix[u] & pix[u + S]), (v, u, S)


def test_art_order_visits_every_ray_once():
    og = O.Geometry(16, V=7, U=23)
    order = O.art_order(og)
    assert sorted(order.tolist()) == list(range(og.m))
    # views in order, and within a view the residue classes of S in turn
    S = O.art_spacing(og)
    first = order[:og.U]
    assert list(first[: (og.U + S - 1) // S]) == list(range(0, og.U, S))


def test_relaxation_one_lands_on_the_ray_hyperplane():
    """With lambda = 1 a step makes ray i's equation r (b_i - <R_i, x>) - u_i = 0
    hold exactly (Kaczmarz projection), and touches only that ray's pixels and u_i."""
    og, R, x, b = small_problem()
    r = 5.0
    rng = np.random.default_rng(1)
    x0 = rng.uniform(size=(og.ny, og.nx))
    u0 = rng.standard_normal((og.V, og.U))
    for i in (0, 17, og.m // 2, og.m - 1):
        res = O.art(R, b, r=r, lam=1.0, cycles=1, x0=x0, u0=u0, order=[i])
        xi, ui = res["x"].ravel(), res["u"].ravel()
        row = slice(R.rp[i], R.rp[i + 1])
        resid = r * (b.ravel()[i] - R.va[row] @ xi[R.ci[row]]) - ui[i]
        assert abs(resid) <= 1e-12 * max(1.0, r * abs(b.ravel()[i]))
        moved = np.flatnonzero(xi != x0.ravel())
        assert set(moved.tolist()) <= set(R.ci[row].tolist())
        assert np.count_nonzero(ui != u0.ravel()) <= 1


@pytest.mark.parametrize("lam,cycles", [(1.0, 300), (0.5, 600), (1.5, 300)])
def test_art_converges_to_the_bayesian_minimiser(lam, cycles):
    """For 0 < lambda < 2 the cycles converge to the minimiser of Eq. (2.3), the
    solution of (r^2 R^T R + I) x = r^2 R^T b + mu_X (dense direct solve), and the
    auxiliary values to the scaled residual r (b - R x*)."""
    og, R, x, b = small_problem(N=6, V=8, U=9)
    r, mu = 2.0, O.gray_level(og, b)
    A = R.dense()
    xs = np.linalg.solve(r * r * A.T @ A + np.eye(og.n), r * r * A.T @ b.ravel() + mu)
    res = O.art(R, b, r=r, lam=lam, cycles=cycles, mu=mu)
    assert np.linalg.norm(res["x"].ravel() - xs) <= 1e-10 * np.linalg.norm(xs)
    us = r * (b.ravel() - A @ xs)
    assert np.linalg.norm(res["u"].ravel() - us) <= 1e-9 * np.linalg.norm(us)


def test_order_inside_a_class_does_not_matter():
    """Rays of one class touch disjoint pixels: visiting each class backwards gives
    bit-identical x and u."""
    og, R, x, b = small_problem(N=16, V=10, U=23)
    S = O.art_spacing(og)
    order = O.art_order(og)
    rev = np.concatenate([np.arange(v * og.U + c, (v + 1) * og.U, S)[::-1]
                          for v in range(og.V) for c in range(S)])
    assert sorted(rev.tolist()) == sorted(order.tolist())
    a = O.art(R, b, r=5.0, lam=0.3, cycles=2, order=order)
    c = O.art(R, b, r=5.0, lam=0.3, cycles=2, order=rev)
    assert np.array_equal(a["x"], c["x"]) and np.array_equal(a["u"], c["u"])


def test_supart_with_zero_steps_is_art():
    """SupART perturbs with S_TV before each cycle; gamma = 0 makes every
    perturbation zero (each trial is accepted at once), so the iterates are ART's
    bit for bit while l still advances by K per cycle."""
    og, R, x, b = small_problem()
    a = O.art(R, b, r=5.0, lam=5e-2, cycles=3)
    s = O.art(R, b, r=5.0, lam=5e-2, cycles=3, K=4, gamma=0.0)
    assert np.array_equal(a["x"], s["x"]) and np.array_equal(a["u"], s["u"])
    assert s["ell"] == 3 * 4 and s["status"] == 0


def test_supart_perturbations_do_not_raise_tv():
    """Every SupART perturbation is S_TV's: TV after it is at most TV before
    (Algorithm 1 accepts only nonascending trials)."""
    og, R, x, b = small_problem(N=16, V=20, U=23)
    state = O.art(R, b, r=5.0, lam=5e-2, cycles=1)
    xk, ell = state["x"], 0
    for _ in range(3):
        rc, s, ell, _ = O.stv(xk, ell, 1 - 1e-5, 1e-2, 10)
        assert rc == 0
        assert O.tv(xk + s) <= O.tv(xk)
        xk = O.art(R, b, r=5.0, lam=5e-2, cycles=1, x0=xk + s)["x"]
