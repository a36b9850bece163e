"""Pins of the oracle's preconditioner M = F^-1 D F (Eq. (3.2)), of U_PCG /
PCG (Algorithm 2) and of SupPCG (Algorithm 3, Theorems 1 and 2, and the
SupTPCG equivalence of Sec. 5, Algorithms 4-5, Table 2)."""
import math

import numpy as np
import pytest

from oracle import oracle as O


# ---------------------------------------------------------------- preconditioner

def test_D_special_values():
    mu, rho, N = 1e-3, 0.6, 16
    D = O.precond_D(N, N, mu, rho)
    assert D[0, 0] == pytest.approx(mu * 1.0, rel=1e-15)                       # h(0) = mu
    assert D[0, N // 4] == pytest.approx((math.pi / 2 + mu) * rho, rel=1e-14)  # w = pi/2
    assert D[N // 4, 0] == pytest.approx((math.pi / 2 + mu) * rho, rel=1e-14)
    assert D[0, N // 2] == pytest.approx((math.pi + mu) * (2 * rho - 1), rel=1e-14)  # w = pi
    assert D[N // 2, N // 2] == pytest.approx((math.pi + mu) * (2 * rho - 1), rel=1e-14)  # clamped
    assert D[0, 3 * N // 4] == D[0, N // 4]                                    # |w| symmetric


def test_fourier_diag_identity_and_numpy_cross_check():
    rng = np.random.default_rng(0)
    for ny, nx in ((8, 8), (6, 10), (7, 5)):
        g = rng.standard_normal((ny, nx))
        np.testing.assert_allclose(O.fourier_diag(np.ones((ny, nx)), g), g, atol=1e-12)
        D = O.precond_D(ny, nx, 1e-5, 0.8)
        ref = np.real(np.fft.ifft2(D * np.fft.fft2(g)))
        np.testing.assert_allclose(O.fourier_diag(D, g), ref, atol=1e-12)


def test_cosine_mode_is_eigenvector():
    ny, nx, k1, k2 = 12, 16, 2, 3
    I, J = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    mode = np.cos(2 * np.pi * (k1 * I / ny + k2 * J / nx))
    mu, rho = 1e-4, 0.8
    w = math.hypot(2 * math.pi * k1 / ny, 2 * math.pi * k2 / nx)
    lam = (w + mu) * (rho + (1 - rho) * math.cos(w))
    np.testing.assert_allclose(O.precondition(mode, mu, rho), lam * mode, atol=1e-12)


def test_M_symmetric_positive_definite_for_rho_above_half():
    rng = np.random.default_rng(1)
    u, v = rng.standard_normal((2, 9, 9))
    Mu, Mv = O.precondition(u, 1e-5, 0.8), O.precondition(v, 1e-5, 0.8)
    assert np.sum(Mu * v) == pytest.approx(np.sum(u * Mv), rel=1e-12)
    assert np.sum(Mu * u) > 0
    assert O.precond_D(9, 9, 1e-5, 0.8).min() > 0
    assert O.precond_D(8, 8, 1e-5, 0.4).min() < 0  # rho <= 1/2 makes M indefinite


# ---------------------------------------------------------------- PCG / SupPCG

def tiny_problem(N=6, V=8, U=9, seed=0):
    g = O.Geometry(N, V=V, U=U)
    R = O.CSR(g)
    rng = np.random.default_rng(seed)
    x = rng.uniform(size=(N, N))
    b = R.project(x) + 0.01 * rng.standard_normal((V, U))
    return g, R, b


def textbook_cgls(A, b, iters):
    """CGLS (CG on A^T A x = A^T b) in its residual-recurrence form."""
    x = np.zeros(A.shape[1])
    r = b.copy()
    s = A.T @ r
    p = s.copy()
    gam = s @ s
    xs = []
    for _ in range(iters):
        q = A @ p
        al = gam / (q @ q)
        x = x + al * p
        r = r - al * q
        s = A.T @ r
        gnew = s @ s
        p = s + (gnew / gam) * p
        gam = gnew
        xs.append(x.copy())
    return xs


def test_unperturbed_cg_equals_textbook_cgls():
    g, R, b = tiny_problem()
    A = R.dense()
    ref = textbook_cgls(A, b.ravel(), 12)
    for it in range(1, 8):
        out = O.suppcg(R, b, perturb=False, max_iter=it, D=np.ones((g.ny, g.nx)))
        # x_{k-1/2} after `it` bodies equals x_it of CG; x_last = x_{it+1}
        np.testing.assert_allclose(out["x_half"].ravel(), ref[it - 1], rtol=1e-8, atol=1e-10)
        np.testing.assert_allclose(out["x_last"].ravel(), ref[it], rtol=1e-8, atol=1e-10)


def test_cg_reaches_least_squares_solution():
    g, R, b = tiny_problem(N=5, V=9, U=9, seed=3)
    A = R.dense()
    xls = np.linalg.lstsq(A, b.ravel(), rcond=None)[0]
    out = O.suppcg(R, b, perturb=False, max_iter=g.n + 5, D=np.ones((g.ny, g.nx)))
    np.testing.assert_allclose(out["x_half"].ravel(), xls, rtol=1e-6, atol=1e-7)
    pcg = O.suppcg(R, b, perturb=False, max_iter=g.n + 5, mu=1e-3, rho=0.6)
    np.testing.assert_allclose(pcg["x_half"].ravel(), xls, rtol=1e-6, atol=1e-7)


def test_residual_monotone_for_cg_and_pcg():
    g, R, b = tiny_problem(N=8, V=10, U=13, seed=4)
    for D in (np.ones((8, 8)), O.precond_D(8, 8, 1e-3, 0.6)):
        out = O.suppcg(R, b, perturb=False, max_iter=20, D=D)
        f = np.concatenate([[out["f0"]], out["f"]])
        assert np.all(np.diff(f) <= 1e-12 * f[0])


def test_scaling_M_leaves_iterates_unchanged():
    g, R, b = tiny_problem(N=7, V=9, U=11, seed=5)
    D = O.precond_D(7, 7, 1e-4, 0.8)
    o1 = O.suppcg(R, b, max_iter=6, D=D, K=2, gamma=0.05, a=0.9, perturb=False)
    o2 = O.suppcg(R, b, max_iter=6, D=3.7 * D, K=2, gamma=0.05, a=0.9, perturb=False)
    np.testing.assert_allclose(o1["x_half"], o2["x_half"], rtol=1e-9, atol=1e-12)


def test_suppcg_theorem1_and_tv_nonascent():
    g, R, b = tiny_problem(N=10, V=12, U=15, seed=6)
    a, gamma, K = 0.9, 0.2, 3
    out = O.suppcg(R, b, a=a, gamma=gamma, K=K, max_iter=15)
    assert out["status"] == 0 and out["iters"] == 15
    for k in range(1, 16):   # body k: ||s_k|| <= K gamma a^((k-1)K), l_{k+1} >= kK
        assert out["snorm"][k - 1] <= K * gamma * a ** ((k - 1) * K) * (1 + 1e-12)
        assert out["ell_log"][k - 1] >= k * K
        assert out["tv_half"][k - 1] <= out["tv_k"][k - 1] * (1 + 1e-15)


def test_suppcg_equals_suptpcg_table2():
    """Algorithms 3 and 5 are equivalent through x = N^T xhat, N = F^-1 D^1/2 F."""
    g, R, b = tiny_problem(N=8, V=10, U=13, seed=7)
    D = O.precond_D(8, 8, 1e-3, 0.8)
    a, gamma, K, iters = 0.8, 0.1, 2, 6
    ref = O.suppcg(R, b, a=a, gamma=gamma, K=K, max_iter=iters, D=D)

    sq, isq = np.sqrt(D), 1.0 / np.sqrt(D)
    Nop = lambda v: O.fourier_diag(sq, v)          # N = N^T (D real and even)
    NinvT = lambda v: O.fourier_diag(isq, v)
    y = R.backproject(b)
    NAN = lambda v: Nop(R.backproject(R.project(Nop(v))))
    # SupTPCG(N^-T x0) with x0 = 0, Algorithm 5 with U_TPCG = Algorithm 4
    xh = np.zeros((8, 8))
    gh = NAN(xh) - Nop(y)
    ph = -gh
    hh = NAN(ph)
    al = -np.sum(gh * ph) / np.sum(ph * hh)
    xh = xh + al * ph
    ell = 0
    for k in range(iters):
        rc, s, ell, _ = O.stv(Nop(xh), ell, a, gamma, K)
        xhh = xh + NinvT(s)
        gh = NAN(xhh) - Nop(y)
        be = np.sum(gh * hh) / np.sum(ph * hh)
        ph = -gh + be * ph
        hh = NAN(ph)
        al = -np.sum(gh * ph) / np.sum(ph * hh)
        xh = xhh + al * ph
    np.testing.assert_allclose(Nop(xhh), ref["x_half"], rtol=0, atol=1e-10)
    assert ell == ref["ell"]


def test_epsilon_mode_terminates_theorem2():
    g, R, b = tiny_problem(N=6, V=8, U=9, seed=8)
    A = R.dense()
    xls = np.linalg.lstsq(A, b.ravel(), rcond=None)[0]
    eps0 = np.sum((A @ xls - b.ravel()) ** 2)
    out = O.suppcg(R, b, a=0.9, gamma=0.1, K=2, eps=eps0 * 1.05 + 1e-12, max_iter=500)
    assert out["status"] == 0 and out["iters"] < 500
    f_ret = np.sum((A @ out["x_half"].ravel() - b.ravel()) ** 2)
    assert f_ret <= eps0 * 1.05 + 1e-12
