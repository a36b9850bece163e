"""GPU (C-ABI) vs FP64 oracle parity for every step of the SupPCG hot path.

Tolerances: projections and backprojections 1e-5 relative L2 (FP32
accumulation of exact intersection lengths), adjoint identity 1e-6, iterates
after 50 SupPCG iterations 1e-4 relative L2 with an identical l sequence.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1807_10151_gb300 import synth

from gpu_cases import F_LAST_REL, F_OF_IMAGE_REL, config1_problem, gpu_geometry, rel_l2, residual_energy, to_dev

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


GEOMS = [
    # (nx, ny, V, U, off, ds-factor): spans several tiles, ragged tails, odd sizes
    (64, 64, 90, 95, 0.0, 1.0),
    (37, 23, 41, 47, 0.013, 1.0),
    (7, 7, 5, 11, 0.0, 1.0),
    (2, 3, 4, 5, 0.0, 1.0),
    (1, 1, 3, 3, 0.0, 1.0),
    (243, 243, 360, 345, 0.0, 1.0),
    (130, 96, 77, 181, -0.02, 1.0),
    (50, 50, 33, 50, 0.0, 1.4),
    (64, 64, 16, 200, 0.0, 0.6),
    (96, 80, 45, 150, 0.0, 0.7),
    (200, 200, 64, 300, 0.0, 1.0),
]


@pytest.mark.parametrize("nx,ny,V,U,off,dsf", GEOMS)
def test_project_and_backproject_match_oracle(nx, ny, V, U, off, dsf):
    d = 1.0 / max(nx, ny)
    og = O.Geometry(nx, ny=ny, V=V, U=U, off=off, ds=d * dsf)
    R = O.CSR(og)
    G = gpu_geometry(og)
    rng = np.random.default_rng(nx * 1000 + V)
    x = f32(rng.uniform(size=(ny, nx)))
    y = f32(rng.standard_normal((V, U)))
    gx = G.project(to_dev(x)).double().cpu().numpy()
    gy = G.backproject(to_dev(y)).double().cpu().numpy()
    assert rel_l2(gx, R.project(x)) <= 1e-5
    assert rel_l2(gy, R.backproject(y)) <= 1e-5
    # adjoint identity of the GPU pair, with y correlated to R x and independent
    for yy in (y, f32(R.project(x) + 0.1 * y)):
        lhs = float(np.sum(gx * yy))
        rhs = float(np.sum(x * G.backproject(to_dev(yy)).double().cpu().numpy()))
        assert abs(lhs - rhs) <= 1e-6 * np.linalg.norm(gx) * np.linalg.norm(yy)


@pytest.mark.parametrize("V,pairs", [(720, 359), (90, 44), (13, 6), (5, 2), (2, 0), (1, 0)])
def test_mirror_pairs_of_the_default_angles(V, pairs):
    """Views v pi / V and (V - v) pi / V pair up; 0 and pi / 2 stay single."""
    og = O.Geometry(16, V=V, U=23)
    assert gpu_geometry(og).mirror_pairs() == pairs


def test_projection_with_paired_and_single_views_matches_oracle():
    """A view set with one mirror pair (0.3, pi - 0.3) among single views, at
    angles the default set does not have: the paired kernel sums the pair's
    rays together, the others alone, every ray within 1e-5 of the oracle's
    explicit R, and the pair still the exact transpose of the backprojector."""
    angles = np.array([0.3, 0.9, np.pi - 0.3, 1.7, 2.2])
    og = O.Geometry(53, ny=41, V=5, U=71, theta=angles)
    R = O.CSR(og)
    G = gpu_geometry(og)
    assert G.mirror_pairs() == 1
    rng = np.random.default_rng(77)
    x = f32(rng.uniform(size=(41, 53)))
    gx = G.project(to_dev(x)).double().cpu().numpy()
    assert rel_l2(gx, R.project(x)) <= 1e-5
    for v in range(5):
        assert rel_l2(gx[v], R.project(x)[v]) <= 1e-5
    e = np.zeros((41, 53), np.float32)
    e[20, 7] = 1
    col = G.project(to_dev(e)).cpu().numpy()
    for v in range(5):
        u = int(np.argmax(col[v]))
        assert col[v, u] > 0
        s = np.zeros((5, 71), np.float32)
        s[v, u] = 1
        assert G.backproject(to_dev(s)).cpu().numpy()[20, 7] == col[v, u]


def test_bin_size_limits():
    """Bins up to about 2.5 times coarser than pixels are projected with oracle parity;
    much coarser or much finer bins are refused (SUPCG_ERR_UNSUPPORTED), not computed wrongly.
    (2.3: with 2.4 or 1.6 some axis-view rays lie on pixel edges up to the FP64 rounding
    of the spacing, and the tie rule then sees a boundary edge on one side only.)"""
    import paper_1807_10151_gb300 as S
    d = 1.0 / 48
    og = O.Geometry(48, V=40, U=31, ds=2.3 * d)
    R = O.CSR(og)
    G = gpu_geometry(og)
    rng = np.random.default_rng(48)
    x = f32(rng.uniform(size=(og.ny, og.nx)))
    y = f32(rng.standard_normal((og.V, og.U)))
    assert rel_l2(G.project(to_dev(x)).double().cpu().numpy(), R.project(x)) <= 1e-5
    assert rel_l2(G.backproject(to_dev(y)).double().cpu().numpy(), R.backproject(y)) <= 1e-5
    for dsf in (3.0, 0.45):
        with pytest.raises(S.SupcgError) as e:
            S.Geometry(48, n_views=40, n_bins=int(1.5 * 48 / dsf) + 2, pixel_size=d, bin_spacing=dsf * d)
        assert e.value.code == -8


@pytest.mark.parametrize("parts", [1, 2, 3, 4, 5, 8])
def test_backprojector_is_exact_transpose_bitwise(parts):
    """Entries of R read from forward columns equal entries read from backward rows,
    bit for bit, for every split of the views among a tile's blocks."""
    og = O.Geometry(24, ny=20, V=13, U=33, off=0.004)
    G = gpu_geometry(og)
    assert G.set_bwd_parts(parts) == 0 and G.get_bwd_parts() == parts
    pix = [(0, 0), (7, 11), (19, 23), (10, 3)]
    rays = [(0, 16), (3, 5), (6, 20), (12, 31), (9, 0)]
    cols = {}
    for (i, j) in pix:
        e = np.zeros((og.ny, og.nx), np.float32)
        e[i, j] = 1
        cols[(i, j)] = G.project(to_dev(e)).cpu().numpy()
    for (v, u) in rays:
        e = np.zeros((og.V, og.U), np.float32)
        e[v, u] = 1
        row = G.backproject(to_dev(e)).cpu().numpy()
        for (i, j) in pix:
            assert row[i, j] == cols[(i, j)][v, u]


def test_full_size_projection_sampled():
    """512 x 512, 720 views, 725 bins (the benchmark's workload): sampled rays and pixels."""
    og = O.Geometry(512, V=720, U=725)
    G = gpu_geometry(og)
    x = f32(synth.ellipse_phantom(512, 20, 2001))
    gy = G.project(to_dev(x)).double().cpu().numpy().ravel()
    rng = np.random.default_rng(7)
    rays = rng.choice(og.m, 500, replace=False)
    ref = O.project_rays(og, x, rays)
    assert rel_l2(gy[rays], ref) <= 1e-5
    yy = f32(rng.standard_normal((og.V, og.U)))
    gb = G.backproject(to_dev(yy)).double().cpu().numpy().ravel()
    pix = rng.choice(og.n, 48, replace=False)
    assert rel_l2(gb[pix], O.backproject_pixels(og, yy, pix)) <= 1e-5


def test_bf16_storage_error_is_bounded():
    og = O.Geometry(64, V=90, U=95)
    R = O.CSR(og)
    G = gpu_geometry(og, storage="bf16")
    x = synth.ellipse_phantom(64, 10, 3)
    xb = torch.tensor(x, dtype=torch.bfloat16, device="cuda")
    ref = R.project(xb.float().cpu().numpy())
    err = rel_l2(G.project(xb).double().cpu().numpy(), ref)
    assert err <= 8e-3   # BF16 output rounding (2^-9 relative per entry)
    yb = torch.tensor(ref, dtype=torch.bfloat16, device="cuda")
    err2 = rel_l2(G.backproject(yb).double().cpu().numpy(), R.backproject(yb.float().cpu().numpy()))
    assert err2 <= 8e-3


@pytest.mark.parametrize("ny,nx,mu,rho", [(64, 64, 1e-5, 0.8), (48, 60, 1e-3, 0.6), (243, 243, 1e-5, 0.8),
                                          (7, 5, 1e-4, 0.9), (1, 1, 1e-5, 0.8), (512, 512, 1e-5, 0.8)])
def test_preconditioner_matches_oracle(ny, nx, mu, rho):
    og = O.Geometry(nx, ny=ny, V=4, U=8)
    G = gpu_geometry(og)
    g = f32(np.random.default_rng(ny + nx).standard_normal((ny, nx)))
    z = G.precondition(to_dev(g), mu, rho).double().cpu().numpy()
    D = O.precond_D(ny, nx, mu, rho)
    ref = O.fourier_diag(D, g) if ny * nx <= 300 * 300 else np.real(np.fft.ifft2(D * np.fft.fft2(g)))
    assert rel_l2(z, ref) <= 1e-5


@pytest.mark.parametrize("ny,nx", [(512, 512), (300, 257), (96, 128)])
def test_preconditioner_keeps_digits_of_damped_low_frequencies(ny, nx):
    """A gradient dominated by its lowest frequencies (as R^T b is): M damps them
    by mu = 1e-5, so z = M g is far smaller than g there.  Each transform step in
    FP32 arithmetic leaves errors of about 2^-24 |g| at every frequency, which
    then dominate z (an FP32 FFT lands 4e-6 from the FP64 one on this input);
    the result must stay near the level of z's own FP32 rounding (2.4e-8)."""
    og = O.Geometry(nx, ny=ny, V=4, U=8)
    G = gpu_geometry(og)
    yy, xx = np.mgrid[0:ny, 0:nx]
    smooth = 1e3 * (2.0 + np.cos(2 * np.pi * xx / nx) + np.sin(2 * np.pi * yy / ny)
                    + 0.5 * np.cos(2 * np.pi * (xx / nx + 2 * yy / ny)))
    g = f32(smooth + np.random.default_rng(7).standard_normal((ny, nx)))
    z = G.precondition(to_dev(g), 1e-5, 0.8).double().cpu().numpy()
    ref = np.real(np.fft.ifft2(O.precond_D(ny, nx, 1e-5, 0.8) * np.fft.fft2(g)))
    assert rel_l2(z, ref) <= 1e-7


def test_preconditioner_rejects_indefinite():
    import paper_1807_10151_gb300 as S
    og = O.Geometry(8, V=4, U=8)
    G = gpu_geometry(og)
    with pytest.raises(S.SupcgError) as e:
        G.precondition(to_dev(np.ones((8, 8))), 1e-5, 0.4)
    assert e.value.code == -7


@pytest.mark.parametrize("shape", [(64, 64), (37, 23), (2, 2), (1, 5), (300, 257)])
def test_tv_and_tbar_match_oracle(shape):
    ny, nx = shape
    og = O.Geometry(nx, ny=ny, V=4, U=8)
    G = gpu_geometry(og)
    y = f32(synth.ellipse_phantom(max(nx, ny), 6, ny)[:ny, :nx] + 0.01 * np.random.default_rng(1).standard_normal(shape))
    y[:3, :3] = 0.25   # a flat patch where partial derivatives are undefined
    tv, nn, tb = G.tv_tbar(to_dev(y))
    rtv, rtb = O.tv_tbar(y)
    assert tv == pytest.approx(rtv, rel=1e-6, abs=1e-12)
    assert nn == pytest.approx(np.sum(rtb ** 2), rel=1e-5, abs=1e-12)
    assert rel_l2(tb.double().cpu().numpy(), rtb) <= 1e-5 or np.all(rtb == 0)
    assert np.all(tb.cpu().numpy()[rtb == 0] == 0)


@pytest.mark.parametrize("K,a,gamma,ell", [(1, 0.995, 0.5, 0), (5, 0.7, 0.3, 4), (40, 1 - 1e-5, 1e-2, 0),
                                           (3, 0.5, 20.0, 0)])
def test_superiorize_matches_algorithm1(K, a, gamma, ell):
    og = O.Geometry(48, ny=40, V=4, U=8)
    G = gpu_geometry(og)
    x = f32(synth.ellipse_phantom(48, 8, 5)[:40, :48] + 0.02 * np.random.default_rng(2).standard_normal((40, 48)))
    xd = to_dev(x)
    rc, ell_g, trials = G.superiorize(xd, ell, a, gamma, K)
    rrc, s, ell_o, tr_o = O.stv(x, ell, a, gamma, K)
    assert rc == 0 and rrc == 0
    assert ell_g == ell_o
    assert trials == list(tr_o)
    assert rel_l2(xd.double().cpu().numpy() - x, s) <= 2e-5


def test_superiorize_backtrack_cap():
    og = O.Geometry(16, V=4, U=8)
    G = gpu_geometry(og)
    x = to_dev(np.random.default_rng(3).uniform(size=(16, 16)))
    rc, ell, _ = G.superiorize(x, 0, 1.0, 1e6, 1, max_trials=7)
    assert rc == -5 and ell == 7


@pytest.mark.parametrize("seed", [1001, 1002, 1003, 1004, 1005])
def test_solve_config1_50_iterations_match_oracle(seed):
    """64 x 64, 90 views, 95 bins, 10 ellipses, 1 % noise, K=1, gamma=0.5, a=0.995:
    50 SupPCG iterations (Algorithm 3).  The l sequence must be identical, the
    returned iterate within 1e-4 (rel. L2) of the oracle's, the logged f and TV
    of every iterate within 1e-4, and the reported final f the residual of the
    returned image and near the oracle's (see gpu_cases.F_LAST_REL)."""
    og, R, x_true, b = config1_problem(seed=seed)
    G = gpu_geometry(og)
    b32 = f32(b)
    kw = dict(K=1, a=0.995, gamma=0.5, mu=1e-5, rho=0.8, max_iter=50)
    ref = O.suppcg(R, b32, **kw)
    errs = []
    for graph in (True, False):
        x, rep, lg = G.solve(to_dev(b32), log=True, graph=graph, **kw)
        assert rep["status"] == 0 and rep["iters"] == 50 and rep["k"] == 51
        assert rep["ell"] == ref["ell"]
        lg = lg.cpu().numpy()
        np.testing.assert_array_equal(lg[:, 3].astype(np.int64), ref["ell_log"])
        errs.append(rel_l2(x.double().cpu().numpy(), ref["x_half"]))
        assert rel_l2(lg[:, 2], ref["tv_half"]) <= 1e-4
        assert rel_l2(lg[:, 0], ref["f"]) <= 1e-4
        assert rep["f_last"] == pytest.approx(residual_energy(R, x.double().cpu().numpy(), b32), rel=F_OF_IMAGE_REL)
        assert rep["f_last"] == pytest.approx(ref["f"][-1], rel=F_LAST_REL)
    assert errs[0] == errs[1]   # graph replay and direct launches are bitwise identical
    print(f"\n64^2 seed {seed}: x {errs[0]:.3e}  f_last {rep['f_last']:.9e} vs {ref['f'][-1]:.9e}")
    assert errs[0] <= 1e-4, errs[0]


@pytest.mark.parametrize("perturb,precond,iters", [(False, True, 10), (False, False, 6), (True, False, 50)])
def test_solve_variants_match_oracle(perturb, precond, iters):
    """PCG (no S_TV) over 10 iterations, CG (M = I) over 6 and SupCG (M = I
    with S_TV) over 50.

    Without the TV perturbation, CG with FP32 vectors parts from CG with FP64
    vectors once its residual has collapsed (loss of conjugacy): on this
    problem the GPU's PCG is 1.3e-6 from the oracle at 10 iterations, 3.9e-4 at
    15 and 5.6e-2 at 20, its CG 2.7e-7 at 6 and 1.3e-3 at 10 (the FP32 p, z, q
    and h, not the residual, which is carried in FP64).  So the unperturbed variants' iterate
    parity stops there, and longer runs are checked by properties below.  The
    perturbed SupCG stays within 1e-6 over the 50 iterations."""
    og, R, x_true, b = config1_problem(seed=1002, N=48, V=60, U=70)
    G = gpu_geometry(og)
    b32 = f32(b)
    kw = dict(K=2, a=0.9, gamma=0.05, mu=1e-3, rho=0.6, max_iter=iters)
    D = None if precond else np.ones((og.ny, og.nx))
    ref = O.suppcg(R, b32, perturb=perturb, D=D, **kw)
    x, rep, _ = G.solve(to_dev(b32), perturb=perturb, precondition=precond, **kw)
    assert rep["status"] == 0 and rep["ell"] == ref["ell"]
    assert rel_l2(x.double().cpu().numpy(), ref["x_half"]) <= 1e-4


@pytest.mark.parametrize("precond", [True, False])
def test_unperturbed_long_run_properties(precond):
    """40 iterations of (P)CG: ||R x - b|| never increases, the first iterations
    match the oracle, and the run keeps making progress past them."""
    og, R, x_true, b = config1_problem(seed=1002, N=48, V=60, U=70)
    G = gpu_geometry(og)
    b32 = f32(b)
    kw = dict(mu=1e-3, rho=0.6, max_iter=40)
    D = None if precond else np.ones((og.ny, og.nx))
    ref = O.suppcg(R, b32, perturb=False, D=D, **kw)
    x, rep, lg = G.solve(to_dev(b32), perturb=False, precondition=precond, log=True, **kw)
    f = lg.cpu().numpy()[:, 0]
    assert rep["status"] == 0
    np.testing.assert_allclose(f[:6], ref["f"][:6], rtol=1e-5)
    assert np.all(np.diff(f) <= 1e-6 * f[0])
    assert f[-1] < f[9]


def test_solve_epsilon_mode_terminates_like_oracle():
    og, R, x_true, b = config1_problem(seed=1003, N=32, V=40, U=47)
    G = gpu_geometry(og)
    b32 = f32(b)
    ref0 = O.suppcg(R, b32, max_iter=30, K=1, a=0.995, gamma=0.5)
    eps = float(ref0["f"][9]) * 1.5      # well between two iterates' residuals
    ref = O.suppcg(R, b32, eps=eps, max_iter=200, K=1, a=0.995, gamma=0.5)
    x, rep, _ = G.solve(to_dev(b32), eps=eps, max_iter=200, K=1, a=0.995, gamma=0.5)
    assert rep["iters"] == ref["iters"]
    assert rep["f_last"] <= eps
    assert rel_l2(x.double().cpu().numpy(), ref["x_half"]) <= 1e-4


def test_solve_host_buffers_equal_device_solve():
    og, R, x_true, b = config1_problem(seed=1004, N=40, V=50, U=60)
    G = gpu_geometry(og)
    b32 = np.ascontiguousarray(b, dtype=np.float32)
    xd, rep_d, _ = G.solve(to_dev(b32), max_iter=10)
    xh = np.zeros((og.ny, og.nx), np.float32)
    rep_h = G.solve_host(b32, xh, max_iter=10)
    assert rep_h["status"] == 0 and rep_h["iters"] == 10
    np.testing.assert_array_equal(xh, xd.cpu().numpy())


def test_solve_large_config_properties():
    """512 x 512 / 720 views / 725 bins, Poisson data, 100 iterations: properties that hold at any size
    (TV nonascent of every S_TV call, Theorem 1 bounds) and the reported f re-evaluated by the oracle."""
    from paper_1807_10151_gb300 import synth as Sy
    og = O.Geometry(512, V=720, U=725)
    G = gpu_geometry(og)
    x_true = Sy.ellipse_phantom(512, 20, 2001)
    clean = O.project_rays(og, x_true, np.arange(og.m)).reshape(og.V, og.U)
    b = f32(Sy.poisson_log(clean, 1e5, 2501))
    K, a, gamma = 1, 0.995, 0.5
    x, rep, lg = G.solve(to_dev(b), log=True, K=K, a=a, gamma=gamma, max_iter=100)
    lg = lg.cpu().numpy()
    assert rep["status"] == 0 and rep["iters"] == 100
    for k in range(1, 101):
        assert lg[k - 1, 2] <= lg[k - 1, 1] * (1 + 1e-6)                   # TV(x_{k+1/2}) <= TV(x_k)
        assert math.sqrt(lg[k - 1, 6]) <= K * gamma * a ** ((k - 1) * K) * (1 + 1e-5)
        assert lg[k - 1, 3] >= k * K
    xs = f32(x.cpu().numpy())
    rays = np.random.default_rng(11).choice(og.m, 2000, replace=False)
    r_s = O.project_rays(og, xs, rays) - b.ravel()[rays]
    assert rel_l2(O.project_rays(og, xs, rays), G.project(to_dev(xs)).double().cpu().numpy().ravel()[rays]) <= 1e-5
    # sampled residual energy is consistent with the reported f (unbiased estimate)
    est = np.sum(r_s ** 2) * og.m / rays.size
    assert est == pytest.approx(rep["f_last"], rel=0.15)


@pytest.mark.parametrize("parts", [1, 3, 6, 8])
def test_backprojector_parts_match_oracle(parts):
    """Any view split gives the oracle's R^T y (the sums' order changes, not the terms),
    in the solve's two-sinogram pass too (a short SupPCG run stays on the oracle's path)."""
    og = O.Geometry(130, ny=96, V=77, U=181, off=-0.02)
    R = O.CSR(og)
    G = gpu_geometry(og)
    assert G.set_bwd_parts(parts) == 0
    y = f32(np.random.default_rng(parts).standard_normal((og.V, og.U)))
    assert rel_l2(G.backproject(to_dev(y)).double().cpu().numpy(), R.backproject(y)) <= 1e-5
    og2, R2, x_true, b = config1_problem(seed=1007, N=48, V=60, U=70)
    G2 = gpu_geometry(og2)
    assert G2.set_bwd_parts(parts) == 0
    kw = dict(K=1, a=0.995, gamma=0.5, mu=1e-5, rho=0.8, max_iter=10)
    ref = O.suppcg(R2, f32(b), **kw)
    x, rep, _ = G2.solve(to_dev(f32(b)), **kw)
    assert rep["status"] == 0 and rep["ell"] == ref["ell"]
    assert rel_l2(x.double().cpu().numpy(), ref["x_half"]) <= 1e-4
    assert G2.set_bwd_parts(0) == -1 and G2.set_bwd_parts(9) == -1


def test_batched_workspace_follows_a_changed_tiling():
    """A batched solve after one of its geometries changed its tiling rebuilds the
    batch's scratch (launch shapes, block order) instead of reusing it."""
    import paper_1807_10151_gb300 as S
    geoms, bs = [], []
    for c, (N, V, U) in enumerate(((64, 90, 95), (48, 60, 70))):
        og, R, x_true, b = config1_problem(seed=1300 + c, N=N, V=V, U=U)
        geoms.append(gpu_geometry(og))
        bs.append(to_dev(f32(b)))
    kw = dict(K=1, a=0.995, gamma=0.5, max_iter=6)
    xs = [torch.zeros(g.ny, g.nx, device="cuda") for g in geoms]
    S.solve_batched(geoms, bs, xs, **kw)
    assert geoms[1].set_tiling(32) == 0 and geoms[1].set_bwd_parts(3) == 0
    xs2 = [torch.zeros(g.ny, g.nx, device="cuda") for g in geoms]
    S.solve_batched(geoms, bs, xs2, **kw)
    for g, b, x in zip(geoms, bs, xs2):     # each problem as solved alone with its current tiling
        xr, _, _ = g.solve(b, **kw)
        np.testing.assert_array_equal(x.cpu().numpy(), xr.cpu().numpy())


def test_forward_tiles_give_identical_results_and_autotuner_picks_one(tmp_path):
    from paper_1807_10151_gb300 import autotune
    og = O.Geometry(160, V=120, U=228)
    G = gpu_geometry(og)
    x = to_dev(np.random.default_rng(12).uniform(size=(og.ny, og.nx)))
    outs = []
    for t in (128, 96, 64, 32):
        assert G.set_tiling(t) == 0 and G.get_tiling() == t
        outs.append(G.project(x).cpu().numpy())
    for o in outs[1:]:
        np.testing.assert_array_equal(o, outs[0])
    rec = autotune.tune(G, reps=2, cache=str(tmp_path / "tiling.json"))
    assert rec["tile"] in (128, 96, 64, 32) and G.get_tiling() == rec["tile"]
    assert autotune.tune(G, cache=str(tmp_path / "tiling.json")) == rec      # cached
    b = to_dev(np.random.default_rng(13).standard_normal((og.V, og.U)))
    rb = autotune.tune_bwd(G, b, iters=2, reps=1, cache=str(tmp_path / "tiling.json"))
    assert rb["parts"] in autotune.BWD_CANDIDATES and G.get_bwd_parts() == rb["parts"]
    assert autotune.tune_bwd(G, b, cache=str(tmp_path / "tiling.json")) == rb
