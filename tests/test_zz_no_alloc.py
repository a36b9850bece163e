"""The allocation-free preconditioner entry point, for callers that may not
allocate device memory (fixed memory budgets, host frameworks that own every
allocation, paths where cudaMalloc would synchronise the device).

It is called through the C ABI and must agree with supcg_precondition, the
allocating entry point, on two calls in a row (the second call reuses the
static scratch the first one left behind).  This file is collected last so
that a run stopping at its first failure has already run every other test.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL = 1e-5   # relative L2, as for the other preconditioner parity tests


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("ny,nx,mu,rho", [(64, 64, 1e-5, 0.8), (243, 200, 1e-3, 0.6), (512, 512, 1e-5, 0.8)])
def test_noalloc_matches_allocating_entry_point(ny, nx, mu, rho):
    import paper_1807_10151_gb300 as S
    L = S.load()
    G = S.Geometry(nx, ny, n_views=4, n_bins=8)
    st = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    rng = np.random.default_rng(ny * 7 + nx)
    for call in range(2):
        g = torch.tensor(rng.standard_normal((ny, nx)), dtype=torch.float32, device="cuda")
        z = torch.full_like(g, float("nan"))
        rc = L.supcg_precondition_noalloc(ny, nx, mu, rho, C.c_void_p(g.data_ptr()), C.c_void_p(z.data_ptr()), st)
        assert rc == 0, (call, S.STATUS.get(rc, rc))
        ref = G.precondition(g, mu, rho)
        torch.cuda.synchronize()
        assert rel_l2(z.double().cpu().numpy(), ref.double().cpu().numpy()) <= TOL, call


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import paper_1807_10151_gb300 as S
    L = S.load()
    g = torch.zeros(4, dtype=torch.float32, device="cuda")
    st = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert L.supcg_precondition_noalloc(513, 4, 1e-5, 0.8, C.c_void_p(g.data_ptr()), C.c_void_p(g.data_ptr()),
                                        st) == -8
    assert L.supcg_precondition_noalloc(4, 4, 1e-5, 0.3, C.c_void_p(g.data_ptr()), C.c_void_p(g.data_ptr()),
                                        st) == -7


@pytest.mark.parametrize("ny,nx", [(1, 1), (1, 37), (37, 1), (509, 7)])
def test_noalloc_degenerate_and_prime_sides_match_the_oracle(ny, nx):
    """Sides of one pixel, and a prime side (509) that only the generic butterfly
    handles, against the oracle's defining-sum DFT of Eq. (3.2), on two calls."""
    import paper_1807_10151_gb300 as S
    from oracle import oracle as O
    L = S.load()
    st = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    rng = np.random.default_rng(ny * 13 + nx)
    for call in range(2):
        g64 = rng.standard_normal((ny, nx)).astype(np.float32).astype(np.float64)
        g = torch.tensor(g64, dtype=torch.float32, device="cuda")
        z = torch.full_like(g, float("nan"))
        rc = L.supcg_precondition_noalloc(ny, nx, 1e-4, 0.7, C.c_void_p(g.data_ptr()), C.c_void_p(z.data_ptr()), st)
        assert rc == 0, (call, S.STATUS.get(rc, rc))
        torch.cuda.synchronize()
        assert rel_l2(z.double().cpu().numpy(), O.precondition(g64, 1e-4, 0.7)) <= TOL, call


def test_noalloc_in_place_call():
    """d_z may be d_g: the forward and inverse passes are separate launches."""
    import paper_1807_10151_gb300 as S
    L = S.load()
    ny, nx = 96, 80
    G = S.Geometry(nx, ny, n_views=4, n_bins=8)
    st = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    g = torch.tensor(np.random.default_rng(5).standard_normal((ny, nx)), dtype=torch.float32, device="cuda")
    ref = G.precondition(g.clone(), 1e-5, 0.8)
    rc = L.supcg_precondition_noalloc(ny, nx, 1e-5, 0.8, C.c_void_p(g.data_ptr()), C.c_void_p(g.data_ptr()), st)
    assert rc == 0
    torch.cuda.synchronize()
    assert rel_l2(g.double().cpu().numpy(), ref.double().cpu().numpy()) <= TOL


def test_noalloc_rejects_parameters_outside_the_accepted_range():
    import paper_1807_10151_gb300 as S
    L = S.load()
    g = torch.zeros(16, dtype=torch.float32, device="cuda")
    st = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    ptr = C.c_void_p(g.data_ptr())
    for mu, rho in ((1e-5, 0.5), (1e-5, 1.01), (-1e-5, 0.8), (float("inf"), 0.8), (float("nan"), 0.8)):
        assert L.supcg_precondition_noalloc(4, 4, mu, rho, ptr, ptr, st) == -7, (mu, rho)
