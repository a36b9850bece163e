"""The boundary's failure statuses, forced without faulting or hanging a GPU.

SUPCG_ERR_TIMEOUT: the grid barriers of the cooperative S_TV launch (Algorithm
1's repeat loop runs on the device, unbounded in the paper) and of ART's ray
classes (Sec. 3.4) are bounded waits.  The test hook makes every barrier wait
for one block more than its launch has, so no barrier is released and each
wait runs out after a short poll limit; the blocks only poll a flag, nothing
is in flight.  The call must return SUPCG_ERR_TIMEOUT and the next normal
call on the same geometry must succeed and match the oracle.

SUPCG_ERR_BREAKDOWN: Algorithm 2 divides by p^T h (steps 3 and 6).  b = 0
gives g = 0, p = 0 and p^T h = 0; a NaN in b makes every scalar NaN.  The
oracle reports the same status on the same input.
"""
import numpy as np
import pytest

from oracle import oracle as O

from gpu_cases import config1_problem, gpu_geometry, rel_l2, to_dev

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

KW = dict(K=1, a=0.995, gamma=0.5, mu=1e-5, rho=0.8)


def f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


class short_barriers:
    """Every cooperative barrier waits for one block too many, for at most 2^14 polls."""

    def __enter__(self):
        import paper_1807_10151_gb300 as S
        assert S.supcg_set_wait_limit(1 << 14) == 0
        assert S.supcg_set_barrier_shortfall(1) == 0

    def __exit__(self, *exc):
        import paper_1807_10151_gb300 as S
        S.supcg_set_barrier_shortfall(0)
        S.supcg_set_wait_limit(S.DEFAULT_WAIT_LIMIT)


@pytest.mark.parametrize("graph", [True, False])
def test_solve_reports_a_barrier_timeout_and_recovers(graph):
    og, R, x_true, b = config1_problem(seed=1003, N=32, V=40, U=47)
    G = gpu_geometry(og)
    b32 = f32(b)
    with short_barriers():
        x, rep, _ = G.solve(to_dev(b32), max_iter=5, graph=graph, **KW)
    assert rep["rc"] == -6 and rep["status"] == -6
    assert rep["iters"] < 5
    # the same geometry (workspace, barrier words, cached graph) solves normally afterwards
    ref = O.suppcg(R, b32, max_iter=8, **KW)
    x, rep, _ = G.solve(to_dev(b32), max_iter=8, graph=graph, **KW)
    assert rep["rc"] == 0 and rep["status"] == 0 and rep["iters"] == 8
    assert rep["ell"] == ref["ell"]
    assert rel_l2(x.double().cpu().numpy(), ref["x_half"]) <= 1e-4


def test_superiorize_and_art_report_a_barrier_timeout_and_recover():
    import paper_1807_10151_gb300 as S
    og, R, x_true, b = config1_problem(seed=1004, N=32, V=40, U=47)
    G = gpu_geometry(og)
    x0 = f32(x_true + 0.02 * np.random.default_rng(4).standard_normal(x_true.shape))
    with short_barriers():
        with pytest.raises(S.SupcgError) as e:
            G.superiorize(to_dev(x0), 0, 0.995, 0.5, 3)
        assert e.value.code == -6
        with pytest.raises(S.SupcgError) as e:
            G.art(to_dev(f32(b)), cycles=1)
        assert e.value.code == -6
    xd = to_dev(x0)
    rc, ell, trials = G.superiorize(xd, 0, 0.995, 0.5, 3)
    rrc, s, ell_o, tr_o = O.stv(x0, 0, 0.995, 0.5, 3)
    assert rc == 0 and ell == ell_o and trials == list(tr_o)
    assert rel_l2(xd.double().cpu().numpy() - x0, s) <= 2e-5
    x, rep = G.art(to_dev(f32(b)), cycles=1)
    assert rep["status"] == 0


def test_zero_data_breaks_down_like_the_oracle():
    og, R, x_true, b = config1_problem(seed=1005, N=32, V=40, U=47)
    G = gpu_geometry(og)
    zero = np.zeros_like(b)
    ref = O.suppcg(R, zero, max_iter=5, **KW)
    assert ref["status"] == O.ERR_BREAKDOWN
    x, rep, _ = G.solve(to_dev(zero), max_iter=5, **KW)
    assert rep["rc"] == -4 and rep["status"] == -4 and rep["iters"] == 0
    assert np.all(x.cpu().numpy() == 0)   # x_0 = 0 comes back unchanged
    # the geometry keeps working
    x, rep, _ = G.solve(to_dev(f32(b)), max_iter=3, **KW)
    assert rep["status"] == 0 and rep["iters"] == 3


def test_nan_in_data_breaks_down_like_the_oracle():
    og, R, x_true, b = config1_problem(seed=1006, N=32, V=40, U=47)
    G = gpu_geometry(og)
    bad = f32(b)
    bad[7, 11] = np.nan
    ref = O.suppcg(R, bad, max_iter=5, **KW)
    assert ref["status"] == O.ERR_BREAKDOWN
    x, rep, _ = G.solve(to_dev(bad), max_iter=5, **KW)
    assert rep["rc"] == -4 and rep["status"] == -4 and rep["iters"] == 0
    x, rep, _ = G.solve(to_dev(f32(b)), max_iter=3, **KW)
    assert rep["status"] == 0 and rep["iters"] == 3
