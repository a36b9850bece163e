"""Parameter sweep (supcg_solve_sweep, Sec. 4.2): solves of one problem with
different S_TV / preconditioner parameters in one batched schedule, and the
selective error of Eq. (4.1) of every iterate against the phantom."""
import numpy as np
import pytest

from oracle import oracle as O
import paper_1807_10151_gb300 as S

from gpu_cases import config1_problem, gpu_geometry, rel_l2, to_dev

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

AX = S.SE_AXES


def f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


GRID = [dict(K=1, a=0.995, gamma=0.5, mu=1e-5, rho=0.8),
        dict(K=3, a=0.9, gamma=0.05, mu=1e-3, rho=0.6),
        dict(K=2, a=0.99, gamma=0.2, mu=1e-4, rho=0.8)]


def test_sweep_equals_the_individual_solves_and_the_oracle():
    og, R, x_true, b = config1_problem(seed=1301, N=48, V=60, U=70)
    G = gpu_geometry(og)
    b32 = f32(b)
    bd = to_dev(b32)
    its = 10
    params = [dict(q, max_iter=its) for q in GRID]
    xs, reps, se = S.solve_sweep(G, bd, params, ref=to_dev(x_true))
    se = se.cpu().numpy()
    for c, q in enumerate(params):
        assert reps[c]["status"] == 0 and reps[c]["iters"] == its
        x1, r1, _ = G.solve(bd, **q)
        np.testing.assert_array_equal(xs[c].cpu().numpy(), x1.cpu().numpy())   # same kernels, same bits
        assert reps[c]["ell"] == r1["ell"]
        ref = O.suppcg(R, b32, **q)
        assert reps[c]["ell"] == ref["ell"]
        assert rel_l2(xs[c].double().cpu().numpy(), ref["x_half"]) <= 1e-4
        # SE of x_{k+1/2} of body k = SE of the image a k-iteration solve returns
        for k in (1, its // 2, its):
            xk, _, _ = G.solve(bd, **dict(q, max_iter=k))
            want = O.selective_error(xk.double().cpu().numpy(), x_true.astype(np.float32), *AX)
            assert se[c, k - 1] == pytest.approx(want, rel=1e-9)


def test_sweep_rejects_differing_shared_settings():
    og, R, x_true, b = config1_problem(seed=1302, N=32, V=30, U=47)
    G = gpu_geometry(og)
    bd = to_dev(f32(b))
    with pytest.raises(S.SupcgError) as e:
        S.solve_sweep(G, bd, [dict(max_iter=4), dict(max_iter=5)])
    assert e.value.code == -1
    with pytest.raises(S.SupcgError) as e:
        S.solve_sweep(G, bd, [dict(max_iter=4), dict(max_iter=4, precondition=False)])
    assert e.value.code == -1
