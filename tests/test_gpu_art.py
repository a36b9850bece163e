"""GPU (C-ABI) ART and SupART (Sec. 3.4) against the FP64 oracle.

The GPU runs each class of rays (one view, u = c mod S) in parallel; the
oracle visits the same rays one after another in the order of art_order.
Rays of one class touch disjoint pixels, so the two orders give the same
iterates up to rounding: the GPU sums <R_i, x> in FP64 and keeps x in FP32,
about 2 V updates of each pixel per cycle."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1807_10151_gb300 import synth

from gpu_cases import config1_problem, gpu_geometry, rel_l2, to_dev

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


@pytest.mark.parametrize("lam,cycles,mu", [(1e-2, 2, None), (0.5, 2, 0.3), (1.5, 1, None)])
def test_art_matches_oracle_config1(lam, cycles, mu):
    """64 x 64, 90 views, 95 bins (r = 5 as in Table 1)."""
    og, R, x_true, b = config1_problem(seed=1001)
    G = gpu_geometry(og)
    b32 = f32(b)
    ref = O.art(R, b32, r=5.0, lam=lam, cycles=cycles, mu=mu)
    x, rep = G.art(to_dev(b32), r=5.0, lam=lam, cycles=cycles, mu=mu)
    assert rep["status"] == 0 and rep["cycles"] == cycles
    assert rep["mu"] == pytest.approx(ref["mu"], rel=1e-12, abs=1e-15)
    assert rel_l2(x.double().cpu().numpy(), ref["x"]) <= 2e-5


@pytest.mark.parametrize("nx,ny,V,U,off,dsf", [(37, 23, 41, 47, 0.013, 1.0), (48, 48, 30, 110, 0.0, 0.6),
                                               (40, 40, 25, 40, 0.0, 1.4), (40, 40, 25, 29, 0.0, 2.0),
                                               (7, 7, 5, 11, 0.0, 1.0)])
def test_art_matches_oracle_on_other_geometries(nx, ny, V, U, off, dsf):
    """Ragged sizes, a shifted detector, bins finer and coarser than pixels (so
    other class spacings S: 2, 3 and 1).  The coarse spacings keep axis-view rays
    off pixel edges (an even bin count at 1.4 d), where the oracle's FP64 spacing
    and the GPU's tie rule would disagree about edge rays (a property of the tie
    rule, seen in the projectors as well)."""
    d = 1.0 / max(nx, ny)
    og = O.Geometry(nx, ny=ny, V=V, U=U, off=off, ds=d * dsf)
    R = O.CSR(og)
    x = synth.ellipse_phantom(max(nx, ny), 5, nx + V)[:ny, :nx]
    b = f32(R.project(x) + 0.01 * np.random.default_rng(nx).standard_normal((V, U)))
    ref = O.art(R, b, r=5.0, lam=0.3, cycles=2)
    G = gpu_geometry(og)
    xg, rep = G.art(to_dev(b), r=5.0, lam=0.3, cycles=2)
    assert rep["status"] == 0
    assert rel_l2(xg.double().cpu().numpy(), ref["x"]) <= 2e-5


def test_supart_matches_oracle():
    """SupART with Table 1's parameters (K = 10, a = 1 - 1e-5, gamma = 1e-2, r = 5,
    lambda = 5e-2): identical l, iterates within 1e-4."""
    og, R, x_true, b = config1_problem(seed=1002)
    G = gpu_geometry(og)
    b32 = f32(b)
    kw = dict(r=5.0, lam=5e-2, cycles=3, K=10, a=1 - 1e-5, gamma=1e-2)
    ref = O.art(R, b32, **kw)
    x, rep = G.art(to_dev(b32), **kw)
    assert rep["status"] == 0 and ref["status"] == 0
    assert rep["ell"] == ref["ell"]
    assert rel_l2(x.double().cpu().numpy(), ref["x"]) <= 1e-4


def test_art_full_size_cycle():
    """512 x 512, 720 views, 725 bins (the benchmark's geometry): one cycle with
    Table 1's ART parameters against the oracle's cycle."""
    og = O.Geometry(512, V=720, U=725)
    R = O.CSR(og)
    x = synth.ellipse_phantom(512, 20, 2001)
    b = f32(R.project(x))
    ref = O.art(R, b, r=5.0, lam=1e-2, cycles=1)
    G = gpu_geometry(og)
    xg, rep = G.art(to_dev(b), r=5.0, lam=1e-2, cycles=1)
    assert rep["status"] == 0
    assert rel_l2(xg.double().cpu().numpy(), ref["x"]) <= 1e-4


def test_art_rejects_bad_parameters():
    import paper_1807_10151_gb300 as S
    og = O.Geometry(16, V=8, U=23)
    G = gpu_geometry(og)
    b = to_dev(np.zeros((og.V, og.U)))
    for kw in (dict(lam=2.0), dict(lam=0.0), dict(r=0.0), dict(r=math.inf), dict(cycles=-1), dict(K=2, a=1.5)):
        with pytest.raises(S.SupcgError) as e:
            G.art(b, **kw)
        assert e.value.code == -1
