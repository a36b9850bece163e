"""Pins of the oracle's TV, nonascending vector and S_TV (Sec. 3.1,
Algorithm 1) against closed forms, finite differences and a hand-derived
example (tests/golden/stv_2x2.json)."""
import json
import math
import os

import numpy as np
import pytest

from oracle import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_tv_closed_forms():
    l, c = 7, 9
    assert O.tv(np.full((l, c), 3.25)) == 0.0
    al, be = 0.3, -1.7
    I, J = np.meshgrid(np.arange(l), np.arange(c), indexing="ij")
    assert O.tv(al * I + be * J) == pytest.approx((l - 1) * (c - 1) * math.hypot(al, be), rel=1e-13)
    h = 2.5
    step = np.where(J >= 4, h, 0.0)
    assert O.tv(step) == pytest.approx((l - 1) * h, rel=1e-14)
    chk = (-1.0) ** (I + J)
    assert O.tv(chk) == pytest.approx((l - 1) * (c - 1) * 2 * math.sqrt(2), rel=1e-13)
    # the last row and column only enter as neighbours: changing pixel (l-1, c-1) does nothing
    y = np.random.default_rng(1).standard_normal((l, c))
    y2 = y.copy()
    y2[-1, -1] += 10.0
    assert O.tv(y) == O.tv(y2)


def test_tbar_matches_central_differences():
    y = np.random.default_rng(2).standard_normal((6, 5))
    tv, tbar = O.tv_tbar(y)
    assert tv == pytest.approx(O.tv(y), rel=1e-15)
    eps = 1e-6
    for p in range(y.size):
        e = np.zeros(y.size)
        e[p] = eps
        e = e.reshape(y.shape)
        fd = (O.tv(y + e) - O.tv(y - e)) / (2 * eps)
        assert -tbar.ravel()[p] == pytest.approx(fd, abs=1e-7)


def test_tbar_zero_where_partial_undefined():
    y = np.zeros((5, 5))
    y[0, 0] = 1.0  # term (0,0) nonzero; every other term touching a zero-only region has root 0
    tv, tbar = O.tv_tbar(y)
    assert tv == pytest.approx(math.sqrt(2))
    # y[0,1] is in term (0,0) (root sqrt(2)) and term (0,1) (root 0): undefined -> 0
    assert tbar[0, 1] == 0.0 and tbar[1, 0] == 0.0
    # y[0,0] only in term (0,0): defined, -(a+b)/T = -(1+1)/sqrt(2)
    assert tbar[0, 0] == pytest.approx(-math.sqrt(2))
    assert np.all(O.tv_tbar(np.ones((4, 4)))[1] == 0.0)
    assert np.all(O.tv_direction(np.ones((4, 4))) == 0.0)


def test_direction_is_unit_and_nonascending():
    y = np.random.default_rng(4).standard_normal((8, 8))
    t = O.tv_direction(y)
    assert np.linalg.norm(t) == pytest.approx(1.0, rel=1e-14)
    tv0 = O.tv(y)
    for delta in (1e-2, 1e-3, 1e-4):
        assert O.tv(y + delta * t) <= tv0


def test_stv_golden_2x2():
    g = json.load(open(os.path.join(GOLDEN, "stv_2x2.json")))
    y = np.array(g["image"])
    tv, tbar = O.tv_tbar(y)
    assert tv == pytest.approx(g["tv"], rel=1e-15)
    np.testing.assert_allclose(tbar, np.array(g["tbar"]), atol=1e-15)
    for case in g["cases"]:
        rc, s, ell, trials = O.stv(y, case["ell_in"], case["a"], case["gamma"], case["K"])
        assert rc == 0
        assert ell == case["ell_out"]
        assert list(trials) == case["trials"]
        np.testing.assert_allclose(s, np.array(case["s"]), atol=1e-15)


def test_stv_invariants_theorem1():
    """Algorithm 1: l grows by at least K, every accepted step is nonascending,
    ||s|| <= K gamma a^l_in (the per-call bound behind Theorem 1)."""
    x = np.random.default_rng(6).uniform(size=(10, 12))
    a, gamma, K = 0.7, 0.3, 5
    ell = 4
    rc, s, ell2, trials = O.stv(x, ell, a, gamma, K)
    assert rc == 0
    assert ell2 - ell == trials.sum() >= K
    assert O.tv(x + s) <= O.tv(x)
    assert np.linalg.norm(s) <= K * gamma * a ** ell * (1 + 1e-12)


def test_stv_backtrack_cap_reports_error():
    x = np.random.default_rng(6).uniform(size=(6, 6))
    # a = 1 keeps the step at gamma; a huge gamma never decreases TV -> cap
    rc, s, ell2, trials = O.stv(x, 0, 1.0, 1e6, 1, max_trials=7)
    assert rc == O.ERR_BACKTRACK and ell2 == 7


def test_directional_derivative():
    rng = np.random.default_rng(8)
    y = rng.standard_normal((7, 6))
    t = rng.standard_normal((7, 6))
    dd = O.tv_dirderiv(y, t)
    eps = 1e-7
    assert dd == pytest.approx((O.tv(y + eps * t) - O.tv(y)) / eps, abs=1e-5)
    # at a constant image every root is 0: derivative = TV(t)
    assert O.tv_dirderiv(np.ones((7, 6)), t) == pytest.approx(O.tv(t), rel=1e-14)
    # the normalised -grad direction has negative derivative
    assert O.tv_dirderiv(y, O.tv_direction(y)) < 0
