"""Pins of the oracle's projector R and its transpose (Sec. 2 data model,
Sec. 4.1 acquisition shape), against closed forms that do not use the
oracle's own clipping code."""
import math

import numpy as np
import pytest

from oracle import oracle as O


def chord_of_rect(c, s, sv, W, H):
    """Length of the line x c + y s = sv inside [-W/2, W/2] x [-H/2, H/2],
    from the points where it crosses the four edge lines (not slab clipping).
    A line running along the rectangle's edge counts half (edge rule)."""
    if s == 0.0:
        x = sv / c
        return H if abs(x) < W / 2 else (H / 2 if abs(x) == W / 2 else 0.0)
    if c == 0.0:
        y = sv / s
        return W if abs(y) < H / 2 else (W / 2 if abs(y) == H / 2 else 0.0)
    pts = []
    for x in (-W / 2, W / 2):
        y = (sv - x * c) / s
        if -H / 2 - 1e-15 <= y <= H / 2 + 1e-15:
            pts.append((x, y))
    for y in (-H / 2, H / 2):
        x = (sv - y * s) / c
        if -W / 2 - 1e-15 <= x <= W / 2 + 1e-15:
            pts.append((x, y))
    best = 0.0
    for p in pts:
        for q in pts:
            best = max(best, math.hypot(p[0] - q[0], p[1] - q[1]))
    return best


def exact_cs(th):
    q = th / (math.pi / 2)
    if abs(q - round(q)) < 1e-12:
        k = int(round(q)) % 4
        return [(1.0, 0.0), (0.0, 1.0), (-1.0, 0.0), (0.0, -1.0)][k]
    return math.cos(th), math.sin(th)


@pytest.mark.parametrize("N,V,U", [(16, 12, 25), (15, 12, 21), (8, 7, 13), (6, 4, 9)])
def test_all_ones_gives_chord_lengths(N, V, U):
    g = O.Geometry(N, V=V, U=U)
    R = O.CSR(g)
    y = R.project(np.ones((N, N)))
    for v in range(V):
        c, s = exact_cs(g.theta[v])
        for u in range(U):
            sv = (u - (U - 1) / 2) * g.ds
            assert y[v, u] == pytest.approx(chord_of_rect(c, s, sv, 1.0, 1.0), abs=1e-13)


def trapezoid(delta, c, s, d):
    """Intersection length of a line with a d x d square at signed distance
    delta from its centre (closed form; half value on an edge)."""
    a, b = max(abs(c), abs(s)), min(abs(c), abs(s))
    if b == 0.0:
        if abs(delta) < d / 2:
            return d
        return d / 2 if abs(delta) == d / 2 else 0.0
    return min(d / a, max(0.0, (d * (a + b) / 2 - abs(delta)) / (a * b)))


@pytest.mark.parametrize("pix", [(0, 0), (3, 5), (7, 7), (5, 2)])
def test_single_pixel_trapezoid(pix):
    N, V, U = 8, 16, 13
    g = O.Geometry(N, V=V, U=U, off=0.013)
    img = np.zeros((N, N))
    img[pix] = 1.0
    y = O.CSR(g).project(img)
    i, j = pix
    xj, yi = (j - (N - 1) / 2) * g.d, ((N - 1) / 2 - i) * g.d
    for v in range(V):
        c, s = exact_cs(g.theta[v])
        for u in range(U):
            sv = (u - (U - 1) / 2) * g.ds + g.off
            assert y[v, u] == pytest.approx(trapezoid(sv - (xj * c + yi * s), c, s, g.d), abs=1e-14)


def disk_image(N, r, sub=8):
    """Area fraction of the disk of radius r in each pixel (sub x sub samples)."""
    d = 1.0 / N
    off = (np.arange(sub) + 0.5) / sub * d
    xj = -0.5 + np.arange(N) * d
    X = (xj[None, :, None, None] + off[None, None, None, :])
    Y = (0.5 - np.arange(N) * d)[:, None, None, None] - off[None, None, :, None]
    inside = (X ** 2 + Y ** 2) <= r * r
    return inside.mean(axis=(2, 3))


def test_disk_projection_converges_to_chords():
    r = 0.3
    errs = []
    for N in (32, 64, 128):
        g = O.Geometry(N, V=8, U=N + 1)
        y = O.CSR(g).project(disk_image(N, r))
        su = (np.arange(g.U) - (g.U - 1) / 2) * g.ds
        keep = np.abs(su) <= 0.8 * r   # away from tangency, where the chord has infinite slope
        exact = 2 * np.sqrt(r * r - su[keep] ** 2)
        errs.append(np.sqrt(np.mean((y[:, keep] - exact[None, :]) ** 2)))
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 2e-3


def test_rotation_by_quarter_turn_permutes_views():
    N, V, U = 12, 8, 17
    g = O.Geometry(N, V=V, U=U)
    R = O.CSR(g)
    x = np.random.default_rng(3).uniform(size=(N, N))
    y = R.project(x)
    yr = R.project(np.rot90(x))  # counter-clockwise quarter turn
    for v in range(V):
        if v < V // 2:
            np.testing.assert_allclose(yr[v], y[v + V // 2][::-1], rtol=0, atol=1e-12)
        else:
            np.testing.assert_allclose(yr[v], y[v - V // 2], rtol=0, atol=1e-12)


def test_adjoint_identity_fp64():
    g = O.Geometry(20, ny=14, V=17, U=31, off=0.021)
    R = O.CSR(g)
    rng = np.random.default_rng(5)
    x = rng.standard_normal((g.ny, g.nx))
    y = rng.standard_normal((g.V, g.U))
    lhs = np.sum(R.project(x) * y)
    rhs = np.sum(x * R.backproject(y))
    assert abs(lhs - rhs) <= 1e-13 * (abs(lhs) + np.linalg.norm(x) * np.linalg.norm(y))


def test_three_routes_agree():
    """CSR rows, ray-by-ray walk and pixel-by-pixel clipping of every ray."""
    g = O.Geometry(10, V=9, U=15, off=-0.02)
    R = O.CSR(g)
    rng = np.random.default_rng(7)
    x = rng.standard_normal((g.ny, g.nx))
    y = rng.standard_normal((g.V, g.U))
    rays = np.arange(g.m)
    np.testing.assert_allclose(O.project_rays(g, x, rays), R.project(x).ravel(), atol=1e-13)
    pix = np.arange(g.n)
    np.testing.assert_allclose(O.backproject_pixels(g, y, pix), R.backproject(y).ravel(), atol=1e-12)


def test_row_sums_and_nnz_scale():
    """Every ray through the image interior has a row sum equal to its chord,
    and nnz grows like (4/pi) n V for ds = d."""
    g = O.Geometry(64, V=90, U=95)
    R = O.CSR(g)
    assert abs(R.nnz / ((4 / math.pi) * g.n * g.V) - 1) < 0.05
