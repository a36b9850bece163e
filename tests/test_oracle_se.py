"""Oracle pins for the selective error of Eq. (4.1) (C = 1, centred ellipse S)."""
import math

import numpy as np
import pytest

from oracle import oracle as O


def test_constant_offset_gives_the_root_of_the_ellipse_pixel_count():
    """SE(ref + c, ref) = |c| sqrt(|S|), and |S| for a disk of radius R pixels is the
    lattice count pi R^2 up to the Gauss circle bound (a few R)."""
    n = 64
    rng = np.random.default_rng(0)
    ref = rng.uniform(size=(n, n))
    c = 0.125
    se = O.selective_error(ref + c, ref, 0.3, 0.3)
    count = (se / c) ** 2
    R = 0.3 * n
    assert abs(count - math.pi * R * R) <= 4 * R
    assert abs(count - round(count)) < 1e-9            # a whole number of pixels
    assert O.selective_error(ref - c, ref, 0.3, 0.3) == pytest.approx(se, rel=1e-12)


def test_pixels_outside_the_ellipse_do_not_count():
    n = 48
    ref = np.zeros((n, n))
    x = ref.copy()
    x[0, 0] = x[n - 1, n - 1] = x[0, n - 1] = 5.0      # corners: outside any inscribed ellipse
    assert O.selective_error(x, ref, 0.27, 0.38) == 0.0
    x[n // 2, n // 2] = 2.0                            # the centre counts
    assert O.selective_error(x, ref, 0.27, 0.38) == pytest.approx(2.0)


def test_axes_orientation_and_central_symmetry():
    """The horizontal semi-axis runs along the columns j, the vertical one along the rows i;
    S is symmetric under the half turn about the image centre."""
    n = 40
    ref = np.zeros((n, n))
    x = ref.copy()
    i0, j = n // 2, int(0.5 * (n - 1) + 0.35 * n)     # 0.35 n from the centre along a row
    x[i0, j] = 1.0
    assert O.selective_error(x, ref, 0.4, 0.2) == 1.0   # inside the wide horizontal axis
    assert O.selective_error(x, ref, 0.2, 0.4) == 0.0   # outside the narrow one
    rng = np.random.default_rng(1)
    y = rng.standard_normal((n, n))
    assert O.selective_error(y, ref, 0.27, 0.38) == pytest.approx(
        O.selective_error(y[::-1, ::-1], ref, 0.27, 0.38), rel=1e-12)
