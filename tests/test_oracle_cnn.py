"""Pins of the oracle's 3x3 convolution layers used to check the learned
perturbation network (the paper has no learned part): shifts, the adjoint
identity of the backward pass, finite-difference gradients."""
import numpy as np
import pytest

from oracle import oracle as O


def test_delta_and_shift_kernels():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((1, 6, 7))
    W = np.zeros((1, 1, 3, 3))
    W[0, 0, 1, 1] = 1.0
    np.testing.assert_array_equal(O.conv3x3(x, W), x)
    W = np.zeros((1, 1, 3, 3))
    W[0, 0, 1, 2] = 1.0          # y[i][j] = x[i][j+1], zero past the right edge
    y = O.conv3x3(x, W)
    np.testing.assert_array_equal(y[0, :, :-1], x[0, :, 1:])
    assert np.all(y[0, :, -1] == 0)
    y = O.conv3x3(x, W, bias=np.array([2.0]), relu=True)
    assert np.all(y >= 0) and y[0, 0, -1] == 2.0


def test_backward_is_the_adjoint_and_matches_finite_differences():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((3, 5, 4))
    W = rng.standard_normal((2, 3, 3, 3))
    g = rng.standard_normal((2, 5, 4))
    dx, dW, db = O.conv3x3_backward(x, W, g)
    assert np.sum(O.conv3x3(x, W) * g) == pytest.approx(np.sum(x * dx), rel=1e-12)
    np.testing.assert_allclose(db, g.sum(axis=(1, 2)), rtol=1e-13)
    eps = 1e-6
    for idx in [(0, 0, 0, 0), (1, 2, 1, 1), (0, 1, 2, 0), (1, 0, 0, 2)]:
        Wp, Wm = W.copy(), W.copy()
        Wp[idx] += eps
        Wm[idx] -= eps
        fd = (np.sum(O.conv3x3(x, Wp) * g) - np.sum(O.conv3x3(x, Wm) * g)) / (2 * eps)
        assert dW[idx] == pytest.approx(fd, rel=1e-7, abs=1e-9)
