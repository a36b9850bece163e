"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle runs.

This module holds no arithmetic of the reconstruction method: it draws random
ellipse phantoms (sampled at pixel centres), optional smooth background
texture, and measurement noise for a given noiseless sinogram.  The phantoms
stand in for the head phantom of Sec. 4.1 of arXiv 1807.10151, which is not
available; they keep its acquisition shape (see the benchmark configurations).

Seed convention: configuration c, problem b -> seed 1000*c + b.
"""
from __future__ import annotations

import numpy as np


def pixel_centres(nx: int, ny: int, d: float):
    """Centres (x_j, y_i) of an ny x nx image of pixel side d centred on 0,
    row 0 at the top."""
    xj = (np.arange(nx) - 0.5 * (nx - 1)) * d
    yi = (0.5 * (ny - 1) - np.arange(ny)) * d
    return xj, yi


def ellipse_params(n_ellipses: int, seed: int, r_centre=0.35, axes=(0.03, 0.25)):
    """Random ellipses in unit-square coordinates: (cx, cy, ax, ay, angle, density)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n_ellipses):
        rad = r_centre * np.sqrt(rng.uniform())
        phi = rng.uniform(0, 2 * np.pi)
        out.append((rad * np.cos(phi), rad * np.sin(phi), rng.uniform(*axes), rng.uniform(*axes),
                    rng.uniform(0, np.pi), rng.uniform(0, 1)))
    return out


def ellipse_phantom(N: int, n_ellipses: int, seed: int, nx: int | None = None, ny: int | None = None,
                    d: float | None = None, dtype=np.float64) -> np.ndarray:
    """Random-ellipse phantom on the unit square, values in [0, 1].

    Later ellipses overwrite earlier ones; each pixel takes the value at its
    centre.
    """
    nx = N if nx is None else nx
    ny = N if ny is None else ny
    d = 1.0 / max(nx, ny) if d is None else d
    xj, yi = pixel_centres(nx, ny, d)
    X, Y = np.meshgrid(xj, yi)
    img = np.zeros((ny, nx))
    for cx, cy, ax, ay, ang, rho in ellipse_params(n_ellipses, seed):
        ca, sa = np.cos(ang), np.sin(ang)
        u = (X - cx) * ca + (Y - cy) * sa
        v = -(X - cx) * sa + (Y - cy) * ca
        img[(u / ax) ** 2 + (v / ay) ** 2 <= 1.0] = rho
    return img.astype(dtype)


def head_standin(N: int, seed: int, n_inner: int = 8) -> np.ndarray:
    """Stand-in for the head phantom of Sec. 4.1 (not available): a dense
    elliptical annulus ("skull", value 1.0, outer semi-axes 0.44 x 0.48 of the
    unit square, 0.035 thick) around a soft-tissue interior (0.2) holding
    n_inner small low-contrast ellipses (0.2 +- 0.01 .. 0.05), values at pixel
    centres."""
    rng = np.random.default_rng(seed)
    xj, yi = pixel_centres(N, N, 1.0 / N)
    X, Y = np.meshgrid(xj, yi)
    img = np.zeros((N, N))
    outer = (X / 0.44) ** 2 + (Y / 0.48) ** 2 <= 1.0
    inner = (X / 0.405) ** 2 + (Y / 0.445) ** 2 <= 1.0
    img[outer] = 1.0
    img[inner] = 0.2
    for _ in range(n_inner):
        r, t = 0.25 * np.sqrt(rng.uniform()), rng.uniform(0.0, 2.0 * np.pi)
        cx, cy = r * np.cos(t), r * np.sin(t)
        ax, ay, ang = rng.uniform(0.02, 0.08), rng.uniform(0.02, 0.08), rng.uniform(0.0, np.pi)
        val = 0.2 + rng.choice([-1.0, 1.0]) * rng.uniform(0.01, 0.05)
        ca, sa = np.cos(ang), np.sin(ang)
        u = (X - cx) * ca + (Y - cy) * sa
        v = -(X - cx) * sa + (Y - cy) * ca
        img[((u / ax) ** 2 + (v / ay) ** 2 <= 1.0) & inner] = val
    return img


def textured_background(N: int, seed: int, sigma_px: float = 8.0, amplitude: float = 0.05,
                        support_radius: float = 0.45) -> np.ndarray:
    """Seeded white noise blurred by a Gaussian of sigma_px pixels (FFT
    convolution, periodic), scaled to +-amplitude, inside a centred disk."""
    rng = np.random.default_rng(seed)
    w = rng.standard_normal((N, N))
    k = np.fft.fftfreq(N)
    g = np.exp(-2.0 * (np.pi * sigma_px) ** 2 * (k[:, None] ** 2 + k[None, :] ** 2))
    sm = np.real(np.fft.ifft2(np.fft.fft2(w) * g))
    sm *= amplitude / max(np.max(np.abs(sm)), 1e-30)
    xj, yi = pixel_centres(N, N, 1.0 / N)
    X, Y = np.meshgrid(xj, yi)
    return np.where(X ** 2 + Y ** 2 <= support_radius ** 2, sm, 0.0)


def ellipse_sinogram(n_ellipses: int, seed: int, V: int, U: int, ds: float, off: float = 0.0,
                     half_width: float = 0.5) -> np.ndarray:
    """Exact line integrals of the continuous ellipse phantom of ellipse_params
    (later ellipses overwrite earlier ones) restricted to the image square
    [-half_width, half_width]^2, for the parallel-beam rays x cos(theta_v) +
    y sin(theta_v) = s_u, theta_v = v pi / V, s_u = (u - (U-1)/2) ds + off.

    This is the measurement model of the paper's simulations (the data are
    line integrals through a continuous phantom, Sec. 4.1), not the
    reconstruction's pixel matrix: the phantom's ellipses are not pixelated.
    Returns [V][U] (float64)."""
    return ellipses_sinogram(ellipse_params(n_ellipses, seed), V, U, ds, off, half_width)


def ellipses_sinogram(ell, V: int, U: int, ds: float, off: float = 0.0, half_width: float = 0.5) -> np.ndarray:
    """ellipse_sinogram for an explicit list of ellipses (cx, cy, ax, ay, angle, density)."""
    th = np.arange(V) * (np.pi / V)
    s = (np.arange(U) - 0.5 * (U - 1)) * ds + off
    c = np.cos(th)[:, None] * np.ones((1, U))
    sn = np.sin(th)[:, None] * np.ones((1, U))
    q = np.pi / 2
    axis = np.abs(th / q - np.round(th / q)) < 1e-12     # exact cos/sin on the axes
    c[axis] = np.where(np.round(th[axis] / q) % 2 == 0, 1.0, 0.0)[:, None]
    sn[axis] = np.where(np.round(th[axis] / q) % 2 == 0, 0.0, 1.0)[:, None]
    S = np.broadcast_to(s[None, :], (V, U))
    c, sn, S = c.ravel(), sn.ravel(), S.ravel()
    # point of ray r at parameter t: S (c, sn) + t (-sn, c); the square's chord [lo, hi]
    px, py = S * c, S * sn
    lo, hi = np.full(S.shape, -np.inf), np.full(S.shape, np.inf)
    for p0, dirn in ((px, -sn), (py, c)):
        with np.errstate(divide="ignore", invalid="ignore"):
            ta = (-half_width - p0) / dirn
            tb = (half_width - p0) / dirn
        par = dirn == 0.0
        inside = np.abs(p0) <= half_width
        lo = np.where(par, np.where(inside, lo, np.inf), np.maximum(lo, np.minimum(ta, tb)))
        hi = np.where(par, np.where(inside, hi, -np.inf), np.minimum(hi, np.maximum(ta, tb)))
    E = len(ell)
    t1 = np.empty((S.size, E))
    t2 = np.empty((S.size, E))
    for e, (cx, cy, ax, ay, ang, _) in enumerate(ell):
        ca, sa = np.cos(ang), np.sin(ang)
        u0 = (px - cx) * ca + (py - cy) * sa
        v0 = -(px - cx) * sa + (py - cy) * ca
        u1 = -sn * ca + c * sa
        v1 = sn * sa + c * ca
        A = u1 * u1 / ax ** 2 + v1 * v1 / ay ** 2
        B = 2.0 * (u0 * u1 / ax ** 2 + v0 * v1 / ay ** 2)
        Cq = u0 * u0 / ax ** 2 + v0 * v0 / ay ** 2 - 1.0
        disc = B * B - 4.0 * A * Cq
        rt = np.sqrt(np.maximum(disc, 0.0))
        a_ = np.where(disc > 0, (-B - rt) / (2.0 * A), np.inf)
        b_ = np.where(disc > 0, (-B + rt) / (2.0 * A), -np.inf)
        t1[:, e] = np.clip(a_, lo, hi)
        t2[:, e] = np.clip(b_, lo, hi)
    # segments between consecutive breakpoints; each takes the last ellipse containing its midpoint
    bp = np.concatenate([t1, t2, lo[:, None], hi[:, None]], axis=1)
    bp = np.where(np.isfinite(bp), bp, 0.0)
    bp = np.clip(bp, np.where(np.isfinite(lo), lo, 0.0)[:, None], np.where(np.isfinite(hi), hi, 0.0)[:, None])
    bp.sort(axis=1)
    mid = 0.5 * (bp[:, 1:] + bp[:, :-1])
    val = np.zeros_like(mid)
    for e, (_, _, _, _, _, dens) in enumerate(ell):
        val = np.where((mid >= t1[:, e:e + 1]) & (mid <= t2[:, e:e + 1]), dens, val)
    out = np.sum(np.diff(bp, axis=1) * val, axis=1)
    out[~(hi > lo)] = 0.0
    return out.reshape(V, U)


def gaussian_noise(clean: np.ndarray, level: float, seed: int) -> np.ndarray:
    """b = clean + e, e ~ N(0, sigma^2), sigma = level * ||clean|| / sqrt(m)."""
    rng = np.random.default_rng(seed)
    sigma = level * np.linalg.norm(clean) / np.sqrt(clean.size)
    return clean + sigma * rng.standard_normal(clean.shape)


def poisson_log(clean: np.ndarray, I0: float, seed: int) -> np.ndarray:
    """Photon counts ~ Poisson(I0 exp(-clean)); b = -ln(max(count, 1) / I0)."""
    rng = np.random.default_rng(seed)
    counts = rng.poisson(I0 * np.exp(-np.asarray(clean, dtype=np.float64)))
    return -np.log(np.maximum(counts, 1) / I0)


def random_field(shape, seed: int, dtype=np.float64) -> np.ndarray:
    """Standard normal test vectors (adjoint checks, operator parity)."""
    return np.random.default_rng(seed).standard_normal(shape).astype(dtype)
