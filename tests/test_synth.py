"""The seeded input generator's analytic sinogram (line integrals of the
continuous ellipse phantom, the data model of the paper's simulations),
pinned by closed forms."""
import math

import numpy as np

from paper_1807_10151_gb300 import synth


def chord(r, s):
    return 2.0 * math.sqrt(max(r * r - s * s, 0.0))


def test_centred_disk_gives_chord_lengths():
    V, U, ds = 8, 21, 0.02
    sg = synth.ellipses_sinogram([(0.0, 0.0, 0.3, 0.3, 0.4, 0.7)], V, U, ds)
    s = (np.arange(U) - 0.5 * (U - 1)) * ds
    for v in range(V):
        for u in range(U):
            assert abs(sg[v, u] - 0.7 * chord(0.3, s[u])) <= 1e-12


def test_later_ellipse_overwrites_earlier_one():
    """A disk of 0.2 inside a disk of 0.4 (densities 1 then 3): the inner value
    replaces the outer one, so the integral is 3 c_in + 1 (c_out - c_in)."""
    V, U, ds = 5, 30, 0.025   # no ray tangent to the inner disk
    sg = synth.ellipses_sinogram([(0.0, 0.0, 0.4, 0.4, 0.0, 1.0), (0.0, 0.0, 0.2, 0.2, 0.0, 3.0)], V, U, ds)
    s = (np.arange(U) - 0.5 * (U - 1)) * ds
    for u in range(U):
        ci, co = chord(0.2, s[u]), chord(0.4, s[u])
        assert abs(sg[2, u] - (3.0 * ci + (co - ci))) <= 1e-12


def test_rotated_ellipse_matches_its_support_function():
    """Ellipse of semi-axes (a, b) rotated by phi: at view theta the chord at
    offset s is 2 a b sqrt(w^2 - s^2) / w^2, w^2 = a^2 cos^2(theta - phi) +
    b^2 sin^2(theta - phi)."""
    a, b, phi = 0.3, 0.1, 0.7
    V, U, ds = 12, 41, 0.015
    sg = synth.ellipses_sinogram([(0.0, 0.0, a, b, phi, 1.0)], V, U, ds)
    s = (np.arange(U) - 0.5 * (U - 1)) * ds
    for v in range(V):
        th = v * math.pi / V
        w2 = (a * math.cos(th - phi)) ** 2 + (b * math.sin(th - phi)) ** 2
        for u in range(U):
            ref = 2.0 * a * b * math.sqrt(max(w2 - s[u] ** 2, 0.0)) / w2
            assert abs(sg[v, u] - ref) <= 1e-12


def test_integrals_are_clipped_to_the_image_square():
    """A disk larger than the square: at view 0 (rays x = s) every ray inside
    the square sees the chord clipped to |y| <= 1/2, and rays outside see 0."""
    V, U, ds = 4, 13, 0.1
    sg = synth.ellipses_sinogram([(0.0, 0.0, 0.7, 0.7, 0.0, 1.0)], V, U, ds)
    s = (np.arange(U) - 0.5 * (U - 1)) * ds
    for u in range(U):
        ref = min(chord(0.7, s[u]), 1.0) if abs(s[u]) <= 0.5 else 0.0
        assert abs(sg[0, u] - ref) <= 1e-12


def test_matches_the_pixel_phantom_to_discretisation_error():
    """The pixelated phantom's sums converge to the analytic integrals as the
    grid is refined: the mean ray-sum difference falls with the pixel size."""
    from oracle import oracle as O
    errs = []
    for N in (64, 256):
        og = O.Geometry(N, V=30, U=int(1.42 * N))
        sg = synth.ellipse_sinogram(6, 11, og.V, og.U, og.ds)
        pr = O.CSR(og).project(synth.ellipse_phantom(N, 6, 11))
        errs.append(np.abs(sg - pr).mean())
    assert errs[1] < 0.5 * errs[0]
