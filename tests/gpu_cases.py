"""Seeded problem builders shared by the GPU parity tests.  Inputs come from
paper_1807_10151_gb300.synth; every expected value comes from the oracle."""
import numpy as np

from oracle import oracle as O
from paper_1807_10151_gb300 import synth


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def residual_energy(R, x, b):
    """f(x) = ||R x - b||^2 (Eq. (2.1)) by the oracle's explicit R, in FP64."""
    r = R.project(np.asarray(x, dtype=np.float64)).ravel() - np.asarray(b, dtype=np.float64).ravel()
    return float(r @ r)


# The final f is the residual energy near the noise floor: a change dx of the iterate
# moves it by 2 g^T dx + ||R dx||^2, i.e. by up to kappa_f = 2 ||g|| ||x|| / f (about 60 on
# the 64^2 and 512^2 workloads, measured with the oracle) times the iterate's relative
# change.  So the reported f is checked twice: tightly against the oracle's f of the very
# image returned (it must be that image's residual), and against the oracle's own final
# f at F_LAST_REL, which bounds the iterate's error along the gradient at ~1e-5.
F_LAST_REL = 5e-4
F_OF_IMAGE_REL = 1e-5


def config1_problem(seed=1001, N=64, V=90, U=95, n_ell=10, level=0.01):
    """64x64 unit square, 90 views, 95 bins, 10 ellipses, 1 % Gaussian noise."""
    g = O.Geometry(N, V=V, U=U)
    R = O.CSR(g)
    x = synth.ellipse_phantom(N, n_ell, seed)
    b = synth.gaussian_noise(R.project(x), level, seed + 500)
    return g, R, x, b


def gpu_geometry(og, storage="f32"):
    import paper_1807_10151_gb300 as S
    return S.Geometry(og.nx, og.ny, n_views=og.V, n_bins=og.U, pixel_size=og.d,
                      angles=list(og.theta), bin_spacing=og.ds, offset=og.off, storage=storage)


def to_dev(a, dtype=None):
    import torch
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype or torch.float32, device="cuda")
