"""Python face of the FP64 CPU oracle (``supcg_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by the test suite, by the smoke check and
by the benchmark's CPU-baseline leg, never by the product package.  The oracle
shares no code with the CUDA path; only the seeded input generators are common.

Every function states the passage of arXiv 1807.10151 it follows; the C file
holds the arithmetic.  numpy is used only to hold arrays.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "supcg_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK, ERR_ARG, ERR_NOMEM, ERR_BREAKDOWN, ERR_BACKTRACK = 0, -1, -3, -4, -5


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP when available)."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".{os.getpid()}.tmp"
    base = ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", _SRC, "-o", tmp, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _LIB)
    return _LIB


def _L():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            dp, lp, ip = C.POINTER(C.c_double), C.POINTER(C.c_long), C.POINTER(C.c_int)
            geo = [C.c_int, C.c_int, C.c_double, C.c_int, dp, C.c_int, C.c_double, C.c_double]
            lib.orc_csr_rowptr.argtypes = geo + [lp]
            lib.orc_csr_rowptr.restype = C.c_long
            lib.orc_csr_fill.argtypes = geo + [lp, ip, dp]
            lib.orc_csr_transpose.argtypes = [C.c_long, C.c_long, lp, ip, dp, lp, ip, dp]
            lib.orc_spmv.argtypes = [C.c_long, lp, ip, dp, dp, dp]
            lib.orc_project_rays.argtypes = geo + [dp, C.c_long, lp, dp]
            lib.orc_backproject_pixels.argtypes = geo + [dp, C.c_long, lp, dp]
            lib.orc_tv.argtypes = [C.c_int, C.c_int, dp]
            lib.orc_tv.restype = C.c_double
            lib.orc_tv_tbar.argtypes = [C.c_int, C.c_int, dp, dp]
            lib.orc_tv_tbar.restype = C.c_double
            lib.orc_tv_dirderiv.argtypes = [C.c_int, C.c_int, dp, dp]
            lib.orc_tv_dirderiv.restype = C.c_double
            lib.orc_stv.argtypes = [C.c_int, C.c_int, dp, C.c_long, C.c_double, C.c_double,
                                    C.c_int, C.c_long, dp, lp, lp]
            lib.orc_precond_D.argtypes = [C.c_int, C.c_int, C.c_double, C.c_double, dp]
            lib.orc_fourier_diag.argtypes = [C.c_int, C.c_int, dp, dp, dp]
            lib.orc_suppcg.argtypes = ([C.c_long, C.c_long, lp, ip, dp, lp, ip, dp,
                                        C.c_int, C.c_int, dp, dp, dp,
                                        C.c_double, C.c_double, C.c_int, C.c_double, C.c_int,
                                        C.c_long, C.c_int,
                                        dp, dp, ip, ip, lp] + [dp, dp, dp, lp, dp, dp, dp, dp]
                                       + [C.c_double, C.c_double])
            lib.orc_art_rays.argtypes = [lp, ip, dp, lp, C.c_long, dp, C.c_double, C.c_double, dp, dp]
            lib.orc_num_threads.restype = C.c_int
            lib.orc_conv3x3.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, dp, dp, dp, C.c_int, dp]
            lib.orc_conv3x3_backward.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, dp, dp, dp, dp, dp, dp]
            _lib = lib
    return _lib


def _d(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _l(a):
    return a.ctypes.data_as(C.POINTER(C.c_long))


def _i(a):
    return a.ctypes.data_as(C.POINTER(C.c_int))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def num_threads() -> int:
    return int(_L().orc_num_threads())


class Geometry:
    """2-D parallel-beam geometry (Sec. 2 data model, Sec. 4.1 acquisition shape).

    Image ny x nx of pixels of side d centred on the origin; view angles theta
    (default: V equally spaced angles v*pi/V in [0, pi)); U bins of spacing ds
    (default d: ray spacing equal to pixel size, as in Sec. 4.1) centred on
    the detector centre shifted by ``off``.
    """

    def __init__(self, nx, ny=None, d=None, V=90, U=None, ds=None, off=0.0, theta=None):
        self.nx = int(nx)
        self.ny = int(ny if ny is not None else nx)
        self.d = float(d if d is not None else 1.0 / max(self.nx, self.ny))
        self.V = int(V)
        self.U = int(U if U is not None else int(np.ceil(1.42 * max(self.nx, self.ny))))
        self.ds = float(ds if (ds is not None and ds > 0) else self.d)
        self.off = float(off)
        if theta is None:
            theta = np.arange(self.V, dtype=np.float64) * (np.pi / self.V)
        self.theta = _f64(theta)
        assert self.theta.shape == (self.V,)

    @property
    def n(self):
        return self.nx * self.ny

    @property
    def m(self):
        return self.V * self.U

    def _args(self):
        return (self.nx, self.ny, self.d, self.V, _d(self.theta), self.U, self.ds, self.off)


class CSR:
    """Explicit R (rows = rays v*U+u, columns = pixels i*nx+j) and R^T."""

    def __init__(self, geom: Geometry):
        L = _L()
        self.geom = geom
        m, n = geom.m, geom.n
        self.rp = np.zeros(m + 1, dtype=np.int64)
        nnz = L.orc_csr_rowptr(*geom._args(), _l(self.rp))
        self.ci = np.zeros(max(nnz, 1), dtype=np.int32)
        self.va = np.zeros(max(nnz, 1), dtype=np.float64)
        L.orc_csr_fill(*geom._args(), _l(self.rp), _i(self.ci), _d(self.va))
        self.rpt = np.zeros(n + 1, dtype=np.int64)
        self.cit = np.zeros(max(nnz, 1), dtype=np.int32)
        self.vat = np.zeros(max(nnz, 1), dtype=np.float64)
        L.orc_csr_transpose(m, n, _l(self.rp), _i(self.ci), _d(self.va),
                            _l(self.rpt), _i(self.cit), _d(self.vat))
        self.nnz = int(nnz)

    def project(self, x):
        """y = R x (Sec. 2)."""
        x = _f64(x).ravel()
        y = np.empty(self.geom.m)
        _L().orc_spmv(self.geom.m, _l(self.rp), _i(self.ci), _d(self.va), _d(x), _d(y))
        return y.reshape(self.geom.V, self.geom.U)

    def backproject(self, y):
        """x = R^T y (Eq. (2.2)), through the explicit transpose."""
        y = _f64(y).ravel()
        x = np.empty(self.geom.n)
        _L().orc_spmv(self.geom.n, _l(self.rpt), _i(self.cit), _d(self.vat), _d(y), _d(x))
        return x.reshape(self.geom.ny, self.geom.nx)

    def dense(self):
        A = np.zeros((self.geom.m, self.geom.n))
        for r in range(self.geom.m):
            for k in range(self.rp[r], self.rp[r + 1]):
                A[r, self.ci[k]] += self.va[k]
        return A


def project_rays(geom: Geometry, x, rays):
    """Ray sums of the rays ``rays`` (ids v*U+u) without storing R (Sec. 2)."""
    x = _f64(x).ravel()
    rays = np.ascontiguousarray(rays, dtype=np.int64)
    out = np.empty(rays.size)
    _L().orc_project_rays(*geom._args(), _d(x), rays.size, _l(rays), _d(out))
    return out


def backproject_pixels(geom: Geometry, y, pix):
    """(R^T y) at pixels ``pix`` (ids i*nx+j), each column of R clipped afresh."""
    y = _f64(y).ravel()
    pix = np.ascontiguousarray(pix, dtype=np.int64)
    out = np.empty(pix.size)
    _L().orc_backproject_pixels(*geom._args(), _d(y), pix.size, _l(pix), _d(out))
    return out


def tv(y):
    """TV(y), Sec. 3.1."""
    y = _f64(y)
    return float(_L().orc_tv(y.shape[0], y.shape[1], _d(y)))


def tv_tbar(y):
    """(TV(y), tbar): tbar = -dTV/dy where defined, else 0 (Sec. 3.1)."""
    y = _f64(y)
    t = np.empty_like(y)
    v = _L().orc_tv_tbar(y.shape[0], y.shape[1], _d(y), _d(t))
    return float(v), t


def tv_direction(y):
    """The nonascending vector t = tbar/||tbar|| or 0 (Sec. 3.1)."""
    v, t = tv_tbar(y)
    nrm = np.sqrt(np.sum(t * t))
    return (t / nrm) if nrm != 0 else np.zeros_like(t)


def tv_dirderiv(y, t):
    """One-sided directional derivative of TV at y along t (nonascent test)."""
    y, t = _f64(y), _f64(t)
    return float(_L().orc_tv_dirderiv(y.shape[0], y.shape[1], _d(y), _d(t)))


def stv(x, ell, a, gamma, K, max_trials=10_000):
    """S_TV(x, l, a, gamma, K), Algorithm 1 -> (status, s, l_new, trials per step)."""
    x = _f64(x)
    s = np.empty_like(x)
    ell_out = np.zeros(1, dtype=np.int64)
    tr = np.zeros(max(K, 1), dtype=np.int64)
    rc = _L().orc_stv(x.shape[0], x.shape[1], _d(x), int(ell), float(a), float(gamma), int(K),
                      int(max_trials), _d(s), _l(ell_out), _l(tr))
    return int(rc), s, int(ell_out[0]), tr[:K].copy()


def precond_D(ny, nx, mu, rho):
    """Diagonal of M = F^-1 D F, Eq. (3.2), radial frequency clamped to pi."""
    D = np.empty((ny, nx))
    _L().orc_precond_D(ny, nx, float(mu), float(rho), _d(D))
    return D


def fourier_diag(D, g):
    """Re(F^-1 diag(D) F g) by the defining DFT sums."""
    D, g = _f64(D), _f64(g)
    z = np.empty_like(g)
    _L().orc_fourier_diag(g.shape[0], g.shape[1], _d(D), _d(g), _d(z))
    return z


def precondition(g, mu, rho):
    """z = M g with M from Eq. (3.2)."""
    g = _f64(g)
    return fourier_diag(precond_D(g.shape[0], g.shape[1], mu, rho), g)


def selective_error(x, ref, ax, ay):
    """SE of Eq. (4.1) with C = 1: sqrt of the sum over the pixels S whose centres
    lie in the centred ellipse of horizontal semi-axis ax * nx and vertical
    semi-axis ay * ny pixels of (x - ref)^2 (Sec. 4.2 uses semi-axes of 5 and
    7 cm, just inside the skull)."""
    x, ref = _f64(x), _f64(ref)
    ny, nx = ref.shape
    s = 0.0
    for i in range(ny):
        for j in range(nx):
            ex = (j - 0.5 * (nx - 1)) / (ax * nx)
            ey = (i - 0.5 * (ny - 1)) / (ay * ny)
            if ex * ex + ey * ey <= 1.0:
                s += (x[i, j] - ref[i, j]) ** 2
    return float(np.sqrt(s))


def gray_level(g: Geometry, b):
    """mu_X of Eq. (2.3): the image's average value estimated from the data
    (Sec. 2).  Each view's sum b_u ds approximates the integral of the image
    (every ray of a view crosses it, spaced ds apart); the mean over views,
    divided by the image area nx ny d^2, is the gray level."""
    b = _f64(b).reshape(g.V, g.U)
    return float(np.mean(b.sum(axis=1)) * g.ds / (g.nx * g.ny * g.d * g.d))


def suppcg(R: CSR, b, x0=None, a=0.995, gamma=0.5, K=1, eps=-1.0, max_iter=50,
           max_trials=10_000, perturb=True, mu=1e-5, rho=0.8, D=None, bayes_r=0.0, bayes_mu=None):
    """SupPCG(x0, a, gamma, K, eps), Algorithm 3 (perturb=False: PCG).

    bayes_r > 0 minimises the Bayesian criterion of Eq. (2.3),
    r^2 ||Rx - b||^2 + ||x - mu_X||^2, instead of ||Rx - b||^2 (mu_X = bayes_mu,
    or gray_level(b) when None).  Returns a dict with the returned image
    x_{k-1/2} ("x_half"), x_k ("x_last"), the count of while-body executions,
    the returned k, l_k and per-body logs.
    """
    g = R.geom
    n, m = g.n, g.m
    b = _f64(b).ravel()
    x0 = np.zeros(n) if x0 is None else _f64(x0).ravel()
    if D is None:
        D = precond_D(g.ny, g.nx, mu, rho)
    D = _f64(D)
    x_half = np.empty(n)
    x_last = np.empty(n)
    iters = np.zeros(1, dtype=np.int32)
    k_out = np.zeros(1, dtype=np.int32)
    ell = np.zeros(1, dtype=np.int64)
    mi = max(int(max_iter), 1)
    logs = {k: np.zeros(mi) for k in ("f", "tv_k", "tv_half", "alpha", "beta", "snorm")}
    log_ell = np.zeros(mi, dtype=np.int64)
    init = np.zeros(3)
    rc = _L().orc_suppcg(m, n, _l(R.rp), _i(R.ci), _d(R.va), _l(R.rpt), _i(R.cit), _d(R.vat),
                         g.ny, g.nx, _d(b), _d(x0), _d(D), float(a), float(gamma), int(K),
                         float(eps), int(max_iter), int(max_trials), int(bool(perturb)),
                         _d(x_half), _d(x_last), _i(iters), _i(k_out), _l(ell),
                         _d(logs["f"]), _d(logs["tv_k"]), _d(logs["tv_half"]), _l(log_ell),
                         _d(logs["alpha"]), _d(logs["beta"]), _d(logs["snorm"]), _d(init),
                         float(bayes_r) ** 2 if bayes_r > 0 else 0.0,
                         float(gray_level(g, b) if (bayes_r > 0 and bayes_mu is None) else (bayes_mu or 0.0)))
    it = int(iters[0])
    out = {"status": int(rc), "x_half": x_half.reshape(g.ny, g.nx),
           "x_last": x_last.reshape(g.ny, g.nx), "iters": it, "k": int(k_out[0]),
           "ell": int(ell[0]), "ell_log": log_ell[:it].copy(),
           "f0": float(init[0]), "alpha0": float(init[1])}
    for k, v in logs.items():
        out[k] = v[:it].copy()
    return out


# ------------------------------------------------------------------ learned perturbation layers
def art_spacing(g: Geometry):
    """Smallest bin spacing S at which two rays of one view share no pixel.

    A pixel meets ray u when its centre projects within E = (d/ds)(|cos| +
    |sin|)/2 bins of u (the footprint of a square pixel; on the boundary only
    for axis-aligned views), so rays S >= 2E + (a little) apart touch disjoint
    pixel sets: S = floor(2 max_v E_v) + 1."""
    r = g.d / g.ds
    E = 0.0
    for th in g.theta:
        q = th / (0.5 * np.pi)
        if abs(q - round(q)) < 1e-12:
            c, s = (1.0, 0.0) if int(round(q)) % 2 == 0 else (0.0, 1.0)
        else:
            c, s = abs(np.cos(th)), abs(np.sin(th))
        E = max(E, r * (c + s) / 2.0)
    return int(np.floor(2.0 * E)) + 1


def art_order(g: Geometry, S=None):
    """One ART cycle's ray order (the paper only says that a cycle visits every
    equation once): views in order; within a view the residue classes u = c
    (mod S), c = 0 .. S-1, each in increasing u.  Rays of one class touch
    disjoint pixels, so their updates commute."""
    S = art_spacing(g) if S is None else S
    order = [v * g.U + u for v in range(g.V) for c in range(S) for u in range(c, g.U, S)]
    return np.asarray(order, dtype=np.int64)


def art(R: CSR, b, r=5.0, lam=1e-2, cycles=1, mu=None, K=0, a=1 - 1e-5, gamma=1e-2, max_trials=10_000,
        x0=None, u0=None, order=None):
    """ART for the Bayesian criterion of Eq. (2.3), Sec. 3.4 (Herman, Hurwitz,
    Lent): `cycles` full cycles over the rays in art_order, from x = mu_X (the
    prior mean; gray_level(b) when None) and u = 0.  K > 0 gives SupART: before
    every cycle x <- S_TV(x, l, a, gamma, K) (Algorithm 1), the perturbation
    step of superiorization.  Returns x, the auxiliary u, l and the status."""
    g = R.geom
    b = _f64(b).ravel()
    if mu is None:
        mu = gray_level(g, b)
    x = np.full(g.n, float(mu)) if x0 is None else _f64(x0).ravel().copy()
    u = np.zeros(g.m) if u0 is None else _f64(u0).ravel().copy()
    order = art_order(g) if order is None else np.ascontiguousarray(order, dtype=np.int64)
    ell, rc = 0, 0
    for _ in range(int(cycles)):
        if K > 0:
            rc, s, ell, _tr = stv(x.reshape(g.ny, g.nx), ell, a, gamma, K, max_trials)
            if rc != 0:
                break
            x = x + s.ravel()
        _L().orc_art_rays(_l(R.rp), _i(R.ci), _d(R.va), _l(order), order.size, _d(b), float(r), float(lam),
                          _d(x), _d(u))
    return {"x": x.reshape(g.ny, g.nx), "u": u.reshape(g.V, g.U), "ell": ell, "status": rc, "mu": float(mu)}


def conv3x3(x, W, bias=None, relu=False):
    """3x3 convolution with zero padding: x [cin][ny][nx], W [cout][cin][3][3]."""
    x, W = _f64(x), _f64(W)
    cin, ny, nx = x.shape
    cout = W.shape[0]
    assert W.shape == (cout, cin, 3, 3)
    y = np.empty((cout, ny, nx))
    b = _f64(bias) if bias is not None else None
    _L().orc_conv3x3(ny, nx, cin, cout, _d(x), _d(W), _d(b) if b is not None else None, int(relu), _d(y))
    return y


def conv3x3_backward(x, W, dy, want_dx=True):
    """(dL/dx, dL/dW, dL/dbias) of conv3x3 (no activation) for dL/dy."""
    x, W, dy = _f64(x), _f64(W), _f64(dy)
    cin, ny, nx = x.shape
    cout = W.shape[0]
    dx = np.empty_like(x) if want_dx else None
    dW = np.empty_like(W)
    db = np.empty(cout)
    _L().orc_conv3x3_backward(ny, nx, cin, cout, _d(x), _d(W), _d(dy), _d(dx) if want_dx else None, _d(dW), _d(db))
    return dx, dW, db


def cnn_forward(x, layers):
    """Network of 3x3 layers [(W, b), ...], ReLU after every layer but the last."""
    a = _f64(x)
    for li, (W, b) in enumerate(layers):
        a = conv3x3(a, W, b, relu=li + 1 < len(layers))
    return a
