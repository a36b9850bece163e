"""GB300 (sm_103a) SupPCG: matrix-free parallel-beam projector pair, Fourier
preconditioner, TV superiorization and the SupPCG iteration of
arXiv 1807.10151, behind the C ABI of ``libsupcg.so`` (include/supcg.h).

This module is a thin ctypes binding: it marshals torch tensors (device
memory, streams) into the C entry points of the same names.  Every step of
the computation runs in the library's CUDA kernels; there is no CPU path.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import threading

__all__ = [
    "load", "lib_path", "SupcgError", "Geometry", "Params", "Report", "solve_batched",
    "supcg_create_geometry", "supcg_destroy_geometry", "supcg_project", "supcg_backproject",
    "supcg_precondition", "supcg_tv_tbar", "supcg_superiorize", "supcg_solve", "supcg_solve_host",
    "supcg_solve_batched", "supcg_status_string", "LOG_STRIDE", "EXPORTED", "solve_sweep", "SE_AXES",
    "ArtParams", "ArtReport", "supcg_art",
]

LOG_STRIDE = 8
F32, BF16 = 0, 1
STATUS = {0: "OK", -1: "ERR_ARG", -2: "ERR_CUDA", -3: "ERR_NOMEM", -4: "ERR_BREAKDOWN",
          -5: "ERR_BACKTRACK", -6: "ERR_TIMEOUT", -7: "ERR_PRECOND", -8: "ERR_UNSUPPORTED"}
EXPORTED = ["supcg_create_geometry", "supcg_destroy_geometry", "supcg_project", "supcg_backproject",
            "supcg_precondition", "supcg_tv_tbar", "supcg_superiorize", "supcg_solve", "supcg_solve_host",
            "supcg_solve_batched", "supcg_status_string", "supcg_solve_profiled", "supcg_kernel_launches",
            "supcg_precondition_noalloc", "supcg_cnn_create", "supcg_cnn_destroy", "supcg_cnn_num_params",
            "supcg_cnn_get_params", "supcg_cnn_set_params", "supcg_cnn_forward", "supcg_cnn_gradients",
            "supcg_cnn_train_step", "supcg_solve_trace", "supcg_solve_learned", "supcg_set_tiling",
            "supcg_get_tiling", "supcg_solve_sweep", "supcg_art", "supcg_set_wait_limit",
            "supcg_set_barrier_shortfall", "supcg_solve_batched_learned", "supcg_set_bwd_parts",
            "supcg_get_bwd_parts", "supcg_get_mirror_pairs"]
KINDS = ["forward", "backward", "fft", "stv", "vector", "cnn"]

_lock = threading.Lock()
_lib = None


class SupcgError(RuntimeError):
    def __init__(self, code, what=""):
        self.code = int(code)
        super().__init__(f"{what}: {STATUS.get(self.code, self.code)} ({self.code})")


class Params(C.Structure):
    """supcg_params (include/supcg.h)."""
    _fields_ = [("K", C.c_int), ("a", C.c_double), ("gamma", C.c_double), ("mu", C.c_double),
                ("rho", C.c_double), ("eps", C.c_double), ("max_iter", C.c_int),
                ("max_trials", C.c_longlong), ("perturb", C.c_int), ("precondition", C.c_int),
                ("graph", C.c_int), ("bayes_r", C.c_double), ("bayes_mu", C.c_double)]


class Report(C.Structure):
    """supcg_report (include/supcg.h)."""
    _fields_ = [("iters", C.c_int), ("k", C.c_int), ("ell", C.c_longlong), ("f_last", C.c_double),
                ("f0", C.c_double), ("tv_last", C.c_double), ("status", C.c_int), ("n_fallback", C.c_int),
                ("n_learned", C.c_int)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class ArtParams(C.Structure):
    """supcg_art_params (include/supcg.h): ART / SupART of Sec. 3.4."""
    _fields_ = [("r", C.c_double), ("lam", C.c_double), ("mu", C.c_double), ("cycles", C.c_int), ("K", C.c_int),
                ("a", C.c_double), ("gamma", C.c_double), ("max_trials", C.c_longlong)]


class ArtReport(C.Structure):
    """supcg_art_report (include/supcg.h)."""
    _fields_ = [("cycles", C.c_int), ("ell", C.c_longlong), ("mu", C.c_double), ("status", C.c_int)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


def lib_path() -> str:
    from . import build as _b
    return _b.LIB


def load(allow_build: bool = True):
    """Load libsupcg.so (building it in-tree with nvcc if it is stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        from . import build as _b
        if allow_build and not _b.up_to_date():
            _b.build()
        if not os.path.exists(_b.LIB):
            raise RuntimeError(f"libsupcg.so not built ({_b.LIB}); run __graft_entry__.build()")
        L = C.CDLL(_b.LIB)
        vp, i, d, ll = C.c_void_p, C.c_int, C.c_double, C.c_longlong
        L.supcg_create_geometry.argtypes = [i, i, d, i, C.POINTER(d), i, d, d, i, C.POINTER(vp)]
        L.supcg_destroy_geometry.argtypes = [vp]
        L.supcg_project.argtypes = [vp, vp, vp, i, vp]
        L.supcg_backproject.argtypes = [vp, vp, vp, i, vp]
        L.supcg_precondition.argtypes = [vp, d, d, vp, vp, i, vp]
        L.supcg_precondition_noalloc.argtypes = [i, i, d, d, vp, vp, vp]
        L.supcg_tv_tbar.argtypes = [vp, vp, vp, C.POINTER(d), vp]
        L.supcg_superiorize.argtypes = [vp, vp, d, d, i, ll, C.POINTER(ll), C.POINTER(i), vp]
        L.supcg_solve.argtypes = [vp, vp, vp, C.POINTER(Params), C.POINTER(Report), vp, vp]
        L.supcg_art.argtypes = [vp, vp, vp, C.POINTER(ArtParams), C.POINTER(ArtReport), vp]
        L.supcg_solve_host.argtypes = [vp, vp, vp, C.POINTER(Params), C.POINTER(Report), vp]
        L.supcg_solve_batched.argtypes = [C.POINTER(vp), C.POINTER(vp), C.POINTER(vp), i,
                                          C.POINTER(Params), C.POINTER(Report), vp]
        L.supcg_solve_sweep.argtypes = [vp, vp, C.POINTER(vp), i, C.POINTER(Params), vp, d, d, vp,
                                        C.POINTER(Report), vp]
        L.supcg_solve_profiled.argtypes = [vp, vp, vp, C.POINTER(Params), C.POINTER(Report),
                                           C.POINTER(d), C.POINTER(ll), vp]
        L.supcg_kernel_launches.argtypes = []
        L.supcg_kernel_launches.restype = ll
        fp = C.POINTER(C.c_float)
        L.supcg_cnn_create.argtypes = [i, i, i, C.c_ulonglong, C.POINTER(vp)]
        L.supcg_cnn_destroy.argtypes = [vp]
        L.supcg_cnn_num_params.argtypes = [vp]
        L.supcg_cnn_get_params.argtypes = [vp, fp]
        L.supcg_cnn_set_params.argtypes = [vp, fp]
        L.supcg_cnn_forward.argtypes = [vp, vp, vp, i, vp, vp]
        L.supcg_cnn_gradients.argtypes = [vp, vp, vp, vp, i, fp, C.POINTER(d), vp]
        L.supcg_cnn_train_step.argtypes = [vp, vp, vp, vp, i, d, C.POINTER(d), vp]
        L.supcg_solve_trace.argtypes = [vp, vp, vp, C.POINTER(Params), C.POINTER(Report), vp, vp, vp]
        L.supcg_solve_learned.argtypes = [vp, vp, vp, vp, C.POINTER(Params), C.POINTER(Report), vp, vp]
        L.supcg_solve_batched_learned.argtypes = [C.POINTER(vp), vp, C.POINTER(vp), C.POINTER(vp), i,
                                                  C.POINTER(Params), C.POINTER(Report), vp]
        L.supcg_set_tiling.argtypes = [vp, i]
        L.supcg_set_bwd_parts.argtypes = [vp, i]
        L.supcg_get_bwd_parts.argtypes = [vp, C.POINTER(i)]
        L.supcg_get_mirror_pairs.argtypes = [vp, C.POINTER(i)]
        L.supcg_get_tiling.argtypes = [vp, C.POINTER(i)]
        L.supcg_set_wait_limit.argtypes = [ll]
        L.supcg_set_barrier_shortfall.argtypes = [i]
        L.supcg_status_string.argtypes = [i]
        L.supcg_status_string.restype = C.c_char_p
        for name in EXPORTED:
            if name not in ("supcg_status_string", "supcg_kernel_launches"):
                getattr(L, name).restype = i
        _lib = L
        return L


# Statuses a solve reports after running its iterations (in the report as well);
# any other code means the call did not run and raises SupcgError.
RUN_STATUSES = (0, -4, -5, -6)


def _check(rc, what):
    if rc != 0:
        raise SupcgError(rc, what)


# ---------------------------------------------------------------- C-ABI mirrors
def supcg_create_geometry(nx, ny, pixel_size, n_views, angles, n_bins, bin_spacing, det_center_offset, storage):
    h = C.c_void_p()
    arr = None
    if angles is not None:
        arr = (C.c_double * n_views)(*[float(a) for a in angles])
    rc = load().supcg_create_geometry(nx, ny, pixel_size, n_views, arr, n_bins, bin_spacing,
                                      det_center_offset, storage, C.byref(h))
    _check(rc, "supcg_create_geometry")
    return h


def supcg_destroy_geometry(g):
    return load().supcg_destroy_geometry(g)


def supcg_project(g, d_x, d_y, batch, stream):
    return load().supcg_project(g, d_x, d_y, batch, stream)


def supcg_backproject(g, d_y, d_x, batch, stream):
    return load().supcg_backproject(g, d_y, d_x, batch, stream)


def supcg_precondition(g, mu, rho, d_g, d_z, batch, stream):
    return load().supcg_precondition(g, mu, rho, d_g, d_z, batch, stream)


def supcg_precondition_noalloc(ny, nx, mu, rho, d_g, d_z, stream):
    return load().supcg_precondition_noalloc(ny, nx, mu, rho, d_g, d_z, stream)


def supcg_tv_tbar(g, d_y, d_tbar, h_out, stream):
    return load().supcg_tv_tbar(g, d_y, d_tbar, h_out, stream)


def supcg_superiorize(g, d_x, a, gamma, K, max_trials, h_ell, h_trials, stream):
    return load().supcg_superiorize(g, d_x, a, gamma, K, max_trials, h_ell, h_trials, stream)


def supcg_art(g, d_b, d_x, params, rep, stream):
    return load().supcg_art(g, d_b, d_x, C.byref(params), C.byref(rep), stream)


def supcg_solve(g, d_b, d_x, params, rep, d_log, stream):
    return load().supcg_solve(g, d_b, d_x, C.byref(params), C.byref(rep), d_log, stream)


def supcg_solve_host(g, h_b, h_x, params, rep, stream):
    return load().supcg_solve_host(g, h_b, h_x, C.byref(params), C.byref(rep), stream)


def supcg_solve_batched(gs, d_b, d_x, count, params, reps, stream):
    return load().supcg_solve_batched(gs, d_b, d_x, count, C.byref(params), reps, stream)


def supcg_solve_profiled(g, d_b, d_x, params, rep, h_ms, h_launches, stream):
    return load().supcg_solve_profiled(g, d_b, d_x, C.byref(params), C.byref(rep), h_ms, h_launches, stream)


def supcg_kernel_launches():
    return int(load().supcg_kernel_launches())


def supcg_status_string(status):
    return load().supcg_status_string(status).decode()


def supcg_set_wait_limit(polls):
    return load().supcg_set_wait_limit(int(polls))


def supcg_set_barrier_shortfall(extra_blocks):
    return load().supcg_set_barrier_shortfall(int(extra_blocks))


DEFAULT_WAIT_LIMIT = 1 << 24


# ---------------------------------------------------------------- torch helpers
def _stream(stream):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


def _ptr(t, dtype=None):
    import torch
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"expected {dtype}, got {t.dtype}")
    return C.c_void_p(t.data_ptr())


def make_params(K=1, a=0.995, gamma=0.5, mu=1e-5, rho=0.8, eps=-1.0, max_iter=50, max_trials=10_000,
                perturb=True, precondition=True, graph=True, bayes_r=0.0, bayes_mu=None) -> Params:
    """supcg_params; bayes_r > 0 selects the Bayesian criterion (bayes_mu None: mu_X from the data)."""
    return Params(int(K), float(a), float(gamma), float(mu), float(rho), float(eps), int(max_iter),
                  int(max_trials), int(bool(perturb)), int(bool(precondition)), int(bool(graph)),
                  float(bayes_r), float("nan") if bayes_mu is None else float(bayes_mu))


class Geometry:
    """2-D parallel-beam geometry (owner of a supcg_geometry handle).

    Defaults follow Sec. 4.1 of the paper: V equally spaced angles in
    [0, pi), bin spacing equal to the pixel size; the image is the unit square
    (pixel size 1/max(nx, ny)).
    """

    def __init__(self, nx, ny=None, n_views=90, n_bins=None, pixel_size=None, angles=None, bin_spacing=0.0,
                 offset=0.0, storage="f32"):
        self.nx = int(nx)
        self.ny = int(ny if ny is not None else nx)
        self.V = int(n_views)
        self.U = int(n_bins if n_bins is not None else math.ceil(1.42 * max(self.nx, self.ny)))
        self.d = float(pixel_size if pixel_size is not None else 1.0 / max(self.nx, self.ny))
        self.storage = BF16 if storage in ("bf16", BF16) else F32
        self.handle = supcg_create_geometry(self.nx, self.ny, self.d, self.V, angles, self.U,
                                            float(bin_spacing), float(offset), self.storage)

    def close(self):
        if getattr(self, "handle", None) is not None and _lib is not None:
            supcg_destroy_geometry(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_tiling(self, fwd_bins_per_block):
        """Forward-projector rays per block (supcg_set_tiling); returns the status."""
        return load().supcg_set_tiling(self.handle, int(fwd_bins_per_block))

    def get_tiling(self):
        v = C.c_int()
        _check(load().supcg_get_tiling(self.handle, C.byref(v)), "supcg_get_tiling")
        return v.value

    def set_bwd_parts(self, parts):
        """Backprojector view parts per pixel tile (supcg_set_bwd_parts); returns the status."""
        return load().supcg_set_bwd_parts(self.handle, int(parts))

    def get_bwd_parts(self):
        v = C.c_int()
        _check(load().supcg_get_bwd_parts(self.handle, C.byref(v)), "supcg_get_bwd_parts")
        return v.value

    def mirror_pairs(self):
        """Mirror pairs of views (theta, pi - theta) the forward projector evaluates together."""
        v = C.c_int()
        _check(load().supcg_get_mirror_pairs(self.handle, C.byref(v)), "supcg_get_mirror_pairs")
        return v.value

    @property
    def _dt(self):
        import torch
        return torch.bfloat16 if self.storage == BF16 else torch.float32

    def project(self, x, out=None, stream=None):
        """R x for x [..., ny, nx] -> [..., V, U] (Sec. 2)."""
        import torch
        batch = x.numel() // (self.nx * self.ny)
        if out is None:
            out = torch.empty(*x.shape[:-2], self.V, self.U, device=x.device, dtype=self._dt)
        _check(supcg_project(self.handle, _ptr(x, self._dt), _ptr(out, self._dt), batch, _stream(stream)),
               "supcg_project")
        return out

    def backproject(self, y, out=None, stream=None):
        """R^T y for y [..., V, U] -> [..., ny, nx] (Eq. (2.2))."""
        import torch
        batch = y.numel() // (self.V * self.U)
        if out is None:
            out = torch.empty(*y.shape[:-2], self.ny, self.nx, device=y.device, dtype=self._dt)
        _check(supcg_backproject(self.handle, _ptr(y, self._dt), _ptr(out, self._dt), batch, _stream(stream)),
               "supcg_backproject")
        return out

    def precondition(self, g, mu=1e-5, rho=0.8, out=None, stream=None):
        """M g with M = F^-1 D F of Eq. (3.2)."""
        import torch
        batch = g.numel() // (self.nx * self.ny)
        if out is None:
            out = torch.empty_like(g)
        _check(supcg_precondition(self.handle, float(mu), float(rho), _ptr(g, torch.float32),
                                  _ptr(out, torch.float32), batch, _stream(stream)), "supcg_precondition")
        return out

    def tv_tbar(self, y, stream=None):
        """(TV(y), ||tbar||^2, tbar) of Sec. 3.1."""
        import torch
        tb = torch.empty_like(y)
        h = (C.c_double * 2)()
        _check(supcg_tv_tbar(self.handle, _ptr(y, torch.float32), _ptr(tb, torch.float32), h, _stream(stream)),
               "supcg_tv_tbar")
        return h[0], h[1], tb

    def superiorize(self, x, ell, a, gamma, K, max_trials=10_000, stream=None):
        """S_TV (Algorithm 1) in place on x; returns (status, new l, trials per step)."""
        import torch
        e = C.c_longlong(int(ell))
        tr = (C.c_int * max(int(K), 1))()
        rc = supcg_superiorize(self.handle, _ptr(x, torch.float32), float(a), float(gamma), int(K),
                               int(max_trials), C.byref(e), tr, _stream(stream))
        if rc not in (0, -5):
            raise SupcgError(rc, "supcg_superiorize")
        return rc, int(e.value), list(tr)[:int(K)]

    def art(self, b, r=5.0, lam=1e-2, cycles=1, mu=None, K=0, a=1 - 1e-5, gamma=1e-2, max_trials=10_000,
            stream=None):
        """ART on the Bayesian criterion of Eq. (2.3) (K = 0) or SupART (K > 0), Sec. 3.4:
        `cycles` full cycles through the rays from x = mu_X (None: estimated from b).
        Returns (x [ny][nx], report dict)."""
        import torch
        x = torch.empty(self.ny, self.nx, device=b.device, dtype=torch.float32)
        p = ArtParams(float(r), float(lam), float("nan") if mu is None else float(mu), int(cycles), int(K),
                      float(a), float(gamma), int(max_trials))
        rep = ArtReport()
        rc = supcg_art(self.handle, _ptr(b, torch.float32), _ptr(x, torch.float32), p, rep, _stream(stream))
        if rc not in (0, -5):
            raise SupcgError(rc, "supcg_art")
        return x, rep.as_dict()

    def solve(self, b, x0=None, log=False, stream=None, **kw):
        """SupPCG (Algorithm 3).  Returns (x_{k-1/2}, report dict, log or None)."""
        import torch
        x = torch.zeros(self.ny, self.nx, device=b.device, dtype=torch.float32) if x0 is None else x0.clone()
        p = make_params(**kw)
        rep = Report()
        lg = torch.zeros(max(p.max_iter, 1), LOG_STRIDE, device=b.device, dtype=torch.float64) if log else None
        rc = supcg_solve(self.handle, _ptr(b, torch.float32), _ptr(x, torch.float32), p, rep,
                         _ptr(lg) if log else None, _stream(stream))
        if rc not in RUN_STATUSES:
            raise SupcgError(rc, "supcg_solve")
        out = rep.as_dict()
        out["rc"] = rc
        return x, out, lg

    def solve_profiled(self, b, x0=None, stream=None, **kw):
        """SupPCG with CUDA events around every launch: (x, report, {kind: (ms, launches)})."""
        import torch
        x = torch.zeros(self.ny, self.nx, device=b.device, dtype=torch.float32) if x0 is None else x0.clone()
        p = make_params(**kw)
        rep = Report()
        ms = (C.c_double * len(KINDS))()
        cnt = (C.c_longlong * len(KINDS))()
        rc = supcg_solve_profiled(self.handle, _ptr(b, torch.float32), _ptr(x, torch.float32), p, rep, ms, cnt,
                                  _stream(stream))
        if rc not in RUN_STATUSES:
            raise SupcgError(rc, "supcg_solve_profiled")
        out = rep.as_dict()
        out["rc"] = rc
        return x, out, {k: (ms[i], cnt[i]) for i, k in enumerate(KINDS)}

    def solve_trace(self, b, x0=None, stream=None, **kw):
        """SupPCG recording x_k of every while body: (x, report, log, trace [max_iter][ny][nx])."""
        import torch
        x = torch.zeros(self.ny, self.nx, device=b.device, dtype=torch.float32) if x0 is None else x0.clone()
        p = make_params(**kw)
        rep = Report()
        lg = torch.zeros(max(p.max_iter, 1), LOG_STRIDE, device=b.device, dtype=torch.float64)
        tr = torch.zeros(max(p.max_iter, 1), self.ny, self.nx, device=b.device, dtype=torch.float32)
        rc = load().supcg_solve_trace(self.handle, _ptr(b, torch.float32), _ptr(x, torch.float32), C.byref(p),
                                      C.byref(rep), _ptr(lg), _ptr(tr), _stream(stream))
        if rc not in RUN_STATUSES:
            raise SupcgError(rc, "supcg_solve_trace")
        out = rep.as_dict()
        out["rc"] = rc
        return x, out, lg, tr

    def solve_learned(self, net, b, x0=None, log=False, stream=None, **kw):
        """SupPCG with the learned direction (supcg_solve_learned)."""
        import torch
        x = torch.zeros(self.ny, self.nx, device=b.device, dtype=torch.float32) if x0 is None else x0.clone()
        p = make_params(**kw)
        rep = Report()
        lg = torch.zeros(max(p.max_iter, 1), LOG_STRIDE, device=b.device, dtype=torch.float64) if log else None
        rc = load().supcg_solve_learned(self.handle, net.handle, _ptr(b, torch.float32), _ptr(x, torch.float32),
                                        C.byref(p), C.byref(rep), _ptr(lg) if log else None, _stream(stream))
        if rc not in RUN_STATUSES:
            raise SupcgError(rc, "supcg_solve_learned")
        out = rep.as_dict()
        out["rc"] = rc
        return x, out, lg

    def solve_host(self, b_host, x_host, stream=None, **kw):
        """SupPCG through host buffers (numpy / CPU tensors, float32); x_host is overwritten."""
        p = make_params(**kw)
        rep = Report()
        rc = supcg_solve_host(self.handle, C.c_void_p(b_host.ctypes.data if hasattr(b_host, "ctypes")
                                                      else b_host.data_ptr()),
                              C.c_void_p(x_host.ctypes.data if hasattr(x_host, "ctypes") else x_host.data_ptr()),
                              p, rep, _stream(stream))
        if rc not in RUN_STATUSES:
            raise SupcgError(rc, "supcg_solve_host")
        out = rep.as_dict()
        out["rc"] = rc
        return out


def solve_batched(geoms, bs, xs, stream=None, **kw):
    """Solve independent problems of different geometries in one batched schedule.
    xs are updated in place (x_0 in, x_{k-1/2} out).  Returns the reports."""
    import torch
    n = len(geoms)
    G = (C.c_void_p * n)(*[g.handle.value for g in geoms])
    B = (C.c_void_p * n)(*[_ptr(b, torch.float32).value for b in bs])
    X = (C.c_void_p * n)(*[_ptr(x, torch.float32).value for x in xs])
    reps = (Report * n)()
    p = make_params(**kw)
    rc = supcg_solve_batched(G, B, X, n, p, reps, _stream(stream))
    if rc not in RUN_STATUSES:
        raise SupcgError(rc, "supcg_solve_batched")
    return [r.as_dict() for r in reps]


def solve_batched_learned(geoms, net, bs, xs, stream=None, **kw):
    """The learned direction over independent problems of the network's image size
    in one batched schedule (supcg_solve_batched_learned); xs updated in place.
    Returns the reports."""
    import torch
    n = len(geoms)
    G = (C.c_void_p * n)(*[g.handle.value for g in geoms])
    B = (C.c_void_p * n)(*[_ptr(b, torch.float32).value for b in bs])
    X = (C.c_void_p * n)(*[_ptr(x, torch.float32).value for x in xs])
    reps = (Report * n)()
    p = make_params(**kw)
    rc = load().supcg_solve_batched_learned(G, net.handle, B, X, n, C.byref(p), reps, _stream(stream))
    if rc not in RUN_STATUSES:
        raise SupcgError(rc, "supcg_solve_batched_learned")
    return [r.as_dict() for r in reps]


# Semi-axes of the selective-error ellipse as fractions of the image side: 5 cm and
# 7 cm in the paper's 243 x 0.0752 cm field (Sec. 4.2, Eq. (4.1)).
SE_AXES = (5.0 / (243 * 0.0752), 7.0 / (243 * 0.0752))


def solve_sweep(G, b, params, ref=None, se_axes=SE_AXES, stream=None):
    """Parameter sweep (supcg_solve_sweep): one solve of (G, b) per dict of
    parameters in `params` (K, a, gamma, mu, rho differ; the rest shared), all in
    one batched schedule.  Returns (images [count][ny][nx], reports, SE) with SE
    [count][max_iter] the selective error of every iteration against `ref`
    (None without a reference)."""
    import torch
    n = len(params)
    ps = (Params * n)(*[make_params(**q) for q in params])
    xs = torch.zeros(n, G.ny, G.nx, device=b.device, dtype=torch.float32)
    X = (C.c_void_p * n)(*[xs[c].data_ptr() for c in range(n)])
    mi = max(int(ps[0].max_iter), 1)
    se = torch.zeros(n, mi, device=b.device, dtype=torch.float64) if ref is not None else None
    reps = (Report * n)()
    rc = load().supcg_solve_sweep(G.handle, _ptr(b, torch.float32), X, n, ps,
                                  _ptr(ref, torch.float32) if ref is not None else None,
                                  float(se_axes[0]), float(se_axes[1]), _ptr(se) if se is not None else None,
                                  reps, _stream(stream))
    if rc not in RUN_STATUSES:
        raise SupcgError(rc, "supcg_solve_sweep")
    return xs, [r.as_dict() for r in reps], se


# ---------------------------------------------------------------- learned perturbation network
CNN_SHAPES = [(32, 2), (32, 32), (32, 32), (32, 32), (1, 32)]   # (cout, cin) of the five 3x3 layers


class CNN:
    """The learned-direction network (supcg_cnn_*): 2 -> 32 -> 32 -> 32 -> 32 -> 1
    channels of 3x3 convolutions on the tensor cores."""

    def __init__(self, ny, nx, max_batch=1, seed=1):
        self.ny, self.nx, self.cap = int(ny), int(nx), int(max_batch)
        h = C.c_void_p()
        _check(load().supcg_cnn_create(self.ny, self.nx, self.cap, int(seed), C.byref(h)), "supcg_cnn_create")
        self.handle = h
        self.nparam = load().supcg_cnn_num_params(h)

    def close(self):
        if getattr(self, "handle", None) is not None and _lib is not None:
            _lib.supcg_cnn_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def get_params(self):
        import numpy as np
        a = np.empty(self.nparam, dtype=np.float32)
        _check(load().supcg_cnn_get_params(self.handle, a.ctypes.data_as(C.POINTER(C.c_float))), "get_params")
        return a

    def set_params(self, a):
        import numpy as np
        a = np.ascontiguousarray(a, dtype=np.float32)
        assert a.size == self.nparam
        _check(load().supcg_cnn_set_params(self.handle, a.ctypes.data_as(C.POINTER(C.c_float))), "set_params")

    @staticmethod
    def unflatten(a):
        """Flat parameters -> [(W [cout][cin][3][3], b [cout]), ...]."""
        out, off = [], 0
        for co, ci in CNN_SHAPES:
            W = a[off:off + co * ci * 9].reshape(co, ci, 3, 3)
            off += co * ci * 9
            b = a[off:off + co]
            off += co
            out.append((W, b))
        return out

    def forward(self, x, tbar, stream=None):
        import torch
        count = x.numel() // (self.ny * self.nx)
        out = torch.empty_like(x)
        _check(load().supcg_cnn_forward(self.handle, _ptr(x, torch.float32), _ptr(tbar, torch.float32), count,
                                        _ptr(out, torch.float32), _stream(stream)), "supcg_cnn_forward")
        return out

    def gradients(self, x, tbar, target, stream=None):
        import numpy as np
        import torch
        count = x.numel() // (self.ny * self.nx)
        g = np.empty(self.nparam, dtype=np.float32)
        loss = C.c_double()
        _check(load().supcg_cnn_gradients(self.handle, _ptr(x, torch.float32), _ptr(tbar, torch.float32),
                                          _ptr(target, torch.float32), count, g.ctypes.data_as(C.POINTER(C.c_float)),
                                          C.byref(loss), _stream(stream)), "supcg_cnn_gradients")
        return g, loss.value

    def train_step(self, x, tbar, target, lr=1e-3, want_loss=True, stream=None):
        import torch
        count = x.numel() // (self.ny * self.nx)
        loss = C.c_double()
        _check(load().supcg_cnn_train_step(self.handle, _ptr(x, torch.float32), _ptr(tbar, torch.float32),
                                           _ptr(target, torch.float32), count, float(lr),
                                           C.byref(loss) if want_loss else None, _stream(stream)),
               "supcg_cnn_train_step")
        return loss.value if want_loss else None
