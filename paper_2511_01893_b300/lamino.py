"""ctypes binding of liblamino.so (C ABI in include/lamino.h).

Argument marshalling only: every step of the operator and of ADMM-TV runs in
the library's CUDA kernels.  PyTorch supplies device memory (tensors) and the
stream (``torch.cuda.current_stream()``).  There is no CPU fallback: if the
library is missing or no GPU is present, the calls raise.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
# LAMINO_LIB selects another build of the same ABI (liblamino_checked.so: the
# LAM_BOUNDS_CHECK variant)
LIB_PATH = os.environ.get("LAMINO_LIB") or os.path.join(_HERE, "liblamino.so")

LAM_F32, LAM_F64 = 0, 1
NSCALARS = 16
SC = dict(rho=0, alpha=1, objective=2, r=3, s=4, iter=5, data2=6, tv=7, status=8, memo_hits=9, memo_lookups=10)

_lib = None


class LaminoError(RuntimeError):
    pass


def lib() -> ctypes.CDLL:
    """Load liblamino.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise LaminoError(f"{LIB_PATH} is missing: run `python -m paper_2511_01893_b300.build`")
        L = ctypes.CDLL(LIB_PATH)
        vp, i, d, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
        sig = {
            "lam_plan_create": [ctypes.POINTER(vp), i, i, i, i, i, ctypes.POINTER(d), d, i, i, i],
            "lam_plan_destroy": [vp],
            "lam_plan_set_option": [vp, i, i],
            "lam_forward": [vp, vp, vp, vp, vp],
            "lam_adjoint": [vp, vp, vp, vp, vp],
            "lam_forward_hat": [vp, vp, vp, vp, vp, vp],
            "lam_adjoint_hat": [vp, vp, vp, vp, vp],
            "lam_fft2d": [vp, vp, vp, i, vp],
            "lam_fbp": [vp, vp, vp, vp, vp],
            "tv_grad": [vp, vp, vp, vp],
            "tv_div": [vp, vp, vp, vp],
            "tv_smooth": [vp, vp, d, vp, ctypes.POINTER(d), vp, vp],
            "admm_state_bytes": [vp, ctypes.POINTER(sz)],
            "admm_init": [vp, vp, vp, d, d, i, i, vp, vp],
            "admm_step": [vp, vp, vp, vp],
            "admm_run": [vp, vp, vp, i, i, vp],
            "admm_read_scalars": [vp, vp, ctypes.POINTER(d), vp],
            "admm_read_history": [vp, vp, i, ctypes.POINTER(d), vp],
            "admm_status": [vp, vp, vp],
            "reconstruct": [vp, ctypes.POINTER(d), d, i, i, i, i, i, i, d, d, vp],
            "lamx_u1d_fwd": [vp, vp, vp, vp],
            "lamx_u1d_adj": [vp, vp, vp, vp],
            "lamx_u2d_fwd": [vp, vp, vp, vp, vp, vp],
            "lamx_u2d_adj": [vp, vp, vp, vp, vp],
            "lamx_u2d_fwd_static": [vp, vp, vp, vp, vp],
            "lamx_plan_info": [vp, ctypes.POINTER(i), i],
            "lamx_admm_graph_kernels": [vp, vp, ctypes.POINTER(sz)],
            "lam_plan_autotune": [vp, vp, vp, vp, i, ctypes.POINTER(d), vp],
            "lamx_plane_ffts": [vp, vp, vp, i, i, vp],
            "lamx_fma_peak": [vp, i, ctypes.POINTER(d), vp],
            "lam_batch_create": [ctypes.POINTER(vp), vp, vp, i],
            "lam_batch_destroy": [vp],
            "lam_forward_hat_batched": [vp, vp, vp, vp],
            "lam_adjoint_hat_batched": [vp, vp, vp, vp],
            "lam_forward_batched": [vp, vp, vp, vp],
            "lam_adjoint_batched": [vp, vp, vp, vp],
            "admm_run_batched": [vp, vp, i, i, vp],
            "lam_batch_set_streams": [vp, i],
            "lamx_batch_info": [vp, ctypes.POINTER(i), i],
            "lamx_spread": [vp, vp, vp, i, i, vp],
            "lamx_jobs_per_batch": [vp],
            "lamx_job_planes": [vp, i, i],
            "lam_plan_status": [vp, vp],
            "lamx_admm_layout": [vp, ctypes.POINTER(sz), i],
            "lam_bounds_checked": [],
            "lamx_bounds_selftest": [vp, i, vp],
        }
        for name, args in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = ctypes.c_int
        L.lam_workspace_bytes.argtypes = [vp]
        L.lam_workspace_bytes.restype = sz
        L.lam_workspace_bytes_hat.argtypes = [vp]
        L.lam_workspace_bytes_hat.restype = sz
        L.admm_u.argtypes = [vp, vp]
        L.admm_u.restype = vp
        L.lam_last_error.argtypes = []
        L.lam_last_error.restype = ctypes.c_char_p
        _lib = L
    return _lib


def _check(status: int, what: str):
    if status != 0:
        msg = lib().lam_last_error().decode(errors="replace")
        raise LaminoError(f"{what} failed with status {status}: {msg}")


def _ptr(t) -> ctypes.c_void_p:
    if t is None:
        return None
    if not t.is_cuda:
        raise LaminoError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise LaminoError("expected a contiguous tensor")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream=None) -> ctypes.c_void_p:
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


@dataclass(frozen=True)
class Geometry:
    n: int
    nz: int
    h: int
    w: int
    theta: tuple
    phi: float
    m: int = 4

    @property
    def n_theta(self) -> int:
        return len(self.theta)


class Plan:
    """A plan for one geometry and precision ('f32' or 'f64') on the current device."""

    SPREADS = {"tiles": 0, "atomic": 1, "exact": 2, "halo": 3, "tiles_exact": 4, "tiles2": 5, "sweep": 6}

    def __init__(self, n, nz, h, w, theta, phi, m=4, prec="f32", device=None, fast_adjoint=False, spread=None,
                 workspace="full"):
        """spread: the adjoint's spread variant, "tiles" (default, per-warp tiles,
        reproducible), "atomic" (floating-point atomic adds) or "exact" (exact
        fixed-point atomic adds); fast_adjoint=True is "atomic"."""
        if not torch.cuda.is_available():
            raise LaminoError("no CUDA device: the laminography operators run only on the GPU")
        # the plan's device with its index resolved (a bare "cuda" means the
        # current device), so that arguments can be checked against it exactly
        dev = torch.device("cuda" if device is None else device)
        if dev.type != "cuda":
            raise LaminoError(f"a plan lives on a CUDA device, not {dev}")
        self.device = torch.device("cuda", torch.cuda.current_device() if dev.index is None else dev.index)
        theta = np.ascontiguousarray(np.asarray(theta, dtype=np.float64))
        self.n, self.nz, self.h, self.w, self.T = int(n), int(nz), int(h), int(w), len(theta)
        self.theta, self.phi, self.m = theta, float(phi), int(m)
        self.prec = prec
        self.rdtype = torch.float32 if prec == "f32" else torch.float64
        self.cdtype = torch.complex64 if prec == "f32" else torch.complex128
        h_ = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            _check(lib().lam_plan_create(ctypes.byref(h_), self.n, self.nz, self.h, self.w, self.T,
                                         theta.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), self.phi,
                                         2, self.m, LAM_F32 if prec == "f32" else LAM_F64),
                   "lam_plan_create")
        self._h = h_
        if fast_adjoint:
            _check(lib().lam_plan_set_option(self._h, 1, 1), "lam_plan_set_option")
        if spread is not None:
            if spread not in self.SPREADS:
                raise LaminoError(f"spread must be one of {sorted(self.SPREADS)}")
            _check(lib().lam_plan_set_option(self._h, 2, self.SPREADS[spread]), "lam_plan_set_option")
        # "hat": only the prefix the L_hat / L_hat^H / L calls use (saves a
        # data-sized buffer; adjoint() and ADMM then refuse to run)
        if workspace not in ("full", "hat"):
            raise LaminoError('workspace must be "full" or "hat"')
        self.workspace = workspace
        nbytes = (lib().lam_workspace_bytes if workspace == "full" else lib().lam_workspace_bytes_hat)(self._h)
        self.ws = torch.empty(nbytes, dtype=torch.uint8, device=self.device)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib is not None:
            _lib.lam_plan_destroy(h)
            self._h = None

    # shapes
    @property
    def vol_shape(self):
        return (self.n, self.nz, self.n)

    @property
    def data_shape(self):
        return (self.T, self.h, self.w)

    def _vol(self):
        return torch.empty(self.vol_shape, dtype=self.rdtype, device=self.device)

    def _data(self):
        return torch.empty(self.data_shape, dtype=self.cdtype, device=self.device)

    def _inp(self, t, dtype, shape):
        t = torch.as_tensor(t)
        if t.dtype != dtype or t.device != self.device or not t.is_contiguous():
            t = t.to(device=self.device, dtype=dtype).contiguous()
        if tuple(t.shape) != tuple(shape):
            raise LaminoError(f"expected shape {shape}, got {tuple(t.shape)}")
        return t

    # operators
    def forward(self, u, out=None):
        u = self._inp(u, self.rdtype, self.vol_shape)
        out = self._data() if out is None else out
        _check(lib().lam_forward(self._h, _ptr(u), _ptr(out), _ptr(self.ws), _stream()), "lam_forward")
        return out

    def _need_full(self, what):
        if self.workspace != "full":
            raise LaminoError(f"{what} needs the full workspace (plan created with workspace='hat')")

    def adjoint(self, d, out=None):
        self._need_full("adjoint")
        d = self._inp(d, self.cdtype, self.data_shape)
        out = self._vol() if out is None else out
        _check(lib().lam_adjoint(self._h, _ptr(d), _ptr(out), _ptr(self.ws), _stream()), "lam_adjoint")
        return out

    def forward_hat(self, u, sub=None, out=None):
        u = self._inp(u, self.rdtype, self.vol_shape)
        if sub is not None:
            sub = self._inp(sub, self.cdtype, self.data_shape)
        out = self._data() if out is None else out
        _check(lib().lam_forward_hat(self._h, _ptr(u), _ptr(out), _ptr(sub), _ptr(self.ws), _stream()),
               "lam_forward_hat")
        return out

    def adjoint_hat(self, d_hat, out=None):
        d_hat = self._inp(d_hat, self.cdtype, self.data_shape)
        out = self._vol() if out is None else out
        _check(lib().lam_adjoint_hat(self._h, _ptr(d_hat), _ptr(out), _ptr(self.ws), _stream()),
               "lam_adjoint_hat")
        return out

    def fbp(self, d, out=None):
        """FBP-style single pass: Re L_hat^H of the ramp-filtered F_2D d (lam_fbp)."""
        self._need_full("fbp")
        d = self._inp(d, self.cdtype, self.data_shape)
        out = self._vol() if out is None else out
        _check(lib().lam_fbp(self._h, _ptr(d), _ptr(out), _ptr(self.ws), _stream()), "lam_fbp")
        return out

    def fft2d(self, x, inverse=False, out=None):
        x = self._inp(x, self.cdtype, self.data_shape)
        out = self._data() if out is None else out
        _check(lib().lam_fft2d(self._h, _ptr(x), _ptr(out), int(bool(inverse)), _stream()), "lam_fft2d")
        return out

    def tv_grad(self, u, out=None):
        u = self._inp(u, self.rdtype, self.vol_shape)
        out = torch.empty((3,) + self.vol_shape, dtype=self.rdtype, device=self.device) if out is None else out
        _check(lib().tv_grad(self._h, _ptr(u), _ptr(out), _stream()), "tv_grad")
        return out

    def tv_div(self, g, out=None):
        g = self._inp(g, self.rdtype, (3,) + self.vol_shape)
        out = self._vol() if out is None else out
        _check(lib().tv_div(self._h, _ptr(g), _ptr(out), _stream()), "tv_div")
        return out

    def tv_smooth(self, u, eps, grad=True):
        """(sum sqrt(|grad u|^2 + eps^2), -div(grad u / sqrt(|grad u|^2 + eps^2)) or None)."""
        u = self._inp(u, self.rdtype, self.vol_shape)
        g = self._vol() if grad else None
        val = ctypes.c_double()
        _check(lib().tv_smooth(self._h, _ptr(u), float(eps), _ptr(g), ctypes.byref(val), _ptr(self.ws), _stream()),
               "tv_smooth")
        return val.value, g

    # stages (u1 is complex [h][n][n], plane-major)
    def u1d_fwd(self, u):
        u = self._inp(u, self.rdtype, self.vol_shape)
        out = torch.empty((self.h, self.n, self.n), dtype=self.cdtype, device=self.device)
        _check(lib().lamx_u1d_fwd(self._h, _ptr(u), _ptr(out), _stream()), "lamx_u1d_fwd")
        return out

    def u1d_adj(self, u1):
        u1 = self._inp(u1, self.cdtype, (self.h, self.n, self.n))
        out = self._vol()
        _check(lib().lamx_u1d_adj(self._h, _ptr(u1), _ptr(out), _stream()), "lamx_u1d_adj")
        return out

    def u2d_fwd(self, u1, sub=None):
        u1 = self._inp(u1, self.cdtype, (self.h, self.n, self.n))
        if sub is not None:
            sub = self._inp(sub, self.cdtype, self.data_shape)
        out = self._data()
        _check(lib().lamx_u2d_fwd(self._h, _ptr(u1), _ptr(out), _ptr(sub), _ptr(self.ws), _stream()),
               "lamx_u2d_fwd")
        return out

    def u2d_fwd_static(self, u1, out, sub=None):
        """F_u2D into the caller's `out` through the library's static plane
        scratch (no workspace, no allocation inside the call).  The tensors
        are passed as they are: wrong dtype, device, layout or shape raises."""
        for t, dt, shape in ((u1, self.cdtype, (self.h, self.n, self.n)), (out, self.cdtype, self.data_shape),
                             (sub, self.cdtype, self.data_shape)):
            if t is None:
                continue
            if t.dtype != dt or t.device != self.device or not t.is_contiguous() or tuple(t.shape) != shape:
                raise LaminoError(f"expected a contiguous {dt} tensor of shape {shape} on {self.device}")
        _check(lib().lamx_u2d_fwd_static(self._h, _ptr(u1), _ptr(out), _ptr(sub), _stream()),
               "lamx_u2d_fwd_static")
        return out

    def u2d_adj(self, d_hat):
        d_hat = self._inp(d_hat, self.cdtype, self.data_shape)
        out = torch.empty((self.h, self.n, self.n), dtype=self.cdtype, device=self.device)
        _check(lib().lamx_u2d_adj(self._h, _ptr(d_hat), _ptr(out), _ptr(self.ws), _stream()), "lamx_u2d_adj")
        return out

    def plane_ffts(self, u1, P, j0=0):
        """The forward's plane FFTs alone for planes j0 .. j0 + len(P) - 1 of u1
        (u1 needs at least j0 + len(P) planes) into P [nb][2n][2n]."""
        _check(lib().lamx_plane_ffts(self._h, _ptr(u1), _ptr(P), int(j0), int(P.shape[0]), _stream()),
               "lamx_plane_ffts")
        return P

    def spread(self, d_hat, j0=0, nb=None):
        """The adjoint spread alone for plane jobs j0 .. j0 + nb - 1 (default: one
        operator batch) into the workspace planes; returns nb."""
        nb = lib().lamx_jobs_per_batch(self._h) if nb is None else int(nb)
        d_hat = self._inp(d_hat, self.cdtype, self.data_shape)
        _check(lib().lamx_spread(self._h, _ptr(d_hat), _ptr(self.ws), int(j0), nb, _stream()), "lamx_spread")
        return nb

    def job_planes(self, j0, nb):
        """Data planes (kv rows) plane jobs j0 .. j0 + nb - 1 cover."""
        return lib().lamx_job_planes(self._h, int(j0), int(nb))

    def set_memo(self, tau):
        """Memoization of F*_u2D per plane job in ADMM states created after this
        call (LAM_OPT_MEMO_TAU): reuse a job's cached plane when the cosine
        similarity of its keys exceeds tau; tau = 0 turns it off."""
        v = int(round(float(tau) * 10000))
        _check(lib().lam_plan_set_option(self._h, 8, v), "lam_plan_set_option")
        return self

    def set_exact_centre_jobs(self, count):
        """Plane jobs nearest the centre plane whose adjoint tile spread
        accumulates in exact fixed point (LAM_OPT_EXACT_CENTRE_JOBS)."""
        _check(lib().lam_plan_set_option(self._h, 7, int(count)), "lam_plan_set_option")
        return self

    def set_threads(self, z=None, fft=None):
        """Threads per block (256 or 512) of the z-stage kernels and of the
        plane row / column FFTs; the lines per block are picked again."""
        if z is not None:
            _check(lib().lam_plan_set_option(self._h, 4, int(z)), "lam_plan_set_option")
        if fft is not None:
            _check(lib().lam_plan_set_option(self._h, 5, int(fft)), "lam_plan_set_option")
        return self

    def autotune(self, reps=2):
        """Pick launch shapes by timing L_hat + L_hat^H (scratch buffers are
        allocated here); returns the best pair time in seconds."""
        u = self._vol().normal_()
        d = self._data()
        t = ctypes.c_double()
        _check(lib().lam_plan_autotune(self._h, _ptr(u), _ptr(d), _ptr(self.ws), int(reps), ctypes.byref(t),
                                       _stream()), "lam_plan_autotune")
        return t.value

    def status(self) -> int:
        """The plan's index-check status (lam_plan_status; synchronises):
        0, or LAM_EBOUNDS (-7) once a LAM_BOUNDS_CHECK build caught an index."""
        return lib().lam_plan_status(self._h, _stream())

    def info(self):
        arr = (ctypes.c_int * 14)()
        _check(lib().lamx_plan_info(self._h, arr, 14), "lamx_plan_info")
        keys = ["TY_fwd", "TY_adj", "rows_per_block", "cols_per_block", "tile", "images", "planes_per_batch",
                "jmin", "jmax", "plane_jobs", "gather_tile", "z_threads", "fft_threads", "spread"]
        out = dict(zip(keys, list(arr)))
        out["spread"] = {v: k for k, v in self.SPREADS.items()}[out["spread"]]
        return out


class LamOp(torch.autograd.Function):
    """d = L u as an autograd function; the backward is the hand-written
    adjoint kernel (Re L^H g, PyTorch's convention for a real input and a
    complex output).  Nothing is saved for the backward: the padded Fourier
    grids are recomputed inside the adjoint."""

    @staticmethod
    def forward(ctx, u, plan):
        ctx.plan = plan
        return plan.forward(u.detach())

    @staticmethod
    def backward(ctx, g):
        return ctx.plan.adjoint(g.contiguous()), None


class TVOp(torch.autograd.Function):
    """Smoothed isotropic TV(u) = sum sqrt(|grad u|^2 + eps^2); the backward is
    -div(grad u / sqrt(|grad u|^2 + eps^2)) from the TV kernel."""

    @staticmethod
    def forward(ctx, u, plan, eps):
        ctx.plan, ctx.eps = plan, eps
        ctx.save_for_backward(u)
        val, _ = plan.tv_smooth(u.detach(), eps, grad=False)
        return torch.tensor(val, dtype=torch.float64, device=u.device)

    @staticmethod
    def backward(ctx, g):
        (u,) = ctx.saved_tensors
        _, grad = ctx.plan.tv_smooth(u.detach(), ctx.eps, grad=True)
        return grad * g.to(grad.dtype), None, None


def lam(u, plan):
    """Differentiable L u."""
    return LamOp.apply(u, plan)


def tv(u, plan, eps=1e-3):
    """Differentiable smoothed TV(u) (float64 scalar tensor)."""
    return TVOp.apply(u, plan, eps)


class Admm:
    """ADMM-TV state on the device (caller-allocated through torch)."""

    def __init__(self, plan: Plan):
        plan._need_full("ADMM")
        self.plan = plan
        nb = ctypes.c_size_t()
        _check(lib().admm_state_bytes(plan._h, ctypes.byref(nb)), "admm_state_bytes")
        self.state = torch.empty(nb.value, dtype=torch.uint8, device=plan.device)
        self.iters = 0
        self._ready = None  # event recorded after init, on the stream init ran on

    def _order(self):
        # later calls may come on another stream (a capture stream for graph
        # replay): make it wait for the initialisation, which ran on the
        # stream current at init()
        if self._ready is not None:
            torch.cuda.current_stream(self.plan.device).wait_event(self._ready)

    RESID = {"carry": 0, "refresh": 1, "compensated": 2, "refresh+compensated": 3}

    def init(self, d, alpha, rho, n_inner=4, adapt_rho=True, form=2, resid=None):
        """form: the LSP form, 2 (Algorithm 2, default) or 1 (Algorithm 1).
        resid: how the Algorithm 2 residual is kept (LAM_OPT_RESIDUAL): "carry"
        (by linearity across LSPs), "refresh" (evaluated afresh at each LSP
        start), "compensated" (carried as a hi + lo pair) or both; None keeps
        the plan's setting (compensated for FP32, carry for FP64)."""
        d = self.plan._inp(d, self.plan.cdtype, self.plan.data_shape)
        if resid is not None and resid not in self.RESID:
            raise LaminoError(f"resid must be one of {sorted(self.RESID)}")
        _check(lib().lam_plan_set_option(self.plan._h, 3, int(form)), "lam_plan_set_option")
        if resid is not None:
            _check(lib().lam_plan_set_option(self.plan._h, 6, self.RESID[resid]), "lam_plan_set_option")
        _check(lib().admm_init(self.plan._h, _ptr(self.state), _ptr(d), float(alpha), float(rho), int(n_inner),
                               int(bool(adapt_rho)), _ptr(self.plan.ws), _stream()), "admm_init")
        self.iters = 0
        self._ready = torch.cuda.Event()
        self._ready.record(torch.cuda.current_stream(self.plan.device))
        return self

    def step(self):
        self._order()
        _check(lib().admm_step(self.plan._h, _ptr(self.state), _ptr(self.plan.ws), _stream()), "admm_step")
        self.iters += 1

    def run(self, iters, graph=False):
        self._order()
        _check(lib().admm_run(self.plan._h, _ptr(self.state), _ptr(self.plan.ws), int(iters), int(bool(graph)),
                              _stream()), "admm_run")
        self.iters += iters

    @property
    def u(self) -> torch.Tensor:
        """The volume u inside the state (a view; no copy)."""
        p = self.plan
        off = lib().admm_u(p._h, _ptr(self.state)) - self.state.data_ptr()
        esz = 4 if p.prec == "f32" else 8
        n = p.n * p.nz * p.n
        return self.state[off:off + n * esz].view(p.rdtype).view(p.vol_shape)

    def scalars(self) -> dict:
        arr = (ctypes.c_double * NSCALARS)()
        _check(lib().admm_read_scalars(self.plan._h, _ptr(self.state), arr, _stream()), "admm_read_scalars")
        return {k: arr[i] for k, i in SC.items()}

    def history(self, count=None) -> np.ndarray:
        count = self.iters if count is None else count
        arr = (ctypes.c_double * (4 * max(count, 1)))()
        _check(lib().admm_read_history(self.plan._h, _ptr(self.state), count, arr, _stream()),
               "admm_read_history")
        return np.frombuffer(arr, dtype=np.float64)[: 4 * count].reshape(count, 4).copy()

    LAYOUT = ["sc", "hist", "partials", "counter", "u", "du", "Gd", "G", "G_prev", "p", "e", "lam", "dpsi",
              "d_hat", "r", "Lp", "r_lo", "total"]

    def arrays(self) -> dict:
        """Views (no copies) of the state's pieces by name: the FP64 scalars
        and history, the volumes (u, du, Gd, G, G_prev, p; e, lam, dpsi with a
        leading axis of 3) and the data arrays (d_hat, r, Lp, r_lo)."""
        p = self.plan
        arr = (ctypes.c_size_t * len(self.LAYOUT))()
        _check(lib().lamx_admm_layout(p._h, arr, len(self.LAYOUT)), "lamx_admm_layout")
        off = dict(zip(self.LAYOUT, list(arr)))
        vol, dat = p.vol_shape, p.data_shape
        rsz, csz = (4, 8) if p.prec == "f32" else (8, 16)
        nv, nd = p.n * p.nz * p.n, p.T * p.h * p.w

        def view(name, count, esz, dtype, shape):
            o = off[name]
            return self.state[o:o + count * esz].view(dtype).view(shape)
        out = {"sc": view("sc", 64, 8, torch.float64, (64,)), "hist": view("hist", 4096 * 4, 8, torch.float64,
                                                                           (4096, 4))}
        for k in ("u", "du", "Gd", "G", "G_prev", "p"):
            out[k] = view(k, nv, rsz, p.rdtype, vol)
        for k in ("e", "lam", "dpsi"):
            out[k] = view(k, 3 * nv, rsz, p.rdtype, (3,) + vol)
        for k in ("d_hat", "r", "Lp", "r_lo"):
            out[k] = view(k, nd, csz, p.cdtype, dat)
        return out

    def log_jsonl(self, path, **extra) -> int:
        """Append one JSON line per outer iteration done so far (iteration,
        objective, rho used, primal and dual residuals, plus `extra` keys) to
        `path`; returns the number of lines written (synchronises)."""
        import json
        h = self.history()
        with open(path, "a", encoding="utf-8") as f:
            for k, (obj, rho, r, s) in enumerate(h):
                f.write(json.dumps({"iter": k + 1, "objective": obj, "rho": rho, "r": r, "s": s, **extra}) + "\n")
        return len(h)

    def graph_kernels(self) -> int:
        """Kernel launches per outer iteration in the captured graph (0 before a graph run)."""
        n = ctypes.c_size_t()
        _check(lib().lamx_admm_graph_kernels(self.plan._h, _ptr(self.state), ctypes.byref(n)),
               "lamx_admm_graph_kernels")
        return n.value

    def status(self) -> int:
        return lib().admm_status(self.plan._h, _ptr(self.state), _stream())


def fma_peak(device=None) -> float:
    """Measured FP32 FMA throughput of the device (flop/s)."""
    dev = torch.device("cuda" if device is None else device)
    sink = torch.empty(8 * torch.cuda.get_device_properties(dev).multi_processor_count, dtype=torch.float32,
                       device=dev)
    out = ctypes.c_double()
    with torch.cuda.device(dev):
        _check(lib().lamx_fma_peak(_ptr(sink), sink.numel(), ctypes.byref(out), _stream()), "lamx_fma_peak")
    return out.value


def _ptr_array(items):
    return (ctypes.c_void_p * len(items))(*[t.data_ptr() if isinstance(t, torch.Tensor) else t for t in items])


class Batch:
    """Several plans run together (lam_batch_create): every plane-stage step of
    the batched L_hat / L_hat^H is one persistent launch over all problems;
    admm_run runs the problems concurrently on side streams by default
    (set_streams)."""

    STAGES = ["z_fwd", "row_fwd", "col_fwd", "gather", "spread", "col_adj", "row_adj", "z_adj"]

    def __init__(self, plans):
        self.plans = list(plans)
        hs = (ctypes.c_void_p * len(self.plans))(*[p._h.value for p in self.plans])
        ws = _ptr_array([p.ws for p in self.plans])
        h_ = ctypes.c_void_p()
        _check(lib().lam_batch_create(ctypes.byref(h_), hs, ws, len(self.plans)), "lam_batch_create")
        self._h = h_

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib is not None:
            _lib.lam_batch_destroy(h)

    def _run(self, name, xs, in_kind, out_kind):
        xs = [p._inp(x, p.rdtype if in_kind == "vol" else p.cdtype, p.vol_shape if in_kind == "vol" else p.data_shape)
              for p, x in zip(self.plans, xs)]
        outs = [p._vol() if out_kind == "vol" else p._data() for p in self.plans]
        _check(getattr(lib(), name)(self._h, _ptr_array(xs), _ptr_array(outs), _stream()), name)
        return outs

    def forward_hat(self, us):
        return self._run("lam_forward_hat_batched", us, "vol", "data")

    def adjoint_hat(self, ds):
        return self._run("lam_adjoint_hat_batched", ds, "data", "vol")

    def forward(self, us):
        return self._run("lam_forward_batched", us, "vol", "data")

    def adjoint(self, ds):
        return self._run("lam_adjoint_batched", ds, "data", "vol")

    def admm_run(self, admms, iters, graph=False):
        """`iters` outer iterations of every Admm (one per plan, same order)."""
        if len(admms) != len(self.plans) or any(a.plan is not p for a, p in zip(admms, self.plans)):
            raise LaminoError("one Admm per plan of the batch, in order")
        for a in admms:
            a._order()
        _check(lib().admm_run_batched(self._h, _ptr_array([a.state for a in admms]), int(iters), int(bool(graph)),
                                      _stream()), "admm_run_batched")
        for a in admms:
            a.iters += iters

    def set_streams(self, streams):
        """Concurrent mode of admm_run (lam_batch_set_streams): 0 = persistent
        batched stages; k >= 1 = each problem's own outer iteration, problem i
        on side stream i mod k."""
        _check(lib().lam_batch_set_streams(self._h, int(streams)), "lam_batch_set_streams")
        return self

    def info(self):
        arr = (ctypes.c_int * 17)()
        _check(lib().lamx_batch_info(self._h, arr, 17), "lamx_batch_info")
        out = {st: {"work": arr[2 * k], "grid": arr[2 * k + 1]} for k, st in enumerate(self.STAGES)}
        out["graph_kernels"] = arr[16]
        return out


def reconstruct(data, theta, phi, n, nz, iters, alpha, rho):
    """One-call FP32 ADMM-TV (4 CG steps per iteration) from real data [T][h][w].

    data may be a numpy array (host) or a CUDA tensor; returns u with the same
    kind of storage."""
    theta = np.ascontiguousarray(np.asarray(theta, dtype=np.float64))
    if isinstance(data, torch.Tensor) and data.is_cuda:
        d = data.to(torch.float32).contiguous()
        out = torch.empty((n, nz, n), dtype=torch.float32, device=d.device)
        dp, op = ctypes.c_void_p(d.data_ptr()), ctypes.c_void_p(out.data_ptr())
    else:
        d = np.ascontiguousarray(np.asarray(data, dtype=np.float32))
        out = np.empty((n, nz, n), dtype=np.float32)
        dp, op = ctypes.c_void_p(d.ctypes.data), ctypes.c_void_p(out.ctypes.data)
    T, h, w = d.shape
    _check(lib().reconstruct(dp, theta.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), float(phi), int(n), int(nz),
                             int(h), int(w), int(T), int(iters), float(alpha), float(rho), op), "reconstruct")
    return out
