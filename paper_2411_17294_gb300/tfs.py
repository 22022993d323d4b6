"""Thin ctypes binding of libtfs.so (include/tfs.h) plus a torch-facing wrapper.

Every function of the C ABI is exposed under its own name with the same
arguments (pointers as ints, streams as ints).  ``Solver`` marshals torch
tensors (device memory, streams) into those calls; all arithmetic of the step
runs in the library's CUDA kernels.  There is no CPU fallback: loading fails
with an error when libtfs.so has not been built or no CUDA device exists.
"""
from __future__ import annotations

import ctypes
import math
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libtfs.so")

# status codes (include/tfs.h)
TFS_OK, TFS_ERR_ARG, TFS_ERR_NOSOE, TFS_ERR_UNSTABLE, TFS_ERR_CUDA, TFS_ERR_STATE, TFS_ERR_NOWORKSPACE, \
    TFS_ERR_FORMAT, TFS_ERR_TOOBIG = range(9)
TFS_FP64, TFS_FP32, TFS_FP32_PLAIN = 0, 1, 2
(TFS_PARAM_RE, TFS_PARAM_EPS, TFS_PARAM_STENCIL, TFS_PARAM_TRANSPORT, TFS_PARAM_UMAX, TFS_PARAM_KRYLOV_TOL,
 TFS_PARAM_KRYLOV_MAXIT, TFS_PARAM_START, TFS_PARAM_FORM) = range(9)
TFS_START_BDF2, TFS_START_SDIRK2 = 0, 1
TFS_FORM_STRESS, TFS_FORM_PAPER = 0, 1
TFS_STENCIL_UPWIND3, TFS_STENCIL_CENTRAL2 = 0, 1
TFS_FLAG_NONFINITE, TFS_FLAG_SINGULAR, TFS_FLAG_COURANT, TFS_FLAG_TIMEOUT, TFS_FLAG_NOCONV = 1, 2, 4, 8, 16

EXPORTS = [
    "tfs_create", "tfs_set_param", "tfs_set_soe", "tfs_transport_limit", "tfs_workspace_bytes", "tfs_bind_workspace",
    "tfs_set_state", "tfs_step", "tfs_get_stress", "tfs_set_step_events", "tfs_step_index", "tfs_last_solve", "tfs_checkpoint_bytes", "tfs_save",
    "tfs_load", "tfs_adjoint_workspace_bytes", "tfs_bind_adjoint_workspace", "tfs_backward", "tfs_status",
    "tfs_strerror", "tfs_destroy", "tfs_run_static", "tfs_static_status", "tfs_check_wait_bound",
    "tfs_halo_bytes", "tfs_get_halo", "tfs_step_slab",
    "tfs_ns_create", "tfs_ns_workspace_bytes", "tfs_ns_bind_workspace", "tfs_ns_set_state", "tfs_ns_step",
    "tfs_ns_destroy",
]


class TfsGrid(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int * 3), ("L", ctypes.c_double * 3)]


class TfsError(RuntimeError):
    def __init__(self, code: int, where: str):
        super().__init__(f"{where}: {strerror(code)} (status {code})")
        self.code = code


_lib = None


def load_library(path: str | None = None):
    """Load libtfs.so and declare the C signatures.  Raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"libtfs.so not built ({p}); run paper_2411_17294_gb300.build.build()")
    lib = ctypes.CDLL(p)
    vp, sz, dp = ctypes.c_void_p, ctypes.c_size_t, ctypes.POINTER(ctypes.c_double)
    H = ctypes.c_void_p
    sig = {
        "tfs_create": (ctypes.c_int, [ctypes.POINTER(H), ctypes.POINTER(TfsGrid), ctypes.c_double, ctypes.c_double,
                                      ctypes.c_double, ctypes.c_int, ctypes.c_double, ctypes.c_int]),
        "tfs_set_param": (ctypes.c_int, [H, ctypes.c_int, ctypes.c_double]),
        "tfs_set_soe": (ctypes.c_int, [H, dp, dp, ctypes.c_int]),
        "tfs_transport_limit": (ctypes.c_int, [H, dp]),
        "tfs_workspace_bytes": (sz, [H]),
        "tfs_bind_workspace": (ctypes.c_int, [H, vp, sz]),
        "tfs_set_state": (ctypes.c_int, [H, vp, vp]),
        "tfs_step": (ctypes.c_int, [H, vp, vp, vp, vp]),
        "tfs_get_stress": (ctypes.c_int, [H, vp, vp]),
        "tfs_set_step_events": (ctypes.c_int, [H, vp, vp]),
        "tfs_step_index": (ctypes.c_long, [H]),
        "tfs_last_solve": (ctypes.c_int, [H, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)]),
        "tfs_checkpoint_bytes": (sz, [H]),
        "tfs_save": (ctypes.c_int, [H, vp, vp]),
        "tfs_load": (ctypes.c_int, [H, vp, vp]),
        "tfs_adjoint_workspace_bytes": (sz, [H, ctypes.c_int]),
        "tfs_bind_adjoint_workspace": (ctypes.c_int, [H, vp, sz]),
        "tfs_backward": (ctypes.c_int, [H, vp, ctypes.POINTER(vp), ctypes.c_int, ctypes.c_int, vp, vp, vp, vp,
                                        dp, dp, vp]),
        "tfs_status": (ctypes.c_int, [H, ctypes.POINTER(ctypes.c_uint)]),
        "tfs_strerror": (ctypes.c_char_p, [ctypes.c_int]),
        "tfs_destroy": (ctypes.c_int, [H]),
        "tfs_check_wait_bound": (ctypes.c_int, [ctypes.POINTER(ctypes.c_uint), dp, vp]),
        "tfs_run_static": (ctypes.c_int, [ctypes.POINTER(TfsGrid), ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                          ctypes.c_int, ctypes.c_double, ctypes.c_int, dp, dp, vp, vp, vp,
                                          ctypes.c_int, vp, vp]),
        "tfs_static_status": (ctypes.c_int, [ctypes.POINTER(ctypes.c_uint), vp]),
        "tfs_halo_bytes": (sz, [H]),
        "tfs_get_halo": (ctypes.c_int, [H, vp, vp, vp]),
        "tfs_step_slab": (ctypes.c_int, [H, vp, vp, vp, vp, vp, vp]),
        "tfs_ns_create": (ctypes.c_int, [ctypes.POINTER(H), ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                         ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                         ctypes.c_int]),
        "tfs_ns_workspace_bytes": (sz, [H]),
        "tfs_ns_bind_workspace": (ctypes.c_int, [H, vp, sz]),
        "tfs_ns_set_state": (ctypes.c_int, [H, vp, vp, vp]),
        "tfs_ns_step": (ctypes.c_int, [H, vp, vp, vp, vp]),
        "tfs_ns_destroy": (ctypes.c_int, [H]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def strerror(code: int) -> str:
    try:
        return load_library().tfs_strerror(code).decode()
    except Exception:  # pragma: no cover - library missing
        return f"status {code}"


def check(code: int, where: str) -> None:
    if code != TFS_OK:
        raise TfsError(code, where)


# ------------------------------------------------------------- torch wrapper
def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("no CUDA device: libtfs runs only on the GPU")
    return torch


def _stream_ptr(stream) -> int:
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


class Solver:
    """One stress problem on the current CUDA device.

    Owns a handle and a torch-allocated workspace; fields are torch tensors of
    the precision's dtype, shaped [nc, N] (stress), [d*d, N] (velocity
    gradient) and [d, N] (velocity).

    transport: False (pointwise law), True (explicit, extrapolated) or
    "implicit" (inside a Krylov solve, eq. FP_discrete); start: "bdf2" (empty
    past) or "sdirk2" (Section 5.1); form: "stress" or "paper" (the paper's
    variable Phi with stress Psi = D^{1-alpha} Phi, Section 3.4; the SOE table
    then approximates g_alpha, i.e. the kernel of order 1 - alpha)."""

    def __init__(self, dim: int, n, alpha: float, Wi: float, beta: float, dt: float, m: int = 0,
                 precision: int = TFS_FP64, L=None, mu=None, w=None, Re: float = 1.0, eps: float = 0.0,
                 stencil: int = TFS_STENCIL_UPWIND3, transport=True, device=None, start: str = "bdf2",
                 form: str = "stress"):
        torch = _torch()
        lib = load_library()
        self.lib = lib
        self.dim = dim
        self.n = tuple(int(k) for k in n)
        self.N = int(math.prod(self.n))
        self.nc = 3 if dim == 2 else 6
        self.precision = precision
        self.dtype = torch.float64 if precision == TFS_FP64 else torch.float32
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        g = TfsGrid()
        g.dim = dim
        Ls = list(L) if L is not None else [2 * math.pi] * dim
        for a in range(3):
            g.n[a] = self.n[a] if a < dim else 1
            g.L[a] = float(Ls[a]) if a < dim else 1.0
        h = ctypes.c_void_p()
        check(lib.tfs_create(ctypes.byref(h), ctypes.byref(g), float(alpha), float(Wi), float(beta), int(m),
                             float(dt), int(precision)), "tfs_create")
        self.h = h
        self.m = m
        # transport: False (pointwise), True (explicit) or "implicit"
        self.implicit = transport == "implicit"
        self.transport = bool(transport)
        check(lib.tfs_set_param(h, TFS_PARAM_RE, float(Re)), "tfs_set_param(Re)")
        check(lib.tfs_set_param(h, TFS_PARAM_EPS, float(eps)), "tfs_set_param(eps)")
        check(lib.tfs_set_param(h, TFS_PARAM_STENCIL, float(stencil)), "tfs_set_param(stencil)")
        check(lib.tfs_set_param(h, TFS_PARAM_TRANSPORT, 2.0 if self.implicit else (1.0 if transport else 0.0)),
              "tfs_set_param(transport)")
        # first step: "bdf2" (empty past) or "sdirk2" (Section 5.1; alpha < 1, transport off or implicit)
        if start not in ("bdf2", "sdirk2"):
            raise ValueError("start must be 'bdf2' or 'sdirk2'")
        self.start = start
        check(lib.tfs_set_param(h, TFS_PARAM_START, float(TFS_START_SDIRK2 if start == "sdirk2" else TFS_START_BDF2)),
              "tfs_set_param(start)")
        # variable carried: "stress" or "paper" (Phi with Psi = D^{1-alpha} Phi, Section 3.4; the SOE
        # then approximates g_alpha, i.e. the kernel of order 1 - alpha; transport off)
        if form not in ("stress", "paper"):
            raise ValueError("form must be 'stress' or 'paper'")
        self.form = form
        check(lib.tfs_set_param(h, TFS_PARAM_FORM, float(TFS_FORM_PAPER if form == "paper" else TFS_FORM_STRESS)),
              "tfs_set_param(form)")
        if mu is not None:
            self.set_soe(mu, w)
        nbytes = lib.tfs_workspace_bytes(h)
        with torch.cuda.device(self.device):
            self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        base = self.workspace.data_ptr()
        off = (-base) % 256
        check(lib.tfs_bind_workspace(h, ctypes.c_void_p(base + off), nbytes), "tfs_bind_workspace")
        self._adj_ws = None

    def set_soe(self, mu, w):
        import numpy as np
        mu = np.ascontiguousarray(mu, dtype=np.float64)
        w = np.ascontiguousarray(w, dtype=np.float64)
        dp = ctypes.POINTER(ctypes.c_double)
        check(self.lib.tfs_set_soe(self.h, mu.ctypes.data_as(dp), w.ctypes.data_as(dp), len(mu)), "tfs_set_soe")

    def transport_limit(self) -> float:
        """Largest stable velocity bound U (see tfs_transport_limit)."""
        v = ctypes.c_double(0.0)
        check(self.lib.tfs_transport_limit(self.h, ctypes.byref(v)), "tfs_transport_limit")
        return v.value

    def _field(self, t, rows):
        if t is None:
            return None
        torch = _torch()
        if not isinstance(t, torch.Tensor):
            t = torch.as_tensor(t)
        t = t.to(device=self.device, dtype=self.dtype).reshape(rows, self.N).contiguous()
        return t

    def set_state(self, sigma0=None, stream=None):
        s0 = self._field(sigma0, self.nc)
        self._keep = s0
        check(self.lib.tfs_set_state(self.h, ctypes.c_void_p(s0.data_ptr() if s0 is not None else 0),
                                     ctypes.c_void_p(_stream_ptr(stream))), "tfs_set_state")

    def step(self, grad_u_n, grad_u_nm1=None, u=None, stream=None):
        """One step.  Tensors must already be contiguous device tensors of the
        right dtype (no copies are made here on the hot path)."""
        kn = grad_u_n.data_ptr()
        knm1 = grad_u_nm1.data_ptr() if grad_u_nm1 is not None else 0
        up = u.data_ptr() if u is not None else 0
        check(self.lib.tfs_step(self.h, ctypes.c_void_p(kn), ctypes.c_void_p(knm1), ctypes.c_void_p(up),
                                ctypes.c_void_p(_stream_ptr(stream))), "tfs_step")

    def halo_buffers(self):
        """Two halo buffers (lo, hi) for a slab of this handle's grid:
        [2 levels][nc][2 planes][plane points] tensors of the handle's dtype."""
        torch = _torch()
        count = self.lib.tfs_halo_bytes(self.h) // (8 if self.dtype == torch.float64 else 4)
        return (torch.empty(count, dtype=self.dtype, device=self.device),
                torch.empty(count, dtype=self.dtype, device=self.device))

    def get_halo(self, lo, hi, stream=None):
        """The slab's own boundary planes as its neighbours need them (tfs_get_halo)."""
        check(self.lib.tfs_get_halo(self.h, ctypes.c_void_p(lo.data_ptr() if lo is not None else 0),
                                    ctypes.c_void_p(hi.data_ptr() if hi is not None else 0),
                                    ctypes.c_void_p(_stream_ptr(stream))), "tfs_get_halo")

    def step_slab(self, grad_u_n, grad_u_nm1, u, halo_lo, halo_hi, stream=None):
        """One step of a slab with the neighbours' boundary planes (tfs_step_slab)."""
        knm1 = grad_u_nm1.data_ptr() if grad_u_nm1 is not None else 0
        up = u.data_ptr() if u is not None else 0
        check(self.lib.tfs_step_slab(self.h, ctypes.c_void_p(grad_u_n.data_ptr()), ctypes.c_void_p(knm1),
                                     ctypes.c_void_p(up), ctypes.c_void_p(halo_lo.data_ptr()),
                                     ctypes.c_void_p(halo_hi.data_ptr()), ctypes.c_void_p(_stream_ptr(stream))),
              "tfs_step_slab")

    def stress(self, stream=None):
        torch = _torch()
        out = torch.empty((self.nc, self.N), dtype=self.dtype, device=self.device)
        check(self.lib.tfs_get_stress(self.h, ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(_stream_ptr(stream))),
              "tfs_get_stress")
        return out

    def set_step_events(self, ev_before, ev_after):
        """Record torch.cuda.Event objects around the step kernel of each later
        step (None, None turns it off).  torch creates an event's handle on its
        first record, so each event must have been recorded once before."""
        def handle(ev):
            if ev is None:
                return 0
            if not ev.cuda_event:
                raise ValueError("set_step_events: record the event once first (torch creates it lazily)")
            return ev.cuda_event
        b = ctypes.c_void_p(handle(ev_before))
        a = ctypes.c_void_p(handle(ev_after))
        check(self.lib.tfs_set_step_events(self.h, b, a), "tfs_set_step_events")

    def last_solve(self):
        """(iterations, relative residual) of the last implicit-transport solve:
        a step's, or after backward() the last reverse step's transposed solve."""
        it = ctypes.c_int(0)
        rr = ctypes.c_double(0.0)
        check(self.lib.tfs_last_solve(self.h, ctypes.byref(it), ctypes.byref(rr)), "tfs_last_solve")
        return it.value, rr.value

    def set_krylov(self, tol=None, maxit=None):
        """Implicit transport: relative residual target and iteration limit."""
        if tol is not None:
            check(self.lib.tfs_set_param(self.h, TFS_PARAM_KRYLOV_TOL, float(tol)), "tfs_set_param(tol)")
        if maxit is not None:
            check(self.lib.tfs_set_param(self.h, TFS_PARAM_KRYLOV_MAXIT, float(maxit)), "tfs_set_param(maxit)")

    def step_index(self) -> int:
        return int(self.lib.tfs_step_index(self.h))

    def status(self) -> int:
        v = ctypes.c_uint(0)
        check(self.lib.tfs_status(self.h, ctypes.byref(v)), "tfs_status")
        return int(v.value)

    def checkpoint_bytes(self) -> int:
        return int(self.lib.tfs_checkpoint_bytes(self.h))

    def new_checkpoint(self):
        torch = _torch()
        return torch.empty(self.checkpoint_bytes(), dtype=torch.uint8, device=self.device)

    def save(self, buf, stream=None):
        check(self.lib.tfs_save(self.h, ctypes.c_void_p(buf.data_ptr()), ctypes.c_void_p(_stream_ptr(stream))),
              "tfs_save")

    def load(self, buf, stream=None):
        check(self.lib.tfs_load(self.h, ctypes.c_void_p(buf.data_ptr()), ctypes.c_void_p(_stream_ptr(stream))),
              "tfs_load")

    def ensure_adjoint_workspace(self, segment_steps: int):
        torch = _torch()
        need = int(self.lib.tfs_adjoint_workspace_bytes(self.h, int(segment_steps)))
        if self._adj_ws is None or self._adj_ws.numel() < need + 256:
            self._adj_ws = torch.empty(need + 256, dtype=torch.uint8, device=self.device)
        base = self._adj_ws.data_ptr()
        off = (-base) % 256
        check(self.lib.tfs_bind_adjoint_workspace(self.h, ctypes.c_void_p(base + off), need),
              "tfs_bind_adjoint_workspace")

    def backward(self, dJ_dsigma_T, checkpoints, K: int, steps: int, grad_u, u=None, stream=None):
        """Gradients of J for a frozen-gradient run of `steps` steps; returns
        (dJ/dsigma0 [nc,N] f64, dJ/dgrad_u [d*d,N] f64, dJ/dWi, dJ/dbeta)."""
        torch = _torch()
        self.ensure_adjoint_workspace(K)
        g_s0 = torch.empty((self.nc, self.N), dtype=torch.float64, device=self.device)
        g_k = torch.empty((self.dim * self.dim, self.N), dtype=torch.float64, device=self.device)
        dJ = self._field(dJ_dsigma_T, self.nc)
        arr = (ctypes.c_void_p * len(checkpoints))(*[ctypes.c_void_p(c.data_ptr()) for c in checkpoints])
        gWi = ctypes.c_double(0.0)
        gb = ctypes.c_double(0.0)
        check(self.lib.tfs_backward(self.h, ctypes.c_void_p(dJ.data_ptr()), arr, int(K), int(steps),
                                    ctypes.c_void_p(grad_u.data_ptr()),
                                    ctypes.c_void_p(u.data_ptr() if u is not None else 0),
                                    ctypes.c_void_p(g_s0.data_ptr()), ctypes.c_void_p(g_k.data_ptr()),
                                    ctypes.byref(gWi), ctypes.byref(gb), ctypes.c_void_p(_stream_ptr(stream))),
              "tfs_backward")
        return g_s0, g_k, gWi.value, gb.value

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            self.lib.tfs_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass


class NSSolver:
    """The Navier-Stokes projection step on the periodic square (tfs_ns_*): the
    velocity the stress is coupled to.  Fields are torch tensors of the
    precision's dtype: velocity [2, N], gradient [4, N], stress [3, N]."""

    def __init__(self, n, L, beta: float, Re: float, dt: float, precision: int = TFS_FP64, device=None):
        torch = _torch()
        lib = load_library()
        self.lib = lib
        self.n = (int(n[0]), int(n[1]))
        self.N = self.n[0] * self.n[1]
        self.dtype = torch.float64 if precision == TFS_FP64 else torch.float32
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        h = ctypes.c_void_p()
        check(lib.tfs_ns_create(ctypes.byref(h), self.n[0], self.n[1], float(L[0]), float(L[1]), float(beta),
                                float(Re), float(dt), int(precision)), "tfs_ns_create")
        self.h = h
        nbytes = lib.tfs_ns_workspace_bytes(h)
        with torch.cuda.device(self.device):
            self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        base = self.workspace.data_ptr()
        check(lib.tfs_ns_bind_workspace(h, ctypes.c_void_p(base + (-base) % 256), nbytes), "tfs_ns_bind_workspace")

    def _dev(self, t, rows):
        torch = _torch()
        return torch.as_tensor(t).to(device=self.device, dtype=self.dtype).reshape(rows, self.N).contiguous()

    def set_state(self, u0, u_prev=None, stream=None):
        u0 = self._dev(u0, 2)
        up = None if u_prev is None else self._dev(u_prev, 2)
        check(self.lib.tfs_ns_set_state(self.h, ctypes.c_void_p(u0.data_ptr()),
                                        ctypes.c_void_p(up.data_ptr() if up is not None else 0),
                                        ctypes.c_void_p(_stream_ptr(stream))), "tfs_ns_set_state")
        self._keep = (u0, up)

    def step(self, sigma=None, u_out=None, grad_u_out=None, stream=None):
        """One step with the stress sigma^n (None: no stress); returns (u, kappa)."""
        torch = _torch()
        if u_out is None:
            u_out = torch.empty((2, self.N), dtype=self.dtype, device=self.device)
        if grad_u_out is None:
            grad_u_out = torch.empty((4, self.N), dtype=self.dtype, device=self.device)
        sp = 0 if sigma is None else sigma.data_ptr()
        check(self.lib.tfs_ns_step(self.h, ctypes.c_void_p(sp), ctypes.c_void_p(u_out.data_ptr()),
                                   ctypes.c_void_p(grad_u_out.data_ptr()), ctypes.c_void_p(_stream_ptr(stream))),
              "tfs_ns_step")
        return u_out, grad_u_out

    def close(self):
        if self.h:
            self.lib.tfs_ns_destroy(self.h)
            self.h = None
