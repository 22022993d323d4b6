"""ctypes wrapper around the plain-C FP64 oracle (test infrastructure only).

``Oracle`` holds the state of the discrete scheme stated in ``tfs_oracle.c``
(stress levels n and n-1, SOE modes at levels n and n-1, step counter) as FP64
NumPy arrays and advances it with ``orc_step``.  ``gradients`` runs the forward
scheme while keeping the stress history and then applies ``orc_adjoint_step``
backwards, giving the derivatives of a functional of the final stress with
respect to Wi, beta, sigma0 and the velocity gradient.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys
from dataclasses import dataclass, field

import numpy as np

from .paper_form import packed_pairs, transport_op, upper_convected

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tfs_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libtfs_oracle.so")


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (-O2, no FP contraction, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC",
               "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class _Params(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int),
        ("n", ctypes.c_int * 3),
        ("L", ctypes.c_double * 3),
        ("alpha", ctypes.c_double),
        ("Wi", ctypes.c_double),
        ("beta", ctypes.c_double),
        ("Re", ctypes.c_double),
        ("eps", ctypes.c_double),
        ("dt", ctypes.c_double),
        ("m", ctypes.c_int),
        ("stencil", ctypes.c_int),
        ("transport", ctypes.c_int),
        ("full", ctypes.c_int),
    ]


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        lib.orc_step.restype = ctypes.c_int
        lib.orc_step.argtypes = [ctypes.POINTER(_Params), dp, dp, ctypes.c_long,
                                 dp, dp, dp, dp, dp, dp, dp, dp, dp, dp]
        lib.orc_first_step_sdirk2.restype = ctypes.c_int
        lib.orc_first_step_sdirk2.argtypes = [ctypes.POINTER(_Params), dp, dp, dp, dp, dp, dp, dp, dp, dp]
        lib.orc_step_implicit.restype = ctypes.c_int
        lib.orc_step_implicit.argtypes = lib.orc_step.argtypes
        lib.orc_adjoint_step.restype = ctypes.c_int
        lib.orc_adjoint_step.argtypes = [ctypes.POINTER(_Params), dp, dp, ctypes.c_long,
                                         dp, dp, dp, dp, dp,
                                         dp, dp, dp, dp,
                                         dp, dp, dp, dp,
                                         dp, dp, dp, dp, dp]
        _lib = lib
    return _lib


def _ptr(a):
    if a is None:
        return ctypes.POINTER(ctypes.c_double)()
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


@dataclass
class Problem:
    """Parameters of the discrete scheme (names follow the paper)."""
    dim: int
    n: tuple                    # grid points per axis (len dim)
    alpha: float
    Wi: float
    beta: float
    dt: float
    mu: np.ndarray = field(default_factory=lambda: np.zeros(0))   # SOE exponents
    w: np.ndarray = field(default_factory=lambda: np.zeros(0))    # SOE weights
    L: tuple = None             # box lengths, default 2*pi per axis
    Re: float = 1.0
    eps: float = 0.0
    stencil: int = 0            # 0 upwind3 (radius 2), 1 central2 (radius 1)
    transport: bool = False
    full: bool = False          # store the full d x d tensor instead of packed
    implicit: bool = False      # transport at t_{n+1} inside a global solve (small grids)
    start: str = "bdf2"         # first step: "bdf2" (empty past) or "sdirk2" (Section 5.1; alpha < 1)

    @property
    def N(self) -> int:
        return int(np.prod(self.n))

    @property
    def nc(self) -> int:
        if self.full:
            return self.dim * self.dim
        return 3 if self.dim == 2 else 6

    @property
    def m(self) -> int:
        return 0 if self.alpha == 1.0 else int(len(self.mu))

    def cparams(self) -> _Params:
        p = _Params()
        p.dim = self.dim
        nn = list(self.n) + [1] * (3 - len(self.n))
        L = list(self.L) if self.L is not None else [2 * np.pi] * self.dim
        L = L + [1.0] * (3 - len(L))
        for i in range(3):
            p.n[i] = int(nn[i])
            p.L[i] = float(L[i])
        p.alpha, p.Wi, p.beta, p.Re, p.eps, p.dt = (float(self.alpha), float(self.Wi), float(self.beta),
                                                    float(self.Re), float(self.eps), float(self.dt))
        p.m = self.m
        p.stencil = int(self.stencil)
        p.transport = int(bool(self.transport))
        p.full = int(bool(self.full))
        return p


class Oracle:
    """FP64 state of the scheme on the whole grid, advanced step by step."""

    def __init__(self, prob: Problem, sigma0: np.ndarray | None = None):
        self.prob = prob
        self._p = prob.cparams()
        self.mu = np.ascontiguousarray(prob.mu, dtype=np.float64)
        self.w = np.ascontiguousarray(prob.w, dtype=np.float64)
        nc, N, m = prob.nc, prob.N, prob.m
        self.sigma0 = (np.zeros((nc, N)) if sigma0 is None
                       else np.ascontiguousarray(sigma0, dtype=np.float64).reshape(nc, N).copy())
        # zero past: sigma^0 = sigma^{-1} = sigma0, modes^0 = modes^{-1} = 0
        self.sig_n = self.sigma0.copy()
        self.sig_nm1 = self.sigma0.copy()
        self.modes_n = np.zeros((max(m, 1), nc, N))
        self.modes_nm1 = np.zeros((max(m, 1), nc, N))
        self.n = 0
        self._kap_prev = None

    def step(self, kap_n: np.ndarray, kap_nm1: np.ndarray | None = None, u: np.ndarray | None = None) -> None:
        """Advance t_n -> t_{n+1}.  kap_nm1 defaults to the previous call's kap_n
        (first call: kap_n itself)."""
        prob = self.prob
        d, N = prob.dim, prob.N
        kap_n = np.ascontiguousarray(kap_n, dtype=np.float64).reshape(d * d, N)
        if kap_nm1 is None:
            kap_nm1 = self._kap_prev if self._kap_prev is not None else kap_n
        kap_nm1 = np.ascontiguousarray(kap_nm1, dtype=np.float64).reshape(d * d, N)
        if prob.transport:
            if u is None:
                raise ValueError("transport needs u")
            u = np.ascontiguousarray(u, dtype=np.float64).reshape(d, N)
        else:
            u = None
        sig_np1 = np.empty_like(self.sig_n)
        modes_np1 = np.zeros_like(self.modes_n)
        if prob.start == "sdirk2" and self.n == 0:
            sig_np1 = np.empty_like(self.sig_n)
            modes_np1 = np.zeros_like(self.modes_n)
            if _load().orc_first_step_sdirk2(ctypes.byref(self._p), _ptr(self.mu), _ptr(self.w), _ptr(self.sig_n),
                                             _ptr(self.modes_n), _ptr(self.sigma0), _ptr(kap_n), _ptr(u),
                                             _ptr(sig_np1), _ptr(modes_np1)):
                raise FloatingPointError("SDIRK2 start failed (alpha = 1, or a singular system)")
            self.sig_nm1, self.sig_n = self.sig_n, sig_np1
            self.modes_nm1, self.modes_n = self.modes_n, modes_np1
            self._kap_prev = kap_n
            self.n += 1
            return
        fn = _load().orc_step_implicit if prob.implicit else _load().orc_step
        fails = fn(ctypes.byref(self._p), _ptr(self.mu), _ptr(self.w), self.n,
                                 _ptr(self.sig_n), _ptr(self.sig_nm1), _ptr(self.modes_n), _ptr(self.modes_nm1),
                                 _ptr(self.sigma0), _ptr(kap_n), _ptr(kap_nm1), _ptr(u),
                                 _ptr(sig_np1), _ptr(modes_np1))
        if fails:
            raise FloatingPointError(f"{fails} singular point systems")
        self.sig_nm1, self.sig_n = self.sig_n, sig_np1
        self.modes_nm1, self.modes_n = self.modes_n, modes_np1
        self._kap_prev = kap_n
        self.n += 1

    def run(self, steps: int, kap, u=None) -> np.ndarray:
        """Run `steps` steps with a frozen velocity gradient (kap) or a callable
        n -> kap^n; returns the final stress [nc][N]."""
        for _ in range(steps):
            k = kap(self.n) if callable(kap) else kap
            km1 = (kap(self.n - 1) if self.n > 0 else k) if callable(kap) else kap
            self.step(k, km1, u)
        return self.sig_n.copy()


def forward(prob: Problem, sigma0, kap, u, steps: int) -> np.ndarray:
    """Final stress after `steps` steps with a frozen velocity gradient."""
    o = Oracle(prob, sigma0)
    return o.run(steps, kap, u)


def gradients(prob: Problem, sigma0, kap, u, steps: int, dJ_dsigma_T) -> dict:
    """Reverse-mode derivatives of J with dJ/dsigma(T) = dJ_dsigma_T (packed
    [nc][N]) for a frozen velocity gradient kap [d*d][N] (and u when transport
    is on).  Returns dict(sigma_T, sigma0, kappa, Wi, beta)."""
    d, N, nc = prob.dim, prob.N, prob.nc
    m = prob.m
    o = Oracle(prob, sigma0)
    kap = np.ascontiguousarray(kap, dtype=np.float64).reshape(d * d, N)
    hist = []
    for _ in range(steps):
        o.step(kap, kap, u)
        hist.append(o.sig_n.copy())
    lib = _load()
    p = prob.cparams()
    mu = np.ascontiguousarray(prob.mu, dtype=np.float64)
    w = np.ascontiguousarray(prob.w, dtype=np.float64)
    s1 = np.ascontiguousarray(dJ_dsigma_T, dtype=np.float64).reshape(nc, N).copy()
    s0 = np.zeros((nc, N))
    z1 = np.zeros((max(m, 1), nc, N))
    z0 = np.zeros((max(m, 1), nc, N))
    g_sigma0 = np.zeros((nc, N))
    g_kap = np.zeros((d * d, N))
    g_Wi = ctypes.c_double(0.0)
    g_beta = ctypes.c_double(0.0)
    uu = None if not prob.transport else np.ascontiguousarray(u, dtype=np.float64).reshape(d, N)
    sig0 = o.sigma0
    for n in range(steps - 1, -1, -1):
        s1o, s0o = np.empty_like(s1), np.empty_like(s0)
        z1o, z0o = np.zeros_like(z1), np.zeros_like(z0)
        gk_n = np.zeros((d * d, N))
        gk_nm1 = np.zeros((d * d, N))
        fails = lib.orc_adjoint_step(ctypes.byref(p), _ptr(mu), _ptr(w), n,
                                     _ptr(hist[n]), _ptr(sig0), _ptr(kap), _ptr(kap), _ptr(uu),
                                     _ptr(s1), _ptr(s0), _ptr(z1), _ptr(z0),
                                     _ptr(s1o), _ptr(s0o), _ptr(z1o), _ptr(z0o),
                                     _ptr(g_sigma0), _ptr(gk_n), _ptr(gk_nm1),
                                     ctypes.byref(g_Wi), ctypes.byref(g_beta))
        if fails:
            raise FloatingPointError("singular adjoint system")
        g_kap += gk_n + gk_nm1
        s1, s0, z1, z0 = s1o, s0o, z1o, z0o
    # initial state: sigma^0 = sigma^{-1} = sigma0, modes zero
    g_sigma0 = g_sigma0 + s1 + s0
    return dict(sigma_T=hist[-1] if hist else o.sigma0.copy(), sigma0=g_sigma0, kappa=g_kap,
                Wi=g_Wi.value, beta=g_beta.value)


def gradients_implicit(prob: Problem, sigma0, kap, u, steps: int, dJ_dsigma_T) -> dict:
    """Reverse-mode derivatives of J with dJ/dsigma(T) = dJ_dsigma_T for the
    implicit-transport step (orc_step_implicit, BDF2 start, frozen kap [d*d][N]),
    small grids.  Plain reverse sweep of the step, in numpy:

        R   = eta sigma0 - H + dt G k g,   H = sum_j eta_j (b1 sigma_j^n + b2 sigma_j^{n-1})
              (alpha = 1: H = b1 sigma^n + b2 sigma^{n-1} + b0 sigma0)
        A sigma^{n+1} = R,   A = a I - dt L(kappa) + dt (u.grad - eps Lap)   (dense, over the grid)
        sigma_j^{n+1} = c_j (-b1 sigma_j^n - b2 sigma_j^{n-1}) + rho_j (sigma^{n+1} - sigma0)

    (a = eta + dt/Wi, k = kappa + kappa^T, G = (1 - beta)/(Wi Re), g = g_alpha(t_{n+1})),
    with the transport matrix assembled from unit vectors by the stencils of
    oracle.paper_form.transport_op.  Returns dict(sigma_T, sigma0, kappa, Wi, beta)."""
    from scipy.special import gamma as Gamma
    d, N, nc, m = prob.dim, prob.N, prob.nc, prob.m
    dt, Wi, Re = prob.dt, prob.Wi, prob.Re
    B0, B1, B2 = 1.5, -2.0, 0.5
    classic = prob.alpha == 1.0
    mu = np.asarray(prob.mu, float)[:m]
    w = np.asarray(prob.w, float)[:m]
    c = 1.0 / (B0 + mu * dt)
    eta_j = mu * dt * c
    rho = w * dt * c
    eta = B0 if classic else float(np.sum(B0 * w * dt * c))
    a = eta + dt / Wi
    G = (1.0 - prob.beta) / (Wi * Re)
    kap = np.asarray(kap, float).reshape(d * d, N)
    K = kap.T.reshape(N, d, d)
    P = packed_pairs(d)
    KS = K + np.swapaxes(K, 1, 2)
    ks = np.stack([KS[:, i, j] for (i, j) in P])
    s0 = np.zeros((nc, N)) if sigma0 is None else np.asarray(sigma0, float).reshape(nc, N)
    # forward, keeping sigma^{n+1}
    o = Oracle(prob, sigma0)
    hist = []
    for _ in range(steps):
        o.step(kap, kap, u)
        hist.append(o.sig_n.copy())
    # the dense operator and its transpose
    L = prob.L if prob.L is not None else (2 * np.pi,) * d
    nn = nc * N
    A = np.zeros((nn, nn))
    for k in range(nn):
        e = np.zeros((nc, N))
        e.flat[k] = 1.0
        img = a * e - dt * upper_convected(d, K, e) + dt * transport_op(d, prob.n, L, prob.eps, prob.stencil, e, u)
        A[:, k] = img.ravel()
    AT = A.T

    def dL_dot(v, X):
        out = np.zeros((d * d, N))
        for ia in range(d):
            for ib in range(d):
                E = np.zeros((N, d, d))
                E[:, ia, ib] = 1.0
                out[ia * d + ib] = np.sum(v * upper_convected(d, E, X), axis=0)
        return out

    a1 = np.asarray(dJ_dsigma_T, float).reshape(nc, N).copy()   # adjoint of sigma^{n+1} (full)
    a0 = np.zeros((nc, N))                                     # partial adjoint of sigma^n
    z1 = np.zeros((m, nc, N))                                  # adjoint of sigma_j^{n+1}
    z0 = np.zeros((m, nc, N))                                  # partial adjoint of sigma_j^n
    g_s0 = np.zeros((nc, N))
    g_kap = np.zeros((d * d, N))
    gWi = gbeta = 0.0
    for n in range(steps - 1, -1, -1):
        sig_new = hist[n]
        g = 1.0 if classic else (n + 1) ** (prob.alpha - 1.0) * dt ** (prob.alpha - 1.0) / Gamma(prob.alpha)
        # sigma_j^{n+1} = c_j (...) + rho_j (sigma^{n+1} - sigma0)
        a_sig = a1 + np.tensordot(rho, z1, axes=(0, 0))
        g_s0 -= np.tensordot(rho, z1, axes=(0, 0))
        # A sigma^{n+1} = R
        ar = np.linalg.solve(AT, a_sig.ravel()).reshape(nc, N)
        # R = eta sigma0 - H + dt G k g
        g_s0 += eta * ar
        if classic:
            new_a1 = a0 - B1 * ar
            new_a0 = -B2 * ar
            g_s0 -= B0 * ar
        else:
            new_a1 = a0.copy()
            new_a0 = np.zeros((nc, N))
        new_z1 = z0 - B1 * eta_j[:, None, None] * ar[None] - B1 * c[:, None, None] * z1
        new_z0 = -B2 * eta_j[:, None, None] * ar[None] - B2 * c[:, None, None] * z1
        # parameters: A through kappa and Wi (a), R through G and k
        g_kap += dt * dL_dot(ar, sig_new)
        for ia in range(d):
            for ib in range(d):
                dks = np.zeros((nc, N))
                for cc, (i, j) in enumerate(P):
                    dks[cc] = (1.0 if (i, j) == (ia, ib) else 0.0) + (1.0 if (j, i) == (ia, ib) else 0.0)
                g_kap[ia * d + ib] += dt * G * g * np.sum(ar * dks, axis=0)
        gWi += dt / Wi ** 2 * np.sum(ar * sig_new) - dt * (G / Wi) * g * np.sum(ar * ks)
        gbeta += -dt * g * np.sum(ar * ks) / (Wi * Re)
        a1, a0, z1, z0 = new_a1, new_a0, new_z1, new_z0
    g_s0 += a1 + a0            # sigma^0 = sigma^{-1} = sigma0
    return dict(sigma_T=hist[-1], sigma0=g_s0, kappa=g_kap, Wi=gWi, beta=gbeta)


if __name__ == "__main__":   # pragma: no cover
    build(force=True)
    print(_LIB, file=sys.stderr)
