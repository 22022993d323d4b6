"""P10: von Neumann analysis of the explicit transport in the fractional
scheme, and the library's Courant limits checked against it (no GPU).

For one Fourier mode e^{i theta x/h} advected by a constant u (kappa = 0, no
relaxation, eps = 0) the scheme is a linear recurrence on
(sigma^n, sigma^{n-1}, modes^n, modes^{n-1}) with the stencil symbol in place
of u.grad.  Its spectral radius is <= 1 for every theta exactly when
C = (dt/b0)^alpha |u|/h is below a limit that does not depend on dt (the
fractional derivative weighs the transport like a step dt^alpha/b0^alpha).
"""
import ctypes
import math

import numpy as np
import pytest

from helpers import ensure_lib
from oracle import soe

B0, B1, B2 = 1.5, -2.0, 0.5


def recurrence(z, mu, w, dt, classic):
    if classic:
        T = np.zeros((2, 2), complex)
        T[0, 0] = (-B1 - 2 * z) / B0
        T[0, 1] = (-B2 + z) / B0
        T[1, 0] = 1
        return T
    m = len(mu)
    c = 1 / (B0 + mu * dt)
    rho = w * dt * c
    etaj = mu * dt * c
    eta = B0 * rho.sum()
    D = 2 + 2 * m
    T = np.zeros((D, D), complex)
    row = np.zeros(D, complex)
    row[0], row[1] = -2 * z, z                      # -(dt u s)(2 sigma^n - sigma^{n-1})
    row[2:2 + m] = -etaj * B1
    row[2 + m:] = -etaj * B2
    row /= eta
    T[0] = row
    T[1, 0] = 1
    for j in range(m):
        T[2 + j] = rho[j] * row
        T[2 + j, 2 + j] += -c[j] * B1
        T[2 + j, 2 + m + j] += -c[j] * B2
        T[2 + m + j, 2 + j] = 1
    return T


def symbol(theta, stencil):
    e = np.exp(1j * theta)
    if stencil == 0:
        return (e ** -2 - 6 / e + 3 + 2 * e) / 6
    return (e - 1 / e) / 2


def radius(alpha, dt, m, stencil, lam, soe_tab=None):
    """Spectral radius of the one-mode recurrence, maximised over theta,
    for lam = dt |u| / h."""
    classic = alpha == 1.0
    if classic:
        mu, w = np.zeros(0), np.zeros(0)
    else:
        mu, w = soe_tab if soe_tab is not None else soe.soe_nnls(alpha, dt, 200 * dt, m)
    th = np.linspace(0, 2 * np.pi, 361)[1:]
    return max(np.max(np.abs(np.linalg.eigvals(recurrence(lam * symbol(t, stencil), mu, w, dt, classic))))
               for t in th)


def library_lambda(stencil, alpha, dt, m, soe_tab):
    """lambda* = dt U sum_a 1/h_a / 0.9 from tfs_transport_limit (2D, h equal)."""
    ensure_lib()
    from paper_2411_17294_gb300 import tfs
    lib = tfs.load_library()
    g = tfs.TfsGrid()
    g.dim = 2
    for a in range(3):
        g.n[a] = 64 if a < 2 else 1
        g.L[a] = 2 * math.pi
    h = ctypes.c_void_p()
    assert lib.tfs_create(ctypes.byref(h), ctypes.byref(g), alpha, 1.0, 0.5, m, dt, 1) == 0
    assert lib.tfs_set_param(h, tfs.TFS_PARAM_STENCIL, float(stencil)) == 0
    U = ctypes.c_double(0)
    dp = ctypes.POINTER(ctypes.c_double)
    if alpha < 1:
        assert lib.tfs_transport_limit(h, ctypes.byref(U)) == tfs.TFS_ERR_NOSOE
        mu, w = [np.ascontiguousarray(a) for a in soe_tab]
        assert lib.tfs_set_soe(h, mu.ctypes.data_as(dp), w.ctypes.data_as(dp), m) == 0
    assert lib.tfs_transport_limit(h, ctypes.byref(U)) == 0
    inv_h = 64 / (2 * math.pi)
    lam_lib = dt * U.value * inv_h          # per-axis lambda at the accepted bound, both axes at U
    # declared bounds just below / above are accepted / refused
    assert lib.tfs_set_param(h, tfs.TFS_PARAM_UMAX, U.value * 0.999) == 0
    assert lib.tfs_set_param(h, tfs.TFS_PARAM_UMAX, U.value * 1.001) == tfs.TFS_ERR_UNSTABLE
    lib.tfs_destroy(h)
    return 2 * lam_lib / 0.9


CASES = [(0.2, 12, 0), (0.6, 8, 0), (0.6, 32, 0), (0.8, 12, 0), (0.9, 16, 0), (1.0, 0, 0), (0.5, 16, 1)]


@pytest.mark.parametrize("alpha,m,stencil", CASES)
def test_library_limit_matches_eigenvalue_scan(alpha, m, stencil):
    dt = 2e-4
    tab = None if alpha == 1.0 else soe.soe_nnls(alpha, dt, 200 * dt, m)
    lam_star = library_lambda(stencil, alpha, dt, m, tab)
    # stable at the accepted bound (0.9 lambda*) and at lambda* itself within the scan's resolution,
    # unstable a little beyond lambda*
    assert radius(alpha, dt, m, stencil, 0.9 * lam_star, tab) <= 1 + 1e-9
    assert radius(alpha, dt, m, stencil, 0.995 * lam_star, tab) <= 1 + 1e-6
    assert radius(alpha, dt, m, stencil, 1.05 * lam_star, tab) > 1 + 1e-6


def test_fractional_courant_scaling():
    # with a fixed SOE accuracy the boundary scales like (b0/dt)^alpha dt, i.e.
    # C = (dt/b0)^alpha |u|/h is dt-independent
    Cs = []
    for dt in (1e-3, 1e-4):
        tab = soe.soe_nnls(0.5, dt, 200 * dt, 16)
        lam = library_lambda(0, 0.5, dt, 16, tab)
        Cs.append(lam * (1.5 / dt) ** 0.5)
    assert abs(Cs[0] / Cs[1] - 1) < 0.02


def test_central2_alpha1_unstable():
    lam = library_lambda(1, 1.0, 2e-4, 0, None)
    assert lam < 0.02
    assert radius(1.0, 2e-4, 0, 1, 0.05) > 1 + 1e-6


def test_explicit_diffusion_bound():
    # eps alone: accepted while 4 eps dt sum_a 1/h_a^2 <= 0.9 z*; the eigenvalues of
    # the recurrence with the diffusion symbol z = 4 nu sin^2(theta/2) confirm z*
    ensure_lib()
    from paper_2411_17294_gb300 import tfs
    lib = tfs.load_library()
    alpha, dt, m = 0.3, 2e-3, 12
    mu, w = soe.soe_nnls(alpha, dt, 200 * dt, m)
    g = tfs.TfsGrid()
    g.dim = 2
    for a in range(3):
        g.n[a] = 64 if a < 2 else 1
        g.L[a] = 2 * math.pi
    h = ctypes.c_void_p()
    assert lib.tfs_create(ctypes.byref(h), ctypes.byref(g), alpha, 1.0, 0.5, m, dt, 1) == 0
    dp = ctypes.POINTER(ctypes.c_double)
    mu_c, w_c = np.ascontiguousarray(mu), np.ascontiguousarray(w)
    assert lib.tfs_set_soe(h, mu_c.ctypes.data_as(dp), w_c.ctypes.data_as(dp), m) == 0
    lo, hi = 0.0, 10.0
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        if lib.tfs_set_param(h, tfs.TFS_PARAM_EPS, mid) == tfs.TFS_OK:
            lo = mid
        else:
            hi = mid
    U = ctypes.c_double(1.0)
    assert lib.tfs_transport_limit(h, ctypes.byref(U)) == 0
    assert U.value < 1e-6 * (1 + lo)           # eps at its bound leaves no room for velocity
    lib.tfs_destroy(h)
    inv_h2 = (64 / (2 * math.pi)) ** 2
    z_star = 4 * lo * dt * 2 * inv_h2 / 0.9   # both axes

    def rad(zmax):
        th = np.linspace(0, 2 * np.pi, 361)[1:]
        return max(np.max(np.abs(np.linalg.eigvals(recurrence(zmax * np.sin(t / 2) ** 2, mu, w, dt, False))))
                   for t in th)
    assert rad(0.9 * z_star) <= 1 + 1e-9
    assert rad(1.1 * z_star) > 1 + 1e-6


def paper_recurrence(z, mu, w, dt):
    """One Fourier mode of the scheme in the paper's variable (Phi, the modes
    phi_j of Phi, Psi = xi Phi + h), the transport z (2 Psi^n - Psi^{n-1})
    explicit, no relaxation: state (Phi^n, Phi^{n-1}, Psi^n, Psi^{n-1}, phi^n,
    phi^{n-1})."""
    m = len(mu)
    c = 1 / (B0 + mu * dt)
    xi = B0 * np.sum(w * c)
    D = 4 + 2 * m
    T = np.zeros((D, D), complex)
    # Phi^{n+1} = (-b1 Phi^n - b2 Phi^{n-1} - z (2 Psi^n - Psi^{n-1})) / b0
    phi_row = np.zeros(D, complex)
    phi_row[0], phi_row[1] = -B1 / B0, -B2 / B0
    phi_row[2], phi_row[3] = -2 * z / B0, z / B0
    T[0] = phi_row
    T[1, 0] = 1
    # h^n = sum_j w_j mu_j c_j (b1 phi_j^n + b2 phi_j^{n-1});  Psi^{n+1} = xi Phi^{n+1} + h^n
    T[2] = xi * phi_row
    T[2, 4:4 + m] += w * mu * c * B1
    T[2, 4 + m:] += w * mu * c * B2
    T[3, 2] = 1
    for j in range(m):
        T[4 + j] = c[j] * dt * phi_row
        T[4 + j, 4 + j] += -c[j] * B1
        T[4 + j, 4 + m + j] += -c[j] * B2
        T[4 + m + j, 4 + j] = 1
    return T


def paper_library_lambda(stencil, alpha, dt, m, soe_tab):
    ensure_lib()
    from paper_2411_17294_gb300 import tfs
    lib = tfs.load_library()
    g = tfs.TfsGrid()
    g.dim = 2
    for a in range(3):
        g.n[a] = 64 if a < 2 else 1
        g.L[a] = 2 * math.pi
    h = ctypes.c_void_p()
    assert lib.tfs_create(ctypes.byref(h), ctypes.byref(g), alpha, 1.0, 0.5, m, dt, 1) == 0
    assert lib.tfs_set_param(h, tfs.TFS_PARAM_STENCIL, float(stencil)) == 0
    assert lib.tfs_set_param(h, tfs.TFS_PARAM_FORM, float(tfs.TFS_FORM_PAPER)) == 0
    dp = ctypes.POINTER(ctypes.c_double)
    mu, w = [np.ascontiguousarray(a) for a in soe_tab]
    assert lib.tfs_set_soe(h, mu.ctypes.data_as(dp), w.ctypes.data_as(dp), m) == 0
    U = ctypes.c_double(0)
    assert lib.tfs_transport_limit(h, ctypes.byref(U)) == 0
    lam_lib = dt * U.value * 64 / (2 * math.pi)
    assert lib.tfs_set_param(h, tfs.TFS_PARAM_UMAX, U.value * 0.999) == 0
    assert lib.tfs_set_param(h, tfs.TFS_PARAM_UMAX, U.value * 1.001) == tfs.TFS_ERR_UNSTABLE
    lib.tfs_destroy(h)
    return 2 * lam_lib / 0.9


@pytest.mark.parametrize("alpha,m", [(0.3, 8), (0.5, 12), (0.8, 8)])
def test_paper_variable_limit_matches_eigenvalue_scan(alpha, m):
    # The Courant bound of the explicit transport in the paper's variable (the
    # transport acts on Psi = V(zeta) Phi) against the spectral radius of its
    # one-mode recurrence: stable at 0.9 lambda*, unstable just beyond lambda*.
    dt = 2e-4
    tab = soe.soe_nnls(1 - alpha, dt, 200 * dt, m)
    lam_star = paper_library_lambda(0, alpha, dt, m, tab)
    th = np.linspace(0, 2 * np.pi, 361)[1:]
    rad = lambda lam: max(np.max(np.abs(np.linalg.eigvals(paper_recurrence(lam * symbol(t, 0), *tab, dt))))
                          for t in th)
    assert rad(0.9 * lam_star) <= 1 + 1e-9
    assert rad(0.995 * lam_star) <= 1 + 1e-6
    assert rad(1.05 * lam_star) > 1 + 1e-6
