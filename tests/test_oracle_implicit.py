"""Pins of the oracle's implicit-transport step (transport at t_{n+1} inside a
global solve, the form of eq. FP_discrete), on CPU.

1. One Fourier mode advected by a constant velocity with kappa = 0: the
   components decouple and the fully discrete scheme reduces to a complex
   scalar recurrence per mode,
       (eta + dt/Wi + dt s(k)) S^{n+1} = eta S0 - H^n,
   s(k) = U D(k) + eps 4 sin^2(k h/2)/h^2 with D(k) the symbol of the first-
   derivative stencil, and the SOE modes follow their own scalar BDF2 update.
   The oracle's dense global solve must reproduce Re(S^n e^{ikx}) to rounding.
2. Without velocity the implicit and explicit steps coincide.
3. Far above the explicit Courant limit the implicit step stays bounded where
   the explicit one grows.
"""
import math

import numpy as np
import pytest

from oracle import orc, soe


def fourier_recurrence(alpha, Wi, dt, mu, w, U, eps, k, h, stencil, steps):
    b0, b1, b2 = 1.5, -2.0, 0.5
    th = k * h
    if stencil == 1:
        D = 1j * math.sin(th) / h
    elif U >= 0:
        D = (np.exp(-2j * th) - 6 * np.exp(-1j * th) + 3 + 2 * np.exp(1j * th)) / (6 * h)
    else:
        D = (-2 * np.exp(-1j * th) - 3 + 6 * np.exp(1j * th) - np.exp(2j * th)) / (6 * h)
    s = U * D + eps * 4.0 * math.sin(th / 2) ** 2 / h ** 2
    S0 = 1.0 + 0j
    if alpha == 1.0:
        eta = b0
        Sn = Snm1 = S0
        for _ in range(steps):
            H = b1 * Sn + b2 * Snm1 + b0 * S0
            Snp1 = (eta * S0 - H) / (eta + dt / Wi + dt * s)
            Snm1, Sn = Sn, Snp1
        return Sn
    c = 1.0 / (b0 + mu * dt)
    rho = w * dt * c
    etaj = mu * dt * c
    eta = b0 * np.sum(rho)
    Mn = np.zeros(len(mu), complex)
    Mnm1 = np.zeros(len(mu), complex)
    Sn = S0
    for _ in range(steps):
        H = np.sum(etaj * (b1 * Mn + b2 * Mnm1))
        Sn = (eta * S0 - H) / (eta + dt / Wi + dt * s)
        Mnp1 = c * (-b1 * Mn - b2 * Mnm1) + rho * (Sn - S0)
        Mnm1, Mn = Mn, Mnp1
    return Sn


@pytest.mark.parametrize("alpha,m", [(0.5, 8), (1.0, 0)])
@pytest.mark.parametrize("stencil,U,eps", [(0, 6.0, 0.0), (0, -6.0, 0.05), (1, 6.0, 0.02)])
def test_implicit_single_fourier_mode(alpha, m, stencil, U, eps):
    n, kx, Wi, dt, steps = (16, 3), 3, 1.7, 0.02, 12
    h = 2 * math.pi / n[0]
    mu, w = (soe.soe_nnls(alpha, dt, steps * dt, m) if m else (np.zeros(0), np.zeros(0)))
    prob = orc.Problem(dim=2, n=n, alpha=alpha, Wi=Wi, beta=0.5, dt=dt, mu=mu, w=w, eps=eps, stencil=stencil,
                       transport=True, implicit=True)
    N = n[0] * n[1]
    x = (np.arange(N) % n[0]) * h
    sigma0 = np.zeros((3, N))
    sigma0[0] = np.cos(kx * x)
    u = np.zeros((2, N))
    u[0] = U
    # the explicit step would be far outside its stability region here
    assert abs(U) * dt / h > 0.25
    got = orc.forward(prob, sigma0, np.zeros((4, N)), u, steps)
    S = fourier_recurrence(alpha, Wi, dt, mu, w, U, eps, kx, h, stencil, steps)
    ref = (S * np.exp(1j * kx * x)).real
    assert np.max(np.abs(got[0] - ref)) < 1e-12
    assert np.max(np.abs(got[1:])) == 0.0


def test_implicit_equals_explicit_without_flow():
    dim, n, alpha, m, dt, steps = 3, (4, 3, 5), 0.6, 6, 2e-3, 8
    rng = np.random.default_rng(5)
    N = int(np.prod(n))
    mu, w = soe.soe_nnls(alpha, dt, steps * dt, m)
    kap = rng.normal(size=(9, N))
    sigma0 = rng.normal(size=(6, N))
    u = np.zeros((3, N))
    kw = dict(dim=dim, n=n, alpha=alpha, Wi=1.2, beta=0.3, dt=dt, mu=mu, w=w, transport=True)
    a = orc.forward(orc.Problem(**kw, implicit=True), sigma0, kap, u, steps)
    b = orc.forward(orc.Problem(**kw, implicit=False), sigma0, kap, u, steps)
    assert np.max(np.abs(a - b)) < 1e-13 * np.max(np.abs(b))


def test_implicit_bounded_where_explicit_grows():
    n, alpha, m, dt, steps = (12, 12), 0.5, 8, 0.05, 40
    N = n[0] * n[1]
    mu, w = soe.soe_nnls(alpha, dt, steps * dt, m)
    rng = np.random.default_rng(9)
    sigma0 = rng.normal(size=(3, N))
    u = np.zeros((2, N))
    u[0], u[1] = 5.0, -3.0
    kw = dict(dim=2, n=n, alpha=alpha, Wi=1.0, beta=0.5, dt=dt, mu=mu, w=w, transport=True)
    imp = orc.forward(orc.Problem(**kw, implicit=True), sigma0, np.zeros((4, N)), u, steps)
    exp_ = orc.forward(orc.Problem(**kw, implicit=False), sigma0, np.zeros((4, N)), u, steps)
    assert np.max(np.abs(imp)) <= 1.01 * np.max(np.abs(sigma0))
    assert not np.all(np.isfinite(exp_)) or np.max(np.abs(exp_)) > 1e3 * np.max(np.abs(sigma0))
