"""Pins of the FP64 Navier-Stokes oracle (oracle/ns.py, the projection step of
Section 4.1) against closed forms (no GPU).

TG   Taylor-Green decay u = (sin x cos y, -cos x sin y) exp(-2 nu t): the
     convective term is a gradient, so the projection removes it and the scheme
     is BDF2 for the viscous decay: second order in dt when the level u^{-1} is
     the exact one, first order with the empty past.
KF   a shear stress sigma_xy = A sin(k y) drives u = (U(y), 0), for which the
     convective term vanishes; the steady state of nu U'' + dsigma_xy/dy = 0 is
     U = A cos(k y) / (nu k).  Checks the stress divergence (sign, index) and
     the implicit viscous term.
DIV  for random velocity and stress fields every step leaves a divergence-free
     field (the discrete divergence vanishes to rounding).
"""
import numpy as np
import pytest

from oracle.ns import NSOracle


def grid(n, L=2 * np.pi):
    x = np.arange(n) * L / n
    return np.meshgrid(x, x)


def taylor_green(X, Y, nu, t):
    return np.stack([np.sin(X) * np.cos(Y), -np.cos(X) * np.sin(Y)]).reshape(2, -1) * np.exp(-2 * nu * t)


@pytest.mark.parametrize("start,order", [("exact", 2.0), ("empty", 1.0)])
def test_taylor_green_decay_order(start, order):
    n, beta, Re, T = 32, 0.5, 10.0, 1.0
    nu = beta / Re
    X, Y = grid(n)
    errs = []
    for steps in (20, 40, 80):
        dt = T / steps
        o = NSOracle((n, n), (2 * np.pi, 2 * np.pi), beta, Re, dt)
        o.set_state(taylor_green(X, Y, nu, 0.0), taylor_green(X, Y, nu, -dt) if start == "exact" else None)
        for _ in range(steps):
            u, kap = o.step()
        errs.append(np.max(np.abs(u - taylor_green(X, Y, nu, T))))
        # the gradient is the analytic one of the computed field
        assert np.allclose(kap[1].reshape(n, n), -np.sin(X) * np.sin(Y) * u[0].reshape(n, n).max()
                           / np.sin(X).max(), atol=1e-6)
    rates = [np.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(abs(r - order) < 0.05 for r in rates), (errs, rates)
    assert errs[0] < (1e-6 if start == "exact" else 3e-3)


def test_shear_stress_drives_the_steady_kolmogorov_profile():
    n, beta, Re, dt, k, A = 32, 0.8, 4.0, 0.02, 2, 0.3
    nu = beta / Re
    X, Y = grid(n)
    sigma = np.stack([np.zeros_like(X), A * np.sin(k * Y), np.zeros_like(X)]).reshape(3, -1)
    o = NSOracle((n, n), (2 * np.pi, 2 * np.pi), beta, Re, dt)
    o.set_state(np.zeros((2, n * n)))
    for _ in range(3000):
        u, _ = o.step(sigma)
    U = (A * np.cos(k * Y) / (nu * k)).reshape(-1)
    assert np.max(np.abs(u[0] - U)) < 1e-9 * np.max(np.abs(U))
    assert np.max(np.abs(u[1])) < 1e-12


def test_every_step_is_divergence_free():
    n, beta, Re, dt = 24, 0.6, 50.0, 1e-2
    rng = np.random.default_rng(5)
    o = NSOracle((n, n), (2 * np.pi, 2 * np.pi), beta, Re, dt)
    o.set_state(rng.normal(size=(2, n * n)))
    for _ in range(6):
        o.step(0.1 * rng.normal(size=(3, n * n)))
        div = o.DX * o.uh[0] + o.DY * o.uh[1]
        assert np.max(np.abs(div)) < 1e-10 * np.max(np.abs(o.uh[0]))
