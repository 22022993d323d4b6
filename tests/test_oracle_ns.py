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
ROT  the scheme's velocity equals the projection of its explicit terms without
     the rotational term (k.(curl curl u) = 0), formed independently with NumPy.
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


def test_rotational_term_leaves_the_velocity_unchanged_on_the_periodic_box():
    """ROT  k.(curl curl u) = k.(k^2 u - k (k.u)) = 0 for every wavevector, so on the
    periodic box the velocity of the scheme is -(w - k (k.w)/k^2)/(b0/dt + nu k^2)
    with w = (b1 u^n + b2 u^{n-1})/dt + E((u.grad)u - div sigma): the projection of
    the explicit terms without the rotational term (the form the library's GPU step
    evaluates).  Formed here from the grid levels with NumPy's FFT and compared
    with the oracle's step, which keeps every term, over several steps of random
    velocity and stress."""
    n, L, beta, Re, dt = 32, 2 * np.pi, 0.4, 7.0, 2e-2
    nu = beta / Re
    rng = np.random.default_rng(11)
    o = NSOracle((n, n), (L, L), beta, Re, dt)
    o.set_state(rng.normal(size=(2, n * n)), rng.normal(size=(2, n * n)))
    k = np.fft.fftfreq(n, d=1.0 / n) * (2 * np.pi / L)
    k[n // 2] = 0.0                                   # first derivative zero at the Nyquist wavenumber
    KX, KY = np.meshgrid(k, k)                        # [y][x]
    K2 = KX ** 2 + KY ** 2
    fft = lambda f: np.fft.fft2(np.asarray(f).reshape(n, n))

    def terms(u, sigma):
        """spectral (u.grad)u - div sigma of grid fields u [2][N], sigma [3][N] (or None)"""
        uh = [fft(u[0]), fft(u[1])]
        g = [np.real(np.fft.ifft2(1j * K * uh[a])).reshape(-1) for a in range(2) for K in (KX, KY)]
        conv = [fft(u[0] * g[0] + u[1] * g[1]), fft(u[0] * g[2] + u[1] * g[3])]
        if sigma is None:
            return conv
        sh = [fft(s) for s in sigma]
        return [conv[0] - (1j * KX * sh[0] + 1j * KY * sh[1]), conv[1] - (1j * KX * sh[1] + 1j * KY * sh[2])]

    u_prev = o.velocity(o.uh_prev)
    f_prev = terms(u_prev, None)                      # the given level u^{-1} carries no stress
    for _ in range(4):
        sigma = 0.3 * rng.normal(size=(3, n * n))
        u_n = o.velocity()
        f_n = terms(u_n, sigma)
        w = [(-2.0 * fft(u_n[a]) + 0.5 * fft(u_prev[a])) / dt + 2.0 * f_n[a] - f_prev[a] for a in range(2)]
        with np.errstate(divide="ignore", invalid="ignore"):
            kw = np.where(K2 > 0, (KX * w[0] + KY * w[1]) / K2, 0.0)
        den = 1.5 / dt + nu * K2
        expect = np.stack([np.real(np.fft.ifft2(-(w[0] - KX * kw) / den)).reshape(-1),
                           np.real(np.fft.ifft2(-(w[1] - KY * kw) / den)).reshape(-1)])
        got, _ = o.step(sigma)
        assert np.max(np.abs(got - expect)) <= 1e-12 * np.max(np.abs(expect))
        u_prev, f_prev = u_n, f_n
