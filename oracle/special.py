"""Closed forms and convolution-quadrature weights (oracle side).

TEST INFRASTRUCTURE ONLY (see the package docstring).

``mittag_leffler(alpha, z)``  E_alpha(z) = sum_k z^k / Gamma(alpha k + 1), the
    function in which the decoupled analytic solution of Section 5.1 is written
    (zero flow: sigma(t) = sigma0 E_alpha(-t^alpha / Wi)).  Power series for
    complex z, for alpha >= 1 and for |z| <= 0.5.  For real z = -x < -0.5 and
    0 < alpha < 1 the series cancels catastrophically (its terms reach 1e11 at
    alpha = 0.3, x = 3), so there E_alpha(-x) comes from its spectral
    representation as a completely monotone function (Gorenflo and Mainardi),
        E_alpha(-x) = sin(alpha pi)/pi int_0^inf exp(-r x^(1/alpha)) r^(alpha-1)
                      / (r^(2 alpha) + 2 r^alpha cos(alpha pi) + 1) dr,
    which the substitution u = r^alpha turns into
        sin(alpha pi)/(alpha pi) int_0^inf exp(-(u x)^(1/alpha)) / (u^2 + 2 u cos(alpha pi) + 1) du,
    a smooth integrand evaluated by adaptive quadrature.

``cq_weights_power(alpha, dt, n)``  the first n+1 coefficients of
    dt * (delta(zeta)/dt)^alpha, delta(zeta) = 3/2 - 2 zeta + zeta^2/2, i.e. the
    BDF2 convolution quadrature of the exact Caputo symbol s^alpha (times dt).
    delta(zeta) = (1 - zeta)(3 - zeta)/2, so the power factorises into two
    binomial series whose coefficients follow c_k = c_{k-1} (k - 1 - alpha)/k.

``cq_weights_soe(mu, w, dt, n)``  the first n+1 coefficients of
    W(zeta) = delta(zeta) sum_j w_j dt / (delta(zeta) + mu_j dt), the generating
    function of the discrete derivative produced by the BDF2 mode recursion of
    Section 4.1 (eq. BDF_Phi_k_n+1 inserted in eq.
    fractional_modes_fractional_derivative).  The series of
    1/(p0 + p1 zeta + p2 zeta^2) follows y_k = -(p1 y_{k-1} + p2 y_{k-2}) / p0.
"""
from __future__ import annotations

import cmath
import math

import numpy as np

B0, B1, B2 = 1.5, -2.0, 0.5


def _ml_negative_real(alpha: float, x: float) -> float:
    """E_alpha(-x), 0 < alpha < 1, x > 0, by the spectral integral."""
    import scipy.integrate
    c = math.cos(alpha * math.pi)
    f = lambda u: math.exp(-(u * x) ** (1.0 / alpha)) / (u * u + 2.0 * u * c + 1.0)
    # the exponential factor is e^-1 at u = 1/x and below e^-750 (nothing left
    # in double precision) past u = 750^alpha / x: integrate over [0, 1/x] and
    # [1/x, 750^alpha / x]
    knot = 1.0 / x
    end = 750.0 ** alpha / x
    a, _ = scipy.integrate.quad(f, 0.0, knot, epsabs=0.0, epsrel=1e-13, limit=400)
    b, _ = scipy.integrate.quad(f, knot, end, epsabs=0.0, epsrel=1e-13, limit=400)
    return math.sin(alpha * math.pi) / (alpha * math.pi) * (a + b)


def mittag_leffler(alpha: float, z, tol: float = 1e-17, kmax: int = 2000):
    """E_alpha(z) (scalar or array, real or complex); see the module docstring."""
    zs = np.asarray(z)
    out = np.empty(zs.shape, dtype=np.complex128 if np.iscomplexobj(zs) else np.float64)
    flat_in = zs.reshape(-1)
    flat_out = out.reshape(-1)
    for i, zi in enumerate(flat_in):
        zi = complex(zi) if np.iscomplexobj(zs) else float(zi)
        if not isinstance(zi, complex) and 0.0 < alpha < 1.0 and zi < -0.5:
            flat_out[i] = _ml_negative_real(alpha, -zi)
            continue
        total = 0.0
        comp = 0.0          # Kahan compensation: the series alternates for z < 0
        for k in range(kmax):
            if zi == 0:
                term = 1.0 if k == 0 else 0.0
            else:
                a = alpha * k + 1.0
                if a < 170.0:
                    term = zi ** k / math.gamma(a)
                elif isinstance(zi, complex):
                    term = cmath.exp(k * cmath.log(zi) - math.lgamma(a))
                else:
                    mag = math.exp(k * math.log(abs(zi)) - math.lgamma(a))
                    term = mag if (zi > 0 or k % 2 == 0) else -mag
            y = term - comp
            t = total + y
            comp = (t - total) - y
            total = t
            if k > 2 and abs(term) <= tol * max(abs(total), 1e-300):
                break
        flat_out[i] = total
    return out if out.shape else out.reshape(()).item()


def _binomial_series(alpha: float, n: int, scale: float = 1.0) -> np.ndarray:
    """Coefficients of (1 - x/scale)^alpha up to x^n."""
    c = np.empty(n + 1)
    c[0] = 1.0
    for k in range(1, n + 1):
        c[k] = c[k - 1] * (k - 1 - alpha) / k / scale
    return c


def cq_weights_power(alpha: float, dt: float, n: int) -> np.ndarray:
    """dt * (delta(zeta)/dt)^alpha, coefficients 0..n."""
    a = _binomial_series(alpha, n)              # (1 - zeta)^alpha
    b = _binomial_series(alpha, n, 3.0)         # (1 - zeta/3)^alpha
    conv = np.convolve(a, b)[: n + 1]
    return dt ** (1.0 - alpha) * (1.5 ** alpha) * conv   # ((1)(3)/2)^alpha = 1.5^alpha


def _inverse_quadratic_series(p0: float, p1: float, p2: float, n: int) -> np.ndarray:
    y = np.empty(n + 1)
    y[0] = 1.0 / p0
    if n >= 1:
        y[1] = -(p1 * y[0]) / p0
    for k in range(2, n + 1):
        y[k] = -(p1 * y[k - 1] + p2 * y[k - 2]) / p0
    return y


def cq_weights_soe(mu, w, dt: float, n: int) -> np.ndarray:
    """Coefficients 0..n of delta(zeta) sum_j w_j dt / (delta(zeta) + mu_j dt)."""
    W = np.zeros(n + 1)
    for mj, wj in zip(np.asarray(mu, dtype=float), np.asarray(w, dtype=float)):
        y = _inverse_quadratic_series(B0 + mj * dt, B1, B2, n)
        # delta/(delta + mu dt) = 1 - mu dt / (delta + mu dt)
        term = -mj * dt * y
        term[0] += 1.0
        W += wj * dt * term
    return W
