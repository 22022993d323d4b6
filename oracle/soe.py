"""Sum-of-exponentials (SOE) approximations of the Caputo kernel (oracle side).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The memory term of the stress law is the Caputo derivative of order alpha with
kernel  k(t) = t^-alpha / Gamma(1-alpha),  whose Laplace transform is
s^(alpha-1).  Section 2.2 (kernel compression) replaces the kernel by
sum_j w_j exp(-mu_j t) with non-negative w_j, mu_j (eq. tf_approximate_kernel),
obtained by a rational approximation in the Laplace variable, partial fractions
and inverse Laplace transform.  To avoid a Dirac term (eq.
tf_approximate_kernel_khristenko with w_inf > 0) the paper applies AAA to the
transform multiplied by s and divides the result by s; the rational function
then has a numerator of lower degree and the Dirac weight vanishes.  For our
kernel that means AAA on s^alpha, then r(s)/s ~ s^(alpha-1).

``soe_aaa``     the construction above, written from the AAA algorithm of
                Nakatsukasa, Sete & Trefethen (2018): greedy support points,
                least-squares weights from the Loewner matrix SVD, removal of
                spurious pole-zero pairs (Froissart doublets) with a refit,
                poles from the barycentric generalised eigenvalue problem.
``soe_nnls``    a positive construction with exactly m terms for any m:
                exponents on a geometric grid, weights by non-negative least
                squares on the relative kernel error over [dt/10, T]; the grid
                size is raised until exactly m weights are positive.  AAA in
                FP64 produces spurious (complex or positive) poles beyond about
                20 terms for the ranges used here, so this is the fit the
                default builder (``soe_build``) completes.
``soe_complete`` appends one term that carries the kernel's mass on [0, T]
                missing from a table (the singular part below the fitted
                times): a Dirac term w_inf delta(t) of the Khristenko form (eq.
                tf_approximate_kernel_khristenko) realised as one exponential
                with mu = 1e12/dt and w = w_inf mu, which the BDF2 mode update
                turns into w_inf times the BDF2 difference quotient of sigma
                up to a relative 1e-12.  ``soe_build`` = ``soe_nnls`` with m - 1
                terms completed this way.
``soe_expquad`` a plain positive construction: the trapezoidal rule on
                k(t) = sin(pi alpha)/pi * int exp(alpha x - t e^x) dx.
``soe_eval``    evaluates sum_j w_j exp(-mu_j t).
``kernel_exact`` the closed form t^-alpha / Gamma(1-alpha).
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg
import scipy.optimize
import scipy.special


def kernel_exact(alpha: float, t):
    """t^-alpha / Gamma(1 - alpha), the Caputo kernel of order alpha."""
    t = np.asarray(t, dtype=np.float64)
    return t ** (-alpha) / scipy.special.gamma(1.0 - alpha)


def soe_eval(mu, w, t):
    """sum_j w_j exp(-mu_j t) at the points t."""
    t = np.asarray(t, dtype=np.float64)
    mu = np.asarray(mu, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    return np.exp(-np.multiply.outer(t, mu)) @ w


def _aaa(Z, F, kmax, tol):
    """AAA rational approximation of samples F at points Z.

    Returns (support points zj, values fj, barycentric weights wj) of the
    approximant r(s) = sum_j wj fj/(s-zj) / sum_j wj/(s-zj)."""
    Z = np.asarray(Z, dtype=np.float64)
    F = np.asarray(F, dtype=np.float64)
    M = len(Z)
    mask = np.ones(M, dtype=bool)          # rows not yet used as support points
    R = np.full(M, F.mean())
    zj, fj = [], []
    wj = None
    scale = np.max(np.abs(F))
    for _ in range(kmax):
        err = np.abs(F - R)
        err[~mask] = -1.0
        j = int(np.argmax(err))
        zj.append(Z[j]); fj.append(F[j]); mask[j] = False
        z = np.array(zj); f = np.array(fj)
        C = 1.0 / (Z[mask, None] - z[None, :])
        A = (F[mask, None] - f[None, :]) * C      # Loewner matrix
        _, _, Vh = np.linalg.svd(A, full_matrices=False)
        wj = Vh[-1, :].conj()
        N = C @ (wj * f)
        D = C @ wj
        R = F.copy()
        R[mask] = N / D
        if np.max(np.abs(F - R)) <= tol * scale:
            break
    return np.array(zj), np.array(fj), wj


def _poles(zj, wj):
    """Zeros of the barycentric denominator sum_j wj/(s-zj)."""
    k = len(zj)
    E = np.zeros((k + 1, k + 1))
    E[0, 1:] = wj
    E[1:, 0] = 1.0
    E[1:, 1:] = np.diag(zj)
    B = np.eye(k + 1)
    B[0, 0] = 0.0
    ev = scipy.linalg.eigvals(E, B)
    return ev[np.isfinite(ev)]


def _residues(zj, fj, wj, poles):
    """Residues of the barycentric r(s) = N(s)/D(s) at simple poles p: N(p)/D'(p)."""
    out = []
    for p in poles:
        c = 1.0 / (p - zj)
        out.append((c @ (wj * fj)) / (-(c * c) @ wj))
    return np.array(out)


def _aaa_cleanup(Z, F, zj, fj, wj, tol=1e-13):
    """Removal of spurious pole-zero pairs (Froissart doublets), the last step
    of the AAA algorithm of Nakatsukasa, Sete & Trefethen: a pole whose residue
    is below tol * max|F| (or that sits on a support point, whose weight has
    vanished) is spurious; the support point nearest to it is dropped and the
    weights of the remaining support points are refitted by least squares
    (the smallest right singular vector of the Loewner matrix on the other
    samples).  Repeated until no such pole is left.  Returns (zj, fj, wj)."""
    Z = np.asarray(Z, dtype=np.float64)
    F = np.asarray(F, dtype=np.float64)
    scale = np.max(np.abs(F))
    for _ in range(len(zj)):
        poles = _poles(zj, wj)
        on_support = np.array([np.min(np.abs(zj - p)) <= 1e-12 * max(abs(p), 1e-300) for p in poles], dtype=bool)
        res = np.zeros(len(poles), dtype=complex)
        if (~on_support).any():
            res[~on_support] = _residues(zj, fj, wj, poles[~on_support])
        spurious = on_support | (np.abs(res) < tol * scale)
        if not spurious.any():
            break
        drop = {int(np.argmin(np.abs(zj - p))) for p in poles[spurious]}
        keep = np.array([k for k in range(len(zj)) if k not in drop], dtype=int)
        zj, fj = zj[keep], fj[keep]
        rows = ~np.isin(Z, zj)
        C = 1.0 / (Z[rows, None] - zj[None, :])
        _, _, Vh = np.linalg.svd((F[rows, None] - fj[None, :]) * C, full_matrices=False)
        wj = Vh[-1, :].conj()
    return zj, fj, wj


def soe_aaa(alpha: float, dt: float, T: float, m: int, samples: int = 2000, decades: float = 1.0):
    """SOE of t^-alpha/Gamma(1-alpha) on [dt, T] with m terms (Section 2.2).

    AAA runs on s^alpha over log-spaced samples of [1/T, 1/dt] widened by
    `decades` on each side, with m support points (m-1 poles).  The rational
    function divided by s has the m-1 poles plus a pole at s = 0 whose residue
    r(0) gives a term with exponent 0; all m residues become the weights.
    Spurious pole-zero pairs are removed first (_aaa_cleanup).  Returns (mu, w)
    sorted by mu, or raises ValueError when the cleanup leaves fewer than m
    terms, a pole is not real and negative or a weight is negative (in FP64 on
    these sample ranges the case beyond about m = 20: the extra degrees of
    freedom give complex or positive poles whose residues are not small
    enough to count as spurious)."""
    if not (0.0 < alpha < 1.0):
        raise ValueError("alpha must lie in (0, 1)")
    lo = math.log10(1.0 / T) - decades
    hi = math.log10(1.0 / dt) + decades
    Z = np.logspace(lo, hi, samples)
    F = Z ** alpha
    zj, fj, wj = _aaa(Z, F, m, 0.0)
    zj, fj, wj = _aaa_cleanup(Z, F, zj, fj, wj)
    if len(zj) < m:
        raise ValueError("spurious poles removed: fewer than m terms remain")
    poles = _poles(zj, wj)
    if np.max(np.abs(poles.imag)) > 1e-8 * np.max(np.abs(poles)):
        raise ValueError("complex poles")
    poles = poles.real
    if np.any(poles >= 0.0):
        raise ValueError("non-negative pole")

    def bary(s, deriv=False):
        c = 1.0 / (s - zj)
        if not deriv:
            return (c @ (wj * fj)), (c @ wj)
        return -(c * c) @ wj

    mu, w = [], []
    for p in poles:
        num, _ = bary(p)
        dden = bary(p, deriv=True)
        res = num / (p * dden)     # residue of r(s)/s at s = p
        mu.append(-p)
        w.append(res)
    num0, den0 = bary(0.0)
    mu.append(0.0)
    w.append(num0 / den0)        # residue of r(s)/s at s = 0
    mu = np.array(mu)
    w = np.array(w)
    order = np.argsort(mu)
    mu, w = mu[order], w[order]
    if np.any(w < 0.0):
        raise ValueError("negative weight")
    return mu, w


def soe_expquad(alpha: float, dt: float, T: float, m: int, tail: float = 1e-12):
    """Positive SOE from the trapezoidal rule on
    t^-alpha/Gamma(1-alpha) = sin(pi alpha)/pi * int_R exp(alpha x - t e^x) dx.
    Nodes x_j span [x_lo, x_hi] where the neglected tails are below `tail`
    relative to the kernel on [dt, T]."""
    if not (0.0 < alpha < 1.0):
        raise ValueError("alpha must lie in (0, 1)")
    x_lo = (math.log(tail * alpha * math.gamma(alpha)) + alpha * math.log(1.0 / T)) / alpha
    x_hi = math.log(-math.log(tail) / dt) + 1.0
    x = np.linspace(x_lo, x_hi, m)
    h = x[1] - x[0]
    mu = np.exp(x)
    w = math.sin(math.pi * alpha) / math.pi * h * np.exp(alpha * x)
    return mu, w


def _nnls_on_grid(alpha, dt, T, count, lo_dec, hi_dec):
    mu = np.logspace(math.log10(1.0 / T) - lo_dec, math.log10(1.0 / dt) + hi_dec, count)
    t = np.logspace(math.log10(dt / 10.0), math.log10(T), 1200)
    k = kernel_exact(alpha, t)
    A = np.exp(-np.multiply.outer(t, mu)) / k[:, None]
    w, _ = scipy.optimize.nnls(A, np.ones_like(t), maxiter=50 * count * count)
    keep = w > 0.0
    return mu[keep], w[keep]


def soe_nnls(alpha: float, dt: float, T: float, m: int, max_mass: float = 1.01):
    """Positive SOE with exactly m terms (see the module docstring).

    For each grid extension (lo, hi) in decades beyond [1/T, 1/dt] and each
    grid size from m upwards, NNLS picks the positive weights; among the fits
    with exactly m positive weights (and mass at most max_mass times the
    kernel's) the one with the smallest maximum relative error on [dt, T] is
    returned as (mu, w), sorted by mu."""
    if not (0.0 < alpha < 1.0):
        raise ValueError("alpha must lie in (0, 1)")
    if m < 1:
        raise ValueError("m must be positive")
    best = None
    for lo in (1.0, 1.5, 2.0):
        for hi in (1.0, 2.0, 3.0):
            for count in range(m, 2 * m + 8):
                mu, w = _nnls_on_grid(alpha, dt, T, count, lo, hi)
                if len(mu) != m:
                    continue
                # a term whose decay is complete long before dt is invisible to
                # the error on [dt, T] yet enters the scheme through its mass
                # w_j / mu_j (the per-mode weight rho_j of the BDF2 update);
                # NNLS sometimes gives such terms huge weights, so fits whose
                # mass on [0, T] exceeds max_mass times the kernel's are rejected
                if soe_mass(mu, w, T) > max_mass * kernel_mass(alpha, T):
                    continue
                err = max_rel_error(alpha, mu, w, dt, T)
                if best is None or err < best[0]:
                    best = (err, mu, w)
    if best is None:
        raise ValueError("no positive fit with exactly m terms")
    return best[1], best[2]


DIRAC_RATE = 1e12        # mu dt of the completing term


def soe_complete(alpha: float, mu, w, dt: float, T: float):
    """(mu, w) with one term appended that carries kernel_mass - soe_mass on
    [0, T] (see the module docstring); unchanged when nothing is missing."""
    mu = np.asarray(mu, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    missing = kernel_mass(alpha, T) - soe_mass(mu, w, T)
    if not missing > 1e-12 * kernel_mass(alpha, T):
        return mu.copy(), w.copy()
    rate = DIRAC_RATE / dt
    return np.append(mu, rate), np.append(w, missing * rate)


def soe_build(alpha: float, dt: float, T: float, m: int):
    """Default SOE: ``soe_nnls`` with m - 1 terms and no more mass than the
    kernel, plus the completing term (m terms; the m-term fit when no such fit
    exists or nothing is missing)."""
    if m >= 2:
        try:
            mu, w = soe_complete(alpha, *soe_nnls(alpha, dt, T, m - 1, max_mass=1.0 + 1e-9), dt, T)
            if len(mu) == m:
                return mu, w
        except ValueError:
            pass
    return soe_nnls(alpha, dt, T, m)


def kernel_mass(alpha: float, T: float) -> float:
    """Closed form of int_0^T t^-alpha / Gamma(1-alpha) dt = T^(1-alpha) / Gamma(2-alpha)."""
    return T ** (1.0 - alpha) / math.gamma(2.0 - alpha)


def soe_mass(mu, w, T: float) -> float:
    """int_0^T sum_j w_j exp(-mu_j t) dt."""
    mu = np.asarray(mu, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    return float(np.sum(w * -np.expm1(-mu * T) / mu))


def max_rel_error(alpha: float, mu, w, dt: float, T: float, points: int = 400) -> float:
    """max over 400 log points of [dt, T] of |SOE - kernel| / kernel."""
    t = np.logspace(math.log10(dt), math.log10(T), points)
    ex = kernel_exact(alpha, t)
    return float(np.max(np.abs(soe_eval(mu, w, t) - ex) / ex))
