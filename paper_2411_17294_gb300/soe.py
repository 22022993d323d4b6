"""Host-side FP64 construction of the sum-of-exponentials (SOE) kernel table.

The stress law's memory term is the Caputo derivative of order alpha with kernel
t^-alpha / Gamma(1-alpha).  Kernel compression (Section 2.2) replaces it by
sum_j w_j exp(-mu_j t) with non-negative exponents and weights (completely
monotone by Bernstein's theorem), so each grid point carries m mode tensors.
The table is computed once on the host in FP64 and handed to tfs_set_soe.

``build(alpha, dt, T, m)``  positive table with exactly m terms whose relative
    error is small on [dt, T].  Exponents lie on a geometric grid spanning
    [1/T, 1/dt] widened on both sides; weights are the non-negative least-squares
    fit of the relative kernel error on log-spaced times in [dt/10, T].  The grid
    density is searched so that exactly m weights come out positive.
    By default the last of the m terms is the mass completion below.
``complete(alpha, mu, w, dt, T)``  appends one term holding the part of the
    kernel's integral over [0, T] that the table misses (the singular part
    below the fitted times, 8% of it at alpha = 0.8 and 28% at 0.9 for a fit
    from dt): the Dirac term w_inf delta(t) of the Khristenko form of the
    compressed kernel (eq. tf_approximate_kernel_khristenko), realised as one
    exponential decaying a trillion times faster than dt, which the BDF2 mode
    update turns into w_inf times the BDF2 difference quotient of the stress.
    Without it the step's local weight misses that mass, and the zero-flow
    relaxation at alpha = 0.8 is several percent off its closed form.
``aaa(alpha, dt, T, m)``  the paper's recipe: AAA rational approximation of
    s^alpha (Laplace variable) divided by s, with the removal of spurious
    pole-zero pairs, partial fractions, inverse Laplace transform; valid while
    the poles stay real and negative (about m <= 20: beyond, complex or
    positive poles remain whose residues are too large to count as spurious).
"""
from __future__ import annotations

import math

import numpy as np
from scipy import linalg, optimize, special


def caputo_kernel(alpha: float, t):
    t = np.asarray(t, dtype=np.float64)
    return np.power(t, -alpha) / special.gamma(1.0 - alpha)


def evaluate(mu, w, t):
    t = np.asarray(t, dtype=np.float64)
    return np.exp(-np.outer(t, np.asarray(mu))) @ np.asarray(w)


def relative_error(alpha, mu, w, dt, T, samples=400):
    t = np.geomspace(dt, T, samples)
    k = caputo_kernel(alpha, t)
    return float(np.max(np.abs(evaluate(mu, w, t) / k - 1.0)))


def _fit(alpha, dt, T, count, widen_lo, widen_hi, times):
    exps = np.geomspace(10.0 ** (-widen_lo) / T, 10.0 ** widen_hi / dt, count)
    design = np.exp(-np.outer(times, exps)) / caputo_kernel(alpha, times)[:, None]
    weights, _ = optimize.nnls(design, np.ones(len(times)), maxiter=60 * count * count)
    keep = weights > 0
    return exps[keep], weights[keep]


def mass(alpha: float, T: float) -> float:
    """int_0^T t^-alpha / Gamma(1-alpha) dt."""
    return T ** (1.0 - alpha) / special.gamma(2.0 - alpha)


def complete(alpha: float, mu, w, dt: float, T: float, speed: float = 1e12):
    """The table with one term appended that carries the kernel's missing mass
    on [0, T], at exponent speed/dt (returned unchanged when nothing is
    missing)."""
    mu = np.asarray(mu, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    have = float(np.sum(w * -np.expm1(-mu * T) / mu))
    deficit = mass(alpha, T) - have
    if deficit <= 1e-12 * mass(alpha, T):
        return mu.copy(), w.copy()
    mu_fast = speed / dt
    return np.concatenate([mu, [mu_fast]]), np.concatenate([w, [deficit * mu_fast]])


def build(alpha: float, dt: float, T: float, m: int, complete_mass: bool = True):
    """Positive SOE table (mu, w) with exactly m terms, sorted by mu: the fit of
    m - 1 terms and the mass completion (complete_mass), else m fitted terms."""
    if complete_mass and m >= 2:
        # a fit carrying no more than the kernel's mass, so that the completion
        # can make the total exact
        try:
            mu, w = complete(alpha, *_build_fit(alpha, dt, T, m - 1, 1.0 + 1e-9), dt, T)
            if len(mu) == m:
                return mu, w
        except ValueError:
            pass
    return _build_fit(alpha, dt, T, m, 1.01)


def _build_fit(alpha: float, dt: float, T: float, m: int, max_mass: float):
    if not 0.0 < alpha < 1.0:
        raise ValueError("the SOE table is needed only for 0 < alpha < 1")
    if m < 1 or dt <= 0 or T <= dt:
        raise ValueError("need m >= 1 and 0 < dt < T")
    times = np.geomspace(dt / 10.0, T, 1200)
    best = None
    for widen_hi in (1.0, 2.0, 3.0):
        for widen_lo in (1.0, 1.5, 2.0):
            # the number of positive weights grows with the grid size; scan upwards
            for count in range(m, 2 * m + 8):
                mu, w = _fit(alpha, dt, T, count, widen_lo, widen_hi, times)
                if len(mu) < m:
                    continue
                if len(mu) > m:
                    break
                # NNLS may put a huge weight on an exponent so large that its
                # term has died out before dt: the error on [dt, T] cannot see
                # it, but the step sees its mass w/mu.  Keep only tables whose
                # mass on [0, T] does not exceed max_mass times the kernel's.
                have = float(np.sum(w * -np.expm1(-mu * T) / mu))
                if have > max_mass * mass(alpha, T):
                    continue
                err = relative_error(alpha, mu, w, dt, T)
                if best is None or err < best[0]:
                    best = (err, mu, w)
    if best is None:
        raise ValueError(f"no positive table with exactly {m} terms")
    order = np.argsort(best[1])
    return best[1][order].copy(), best[2][order].copy()


def aaa(alpha: float, dt: float, T: float, m: int, samples: int = 2000):
    """AAA on s^alpha over [0.1/T, 10/dt], divided by s (Section 2.2); m terms
    (m - 1 poles plus the residue at s = 0).  Raises ValueError when the table
    is not real and non-negative."""
    z = np.geomspace(0.1 / T, 10.0 / dt, samples)
    f = z ** alpha
    free = np.ones(samples, dtype=bool)
    approx = np.full(samples, f.mean())
    sup, val = [], []
    bw = None
    for _ in range(m):
        resid = np.where(free, np.abs(f - approx), -1.0)
        i = int(np.argmax(resid))
        sup.append(z[i]); val.append(f[i]); free[i] = False
        zs, fs = np.array(sup), np.array(val)
        cauchy = 1.0 / (z[free][:, None] - zs[None, :])
        loewner = (f[free][:, None] - fs[None, :]) * cauchy
        bw = np.linalg.svd(loewner)[2][-1]
        approx = f.copy()
        approx[free] = (cauchy @ (bw * fs)) / (cauchy @ bw)
    zs, fs = np.array(sup), np.array(val)

    def denominator_zeros(zs, bw):
        k = len(zs)
        A = np.zeros((k + 1, k + 1)); A[0, 1:] = bw; A[1:, 0] = 1.0; A[1:, 1:] = np.diag(zs)
        B = np.eye(k + 1); B[0, 0] = 0.0
        ev = linalg.eigvals(A, B)
        return ev[np.isfinite(ev)]

    # Froissart doublets (the AAA algorithm's cleanup step): a pole with a
    # residue below 1e-13 of max|f|, or one on a support point (zero weight),
    # is spurious; drop the nearest support point, refit the weights by the
    # Loewner least-squares problem on the remaining samples, repeat
    fmax = float(np.max(np.abs(f)))
    while len(zs) > 1:
        poles = denominator_zeros(zs, bw)
        bad = []
        for p in poles:
            gap = np.abs(p - zs)
            if gap.min() <= 1e-12 * abs(p):
                bad.append(int(np.argmin(gap)))
                continue
            c = 1.0 / (p - zs)
            if abs(np.sum(bw * fs * c) / -np.sum(bw * c * c)) < 1e-13 * fmax:
                bad.append(int(np.argmin(gap)))
        if not bad:
            break
        keep = np.setdiff1d(np.arange(len(zs)), np.unique(bad))
        zs, fs = zs[keep], fs[keep]
        rest = ~np.isin(z, zs)
        cauchy = 1.0 / (z[rest][:, None] - zs[None, :])
        bw = np.linalg.svd((f[rest][:, None] - fs[None, :]) * cauchy)[2][-1]
    if len(zs) < m:
        raise ValueError("AAA: spurious poles removed, fewer than m terms remain")
    poles = denominator_zeros(zs, bw)
    if np.any(np.abs(poles.imag) > 1e-8 * np.abs(poles)) or np.any(poles.real >= 0):
        raise ValueError("AAA produced complex or non-negative poles")
    poles = poles.real
    num = lambda s: np.sum(bw * fs / (s - zs))
    den = lambda s: np.sum(bw / (s - zs))
    dden = lambda s: -np.sum(bw / (s - zs) ** 2)
    mu = np.concatenate([-poles, [0.0]])
    w = np.concatenate([[num(p) / (p * dden(p)) for p in poles], [num(0.0) / den(0.0)]])
    if np.any(w < 0):
        raise ValueError("AAA produced a negative weight")
    order = np.argsort(mu)
    return mu[order], w[order]
