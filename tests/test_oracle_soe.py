"""Pins of the oracle's SOE kernels and special functions (no GPU).

P1: the sum of exponentials against the closed-form Caputo kernel
t^-alpha / Gamma(1-alpha) on 400 log points of [dt, T]; two independent
constructions agree within the sum of their errors.  The paper prints no SOE
error, so the bounds below are the achieved accuracies (stated, not pinned by
the paper).
"""
import math

import numpy as np
import pytest
import scipy.special

from oracle import orc, soe, special

# (alpha, dt, T, m, bound on max relative kernel error over [dt, T])
WORKLOAD_SOES = [
    (0.5, 1e-3, 1.0, 16, 1e-4),      # 2D 64^2 FP64 case, SOE on [1e-3, 1]
    (0.3, 5e-4, 0.5, 32, 1e-8),      # 2D 1024^2 cases, 1000 steps
    (0.5, 5e-4, 0.5, 32, 1e-8),
    (0.8, 5e-4, 0.5, 32, 1e-8),
    (0.6, 2e-4, 0.04, 32, 1e-8),     # 3D 256^3, 200 steps
    (0.2, 2e-4, 0.1, 16, 1e-4),      # 3D 192^3 sweep, 500 steps
    (0.5, 2e-4, 0.1, 48, 1e-11),
    (0.9, 2e-4, 0.1, 48, 1e-11),
]


@pytest.mark.parametrize("alpha,dt,T,m,bound", WORKLOAD_SOES)
def test_nnls_soe_matches_closed_form(alpha, dt, T, m, bound):
    mu, w = soe.soe_nnls(alpha, dt, T, m)
    assert len(mu) == m and len(w) == m
    assert np.all(mu >= 0) and np.all(w > 0)            # completely monotone (Section 2.2)
    assert soe.max_rel_error(alpha, mu, w, dt, T) <= bound


def test_aaa_soe_paper_recipe_small_m():
    # Section 2.2: AAA on s^alpha, divided by s -> no Dirac term, positive terms
    alpha, dt, T, m = 0.5, 1e-3, 1.0, 16
    mu, w = soe.soe_aaa(alpha, dt, T, m)
    assert len(mu) == m
    assert np.all(mu >= 0) and np.all(w >= 0)
    e_aaa = soe.max_rel_error(alpha, mu, w, dt, T)
    assert e_aaa < 5e-4
    # independent construction: cross-check within the sum of the two errors
    mu2, w2 = soe.soe_nnls(alpha, dt, T, m)
    e_nnls = soe.max_rel_error(alpha, mu2, w2, dt, T)
    t = np.logspace(math.log10(dt), math.log10(T), 400)
    k = soe.kernel_exact(alpha, t)
    diff = np.max(np.abs(soe.soe_eval(mu, w, t) - soe.soe_eval(mu2, w2, t)) / k)
    assert diff <= (e_aaa + e_nnls) * (1 + 1e-9)


def test_aaa_laplace_identity():
    # the SOE's Laplace transform sum w/(s+mu) approximates s^(alpha-1)
    alpha, dt, T, m = 0.5, 1e-3, 1.0, 16
    mu, w = soe.soe_aaa(alpha, dt, T, m)
    s = np.logspace(0, 3, 50)
    K = (1.0 / (s[:, None] + mu[None, :])) @ w
    assert np.max(np.abs(K / s ** (alpha - 1) - 1)) < 1e-4


def test_trapezoid_soe_converges_and_agrees():
    alpha, dt, T = 0.6, 2e-4, 0.04
    mu, w = soe.soe_expquad(alpha, dt, T, 400, tail=1e-13)
    e_tr = soe.max_rel_error(alpha, mu, w, dt, T)
    assert e_tr < 1e-9
    mu2, w2 = soe.soe_nnls(alpha, dt, T, 32)
    e2 = soe.max_rel_error(alpha, mu2, w2, dt, T)
    t = np.logspace(math.log10(dt), math.log10(T), 400)
    k = soe.kernel_exact(alpha, t)
    diff = np.max(np.abs(soe.soe_eval(mu, w, t) - soe.soe_eval(mu2, w2, t)) / k)
    assert diff <= (e_tr + e2) * (1 + 1e-9)


def test_kernel_exact_gamma_identity():
    # t^-alpha/Gamma(1-alpha) integrates to t^(1-alpha)/Gamma(2-alpha); the
    # algebraic end-point weight of QUADPACK carries the singularity
    import scipy.integrate
    alpha, t = 0.37, 0.8
    g = scipy.special.gamma(1 - alpha)
    val, _ = scipy.integrate.quad(lambda s: 1.0 / g, 0.0, t, weight="alg", wvar=(-alpha, 0.0))
    ref = t ** (1 - alpha) / scipy.special.gamma(2 - alpha)
    assert abs(val - ref) < 1e-12
    # and the closed form itself at a point
    assert abs(soe.kernel_exact(alpha, t) - t ** -alpha / g) < 1e-15


# --------------------------- special functions ---------------------------

def test_mittag_leffler_special_cases():
    x = np.linspace(0.0, 2.0, 11)
    # E_1(z) = exp(z)
    assert np.allclose(special.mittag_leffler(1.0, -x), np.exp(-x), rtol=1e-13, atol=1e-15)
    # E_{1/2}(-x) = exp(x^2) erfc(x)
    assert np.allclose(special.mittag_leffler(0.5, -x), scipy.special.erfcx(x), rtol=1e-12, atol=1e-14)
    # E_2(-x^2) = cos(x)
    assert np.allclose(special.mittag_leffler(2.0, -x ** 2), np.cos(x), rtol=1e-12, atol=1e-12)
    # complex argument: E_1(i y) = exp(i y)
    y = np.linspace(-2, 2, 9)
    assert np.allclose(special.mittag_leffler(1.0, 1j * y), np.exp(1j * y), rtol=1e-13, atol=1e-14)
    # the spectral-integral branch (real z < -0.5, alpha < 1): erfcx far out
    xl = np.linspace(0.6, 40.0, 30)
    assert np.allclose(special.mittag_leffler(0.5, -xl), scipy.special.erfcx(xl), rtol=1e-12, atol=0.0)


@pytest.mark.parametrize("alpha", [0.2, 0.3, 0.7, 0.9])
def test_mittag_leffler_branches_agree_and_large_argument(alpha):
    # near the switch the power series is still accurate: both branches agree
    for x in (0.51, 0.7, 0.9):
        series = math.fsum((-x) ** k / math.gamma(alpha * k + 1.0) for k in range(150))
        assert abs(special._ml_negative_real(alpha, x) / series - 1.0) < 1e-13
    # far out: E_alpha(-x) ~ sum_{k>=1} (-1)^(k+1) x^-k / Gamma(1 - alpha k)
    x = 1e4
    asym = sum((-1) ** (k + 1) * x ** -k * scipy.special.rgamma(1.0 - alpha * k) for k in range(1, 7))
    assert abs(special.mittag_leffler(alpha, -x) / asym - 1.0) < 1e-12
    # the decay case of the paper-variable pin (alpha = 0.3, lambda t^alpha ~ 3),
    # where the power series loses every digit: between the neighbours' bounds
    e = special.mittag_leffler(alpha, -2.97)
    assert 0.0 < e < special.mittag_leffler(alpha, -2.5) < 1.0


def test_mittag_leffler_against_mpmath():
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    # the series cancels badly when alpha is small and |z| large; the oracle
    # only evaluates it where its largest term stays O(10)
    for alpha, z in [(0.3, -0.2), (0.3, -1.0), (0.6, -0.2), (0.6, -1.0), (0.6, -2.5),
                     (0.9, -0.2), (0.9, -1.0), (0.9, -2.5)]:
        ref = mpmath.nsum(lambda k: mpmath.mpf(z) ** k / mpmath.gamma(alpha * k + 1), [0, mpmath.inf])
        assert abs(special.mittag_leffler(alpha, z) - float(ref)) < 1e-13


def test_cq_power_weights():
    dt = 1e-2
    # alpha = 1: the BDF2 coefficients themselves
    W1 = special.cq_weights_power(1.0, dt, 6)
    assert np.allclose(W1, [1.5, -2.0, 0.5, 0, 0, 0, 0], atol=1e-15)
    # alpha = 1/2: the series squared equals dt * delta(zeta)
    Wh = special.cq_weights_power(0.5, dt, 40)
    sq = np.convolve(Wh, Wh)[:41]
    ref = np.zeros(41)
    ref[:3] = np.array([1.5, -2.0, 0.5]) * dt
    assert np.allclose(sq, ref, atol=1e-15)


def test_cq_soe_weights():
    dt = 1e-2
    # one term with mu = 0 and weight w: delta * w dt / delta = w dt
    W = special.cq_weights_soe([0.0], [2.0], dt, 10)
    assert np.allclose(W, np.r_[2.0 * dt, np.zeros(10)], atol=1e-16)
    # mu > 0: delta(1) = 0 so the weights sum to zero (the derivative of a constant)
    W = special.cq_weights_soe([3.0, 40.0], [1.0, 0.5], dt, 4000)
    assert abs(W.sum()) < 1e-12
    # first weight is eta = b0 sum_j w_j dt / (b0 + mu_j dt)
    eta = sum(1.5 * w * dt / (1.5 + m * dt) for m, w in [(3.0, 1.0), (40.0, 0.5)])
    assert abs(W[0] - eta) < 1e-16


def test_kernel_mass_closed_form():
    import scipy.integrate
    for alpha in (0.2, 0.5, 0.9):
        for T in (0.03, 1.0):
            num, _ = scipy.integrate.quad(lambda t: t ** -alpha / scipy.special.gamma(1 - alpha), 0.0, T, limit=200)
            assert abs(soe.kernel_mass(alpha, T) - num) < 1e-8 * num


@pytest.mark.parametrize("alpha", [0.2, 0.3, 0.5, 0.9])
@pytest.mark.parametrize("dt,T", [(2e-4, 0.1), (1e-3, 1.0), (5e-4, 0.5)])
def test_soe_mass_bounded_by_kernel_mass(alpha, dt, T):
    # Each mode enters the BDF2 step through its mass w_j / mu_j; a term that
    # has decayed before dt cannot be seen by the error on [dt, T] but would
    # swamp eta.  The tables must not carry more mass on [0, T] than the kernel
    # (they carry a little less: the singular part below the fitted times).
    # Both builders are checked: the oracle's and the library's (independent code).
    from paper_2411_17294_gb300 import soe as psoe
    for m in (16, 48):
        for mu, w in (soe.soe_nnls(alpha, dt, T, m), psoe.build(alpha, dt, T, m)):
            ratio = soe.soe_mass(mu, w, T) / soe.kernel_mass(alpha, T)
            assert 0.5 < ratio <= 1.01, (alpha, m, ratio)
            assert np.max(w / mu) < 1e3


@pytest.mark.parametrize("alpha", [0.2, 0.5, 0.8, 0.9])
def test_completed_table_carries_the_kernel_mass_and_fits_the_same(alpha):
    # The completing term (a Dirac term of weight = the missing mass, realised as
    # one exponential at 1e12/dt) leaves the table on [dt, T] unchanged and makes
    # its integral over [0, T] that of the kernel.  Both builders.
    from paper_2411_17294_gb300 import soe as psoe
    dt, T, m = 5e-4, 0.5, 32
    base = soe.soe_nnls(alpha, dt, T, m - 1, max_mass=1.0 + 1e-9)
    mu, w = soe.soe_complete(alpha, *base, dt, T)
    assert len(mu) == m and mu[-1] == 1e12 / dt
    t = np.logspace(np.log10(dt), np.log10(T), 50)
    assert np.array_equal(soe.soe_eval(mu, w, t), soe.soe_eval(*base, t))
    for table in ((mu, w), soe.soe_build(alpha, dt, T, m), psoe.build(alpha, dt, T, m)):
        assert len(table[0]) == m
        assert abs(soe.soe_mass(*table, T) / soe.kernel_mass(alpha, T) - 1.0) < 1e-9
        assert soe.max_rel_error(alpha, *table, dt, T) < 1e-3


@pytest.mark.parametrize("alpha", [0.3, 0.7])
def test_dirac_term_is_a_classical_derivative(alpha):
    # A table holding only the completing term (mass M) turns the fractional
    # step into BDF2 for M d sigma/dt = -sigma/Wi + ..., i.e. the alpha = 1 scheme
    # with relaxation time M Wi: the oracle's classical path is the check.
    dt, steps, Wi, M = 1e-2, 40, 0.7, 0.3
    rate = soe.DIRAC_RATE / dt
    rng = np.random.default_rng(3)
    sig0 = rng.normal(size=(3, 5))
    kap = np.zeros((4, 5))
    frac = orc.forward(orc.Problem(dim=2, n=(5, 1), alpha=alpha, Wi=Wi, beta=0.5, dt=dt, mu=[rate], w=[M * rate]),
                       sig0, kap, None, steps)
    classic = orc.forward(orc.Problem(dim=2, n=(5, 1), alpha=1.0, Wi=M * Wi, beta=0.5, dt=dt, mu=[], w=[]),
                          sig0, kap, None, steps)
    assert np.max(np.abs(frac - classic)) < 1e-10 * np.max(np.abs(classic))


@pytest.mark.parametrize("alpha", [0.2, 0.5, 0.8, 0.9])
def test_completed_table_gives_the_mittag_leffler_relaxation(alpha):
    # Zero flow at the 2D 1024^2 workload's step (dt = 5e-4, 1000 steps, m = 32):
    # with the SDIRK2 start the completed table reproduces sigma0 E_alpha(-t^alpha/Wi)
    # to ~1e-6 for every alpha, where the uncompleted fit (missing 8% of the mass
    # at alpha = 0.8, 28% at 0.9) is off by up to 20%.
    dt, steps, Wi = 5e-4, 1000, 1.0
    T = dt * steps
    exact = special.mittag_leffler(alpha, -T ** alpha / Wi)
    errs = []
    for mu, w in (soe.soe_build(alpha, dt, T, 32), soe.soe_nnls(alpha, dt, T, 32)):
        prob = orc.Problem(dim=2, n=(1, 1), alpha=alpha, Wi=Wi, beta=0.5, dt=dt, mu=mu, w=w, start="sdirk2")
        r = orc.forward(prob, np.ones((3, 1)), np.zeros((4, 1)), None, steps)[0, 0]
        errs.append(abs(r - exact) / exact)
    assert errs[0] < 2e-6, errs
    if alpha >= 0.8:
        assert errs[1] > 1e-2, errs


def test_aaa_cleanup_removes_froissart_doublets():
    # f(s) = 1/(s + 2) + 3/(s + 5) is rational of type (1, 2): three support
    # points reproduce it exactly, and AAA run to eight support points adds
    # five spurious poles (pole-zero pairs with negligible residues).  The
    # cleanup of the AAA algorithm (Nakatsukasa, Sete & Trefethen) removes them
    # and leaves the poles -2, -5 with residues 1, 3.
    Z = np.logspace(-1, 2, 400)
    F = 1.0 / (Z + 2.0) + 3.0 / (Z + 5.0)
    zj, fj, wj = soe._aaa(Z, F, 8, 0.0)
    assert len(soe._poles(zj, wj)) == 7
    zj, fj, wj = soe._aaa_cleanup(Z, F, zj, fj, wj)
    poles = soe._poles(zj, wj)
    order = np.argsort(poles.real)
    assert np.allclose(poles[order], [-5.0, -2.0], rtol=1e-10)
    assert np.allclose(soe._residues(zj, fj, wj, poles[order]), [3.0, 1.0], rtol=1e-10)


def test_product_aaa_matches_oracle_aaa():
    # the library's builder and the oracle's are written independently; on the
    # paper's recipe at m = 16 they give the same table
    from paper_2411_17294_gb300 import soe as psoe
    mu, w = psoe.aaa(0.5, 1e-3, 1.0, 16)
    mu2, w2 = soe.soe_aaa(0.5, 1e-3, 1.0, 16)
    assert np.allclose(mu, mu2, rtol=1e-9, atol=0.0) and np.allclose(w, w2, rtol=1e-9)


@pytest.mark.parametrize("alpha,m", [(0.6, 32), (0.5, 48), (0.2, 32), (0.9, 32)])
def test_aaa_beyond_twenty_terms_is_refused(alpha, m):
    # Measured reading of the paper's recipe in FP64 at the workloads' sizes
    # (dt = 2e-4, T = 200 dt): even after the removal of spurious pole-zero
    # pairs, the m-point AAA approximant of s^alpha keeps complex or positive
    # poles (residues ~1e-8 of max|s^alpha|, far above the cleanup's 1e-13), so
    # both builders refuse the table and the NNLS fit serves these m.
    from paper_2411_17294_gb300 import soe as psoe
    dt = 2e-4
    with pytest.raises(ValueError):
        soe.soe_aaa(alpha, dt, 200 * dt, m)
    with pytest.raises(ValueError):
        psoe.aaa(alpha, dt, 200 * dt, m)
    mu, w = soe.soe_nnls(alpha, dt, 200 * dt, m)
    assert len(mu) == m and soe.max_rel_error(alpha, mu, w, dt, 200 * dt) < 1e-7
