"""Pins of the FP64 oracle's stress step against what the paper and the
mathematics fix (no GPU).

P2  zero flow: sigma(t) = sigma0 E_alpha(-t^alpha / Wi)  (Section 5.1 closed form)
P3  (i) the mode recursion equals the full-history convolution with the exact
    generating function of the BDF2 mode scheme; (ii) with an SOE accurate far
    below dt the scheme equals BDF2 convolution quadrature of the exact symbol
P4  alpha = 1: Oldroyd-B relaxation exp(-t/Wi) at second order; the steady
    stress of the Lemma of Section 3.3 (Gaussian with C = I/2 - Wi D) for
    symmetric trace-free D; the Lyapunov steady state for a general kappa;
    alpha = 1 - 10^-k converges to the alpha = 1 path, linearly in 1 - alpha
P5  the full d x d tensor form stays symmetric and equals the packed form
P6  uniform kappa and constant u give the same stress at every point
P7  smooth start from rest: second order in dt for every alpha
P8  one Fourier mode advected by a constant velocity follows
    E_alpha(-(1/Wi + i k u) t^alpha) as dt and h go to zero
P9  the stress is affine in (sigma0, G)
adjoint: the reference adjoint agrees with FP64 central finite differences.

Independent formulations used here (full-tensor Kronecker systems, generating
functions, NumPy solves) share no code with the oracle's step.
"""
import math

import numpy as np
import pytest
import scipy.special

from oracle import orc, soe, special
from paper_2411_17294_gb300 import inputs

PACK2 = [(0, 0), (0, 1), (1, 1)]
PACK3 = [(0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1)]


def pack(S):
    d = S.shape[0]
    pairs = PACK2 if d == 2 else PACK3
    return np.array([S[i, j] for i, j in pairs])


def unpack(v, d):
    pairs = PACK2 if d == 2 else PACK3
    S = np.zeros((d, d))
    for c, (i, j) in enumerate(pairs):
        S[i, j] = S[j, i] = v[c]
    return S


def direct_history_solve(W, kap_of_n, S0, Wi, G, dt, alpha, steps):
    """Full-history scheme  sum_{k=0}^{n+1} W_k (S^{n+1-k} - S0)
         = dt [k* S + S k*^T - S/Wi + G (k* + k*^T) g(t_{n+1})]   (S^k = S0, k <= 0)
    solved with full d x d unknowns (row-major vec, Kronecker products)."""
    d = S0.shape[0]
    I = np.eye(d)
    hist = [S0.copy()]
    for n in range(steps):
        k = 2.0 * kap_of_n(n) - kap_of_n(n - 1 if n > 0 else 0)
        g = 1.0 if alpha == 1.0 else ((n + 1) * dt) ** (alpha - 1) / math.gamma(alpha)
        L = np.kron(k, I) + np.kron(I, k)
        A = (W[0] + dt / Wi) * np.eye(d * d) - dt * L
        rhs = W[0] * S0.ravel() + dt * G * g * (k + k.T).ravel()
        for j in range(1, n + 2):
            rhs -= W[j] * (hist[n + 1 - j] - S0).ravel()
        hist.append(np.linalg.solve(A, rhs).reshape(d, d))
    return hist


def point_problem(dim, alpha, Wi, beta, dt, mu=None, w=None, **kw):
    return orc.Problem(dim=dim, n=(1,) * dim, alpha=alpha, Wi=Wi, beta=beta, dt=dt,
                       mu=np.zeros(0) if mu is None else mu, w=np.zeros(0) if w is None else w, **kw)


# ------------------------------------------------------------------ P3 (i)
@pytest.mark.parametrize("dim,alpha", [(2, 0.5), (3, 0.3), (3, 0.8), (2, 1.0)])
def test_mode_recursion_equals_full_history(dim, alpha):
    rng = np.random.default_rng(7)
    dt, steps, Wi, beta = 2e-3, 80, 1.3, 0.4
    if alpha < 1:
        mu, w = soe.soe_nnls(alpha, dt, steps * dt, 8)
        W = special.cq_weights_soe(mu, w, dt, steps)
    else:
        mu = w = None
        W = np.zeros(steps + 1)
        W[:3] = [1.5, -2.0, 0.5]
    kseq = [rng.normal(scale=2.0, size=(dim, dim)) for _ in range(steps)]
    S0 = unpack(rng.normal(size=3 if dim == 2 else 6), dim)
    G = (1 - beta) / Wi
    hist = direct_history_solve(W, lambda n: kseq[n], S0, Wi, G, dt, alpha, steps)
    prob = point_problem(dim, alpha, Wi, beta, dt, mu, w)
    o = orc.Oracle(prob, pack(S0)[:, None])
    for n in range(steps):
        o.step(kseq[n].reshape(-1, 1), kseq[n - 1 if n > 0 else 0].reshape(-1, 1))
        ref = pack(hist[n + 1])
        assert np.allclose(o.sig_n[:, 0], ref, rtol=1e-11, atol=1e-12 * np.max(np.abs(ref)))


# ------------------------------------------------------------------ P3 (ii)
def test_scheme_is_bdf2_convolution_quadrature_of_exact_symbol():
    alpha, dt, steps = 0.5, 1e-2, 100
    mu, w = soe.soe_expquad(alpha, dt * 1e-14, 10 * steps * dt, 700, tail=1e-14)
    Wsoe = special.cq_weights_soe(mu, w, dt, steps)
    Wex = special.cq_weights_power(alpha, dt, steps)
    # the SOE resolves the kernel down to t_min = 1e-14 dt; the kernel mass it
    # misses below t_min is (t_min/dt)^(1-alpha) = 1e-7 of the first weight
    assert np.max(np.abs(Wsoe - Wex)) < 2e-7 * abs(Wex[0])
    assert np.max(np.abs(Wsoe[3:] - Wex[3:])) < 1e-12 * abs(Wex[0])


# ------------------------------------------------------------------ P2
@pytest.mark.parametrize("alpha", [0.5, 0.8])
def test_zero_flow_mittag_leffler(alpha):
    Wi, T = 1.0, 1.0
    sig0 = np.array([[1.0], [-0.4], [0.7]])

    def closed(t):
        if alpha == 0.5:
            return scipy.special.erfcx(math.sqrt(t) / Wi)
        return special.mittag_leffler(alpha, -t ** alpha / Wi)

    errs = []
    for steps in (100, 200, 400):
        dt = T / steps
        mu, w = soe.soe_expquad(alpha, dt * 1e-14, 10 * T, 700, tail=1e-14)
        o = orc.Oracle(point_problem(2, alpha, Wi, 0.5, dt, mu, w), sig0)
        sT = o.run(steps, np.zeros((4, 1)))
        ratio = sT[:, 0] / sig0[:, 0]
        assert np.allclose(ratio, ratio[0], rtol=1e-12)          # every component decays alike
        errs.append(abs(ratio[0] - closed(T)))
    # zero-past BDF2 with sigma0 != 0: first order at fixed t
    assert errs[0] < 2e-3
    for a, b in zip(errs, errs[1:]):
        assert a / b > 1.8


# ------------------------------------------------------------------ P4
def test_alpha1_exponential_relaxation():
    # Oldroyd-B relaxation exp(-t/Wi).  The scheme starts BDF2 with a zero past
    # (sigma^{-1} = sigma^0): sigma - sigma0 is continued by zero for t <= 0,
    # which has a kink at t = 0 when sigma0 != 0, so the error is first order
    # here (second order from rest: P7 with alpha = 1).
    Wi, T = 0.7, 1.0
    sig0 = np.array([[1.0], [0.5], [-0.2], [0.1], [0.3], [-0.6]])
    errs = []
    for steps in (50, 100, 200):
        o = orc.Oracle(point_problem(3, 1.0, Wi, 0.5, T / steps), sig0)
        sT = o.run(steps, np.zeros((9, 1)))
        errs.append(np.max(np.abs(sT[:, 0] - sig0[:, 0] * math.exp(-T / Wi))))
    assert errs[0] < 5e-3
    for a, b in zip(errs, errs[1:]):
        assert 1.8 < a / b < 2.2


def test_alpha1_lemma_gaussian_steady_state():
    # symmetric trace-free D with I - 2 Wi D positive definite
    D = np.array([[0.2, 0.1, 0.0], [0.1, -0.05, 0.08], [0.0, 0.08, -0.15]])
    Wi, beta = 1.2, 0.3
    G = (1 - beta) / Wi
    ss = G * (np.linalg.inv(np.eye(3) - 2 * Wi * D) - np.eye(3))
    o = orc.Oracle(point_problem(3, 1.0, Wi, beta, 0.05))
    sT = o.run(4000, D.reshape(9, 1))
    assert np.allclose(sT[:, 0], pack(ss), rtol=1e-9, atol=1e-12)


def test_alpha1_lyapunov_steady_state_general_kappa():
    k = np.array([[0.1, 0.4], [-0.3, -0.2]])
    Wi, beta = 0.8, 0.6
    G = (1 - beta) / Wi
    I = np.eye(2)
    L = np.kron(k, I) + np.kron(I, k) - np.eye(4) / Wi
    ss = np.linalg.solve(L, -G * (k + k.T).ravel()).reshape(2, 2)
    o = orc.Oracle(point_problem(2, 1.0, Wi, beta, 0.05))
    sT = o.run(4000, k.reshape(4, 1))
    assert np.allclose(sT[:, 0], pack(ss), rtol=1e-9, atol=1e-12)


@pytest.mark.parametrize("flow", [False, True])
def test_alpha_to_one_limit_recovers_oldroyd_b(flow):
    # alpha -> 1: the Caputo kernel t^-alpha/Gamma(1-alpha) tends to the Dirac
    # delta (its mass on [0, T], T^(1-alpha)/Gamma(2-alpha), tends to 1 while its
    # part on [dt, T] vanishes with 1/Gamma(1-alpha)), so the law becomes the
    # Oldroyd-B equation of the paper's alpha = 1 case (eq.
    # macroscopic_fokker_planck with D^{1-alpha} = identity; Section 5.1's
    # classical runs).  With tables that carry the kernel's whole mass (the
    # completing Dirac term of soe_build) the SOE scheme at alpha = 1 - 10^-k
    # converges to the alpha = 1 scheme (plain BDF2, itself pinned above by
    # exp(-t/Wi) and the steady states), linearly in 1 - alpha: the error drops
    # by a factor 10 per decade.  Zero flow from sigma0 != 0 (the relaxation
    # exp(-t/Wi) in the limit) and a constant kappa from rest (the approach to
    # the Lyapunov steady state).
    dim, Wi, beta, dt, steps, m = 2, 0.8, 0.6, 0.01, 200, 32
    T = dt * steps
    if flow:
        kap, sig0 = np.array([[0.1, 0.4], [-0.3, -0.2]]).reshape(4, 1), None
    else:
        kap, sig0 = np.zeros((4, 1)), np.array([[1.0], [0.3], [0.5]])
    ref = orc.Oracle(point_problem(dim, 1.0, Wi, beta, dt), sig0).run(steps, kap)[:, 0]
    if not flow:
        # the alpha = 1 path is the BDF2 relaxation (first order from sigma0 != 0, P4)
        assert np.max(np.abs(ref - sig0[:, 0] * math.exp(-T / Wi))) < 5e-3 * np.max(np.abs(sig0))
    errs = []
    for k in range(1, 6):
        alpha = 1.0 - 10.0 ** (-k)
        mu, w = soe.soe_build(alpha, dt, T, m)
        out = orc.Oracle(point_problem(dim, alpha, Wi, beta, dt, mu, w), sig0).run(steps, kap)[:, 0]
        errs.append(np.max(np.abs(out - ref)) / np.max(np.abs(ref)))
    ratios = [a / b for a, b in zip(errs, errs[1:])]
    assert all(8.0 < r < 12.0 for r in ratios[1:]), (errs, ratios)
    assert errs[3] < 1e-3 and errs[4] < 1e-4, errs


# ------------------------------------------------------------------ P5
@pytest.mark.parametrize("dim", [2, 3])
def test_full_tensor_symmetric_and_equal_to_packed(dim):
    rng = np.random.default_rng(11)
    n = (5, 4) if dim == 2 else (3, 4, 5)
    alpha, dt, steps = 0.6, 1e-3, 12
    mu, w = soe.soe_nnls(alpha, dt, steps * dt, 6)
    N = int(np.prod(n))
    kap = rng.normal(size=(dim * dim, N))
    u = rng.normal(size=(dim, N)) * 0.5
    sig0 = inputs.random_stress(dim, n, seed=3)
    base = dict(dim=dim, n=n, alpha=alpha, Wi=1.1, beta=0.5, dt=dt, mu=mu, w=w, transport=True, eps=0.05)
    packed = orc.forward(orc.Problem(**base), sig0, kap, u, steps)
    full0 = np.stack([np.stack([unpack(sig0[:, p], dim) for p in range(N)])[:, i, j]
                      for i in range(dim) for j in range(dim)])
    full = orc.forward(orc.Problem(full=True, **base), full0, kap, u, steps)
    F = full.reshape(dim, dim, N)
    assert np.allclose(F, F.transpose(1, 0, 2), rtol=0, atol=1e-13 * np.max(np.abs(F)))
    pairs = PACK2 if dim == 2 else PACK3
    for c, (i, j) in enumerate(pairs):
        assert np.allclose(packed[c], F[i, j], rtol=1e-12, atol=1e-13 * np.max(np.abs(F)))


# ------------------------------------------------------------------ P6
def test_homogeneous_fields_give_uniform_stress():
    n = (6, 5, 4)
    alpha, dt = 0.6, 2e-4
    mu, w = soe.soe_nnls(alpha, dt, 0.01, 8)
    km = np.array([[0.2, 1.0, 0.0], [0.3, -0.1, 0.4], [0.0, 0.2, -0.1]])
    prob = orc.Problem(dim=3, n=n, alpha=alpha, Wi=2.0, beta=0.9, dt=dt, mu=mu, w=w, transport=True, eps=0.01)
    s = orc.forward(prob, None, inputs.uniform_kappa(3, n, km), inputs.uniform_velocity(3, n, [0.3, -1.2, 0.5]), 20)
    assert np.all(s == s[:, :1])
    assert np.max(np.abs(s)) > 0


# ------------------------------------------------------------------ P7
@pytest.mark.parametrize("alpha", [0.3, 0.6, 1.0])
def test_second_order_from_rest_every_alpha(alpha):
    T = 1.0
    if alpha < 1:
        mu, w = soe.soe_expquad(alpha, 1e-9, 10 * T, 300, tail=1e-12)
    else:
        mu = w = None
    k0 = np.array([[0.3, 1.0, 0.2], [-0.4, -0.1, 0.5], [0.1, 0.2, -0.2]])
    res = {}
    for steps in (50, 100, 200, 1600):
        dt = T / steps
        o = orc.Oracle(point_problem(3, alpha, 1.5, 0.5, dt, mu, w))
        res[steps] = o.run(steps, lambda n, dt=dt: (inputs.ramp(n * dt) * k0).reshape(9, 1))
    e = [np.max(np.abs(res[s] - res[1600])) for s in (50, 100, 200)]
    for a, b in zip(e, e[1:]):
        assert 3.6 < a / b < 4.6


# ------------------------------------------------------------------ P8
def test_single_fourier_mode_transport():
    alpha, Wi, T, ux = 0.6, 1.0, 0.2, 0.8
    n = (128, 1)
    kx = 2
    dt = 2.5e-4
    steps = int(round(T / dt))
    mu, w = soe.soe_expquad(alpha, dt * 1e-14, 10 * T, 700, tail=1e-14)
    x = np.arange(n[0]) * (2 * np.pi / n[0])
    sig0 = np.stack([np.cos(kx * x), 0.5 * np.cos(kx * x), -np.cos(kx * x)])
    prob = orc.Problem(dim=2, n=n, alpha=alpha, Wi=Wi, beta=0.5, dt=dt, mu=mu, w=w, transport=True)
    sT = orc.forward(prob, sig0, np.zeros((4, n[0])), inputs.uniform_velocity(2, n, [ux, 0.0]), steps)
    y = special.mittag_leffler(alpha, -(1.0 / Wi + 1j * kx * ux) * T ** alpha)
    exact = np.real(y * np.exp(1j * kx * x))
    assert np.max(np.abs(sT[0] - exact)) < 3e-3
    assert np.max(np.abs(sT[2] + exact)) < 3e-3
    # the decay itself is large compared with the tolerance
    assert np.max(np.abs(exact - np.cos(kx * x))) > 0.2


# ------------------------------------------------------------------ P9
def test_affine_in_sigma0_and_G():
    rng = np.random.default_rng(5)
    n = (6, 7)
    alpha, dt, steps = 0.4, 1e-3, 15
    mu, w = soe.soe_nnls(alpha, dt, steps * dt, 6)
    N = 42
    kap = rng.normal(size=(4, N))
    u = rng.normal(size=(2, N)) * 0.3
    base = dict(dim=2, n=n, alpha=alpha, Wi=1.0, dt=dt, mu=mu, w=w, transport=True)
    s_a = inputs.random_stress(2, n, 1)
    s_b = inputs.random_stress(2, n, 2)
    f = lambda s0, beta: orc.forward(orc.Problem(beta=beta, **base), s0, kap, u, steps)
    lhs = f(s_a + 2.0 * s_b, 0.5)
    rhs = f(s_a, 0.5) + 2.0 * (f(s_b, 0.5) - f(None, 0.5))
    assert np.allclose(lhs, rhs, rtol=1e-11, atol=1e-12)
    # G = (1 - beta)/Wi enters linearly: beta = 0.2, 0.5, 0.8 are equally spaced in G
    assert np.allclose(f(s_a, 0.2) - f(s_a, 0.5), f(s_a, 0.5) - f(s_a, 0.8), rtol=1e-10, atol=1e-12)


# ------------------------------------------------------------------ adjoint
@pytest.mark.parametrize("dim,transport,alpha", [(2, True, 0.5), (3, False, 0.7), (2, False, 1.0)])
def test_reference_adjoint_matches_finite_differences(dim, transport, alpha):
    rng = np.random.default_rng(21)
    n = (5, 4) if dim == 2 else (3, 2, 2)
    N = int(np.prod(n))
    dt, steps = 2e-3, 12
    if alpha < 1:
        mu, w = soe.soe_nnls(alpha, dt, steps * dt, 6)
    else:
        mu, w = np.zeros(0), np.zeros(0)
    kap = rng.normal(size=(dim * dim, N))
    u = rng.normal(size=(dim, N)) * 0.5 if transport else None
    sig0 = inputs.random_stress(dim, n, 9)
    nc = sig0.shape[0]
    target = rng.normal(size=(nc, N))

    def J(Wi, beta, s0, k):
        p = orc.Problem(dim=dim, n=n, alpha=alpha, Wi=Wi, beta=beta, dt=dt, mu=mu, w=w,
                        transport=transport, eps=0.02 if transport else 0.0)
        sT = orc.forward(p, s0, k, u, steps)
        return float(np.sum((sT - target) ** 2))

    Wi, beta = 1.3, 0.4
    p = orc.Problem(dim=dim, n=n, alpha=alpha, Wi=Wi, beta=beta, dt=dt, mu=mu, w=w,
                    transport=transport, eps=0.02 if transport else 0.0)
    sT = orc.forward(p, sig0, kap, u, steps)
    g = orc.gradients(p, sig0, kap, u, steps, 2.0 * (sT - target))
    h = 1e-6

    def fd(fun, x):
        return (fun(x + h) - fun(x - h)) / (2 * h)

    def close(a, b):
        return abs(a - b) <= 1e-6 * max(abs(a), abs(b), 1e-3)

    assert close(g["Wi"], fd(lambda x: J(x, beta, sig0, kap), Wi))
    assert close(g["beta"], fd(lambda x: J(Wi, x, sig0, kap), beta))
    for (c, q) in [(0, 0), (nc - 1, N - 1), (1, N // 2)]:
        def fs(x, c=c, q=q):
            s = sig0.copy(); s[c, q] = x
            return J(Wi, beta, s, kap)
        assert close(g["sigma0"][c, q], fd(fs, sig0[c, q]))
    for (c, q) in [(0, 1), (dim * dim - 1, N - 2), (1, 3)]:
        def fk(x, c=c, q=q):
            k = kap.copy(); k[c, q] = x
            return J(Wi, beta, sig0, k)
        assert close(g["kappa"][c, q], fd(fk, kap[c, q]))


def _paper_case_bochner_errors(start, m, dts, builder=None):
    # default table: soe_build (fitted on [dt, T], mass-completed)
    alpha, Wi, eps, T = 0.5, 1.0, 1e-2, 1.0
    n = (8, 8)
    N = n[0] * n[1]
    h = 1.0 / n[0]
    x = (np.arange(N) % n[0]) * h
    y = (np.arange(N) // n[0]) * h
    shape = np.cos(2 * np.pi * x) * np.cos(4 * np.pi * y)
    sigma0 = np.tile(shape, (3, 1))
    lam_h = 1.0 / Wi + eps * (4 * np.sin(np.pi * h) ** 2 + 4 * np.sin(2 * np.pi * h) ** 2) / h ** 2
    assert abs(lam_h - (1.0 / Wi + 20 * eps * np.pi ** 2)) < 0.5
    errs = []
    for dt in dts:
        steps = int(round(T / dt))
        mu, w = (builder or soe.soe_build)(alpha, dt, T, m)
        prob = orc.Problem(dim=2, n=n, alpha=alpha, Wi=Wi, beta=0.5, dt=dt, mu=mu, w=w, eps=eps, L=(1.0, 1.0),
                           transport=True, implicit=True, start=start)
        o = orc.Oracle(prob, sigma0)
        zero_u, kap = np.zeros((2, N)), np.zeros((4, N))
        acc = 0.0
        for k in range(1, steps + 1):
            o.step(kap, kap, zero_u)
            t = k * dt
            exact = shape * special.mittag_leffler(alpha, -lam_h * t ** alpha)
            e2 = np.mean((o.sig_n[0] - exact) ** 2)          # L2 over the unit square
            acc += (0.5 if k == steps else 1.0) * e2 * t ** (2 * (1 - alpha)) * dt   # trapezoid, e(0) = 0
        errs.append(np.sqrt(acc))
    return errs


def _orders(errs):
    return [float(np.log2(errs[i] / errs[i + 1])) for i in range(len(errs) - 1)]


DTS_PAPER_CASE = [1 / 20, 1 / 40, 1 / 80, 1 / 160]


def test_paper_first_convergence_case_bochner_norm():
    # The paper's convergence case (Section 5.1): no flow, unit square, initial
    # stress cos(2 pi x) cos(4 pi y), eps = 1e-2, De = 0.5 (Wi = 2 De: eq.
    # conf_op_tested gives degree-2 modes the relaxation rate 1/De where the
    # printed matrix has 1/(2 De)), alpha = 0.5, T = 1, error in the weighted Bochner norm of eq.
    # weighted_Bochner_space_norm, diffusion implicit as in the paper.  On the
    # periodic grid the solution is the initial field times E_alpha(-lambda_h
    # t^alpha), lambda_h = 1/Wi + eps x (discrete Laplacian symbol) -> 1/Wi +
    # 20 eps pi^2, so the error is that of time stepping and kernel compression.
    # The paper reports order 1 + alpha (its Fig. 2a) with an SDIRK2 first
    # step.  The stress-form scheme reaches it too, given that start and a
    # table that carries the kernel's whole mass (soe_build's completing term);
    # the same fit without it loses the mass below dt at every step and
    # stalls; the empty-past BDF2 start gives order 1.
    sdirk = _orders(_paper_case_bochner_errors("sdirk2", 32, DTS_PAPER_CASE))
    bdf = _orders(_paper_case_bochner_errors("bdf2", 32, DTS_PAPER_CASE))
    bare = _orders(_paper_case_bochner_errors("sdirk2", 32, DTS_PAPER_CASE, builder=soe.soe_nnls))
    assert all(q > 1.3 for q in sdirk) and sdirk[-1] > 1.38, sdirk
    assert sdirk == sorted(sdirk), sdirk
    assert all(0.95 < q < 1.1 for q in bdf), bdf
    assert bare[-1] < 1.0, bare


def test_paper_variable_scheme_convergence_and_agreement():
    # The scheme in the paper's own variable (oracle.paper_form: BDF2 on Phi,
    # Psi = D^{1-alpha} Phi through kernel compression of g_alpha) on the same
    # decay, one point with the diffusion of the single Fourier mode folded
    # into the rate (exact for an eigenfunction of the Laplacian): order
    # -> 1 + alpha with the SDIRK2 start (alpha = 0.3, 0.5, 0.7).  Then, from rest under the smooth
    # sin^2 ramp of the forcing (Section 5.1), its stress Psi2 and the stress
    # form's sigma approach each other as dt -> 0.
    from oracle.paper_form import PaperForm
    T = 1.0
    lam = 1.0 + 20 * 1e-2 * np.pi ** 2
    for alpha in (0.3, 0.5, 0.7):
        errs = []
        for dt in DTS_PAPER_CASE:
            mu, w = soe.soe_build(1 - alpha, dt, T, 32)
            pf = PaperForm(2, 1, 1.0 / lam, 0.5, dt, mu, w, Phi0=np.ones((3, 1)), start="sdirk2")
            acc = 0.0
            steps = int(round(T / dt))
            for k in range(1, steps + 1):
                pf.step(np.zeros((4, 1)))
                t = k * dt
                e2 = (pf.Phi_n[0, 0] - special.mittag_leffler(alpha, -lam * t ** alpha)) ** 2
                acc += (0.5 if k == steps else 1.0) * e2 * t ** (2 * (1 - alpha)) * dt
            errs.append(np.sqrt(acc))
        q = _orders(errs)
        # order 1 + alpha, approached from below
        assert all(b > a - 0.01 for a, b in zip(q, q[1:])) and 1 + alpha - 0.2 < q[-1] < 1 + alpha + 0.05, (alpha, q)

    rng = np.random.default_rng(4)
    N, Wi, beta, T2 = 6, 1.3, 0.4, 0.5
    K0 = 0.6 * rng.normal(size=(4, N))
    ramp = lambda t: np.sin(0.5 * np.pi * min(max(0.0, 4 * t - 1), 1.0)) ** 2
    diffs = []
    for dt in [1 / 40, 1 / 80, 1 / 160]:
        steps = int(round(T2 / dt))
        mu_s, w_s = soe.soe_build(alpha, dt, T2, 32)
        o = orc.Oracle(orc.Problem(dim=2, n=(N, 1), alpha=alpha, Wi=Wi, beta=beta, dt=dt, mu=mu_s, w=w_s), None)
        mu_p, w_p = soe.soe_build(1 - alpha, dt, T2, 32)
        pf = PaperForm(2, N, Wi, beta, dt, mu_p, w_p)
        for k in range(steps):
            kap, kprev = K0 * ramp(k * dt), K0 * ramp(max(k - 1, 0) * dt)
            o.step(kap, kprev)
            psi = pf.step(kap, kprev)
        diffs.append(np.max(np.abs(o.sig_n - psi)) / np.max(np.abs(o.sig_n)))
    assert diffs[-1] < diffs[0] / 3 and diffs[-1] < 1e-2, diffs


@pytest.mark.parametrize("stencil,U,eps", [(0, 2.0, 0.0), (0, -2.0, 0.05), (1, 2.0, 0.02)])
def test_paper_variable_transport_single_fourier_mode(stencil, U, eps):
    # One Fourier mode advected by a constant velocity with kappa = 0 in the
    # paper's variable: every field is a complex scalar times e^{ikx}; the
    # explicit transport of E = 2 Psi^n - Psi^{n-1} enters through the symbol
    # s(k) = U D(k) + eps 4 sin^2(kh/2)/h^2 of the stencils, so the scheme is a
    # scalar recurrence the grid version must reproduce to rounding.
    from oracle.paper_form import PaperForm
    alpha, m, Wi, dt, steps = 0.5, 8, 1.3, 0.01, 15
    n, kx = (16, 3), 3
    N = n[0] * n[1]
    h = 2 * math.pi / n[0]
    mu, w = soe.soe_nnls(1 - alpha, dt, steps * dt, m)
    x = (np.arange(N) % n[0]) * h
    phi0 = np.zeros((3, N))
    phi0[0] = np.cos(kx * x)
    u = np.zeros((2, N))
    u[0] = U
    pf = PaperForm(2, N, Wi, 0.5, dt, mu, w, Phi0=phi0, grid=n, eps=eps, stencil=stencil)
    for _ in range(steps):
        got = pf.step(np.zeros((4, N)), None, u)
    th = kx * h
    if stencil == 1:
        D = 1j * math.sin(th) / h
    elif U >= 0:
        D = (np.exp(-2j * th) - 6 * np.exp(-1j * th) + 3 + 2 * np.exp(1j * th)) / (6 * h)
    else:
        D = (-2 * np.exp(-1j * th) - 3 + 6 * np.exp(1j * th) - np.exp(2j * th)) / (6 * h)
    sym = U * D + eps * 4.0 * math.sin(th / 2) ** 2 / h ** 2
    b0, b1, b2 = 1.5, -2.0, 0.5
    c = 1.0 / (b0 + mu * dt)
    xi = b0 * np.sum(w * c)
    P_n = P_nm1 = 1.0 + 0j
    q_n = np.zeros(m, complex)
    q_nm1 = np.zeros(m, complex)
    S_n = S_nm1 = 0j
    for _ in range(steps):
        hh = np.sum(w * mu * c * (b1 * q_n + b2 * q_nm1))
        rhs = -b1 * P_n - b2 * P_nm1 - dt * hh / Wi - dt * sym * (2 * S_n - S_nm1)
        P = rhs / (b0 + dt * xi / Wi)
        q = c * (-b1 * q_n - b2 * q_nm1 + dt * P)
        S = xi * P + hh
        P_nm1, P_n, q_nm1, q_n, S_nm1, S_n = P_n, P, q_n, q, S_n, S
    ref = (S_n * np.exp(1j * kx * x)).real
    assert np.max(np.abs(got[0] - ref)) < 1e-12 * np.max(np.abs(ref))
    assert np.max(np.abs(got[1:])) == 0.0


@pytest.mark.parametrize("stencil,U,eps", [(0, 6.0, 0.0), (0, -6.0, 0.05), (1, 6.0, 0.02)])
def test_paper_variable_implicit_transport_single_fourier_mode(stencil, U, eps):
    # As above with the transport inside the solve, acting on Psi^{n+1} = xi Phi + h:
    # (b0 + dt xi/Wi + dt xi s) Phi = -b1 Phi^n - b2 Phi^{n-1} - dt h/Wi - dt s h,
    # at a velocity where the explicit form of the stress variable is unstable.
    from oracle.paper_form import PaperForm
    alpha, m, Wi, dt, steps = 0.5, 8, 1.3, 0.02, 12
    n, kx = (16, 3), 3
    N = n[0] * n[1]
    h = 2 * math.pi / n[0]
    assert abs(U) * dt / h > 0.25
    mu, w = soe.soe_nnls(1 - alpha, dt, steps * dt, m)
    x = (np.arange(N) % n[0]) * h
    phi0 = np.zeros((3, N))
    phi0[0] = np.cos(kx * x)
    u = np.zeros((2, N))
    u[0] = U
    pf = PaperForm(2, N, Wi, 0.5, dt, mu, w, Phi0=phi0, grid=n, eps=eps, stencil=stencil, implicit=True)
    for _ in range(steps):
        got = pf.step(np.zeros((4, N)), None, u)
    th = kx * h
    if stencil == 1:
        D = 1j * math.sin(th) / h
    elif U >= 0:
        D = (np.exp(-2j * th) - 6 * np.exp(-1j * th) + 3 + 2 * np.exp(1j * th)) / (6 * h)
    else:
        D = (-2 * np.exp(-1j * th) - 3 + 6 * np.exp(1j * th) - np.exp(2j * th)) / (6 * h)
    sym = U * D + eps * 4.0 * math.sin(th / 2) ** 2 / h ** 2
    b0, b1, b2 = 1.5, -2.0, 0.5
    c = 1.0 / (b0 + mu * dt)
    xi = b0 * np.sum(w * c)
    P_n = P_nm1 = 1.0 + 0j
    q_n = np.zeros(m, complex)
    q_nm1 = np.zeros(m, complex)
    for _ in range(steps):
        hh = np.sum(w * mu * c * (b1 * q_n + b2 * q_nm1))
        P = (-b1 * P_n - b2 * P_nm1 - dt * hh / Wi - dt * sym * hh) / (b0 + dt * xi / Wi + dt * xi * sym)
        q = c * (-b1 * q_n - b2 * q_nm1 + dt * P)
        S = xi * P + hh
        P_nm1, P_n, q_nm1, q_n = P_n, P, q_n, q
    ref = (S * np.exp(1j * kx * x)).real
    assert np.max(np.abs(got[0] - ref)) < 1e-12 * np.max(np.abs(ref))
    assert np.max(np.abs(got[1:])) == 0.0


def test_paper_variable_sdirk2_start_with_implicit_transport_single_fourier_mode():
    # The SDIRK2 start with the transport inside both stage solves, one Fourier
    # mode, kappa = 0: Psi = W Phi - h at a stage, so (1 + g dt W/Wi + g dt W s) Phi
    # = ZPhi + g dt h/Wi + g dt s h, with h = sum_j w_j mu_j Zphi_j / (1 + g mu_j dt),
    # W = sum_j w_j / (1 + g mu_j dt); then BDF2 steps as in the test above.
    from oracle.paper_form import PaperForm
    alpha, m, Wi, dt, steps, U = 0.5, 8, 1.3, 0.02, 6, 6.0
    n, kx = (16, 3), 3
    N = n[0] * n[1]
    hgrid = 2 * math.pi / n[0]
    mu, w = soe.soe_nnls(1 - alpha, dt, steps * dt, m)
    x = (np.arange(N) % n[0]) * hgrid
    phi0 = np.zeros((3, N))
    phi0[0] = np.cos(kx * x)
    u = np.zeros((2, N))
    u[0] = U
    pf = PaperForm(2, N, Wi, 0.5, dt, mu, w, Phi0=phi0, grid=n, implicit=True, start="sdirk2")
    for _ in range(steps):
        got = pf.step(np.zeros((4, N)), None, u)
    th = kx * hgrid
    s = U * (np.exp(-2j * th) - 6 * np.exp(-1j * th) + 3 + 2 * np.exp(1j * th)) / (6 * hgrid)
    g = 1.0 - math.sqrt(0.5)
    den = 1.0 + g * mu * dt
    W = np.sum(w / den)
    P0, q0 = 1.0 + 0j, np.zeros(m, complex)
    ZP, Zq = P0, q0.copy()
    for stage in (1, 2):
        hh = np.sum(w * mu * Zq / den)
        P = (ZP + g * dt * hh / Wi + g * dt * s * hh) / (1.0 + g * dt * W / Wi + g * dt * W * s)
        q = (Zq + g * dt * P) / den
        if stage == 1:
            ZP = P0 + dt * (1 - g) * (P - P0) / (g * dt)
            Zq = q0 + dt * (1 - g) * (P - mu * q)
    S = W * P - hh
    b0, b1, b2 = 1.5, -2.0, 0.5
    c = 1.0 / (b0 + mu * dt)
    xi = b0 * np.sum(w * c)
    P_n, P_nm1, q_n, q_nm1 = P, P0, q, q0
    for _ in range(steps - 1):
        hh = np.sum(w * mu * c * (b1 * q_n + b2 * q_nm1))
        Pn = (-b1 * P_n - b2 * P_nm1 - dt * hh / Wi - dt * s * hh) / (b0 + dt * xi / Wi + dt * xi * s)
        qn = c * (-b1 * q_n - b2 * q_nm1 + dt * Pn)
        S = xi * Pn + hh
        P_nm1, P_n, q_nm1, q_n = P_n, Pn, q_n, qn
    ref = (S * np.exp(1j * kx * x)).real
    assert np.max(np.abs(got[0] - ref)) < 1e-12 * np.max(np.abs(ref))
