"""The adjoint of the paper's own variable (TFS_FORM_PAPER, Section 3.4;
BDF2 start with the pointwise law, explicit or implicit transport; SDIRK2
start with the pointwise law or implicit transport) through tfs_backward:
J = <dJ, Psi(T)>.

1. Against FP64 central differences of the oracle's scheme in that variable
   (oracle.paper_form.PaperForm), in random directions of Phi(0) (exact: Psi(T)
   is affine in Phi(0)) and of the velocity gradient, and in Wi and beta;
   several checkpoint segments, 2D and 3D, both stencils, with and without
   diffusion, FP64 and FP32 storage.
2. torch.autograd (fractional_stress(form="paper")) against central
   differences of the CUDA forward, 1e-6 relative.
3. A 2D 256^2, m = 32, 200-step run (checkpoint every 50) against central
   differences of the CUDA forward at sampled entries, 1e-6 relative.
4. The SDIRK2 first step (Section 5.1) in this variable: one step alone (the
   adjoint of Psi^1 enters the start's adjoint) and followed by BDF2 steps.
5. Implicit transport (eq. FP_discrete) in this variable, with either start:
   the transposed global solves, against central differences of the oracle's
   dense implicit scheme, above the explicit limit.
6. Element by element against the oracle's reference adjoint
   (oracle.paper_form.paper_gradients, itself pinned to central differences in
   tests/test_oracle_paper_adjoint.py), FP64 storage, to 1e-9 of each field's
   largest entry.

Tolerances: FP64 1e-6 relative to the largest entry of each gradient (the
central differences carry O(h^2) truncation, h = 1e-5); FP32 storage 5e-4
(the float mode ring and the float Psi levels; Psi = xi Phi + h cancels by a
few tens here, as in the forward).
"""
import numpy as np
import pytest

from helpers import ensure_lib
from oracle import soe
from oracle.paper_form import PaperForm, paper_gradients
from paper_2411_17294_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_lib()


def oracle_J(dim, n, Wi, beta, dt, mu, w, P0, kap, steps, dJ, u=None, eps=0.0, stencil=0, start="bdf2",
             implicit=False):
    N = int(np.prod(n))
    pf = PaperForm(dim, N, Wi, beta, dt, mu, w, Phi0=P0, grid=n, eps=eps, stencil=stencil, start=start,
                   implicit=implicit)
    for _ in range(steps):
        psi = pf.step(kap, kap, u)
    return float(np.sum(dJ * psi))


def gpu_grads(dim, n, alpha, Wi, beta, dt, mu, w, P0, kap, steps, K, dJ, precision, u=None, eps=0.0, stencil=0,
              start="bdf2", implicit=False):
    import torch
    from paper_2411_17294_gb300 import tfs
    s = tfs.Solver(dim, n, alpha, Wi, beta, dt, m=len(mu), precision=precision, mu=mu, w=w,
                   transport=("implicit" if implicit else True) if u is not None else False, eps=eps,
                   stencil=stencil, form="paper", start=start)
    if implicit:
        s.set_krylov(maxit=2000)
    kt = torch.as_tensor(kap, dtype=s.dtype, device=s.device).contiguous()
    ut = None if u is None else torch.as_tensor(u, dtype=s.dtype, device=s.device).contiguous()
    s.set_state(torch.as_tensor(P0, dtype=s.dtype, device=s.device))
    ckpts = []
    for k in range(steps):
        if k % K == 0:
            c = s.new_checkpoint()
            s.save(c)
            ckpts.append(c)
        s.step(kt, kt, ut)
    g_p0, g_k, gWi, gb = s.backward(torch.as_tensor(dJ, dtype=s.dtype, device=s.device), ckpts, K, steps, kt, ut)
    flags = s.status()
    s.close()
    assert not (flags & (tfs.TFS_FLAG_NONFINITE | tfs.TFS_FLAG_SINGULAR | tfs.TFS_FLAG_TIMEOUT | tfs.TFS_FLAG_NOCONV))
    return g_p0.cpu().numpy(), g_k.cpu().numpy(), gWi, gb


CASES = [
    # dim, n, alpha, m, steps, K, transport, stencil, eps
    (2, (11, 7), 0.5, 8, 12, 5, False, 0, 0.0),
    (3, (4, 3, 5), 0.3, 12, 9, 4, False, 0, 0.0),
    (2, (40, 1), 0.7, 6, 7, 7, False, 0, 0.0),
    (3, (3, 3, 3), 0.6, 32, 10, 3, False, 0, 0.0),
    (2, (37, 5), 0.4, 40, 6, 4, False, 0, 0.0),        # more than 32 modes: 16 per FP32 thread
    (2, (12, 10), 0.5, 8, 11, 4, True, 0, 0.0),
    (2, (16, 9), 0.4, 8, 9, 9, True, 1, 0.005),
    (3, (5, 4, 6), 0.6, 6, 8, 3, True, 1, 0.01),
    (3, (4, 5, 3), 0.35, 16, 7, 7, True, 0, 0.0),
]
SDIRK2_CASES = [
    (2, (11, 7), 0.5, 8, 1, 1, False, 0, 0.0),
    (2, (9, 6), 0.3, 12, 8, 3, False, 0, 0.0),
    (3, (4, 3, 5), 0.7, 6, 6, 6, False, 0, 0.0),
    (3, (3, 3, 3), 0.45, 32, 2, 1, False, 0, 0.0),
]


@pytest.mark.parametrize("dim,n,alpha,m,steps,K,transport,stencil,eps,start",
                         [c + ("bdf2",) for c in CASES] + [c + ("sdirk2",) for c in SDIRK2_CASES])
@pytest.mark.parametrize("precision", [0, 1])
def test_paper_adjoint_against_oracle_differences(dim, n, alpha, m, steps, K, transport, stencil, eps, start,
                                                  precision):
    dt, Wi, beta = 4e-3, 1.3, 0.4
    mu, w = soe.soe_nnls(1 - alpha, dt, 50 * dt, m)
    _, kap = inputs.spectral_velocity(dim, n, 2, seed=81)
    kap = 0.6 * np.asarray(kap)
    P0 = inputs.random_stress(dim, n, 82)
    rng = np.random.default_rng(83)
    dJ = rng.normal(size=P0.shape)
    u = 0.3 * np.asarray(inputs.spectral_velocity(dim, n, 2, seed=84)[0]) if transport else None
    if precision == 1:
        cast = lambda a: np.asarray(a, np.float32).astype(np.float64)
        kap, P0, dJ = cast(kap), cast(P0), cast(dJ)
        u = None if u is None else cast(u)
    g_p0, g_k, gWi, gb = gpu_grads(dim, n, alpha, Wi, beta, dt, mu, w, P0, kap, steps, K, dJ, precision, u, eps,
                                   stencil, start)
    J = lambda P, k, Wi_, b_: oracle_J(dim, n, Wi_, b_, dt, mu, w, P, k, steps, dJ, u, eps, stencil, start)
    if start == "sdirk2":
        # the start changes the gradient (else the test would not see its adjoint)
        Jb = lambda P: oracle_J(dim, n, Wi, beta, dt, mu, w, P, kap, steps, dJ)
        d = np.random.default_rng(6).normal(size=P0.shape)
        assert abs((Jb(P0 + d) - Jb(P0 - d)) / 2.0 - float(np.sum(g_p0 * d))) > 1e-4 * np.sum(np.abs(g_p0 * d))
    if transport:
        # the transport changes the gradient (else the test would not see its adjoint)
        Jp = lambda P: oracle_J(dim, n, Wi, beta, dt, mu, w, P, kap, steps, dJ)
        d = np.random.default_rng(5).normal(size=P0.shape)
        assert abs((Jp(P0 + d) - Jp(P0 - d)) / 2.0 - float(np.sum(g_p0 * d))) > 1e-3 * np.sum(np.abs(g_p0 * d))
    tol = 1e-6 if precision == 0 else 5e-4
    h = 1e-5

    def check(got, fd, scale):
        assert abs(got - fd) <= tol * scale, (got, fd, scale)

    # Phi(0): affine, so a unit step gives the exact directional derivative
    for seed in (1, 2):
        d = np.random.default_rng(seed).normal(size=P0.shape)
        fd = (J(P0 + d, kap, Wi, beta) - J(P0 - d, kap, Wi, beta)) / 2.0
        check(float(np.sum(g_p0 * d)), fd, np.sum(np.abs(g_p0) * np.abs(d)))
    for seed in (3, 4):
        d = np.random.default_rng(seed).normal(size=kap.shape)
        fd = (J(P0, kap + h * d, Wi, beta) - J(P0, kap - h * d, Wi, beta)) / (2 * h)
        check(float(np.sum(g_k * d)), fd, np.sum(np.abs(g_k) * np.abs(d)))
    fd_wi = (J(P0, kap, Wi + h, beta) - J(P0, kap, Wi - h, beta)) / (2 * h)
    fd_b = (J(P0, kap, Wi, beta + h) - J(P0, kap, Wi, beta - h)) / (2 * h)
    check(gWi, fd_wi, max(abs(fd_wi), 1e-12))
    check(gb, fd_b, max(abs(fd_b), 1e-12))


IMPLICIT_CASES = [
    # dim, n, alpha, m, steps, K, stencil, eps, dt max|u| / h
    (2, (12, 10), 0.5, 8, 8, 3, 0, 0.0, 0.5),
    (2, (10, 8), 0.3, 6, 6, 6, 1, 0.02, 0.08),
    (3, (5, 4, 6), 0.6, 6, 6, 2, 0, 0.01, 0.4),
]


IMPLICIT_SDIRK2_CASES = [
    (2, (12, 10), 0.5, 8, 6, 3, 0, 0.0, 0.5),
    (2, (9, 7), 0.4, 6, 1, 1, 1, 0.01, 0.08),      # central stencil: block Jacobi needs a milder flow
    (3, (5, 4, 6), 0.6, 6, 5, 2, 0, 0.01, 0.4),
]


@pytest.mark.parametrize("dim,n,alpha,m,steps,K,stencil,eps,speed,start",
                         [c + ("bdf2",) for c in IMPLICIT_CASES] + [c + ("sdirk2",) for c in IMPLICIT_SDIRK2_CASES])
@pytest.mark.parametrize("precision", [0, 1])
def test_paper_implicit_adjoint_against_oracle_differences(dim, n, alpha, m, steps, K, stencil, eps, speed, start,
                                                           precision):
    dt, Wi, beta = 2e-3, 1.3, 0.4
    mu, w = soe.soe_nnls(1 - alpha, dt, 50 * dt, m)
    _, kap = inputs.spectral_velocity(dim, n, 2, seed=85)
    kap = 0.6 * np.asarray(kap)
    u, _ = inputs.spectral_velocity(dim, n, 2, seed=86)
    hmin = 2 * np.pi / min(n)
    u = np.asarray(u) * (speed * hmin / dt / np.abs(np.asarray(u)).max())   # far above the explicit limit
    P0 = inputs.random_stress(dim, n, 87)
    dJ = np.random.default_rng(88).normal(size=P0.shape)
    if precision == 1:
        cast = lambda a: np.asarray(a, np.float32).astype(np.float64)
        kap, P0, dJ, u = cast(kap), cast(P0), cast(dJ), cast(u)
    g_p0, g_k, gWi, gb = gpu_grads(dim, n, alpha, Wi, beta, dt, mu, w, P0, kap, steps, K, dJ, precision, u, eps,
                                   stencil, start=start, implicit=True)
    J = lambda P, k, Wi_, b_: oracle_J(dim, n, Wi_, b_, dt, mu, w, P, k, steps, dJ, u, eps, stencil, start=start,
                                       implicit=True)
    tol = 1e-6 if precision == 0 else 5e-4
    h = 1e-5

    def check(got, fd, scale):
        assert abs(got - fd) <= tol * scale, (got, fd, scale)

    for seed in (1, 2):
        d = np.random.default_rng(seed).normal(size=P0.shape)
        fd = (J(P0 + d, kap, Wi, beta) - J(P0 - d, kap, Wi, beta)) / 2.0
        check(float(np.sum(g_p0 * d)), fd, np.sum(np.abs(g_p0) * np.abs(d)))
    for seed in (3, 4):
        d = np.random.default_rng(seed).normal(size=kap.shape)
        fd = (J(P0, kap + h * d, Wi, beta) - J(P0, kap - h * d, Wi, beta)) / (2 * h)
        check(float(np.sum(g_k * d)), fd, np.sum(np.abs(g_k) * np.abs(d)))
    fd_wi = (J(P0, kap, Wi + h, beta) - J(P0, kap, Wi - h, beta)) / (2 * h)
    fd_b = (J(P0, kap, Wi, beta + h) - J(P0, kap, Wi, beta - h)) / (2 * h)
    check(gWi, fd_wi, max(abs(fd_wi), 1e-12))
    check(gb, fd_b, max(abs(fd_b), 1e-12))
    # the transport's adjoint matters
    Jp = lambda P: oracle_J(dim, n, Wi, beta, dt, mu, w, P, kap, steps, dJ)
    d = np.random.default_rng(5).normal(size=P0.shape)
    assert abs((Jp(P0 + d) - Jp(P0 - d)) / 2.0 - float(np.sum(g_p0 * d))) > 1e-3 * np.sum(np.abs(g_p0 * d))


@pytest.mark.parametrize("dim,n,alpha,m,steps,K", [(2, (37, 5), 0.5, 8, 9, 4), (3, (4, 3, 5), 0.35, 12, 7, 3)])
def test_paper_adjoint_fields_match_oracle_adjoint(dim, n, alpha, m, steps, K):
    dt, Wi, beta = 4e-3, 1.3, 0.4
    N = int(np.prod(n))
    mu, w = soe.soe_nnls(1 - alpha, dt, 50 * dt, m)
    _, kap = inputs.spectral_velocity(dim, n, 2, seed=95)
    kap = 0.6 * np.asarray(kap)
    P0 = inputs.random_stress(dim, n, 96)
    dJ = np.random.default_rng(97).normal(size=P0.shape)
    g_p0, g_k, gWi, gb = gpu_grads(dim, n, alpha, Wi, beta, dt, mu, w, P0, kap, steps, K, dJ, 0)
    ref = paper_gradients(dim, N, Wi, beta, dt, mu, w, P0, kap, steps, dJ)
    for got, exp in ((g_p0, ref["Phi0"]), (g_k, ref["kappa"])):
        assert np.max(np.abs(got - exp)) <= 1e-9 * np.max(np.abs(exp))
    assert abs(gWi - ref["Wi"]) <= 1e-9 * abs(ref["Wi"])
    assert abs(gb - ref["beta"]) <= 1e-9 * abs(ref["beta"])


def test_paper_autograd_matches_central_differences():
    import torch
    from paper_2411_17294_gb300.autograd import fractional_stress
    dim, n, alpha, dt, steps, K, m = 2, (8, 8), 0.4, 2e-3, 30, 7, 8
    mu, w = soe.soe_nnls(1 - alpha, dt, steps * dt, m)
    dev = torch.device("cuda", 0)
    _, k_np = inputs.spectral_velocity(dim, n, 2, seed=91)
    s0_np = inputs.random_stress(dim, n, 92)
    target = torch.as_tensor(np.random.default_rng(93).normal(size=s0_np.shape), device=dev)
    kw = dict(dim=dim, n=n, alpha=alpha, dt=dt, steps=steps, K=K, mu=mu, w=w, u=None, form="paper")

    def J(s0, k, Wi, beta):
        sT = fractional_stress(s0, k, Wi, beta, **kw)
        return ((sT - target) ** 2).sum()

    s0 = torch.as_tensor(s0_np, device=dev).requires_grad_(True)
    k = torch.as_tensor(k_np, device=dev).requires_grad_(True)
    Wi = torch.tensor(1.4, dtype=torch.float64, device=dev, requires_grad=True)
    beta = torch.tensor(0.3, dtype=torch.float64, device=dev, requires_grad=True)
    J(s0, k, Wi, beta).backward()
    h = 1e-6

    def fd(fun, x0):
        return (fun(x0 + h) - fun(x0 - h)) / (2 * h)

    def close(a, b):
        return abs(a - b) <= 1e-6 * max(abs(a), abs(b))

    t = lambda x: torch.tensor(x, dtype=torch.float64, device=dev)
    with torch.no_grad():
        s0d, kd = s0.detach(), k.detach()
        assert close(Wi.grad.item(), fd(lambda x: J(s0d, kd, t(x), beta.detach()).item(), 1.4))
        assert close(beta.grad.item(), fd(lambda x: J(s0d, kd, Wi.detach(), t(x)).item(), 0.3))
        for (c, q) in [(0, 0), (2, 63), (1, 17)]:
            def fs(x, c=c, q=q):
                a = s0d.clone()
                a[c, q] = x
                return J(a, kd, Wi.detach(), beta.detach()).item()
            assert close(s0.grad[c, q].item(), fd(fs, s0d[c, q].item()))
        for (c, q) in [(0, 5), (3, 40), (1, 9)]:
            def fk(x, c=c, q=q):
                a = kd.clone()
                a[c, q] = x
                return J(s0d, a, Wi.detach(), beta.detach()).item()
            assert close(k.grad[c, q].item(), fd(fk, kd[c, q].item()))


def test_paper_adjoint_256_against_central_differences():
    # 2D periodic 256^2, m = 32, alpha = 0.5, dt = 1e-3, 200 steps, checkpoint
    # every 50, FP64; J = ||Psi(T) - target||^2, the target from a seeded run at
    # Wi = 1.5; J(x+h) - J(x-h) summed as sum (s+ - s-)(s+ + s- - 2 t).
    import torch
    from paper_2411_17294_gb300 import tfs
    dim, n, alpha, m, dt, steps, K = 2, (256, 256), 0.5, 32, 1e-3, 200, 50
    Wi, beta = 1.0, 0.5
    N = n[0] * n[1]
    mu, w = soe.soe_nnls(1 - alpha, dt, steps * dt, m)
    dev = torch.device("cuda", 0)
    _, kap = inputs.spectral_velocity(dim, n, 32, 2)
    kap = torch.as_tensor(0.05 * kap, device=dev)
    P0 = torch.as_tensor(inputs.random_stress(dim, n, 5, amplitude=0.5), device=dev)

    def run(Wi_, beta_, p0, k, grads_for=None):
        s = tfs.Solver(dim, n, alpha, Wi_, beta_, dt, m=m, precision=tfs.TFS_FP64, mu=mu, w=w, transport=False,
                       form="paper")
        s.set_state(p0)
        ckpts = []
        for i in range(steps):
            if grads_for is not None and i % K == 0:
                c = s.new_checkpoint()
                s.save(c)
                ckpts.append(c)
            s.step(k, k, None)
        out = s.stress()
        if grads_for is not None:
            out = (out, s.backward(2.0 * (out - grads_for), ckpts, K, steps, k, None))
        s.close()
        return out

    target = run(1.5, beta, P0, kap)
    _, (g_p0, g_k, gWi, gbeta) = run(Wi, beta, P0, kap, grads_for=target)

    def dJ(sp, sm):
        return float(torch.sum((sp - sm) * (sp + sm - 2.0 * target)).item())

    def close(a, b):
        return abs(a - b) <= 1e-6 * max(abs(a), abs(b))

    h = 1e-5
    fd_Wi = dJ(run(Wi + h, beta, P0, kap), run(Wi - h, beta, P0, kap)) / (2 * h)
    fd_beta = dJ(run(Wi, beta + h, P0, kap), run(Wi, beta - h, P0, kap)) / (2 * h)
    assert close(gWi, fd_Wi), (gWi, fd_Wi)
    assert close(gbeta, fd_beta), (gbeta, fd_beta)
    for (c, q) in [(0, 1234), (2, N - 77)]:
        pp, pm = P0.clone(), P0.clone()
        pp[c, q] += h
        pm[c, q] -= h
        fd = dJ(run(Wi, beta, pp, kap), run(Wi, beta, pm, kap)) / (2 * h)
        assert close(g_p0[c, q].item(), fd), (c, q, g_p0[c, q].item(), fd)
    for (c, q) in [(1, 4321), (3, N - 5)]:
        kp, km = kap.clone(), kap.clone()
        kp[c, q] += h
        km[c, q] -= h
        fd = dJ(run(Wi, beta, P0, kp), run(Wi, beta, P0, km)) / (2 * h)
        assert close(g_k[c, q].item(), fd), (c, q, g_k[c, q].item(), fd)
