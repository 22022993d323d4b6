"""The adjoint of the implicit-transport step (TFS_PARAM_TRANSPORT = 2, stress
form; BDF2 start, and the SDIRK2 start of Section 5.1) through tfs_backward:
the global solve with the transposed operator (the step's block-Jacobi
BiCGStab on the transposed point blocks and the gathered tap coefficients),
then the pointwise adjoint; for the SDIRK2 start, stage 1 solved again and
both stage systems transposed.

1. Against FP64 central differences of the oracle's implicit scheme (its dense
   global solve, oracle/orc.c), with velocities above the explicit Courant
   limit: random directions of sigma0 (exact: sigma(T) is affine in sigma0) and
   of the velocity gradient, Wi and beta; both stencils, with diffusion,
   alpha < 1 and alpha = 1, 2D and 3D, FP64 and FP32 storage.
2. torch.autograd through fractional_stress(transport="implicit") against
   central differences of the CUDA forward, 1e-6 relative.
(The paper's variable with implicit transport, either start, is covered in
test_gpu_paper_adjoint.py.)

Tolerances: FP64 1e-6 relative (central differences, h = 1e-5; Krylov stopping
at a relative residual of 1e-13 forward and backward); FP32 storage 5e-4 (its
default Krylov tolerance is 1e-9, the mode ring is float).
"""
import numpy as np
import pytest

from helpers import courant_fraction, ensure_lib
from oracle import orc, soe
from paper_2411_17294_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_lib()


CASES = [
    # dim, n, alpha, m, steps, K, stencil, eps, speed (x the explicit limit)
    (2, (12, 10), 0.5, 8, 8, 3, 0, 0.0, 3.0),
    (2, (9, 9), 1.0, 0, 7, 4, 0, 0.0, 3.0),
    (2, (16, 6), 0.3, 12, 6, 6, 1, 0.02, 2.0),
    (3, (5, 4, 6), 0.6, 6, 6, 2, 1, 0.01, 2.0),
    (3, (4, 5, 3), 0.45, 16, 5, 5, 0, 0.0, 3.0),
]


SDIRK2_CASES = [
    (2, (12, 10), 0.5, 8, 8, 3, 0, 0.0, 3.0),
    (2, (9, 7), 0.4, 6, 1, 1, 1, 0.0, 2.0),
    (3, (5, 4, 6), 0.6, 6, 6, 2, 1, 0.01, 2.0),
]


@pytest.mark.parametrize("dim,n,alpha,m,steps,K,stencil,eps,speed,start",
                         [c + ("bdf2",) for c in CASES] + [c + ("sdirk2",) for c in SDIRK2_CASES])
@pytest.mark.parametrize("precision", [0, 1])
def test_implicit_adjoint_against_oracle_differences(dim, n, alpha, m, steps, K, stencil, eps, speed, start,
                                                     precision):
    import torch
    from paper_2411_17294_gb300 import tfs
    dt, Wi, beta = 2e-3, 1.3, 0.4
    mu = w = None
    if alpha < 1:
        mu, w = soe.soe_nnls(alpha, dt, 20 * dt, m)
    case = dict(dim=dim, n=n, alpha=alpha, dt=dt, eps=eps, mu=mu, w=w, transport=True)
    u, kap = inputs.spectral_velocity(dim, n, 2, seed=21)
    u = np.asarray(u) * (speed / courant_fraction(case, u))
    kap = 0.5 * np.asarray(kap)
    s0 = inputs.random_stress(dim, n, 22)
    dJ = np.random.default_rng(23).normal(size=s0.shape)
    if precision == 1:
        cast = lambda a: np.asarray(a, np.float32).astype(np.float64)
        u, kap, s0, dJ = cast(u), cast(kap), cast(s0), cast(dJ)
    # GPU gradients
    s = tfs.Solver(dim, n, alpha, Wi, beta, dt, m=m, precision=precision, mu=mu, w=w, eps=eps, stencil=stencil,
                   transport="implicit", start=start)
    dev, tdt = s.device, s.dtype
    kt = torch.as_tensor(kap, dtype=tdt, device=dev).contiguous()
    ut = torch.as_tensor(u, dtype=tdt, device=dev).contiguous()
    s.set_state(torch.as_tensor(s0, dtype=tdt, device=dev))
    ckpts = []
    for k in range(steps):
        if k % K == 0:
            c = s.new_checkpoint()
            s.save(c)
            ckpts.append(c)
        s.step(kt, kt, ut)
    g_s0, g_k, gWi, gb = s.backward(torch.as_tensor(dJ, dtype=tdt, device=dev), ckpts, K, steps, kt, ut)
    g_s0, g_k = g_s0.cpu().numpy(), g_k.cpu().numpy()
    flags = s.status()
    s.close()
    assert not (flags & (tfs.TFS_FLAG_NOCONV | tfs.TFS_FLAG_NONFINITE | tfs.TFS_FLAG_SINGULAR))

    def J(sig0, k, Wi_, b_):
        p = orc.Problem(dim=dim, n=n, alpha=alpha, Wi=Wi_, beta=b_, dt=dt,
                        mu=mu if mu is not None else np.zeros(0), w=w if w is not None else np.zeros(0),
                        eps=eps, stencil=stencil, transport=True, implicit=True, start=start)
        return float(np.sum(dJ * orc.forward(p, sig0, k, u, steps)))

    tol = 1e-6 if precision == 0 else 5e-4
    h = 1e-5

    def check(got, fd, scale):
        assert abs(got - fd) <= tol * scale, (got, fd, scale)

    for seed in (1, 2):
        d = np.random.default_rng(seed).normal(size=s0.shape)
        fd = (J(s0 + d, kap, Wi, beta) - J(s0 - d, kap, Wi, beta)) / 2.0
        check(float(np.sum(g_s0 * d)), fd, np.sum(np.abs(g_s0 * d)))
    for seed in (3, 4):
        d = np.random.default_rng(seed).normal(size=kap.shape)
        fd = (J(s0, kap + h * d, Wi, beta) - J(s0, kap - h * d, Wi, beta)) / (2 * h)
        check(float(np.sum(g_k * d)), fd, np.sum(np.abs(g_k * d)))
    fd_wi = (J(s0, kap, Wi + h, beta) - J(s0, kap, Wi - h, beta)) / (2 * h)
    fd_b = (J(s0, kap, Wi, beta + h) - J(s0, kap, Wi, beta - h)) / (2 * h)
    check(gWi, fd_wi, max(abs(fd_wi), 1e-12))
    check(gb, fd_b, max(abs(fd_b), 1e-12))
    # the transport's adjoint matters: the explicit-free (pointwise) gradient differs
    p0 = orc.Problem(dim=dim, n=n, alpha=alpha, Wi=Wi, beta=beta, dt=dt,
                     mu=mu if mu is not None else np.zeros(0), w=w if w is not None else np.zeros(0))
    d = np.random.default_rng(1).normal(size=s0.shape)
    fd0 = float(np.sum(dJ * (orc.forward(p0, s0 + d, kap, None, steps) - orc.forward(p0, s0 - d, kap, None, steps))))
    assert abs(fd0 / 2.0 - float(np.sum(g_s0 * d))) > 1e-3 * np.sum(np.abs(g_s0 * d))


def test_implicit_autograd_matches_central_differences():
    import torch
    from paper_2411_17294_gb300.autograd import fractional_stress
    dim, n, alpha, dt, steps, K, m = 2, (8, 8), 0.5, 2e-3, 20, 6, 8
    mu, w = soe.soe_nnls(alpha, dt, steps * dt, m)
    dev = torch.device("cuda", 0)
    u_np, k_np = inputs.spectral_velocity(dim, n, 2, seed=41)
    case = dict(dim=dim, n=n, alpha=alpha, dt=dt, mu=mu, w=w, transport=True)
    u_np = np.asarray(u_np) * (4.0 / courant_fraction(case, u_np))
    s0_np = inputs.random_stress(dim, n, 42)
    target = torch.as_tensor(np.random.default_rng(43).normal(size=s0_np.shape), device=dev)
    kw = dict(dim=dim, n=n, alpha=alpha, dt=dt, steps=steps, K=K, mu=mu, w=w,
              u=torch.as_tensor(u_np, device=dev), transport="implicit", eps=0.01)

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

    def close(a, b, scale=0.0):
        # relative 1e-6; field entries normwise (against the largest entry of
        # their gradient field): the forward's and the adjoint's Krylov solves
        # stop at a relative residual of 1e-13, which leaves an absolute error
        # of ~1e-8 on entries that are small against the field
        return abs(a - b) <= 1e-6 * max(abs(a), abs(b), scale)

    t = lambda x: torch.tensor(x, dtype=torch.float64, device=dev)
    with torch.no_grad():
        s0d, kd = s0.detach(), k.detach()
        gs0, gk = float(s0.grad.abs().max()), float(k.grad.abs().max())
        assert close(Wi.grad.item(), fd(lambda x: J(s0d, kd, t(x), beta.detach()).item(), 1.4))
        assert close(beta.grad.item(), fd(lambda x: J(s0d, kd, Wi.detach(), t(x)).item(), 0.3))
        for (c, q) in [(0, 0), (2, 63), (1, 17)]:
            def fs(x, c=c, q=q):
                a = s0d.clone()
                a[c, q] = x
                return J(a, kd, Wi.detach(), beta.detach()).item()
            assert close(s0.grad[c, q].item(), fd(fs, s0d[c, q].item()), gs0)
        for (c, q) in [(0, 5), (3, 40)]:
            def fk(x, c=c, q=q):
                a = kd.clone()
                a[c, q] = x
                return J(s0d, a, Wi.detach(), beta.detach()).item()
            assert close(k.grad[c, q].item(), fd(fk, kd[c, q].item()), gk)
