"""torch.autograd through the CUDA forward and the hand-written adjoint,
checked against FP64 central finite differences of the CUDA forward itself
(relative agreement 1e-6)."""
import numpy as np
import pytest

from helpers import courant_fraction, ensure_lib, stable_velocity
from oracle import soe
from paper_2411_17294_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_lib()


@pytest.mark.parametrize("transport,start,form", [
    (False, "bdf2", "stress"), (True, "bdf2", "stress"), (False, "sdirk2", "stress"),
    # implicit transport with the paper's first step, and in the paper's variable
    ("implicit", "sdirk2", "stress"), ("implicit", "bdf2", "paper"), ("implicit", "sdirk2", "paper")])
def test_autograd_matches_central_differences(transport, start, form):
    import torch
    from paper_2411_17294_gb300.autograd import fractional_stress
    dim, n, alpha, dt, steps, K, m = 2, (8, 8), 0.5, 2e-3, 30, 7, 8
    mu, w = soe.soe_nnls(1 - alpha if form == "paper" else alpha, dt, steps * dt, m)
    dev = torch.device("cuda", 0)
    u_np, k_np = inputs.spectral_velocity(dim, n, 2, seed=31)
    case = dict(dim=dim, n=n, alpha=alpha, dt=dt, mu=mu, w=w, transport=True)
    if transport == "implicit":
        # twice the explicit stress-form limit (the explicit step would be unstable)
        mu_s, w_s = soe.soe_nnls(alpha, dt, steps * dt, m)
        u_np = np.asarray(u_np) * (2.0 / courant_fraction(dict(case, mu=mu_s, w=w_s), u_np))
    else:
        u_np = stable_velocity(case, u_np)
    s0_np = inputs.random_stress(dim, n, 32)
    target = torch.as_tensor(np.random.default_rng(33).normal(size=s0_np.shape), device=dev)
    kw = dict(dim=dim, n=n, alpha=alpha, dt=dt, steps=steps, K=K, mu=mu, w=w,
              u=torch.as_tensor(u_np, device=dev) if transport else None, start=start, form=form,
              transport=transport if transport == "implicit" else None)

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
        # their gradient field, the error measure of every parity test here):
        # with implicit transport both the forward's and the adjoint's Krylov
        # solves stop at a relative residual of 1e-13, which leaves an absolute
        # error of ~1e-8 on entries that are small against the field
        return abs(a - b) <= 1e-6 * max(abs(a), abs(b), scale)

    with torch.no_grad():
        s0d, kd = s0.detach(), k.detach()
        gs0, gk = float(s0.grad.abs().max()), float(k.grad.abs().max())
        assert close(Wi.grad.item(), fd(lambda x: J(s0d, kd, torch.tensor(x, dtype=torch.float64, device=dev), beta.detach()).item(), 1.4))
        assert close(beta.grad.item(), fd(lambda x: J(s0d, kd, Wi.detach(), torch.tensor(x, dtype=torch.float64, device=dev)).item(), 0.3))
        for (c, q) in [(0, 0), (2, 63), (1, 17)]:
            def fs(x, c=c, q=q):
                t = s0d.clone(); t[c, q] = x
                return J(t, kd, Wi.detach(), beta.detach()).item()
            assert close(s0.grad[c, q].item(), fd(fs, s0d[c, q].item()), gs0)
        for (c, q) in [(0, 5), (3, 40), (1, 9)]:
            def fk(x, c=c, q=q):
                t = kd.clone(); t[c, q] = x
                return J(s0d, t, Wi.detach(), beta.detach()).item()
            assert close(k.grad[c, q].item(), fd(fk, kd[c, q].item()), gk)
