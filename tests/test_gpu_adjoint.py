"""The hand-written adjoint (tfs_backward: checkpoint segments, recompute,
reverse sweep) against the oracle's reference adjoint, which is itself pinned
to FP64 central finite differences (tests/test_oracle_pins.py)."""
import numpy as np
import pytest

from helpers import ensure_lib, stable_velocity
from oracle import orc, soe
from paper_2411_17294_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_lib()


def gpu_gradients(dim, n, alpha, Wi, beta, dt, m, steps, K, sigma0, kap, u, dJ, precision, transport, mu, w,
                  eps=0.0):
    import torch
    from paper_2411_17294_gb300 import tfs
    s = tfs.Solver(dim, n, alpha, Wi, beta, dt, m=m if alpha < 1 else 0, precision=precision, mu=mu, w=w,
                   transport=transport, eps=eps)
    dt_ = s.dtype
    dev = s.device
    kt = torch.as_tensor(kap, dtype=dt_, device=dev).contiguous()
    ut = torch.as_tensor(u, dtype=dt_, device=dev).contiguous() if transport else None
    s.set_state(torch.as_tensor(sigma0, dtype=dt_, device=dev))
    ckpts = []
    for k in range(steps):
        if k % K == 0:
            buf = s.new_checkpoint()
            s.save(buf)
            ckpts.append(buf)
        s.step(kt, kt, ut)
    sT = s.stress().double().cpu().numpy()
    g_s0, g_k, gWi, gb = s.backward(torch.as_tensor(dJ(sT), dtype=dt_, device=dev), ckpts, K, steps, kt, ut)
    out = dict(sigma_T=sT, sigma0=g_s0.cpu().numpy(), kappa=g_k.cpu().numpy(), Wi=gWi, beta=gb)
    s.close()
    return out, mu, w


CASES = [
    # dim, n, alpha, m, steps, K, transport, eps
    (2, (12, 10), 0.5, 6, 20, 7, True, 0.02),
    (3, (5, 4, 6), 0.7, 8, 12, 5, False, 0.0),
    (2, (9, 9), 1.0, 0, 15, 4, True, 0.0),
    (3, (4, 5, 3), 0.35, 16, 10, 10, True, 0.0),
]


@pytest.mark.parametrize("dim,n,alpha,m,steps,K,transport,eps", CASES)
@pytest.mark.parametrize("precision", [0, 1])
def test_adjoint_matches_oracle(dim, n, alpha, m, steps, K, transport, eps, precision):
    Wi, beta, dt = 1.3, 0.4, 2e-3
    N = int(np.prod(n))
    u, kap = inputs.spectral_velocity(dim, n, 2, seed=12)
    mu = w = None
    case = dict(dim=dim, n=n, alpha=alpha, dt=dt, eps=eps)
    if alpha < 1:
        mu, w = soe.soe_nnls(alpha, dt, steps * dt, m)
        case.update(mu=mu, w=w)
    u = stable_velocity(case, u)
    sigma0 = inputs.random_stress(dim, n, 13)
    rng = np.random.default_rng(14)
    target = rng.normal(size=sigma0.shape)
    dJ = lambda sT: 2.0 * (sT - target)
    got, mu, w = gpu_gradients(dim, n, alpha, Wi, beta, dt, m, steps, K, sigma0, kap, u, dJ, precision,
                               transport, mu, w, eps)
    p = orc.Problem(dim=dim, n=n, alpha=alpha, Wi=Wi, beta=beta, dt=dt,
                    mu=mu if mu is not None else np.zeros(0), w=w if w is not None else np.zeros(0),
                    transport=transport, eps=eps)
    sT = orc.forward(p, sigma0, kap, u if transport else None, steps)
    ref = orc.gradients(p, sigma0, kap, u if transport else None, steps, dJ(sT))
    tol = 1e-10 if precision == 0 else 2e-4
    for key in ("sigma0", "kappa"):
        scale = np.max(np.abs(ref[key]))
        assert np.max(np.abs(got[key] - ref[key])) <= tol * scale, key
    for key in ("Wi", "beta"):
        assert abs(got[key] - ref[key]) <= tol * max(abs(ref[key]), 1e-12), key
