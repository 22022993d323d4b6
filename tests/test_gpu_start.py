"""The SDIRK2 first step (TFS_PARAM_START = TFS_START_SDIRK2, Section 5.1)
through the C ABI against the oracle's `orc_first_step_sdirk2`, followed by
BDF2 steps whose history is the initial state.

1. Pointwise law (transport off): the per-point kernel of tfs_start.cu.
2. Implicit transport: both stage systems through the Krylov solver.
3. The paper's convergence case on the GPU (no flow, cos(2 pi x) cos(4 pi y),
   eps = 1e-2, alpha = 0.5, weighted Bochner norm): order -> 1 + alpha with
   the SDIRK2 start and the mass-completed SOE, order 1 with BDF2.
4. Refusals: explicit transport at the first step, alpha = 1 at creation.

Tolerances as for the default step: FP64 1e-11 per component (1e-10 with the
Krylov solve, whose stopping rule is a relative residual of 1e-13), FP32
storage 2e-5 (the start itself is formed in FP64 from the float inputs).
"""
import numpy as np
import pytest

from helpers import courant_fraction, ensure_lib, rel_err_per_component
from oracle import orc, soe, special
from paper_2411_17294_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_lib()


def gpu_run(case, sigma0, kap, u, steps, precision, transport):
    import torch
    from paper_2411_17294_gb300 import tfs
    s = tfs.Solver(case["dim"], case["n"], case["alpha"], case["Wi"], case["beta"], case["dt"], m=len(case["mu"]),
                   precision=precision, mu=case["mu"], w=case["w"], eps=case.get("eps", 0.0),
                   stencil=case.get("stencil", 0), transport=transport, L=case.get("L"), start="sdirk2")
    dt_ = s.dtype
    s.set_state(None if sigma0 is None else torch.as_tensor(sigma0, dtype=dt_, device=s.device))
    kt = torch.as_tensor(kap, dtype=dt_, device=s.device).contiguous()
    ut = None if u is None else torch.as_tensor(u, dtype=dt_, device=s.device).contiguous()
    for _ in range(steps):
        s.step(kt, kt, ut)
    out = s.stress().double().cpu().numpy()
    flags = s.status()
    s.close()
    return out, flags


POINT_CASES = [
    # dim, n, alpha, m, with sigma0
    (2, (20, 17), 0.5, 8, True),
    (2, (13, 11), 0.3, 12, False),
    (3, (7, 6, 5), 0.7, 6, True),
]


@pytest.mark.parametrize("dim,n,alpha,m,with_s0", POINT_CASES)
@pytest.mark.parametrize("steps", [1, 5])
@pytest.mark.parametrize("precision", [0, 1])
def test_sdirk2_start_pointwise_matches_oracle(dim, n, alpha, m, with_s0, steps, precision):
    from paper_2411_17294_gb300 import tfs
    dt, Wi, beta = 5e-3, 1.3, 0.4
    mu, w = soe.soe_nnls(alpha, dt, 8 * dt, m)
    case = dict(dim=dim, n=n, alpha=alpha, Wi=Wi, beta=beta, dt=dt, mu=mu, w=w)
    _, kap = inputs.spectral_velocity(dim, n, 2, seed=31)
    kap = 0.5 * np.asarray(kap)
    sigma0 = inputs.random_stress(dim, n, 32) if with_s0 else None
    if precision == 1:
        kap = np.asarray(kap, np.float32).astype(np.float64)
        sigma0 = None if sigma0 is None else np.asarray(sigma0, np.float32).astype(np.float64)
    prob = orc.Problem(dim=dim, n=n, alpha=alpha, Wi=Wi, beta=beta, dt=dt, mu=mu, w=w, start="sdirk2")
    ref = orc.forward(prob, sigma0, kap, None, steps)
    got, flags = gpu_run(case, sigma0, kap, None, steps, precision, transport=False)
    assert not (flags & (tfs.TFS_FLAG_NONFINITE | tfs.TFS_FLAG_SINGULAR))
    assert np.max(np.abs(ref)) > 1e-3
    assert np.all(rel_err_per_component(got, ref) < (1e-11 if precision == 0 else 2e-5))


IMPLICIT_CASES = [
    (2, (16, 12), 0.5, 8, 0.0, 0, 4.0),
    (3, (6, 5, 4), 0.35, 8, 0.01, 1, 3.0),
]


@pytest.mark.parametrize("dim,n,alpha,m,eps,stencil,speed", IMPLICIT_CASES)
@pytest.mark.parametrize("precision", [0, 1])
def test_sdirk2_start_implicit_transport_matches_oracle(dim, n, alpha, m, eps, stencil, speed, precision):
    from paper_2411_17294_gb300 import tfs
    steps, dt, Wi, beta = 6, 2e-3, 1.3, 0.4
    mu, w = soe.soe_nnls(alpha, dt, steps * dt, m)
    case = dict(dim=dim, n=n, alpha=alpha, Wi=Wi, beta=beta, dt=dt, mu=mu, w=w, eps=eps, stencil=stencil)
    u, kap = inputs.spectral_velocity(dim, n, 2, seed=41)
    u = np.asarray(u) * (speed / courant_fraction(dict(case, transport=True), u))
    sigma0 = inputs.random_stress(dim, n, 42)
    if precision == 1:
        kap, u, sigma0 = (np.asarray(a, np.float32).astype(np.float64) for a in (kap, u, sigma0))
    prob = orc.Problem(dim=dim, n=n, alpha=alpha, Wi=Wi, beta=beta, dt=dt, mu=mu, w=w, eps=eps, stencil=stencil,
                       transport=True, implicit=True, start="sdirk2")
    ref = orc.forward(prob, sigma0, kap, u, steps)
    got, flags = gpu_run(case, sigma0, kap, u, steps, precision, transport="implicit")
    assert not (flags & (tfs.TFS_FLAG_NOCONV | tfs.TFS_FLAG_NONFINITE))
    assert np.all(rel_err_per_component(got, ref) < (1e-10 if precision == 0 else 2e-5))


def _gpu_bochner_errors(start, dts, m=32):
    import torch
    from paper_2411_17294_gb300 import tfs
    alpha, Wi, eps, T = 0.5, 1.0, 1e-2, 1.0
    n = (8, 8)
    N = n[0] * n[1]
    h = 1.0 / n[0]
    x = (np.arange(N) % n[0]) * h
    y = (np.arange(N) // n[0]) * h
    shape = np.cos(2 * np.pi * x) * np.cos(4 * np.pi * y)
    lam_h = 1.0 / Wi + eps * (4 * np.sin(np.pi * h) ** 2 + 4 * np.sin(2 * np.pi * h) ** 2) / h ** 2
    errs = []
    for dt in dts:
        steps = int(round(T / dt))
        mu, w = soe.soe_build(alpha, dt, T, m)
        s = tfs.Solver(2, n, alpha, Wi, 0.5, dt, m=m, precision=tfs.TFS_FP64, mu=mu, w=w, eps=eps, L=(1.0, 1.0),
                       transport="implicit", start=start)
        s.set_state(torch.as_tensor(np.tile(shape, (3, 1)), device=s.device))
        k = torch.zeros((4, N), dtype=torch.float64, device=s.device)
        u = torch.zeros((2, N), dtype=torch.float64, device=s.device)
        acc = 0.0
        for kk in range(1, steps + 1):
            s.step(k, k, u)
            t = kk * dt
            exact = shape * special.mittag_leffler(alpha, -lam_h * t ** alpha)
            e2 = np.mean((s.stress()[0].cpu().numpy() - exact) ** 2)
            acc += (0.5 if kk == steps else 1.0) * e2 * t ** (2 * (1 - alpha)) * dt
        assert not (s.status() & tfs.TFS_FLAG_NOCONV)
        s.close()
        errs.append(np.sqrt(acc))
    return [float(np.log2(errs[i] / errs[i + 1])) for i in range(len(errs) - 1)]


def test_paper_convergence_case_order_on_gpu():
    dts = [1 / 20, 1 / 40, 1 / 80, 1 / 160]
    sdirk = _gpu_bochner_errors("sdirk2", dts)
    bdf = _gpu_bochner_errors("bdf2", dts)
    assert all(q > 1.3 for q in sdirk) and sdirk[-1] > 1.38, sdirk
    assert all(0.95 < q < 1.1 for q in bdf), bdf


def test_sdirk2_start_refusals():
    import torch
    from paper_2411_17294_gb300 import tfs
    n, dt = (8, 8), 1e-2
    mu, w = soe.soe_nnls(0.5, dt, 1.0, 4)
    s = tfs.Solver(2, n, 0.5, 1.0, 0.5, dt, m=4, precision=tfs.TFS_FP64, mu=mu, w=w, transport=True, start="sdirk2")
    s.set_state(torch.ones((3, 64), dtype=torch.float64, device=s.device))
    k = torch.zeros((4, 64), dtype=torch.float64, device=s.device)
    u = torch.zeros((2, 64), dtype=torch.float64, device=s.device)
    with pytest.raises(tfs.TfsError):
        s.step(k, k, u)
    assert s.step_index() == 0
    s.close()
    with pytest.raises(tfs.TfsError):
        tfs.Solver(2, n, 1.0, 1.0, 0.5, dt, m=0, precision=tfs.TFS_FP64, transport=False, start="sdirk2")
