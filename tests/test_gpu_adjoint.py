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
                  eps=0.0, start="bdf2"):
    import torch
    from paper_2411_17294_gb300 import tfs
    s = tfs.Solver(dim, n, alpha, Wi, beta, dt, m=m if alpha < 1 else 0, precision=precision, mu=mu, w=w,
                   transport=transport, eps=eps, start=start)
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


def test_adjoint_workload_512_against_central_differences():
    # The adjoint workload at full size: 2D periodic 512^2, m = 32, alpha = 0.5,
    # dt = 1e-3, 500 steps, checkpoint every 50, transport off, FP64;
    # J = ||sigma(T) - sigma_target||^2 with the target from a seeded run at
    # Wi = 1.5.  Gradients with respect to Wi, beta and sampled entries of
    # sigma0 and grad_u against central differences of the CUDA forward, to
    # 1e-6 relative.  J(x+h) - J(x-h) is summed as sum (s+ - s-)(s+ + s- - 2 t),
    # which has no cancellation (the perturbed runs differ from each other only
    # where the perturbation reaches).
    import torch
    from paper_2411_17294_gb300 import tfs
    dim, n, alpha, m, dt, steps, K = 2, (512, 512), 0.5, 32, 1e-3, 500, 50
    Wi, beta = 1.0, 0.5
    N = n[0] * n[1]
    mu, w = soe.soe_nnls(alpha, dt, steps * dt, m)
    dev = torch.device("cuda", 0)
    _, kap = inputs.spectral_velocity(dim, n, 32, 2)
    kap = torch.as_tensor(0.05 * kap, device=dev)
    sigma0 = torch.as_tensor(inputs.random_stress(dim, n, 5, amplitude=0.5), device=dev)

    def run(Wi_, beta_, s0, k, grads_for=None):
        s = tfs.Solver(dim, n, alpha, Wi_, beta_, dt, m=m, precision=tfs.TFS_FP64, mu=mu, w=w, transport=False)
        s.set_state(s0)
        ckpts = []
        for i in range(steps):
            if grads_for is not None and i % K == 0:
                buf = s.new_checkpoint()
                s.save(buf)
                ckpts.append(buf)
            s.step(k, k, None)
        sT = s.stress()
        out = sT
        if grads_for is not None:
            out = (sT, s.backward(2.0 * (sT - grads_for), ckpts, K, steps, k, None))
        s.close()
        return out

    target = run(1.5, beta, sigma0, kap)
    _, (g_s0, g_k, gWi, gbeta) = run(Wi, beta, sigma0, kap, grads_for=target)

    def dJ(sp, sm):
        return float(torch.sum((sp - sm) * (sp + sm - 2.0 * target)).item())

    def close(a, b):
        return abs(a - b) <= 1e-6 * max(abs(a), abs(b))

    h = 1e-5
    fd_Wi = dJ(run(Wi + h, beta, sigma0, kap), run(Wi - h, beta, sigma0, kap)) / (2 * h)
    fd_beta = dJ(run(Wi, beta + h, sigma0, kap), run(Wi, beta - h, sigma0, kap)) / (2 * h)
    assert close(gWi, fd_Wi), (gWi, fd_Wi)
    assert close(gbeta, fd_beta), (gbeta, fd_beta)
    for (c, q) in [(0, 1234), (2, N - 77)]:
        sp, sm = sigma0.clone(), sigma0.clone()
        sp[c, q] += h
        sm[c, q] -= h
        fd = dJ(run(Wi, beta, sp, kap), run(Wi, beta, sm, kap)) / (2 * h)
        assert close(g_s0[c, q].item(), fd), (c, q, g_s0[c, q].item(), fd)
    for (c, q) in [(1, 4321), (3, 99999)]:
        kp, km = kap.clone(), kap.clone()
        kp[c, q] += h
        km[c, q] -= h
        fd = dJ(run(Wi, beta, sigma0, kp), run(Wi, beta, sigma0, km)) / (2 * h)
        assert close(g_k[c, q].item(), fd), (c, q, g_k[c, q].item(), fd)


@pytest.mark.parametrize("dim,n,alpha,transport", [(2, (20, 17), 0.5, True), (3, (6, 5, 7), 0.3, False),
                                                   (2, (16, 9), 1.0, True)])
def test_adjoint_dot_product_exact_directions(dim, n, alpha, transport):
    # Directions in which the step map is affine give dot-product tests with no
    # finite-difference error: sigma(T) is affine in sigma0 (the initial stress
    # enters every step linearly), so <lambda, sigma(T; sigma0 + d) - sigma(T;
    # sigma0)> = <d, dJ/dsigma0> for J = <lambda, sigma(T)>; and it is affine in G =
    # (1 - beta)/(Wi Re), itself affine in beta, so (J(beta2) - J(beta1))/(beta2 -
    # beta1) = dJ/dbeta.  FP64, to rounding.
    Wi, beta, dt, steps, K = 1.3, 0.4, 2e-3, 14, 4
    m = 0 if alpha == 1.0 else 8
    mu, w = soe.soe_build(alpha, dt, steps * dt, m) if m else (None, None)
    u, kap = inputs.spectral_velocity(dim, n, 2, seed=31)
    case = dict(dim=dim, n=n, alpha=alpha, dt=dt, eps=0.0)
    if m:
        case.update(mu=mu, w=w)
    u = stable_velocity(case, u)
    rng = np.random.default_rng(32)
    nc = 3 if dim == 2 else 6
    N = int(np.prod(n))
    sigma0 = rng.normal(size=(nc, N))
    d = rng.normal(size=(nc, N))
    lam = rng.normal(size=(nc, N))
    run = lambda s0, b: gpu_gradients(dim, n, alpha, Wi, b, dt, m, steps, K, s0, kap, u, lambda sT: lam, 0,
                                      transport, mu, w)[0]
    base = run(sigma0, beta)
    moved = run(sigma0 + d, beta)
    lhs = np.sum(lam * (moved["sigma_T"] - base["sigma_T"]))
    rhs = np.sum(d * base["sigma0"])
    assert abs(lhs - rhs) <= 1e-11 * (abs(lhs) + abs(rhs)), (lhs, rhs)
    b2 = beta + 0.05
    other = run(sigma0, b2)
    dJ = (np.sum(lam * other["sigma_T"]) - np.sum(lam * base["sigma_T"])) / (b2 - beta)
    assert abs(dJ - base["beta"]) <= 1e-9 * abs(dJ), (dJ, base["beta"])



@pytest.mark.parametrize("dim,n,alpha,steps,K", [(2, (9, 7), 0.5, 8, 3), (3, (4, 5, 3), 0.3, 5, 5), (2, (6, 5), 0.7, 1, 1)])
def test_sdirk2_start_adjoint(dim, n, alpha, steps, K):
    # The adjoint of a run that starts with the SDIRK2 step (pointwise law):
    # exact in the affine directions (sigma0, beta), FP64 central differences
    # for Wi and entries of kappa, and the FP32-storage adjoint near the FP64 one.
    Wi, beta, dt, m = 1.3, 0.4, 2e-3, 6
    mu, w = soe.soe_build(alpha, dt, 50 * dt, m)
    _, kap = inputs.spectral_velocity(dim, n, 2, seed=41)
    kap = 0.5 * np.asarray(kap)
    rng = np.random.default_rng(42)
    nc = 3 if dim == 2 else 6
    N = int(np.prod(n))
    sigma0 = rng.normal(size=(nc, N))
    lam = rng.normal(size=(nc, N))
    run = lambda s0, k, wi, b, prec=0: gpu_gradients(dim, n, alpha, wi, b, dt, m, steps, K, s0, k, None,
                                                     lambda sT: lam, prec, False, mu, w, start="sdirk2")[0]
    J = lambda out: float(np.sum(lam * out["sigma_T"]))
    base = run(sigma0, kap, Wi, beta)
    d = rng.normal(size=(nc, N))
    moved = run(sigma0 + d, kap, Wi, beta)
    lhs, rhs = J(moved) - J(base), float(np.sum(d * base["sigma0"]))
    assert abs(lhs - rhs) <= 1e-10 * (abs(lhs) + abs(rhs)), (lhs, rhs)
    db = 0.05
    fd_b = (J(run(sigma0, kap, Wi, beta + db)) - J(base)) / db
    assert abs(fd_b - base["beta"]) <= 1e-9 * abs(fd_b), (fd_b, base["beta"])
    hW = 1e-5 * Wi
    fd_w = (J(run(sigma0, kap, Wi + hW, beta)) - J(run(sigma0, kap, Wi - hW, beta))) / (2 * hW)
    assert abs(fd_w - base["Wi"]) <= 1e-6 * abs(fd_w), (fd_w, base["Wi"])
    for c, q in [(0, 0), (dim * dim - 1, N - 1), (1, N // 2)]:
        hk = 1e-6
        kp, km = kap.copy(), kap.copy()
        kp[c, q] += hk
        km[c, q] -= hk
        fd_k = (J(run(sigma0, kp, Wi, beta)) - J(run(sigma0, km, Wi, beta))) / (2 * hk)
        assert abs(fd_k - base["kappa"][c, q]) <= 1e-6 * max(abs(fd_k), 1e-3), (c, q, fd_k, base["kappa"][c, q])
    f32 = run(sigma0, kap, Wi, beta, prec=1)
    assert np.max(np.abs(f32["sigma0"] - base["sigma0"])) < 1e-4 * np.max(np.abs(base["sigma0"]))
    assert abs(f32["Wi"] - base["Wi"]) < 1e-4 * abs(base["Wi"])
