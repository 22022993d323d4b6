"""The paper's own variable (TFS_PARAM_FORM = TFS_FORM_PAPER, Section 3.4)
through the C ABI against the oracle's scheme in that variable
(oracle.paper_form.PaperForm: BDF2 on Phi, Psi = D^{1-alpha} Phi by kernel
compression of g_alpha, stress = Psi).

1. Grids spanning several 32-point tiles and a ragged tail, 2D and 3D, zero and
   non-zero Phi(0), frozen and time-varying velocity gradients, element by
   element.
2. The 3D 256^3 m = 32 FP32 size in the benchmark's launch configuration, on
   sampled points (every point is independent in this form, so the oracle
   runs on the samples alone).
3. Checkpoint round trip (Psi and the host modes of Phi0 = 1 restored).
4. The SDIRK2 first step in this variable (Section 5.1).
5. Explicit transport of Psi, with the tiled and the per-point pre-pass.
6. Implicit transport of Psi (eq. FP_discrete) through the Krylov solver, far
   above the explicit limit.
   With either start (the SDIRK2 stages solve with the transport inside too).
7. Refusals: alpha = 1, explicit transport with the SDIRK2 start.

Tolerances: FP64 1e-11 per component; FP32 storage 2e-5 (Psi = xi Phi + h
cancels: xi ~ (b0/dt)^(1-alpha), so the float rounding of Phi and of the
mode levels is amplified by xi |Phi| / |Psi|, a few tens here).
"""
import numpy as np
import pytest

from helpers import ensure_lib, rel_err_per_component
from oracle import soe
from oracle.paper_form import PaperForm
from paper_2411_17294_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_lib()


def make_solver(dim, n, alpha, Wi, beta, dt, mu, w, precision, **kw):
    from paper_2411_17294_gb300 import tfs
    return tfs.Solver(dim, n, alpha, Wi, beta, dt, m=len(mu), precision=precision, mu=mu, w=w, transport=False,
                      form="paper", **kw)


def kap_sequence(dim, n, seed, varying):
    _, k0 = inputs.spectral_velocity(dim, n, 2, seed=seed)
    k0 = 0.6 * np.asarray(k0)
    if not varying:
        return lambda k: k0
    _, k1 = inputs.spectral_velocity(dim, n, 2, seed=seed + 1)
    k1 = 0.6 * np.asarray(k1)
    return lambda k: k0 * np.cos(0.3 * k) + k1 * np.sin(0.2 * k)


CASES = [
    # dim, n, alpha, m, phi0, varying
    (2, (37, 29), 0.5, 8, True, False),
    (2, (33, 7), 0.3, 16, False, True),
    (3, (9, 7, 5), 0.6, 12, True, True),
    (3, (8, 8, 4), 0.45, 32, False, False),
]


@pytest.mark.parametrize("dim,n,alpha,m,phi0,varying", CASES)
@pytest.mark.parametrize("precision", [0, 1, 2])
def test_paper_form_matches_oracle(dim, n, alpha, m, phi0, varying, precision):
    import torch
    from paper_2411_17294_gb300 import tfs
    steps, dt, Wi, beta = 7, 4e-3, 1.3, 0.4
    N = int(np.prod(n))
    nc = 3 if dim == 2 else 6
    mu, w = soe.soe_nnls(1 - alpha, dt, 50 * dt, m)
    K = kap_sequence(dim, n, 51, varying)
    P0 = inputs.random_stress(dim, n, 52) if phi0 else None
    if precision != 0:
        cast = lambda a: np.asarray(a, np.float32).astype(np.float64)
        K0 = K
        K = lambda k: cast(K0(k))
        P0 = None if P0 is None else cast(P0)
    pf = PaperForm(dim, N, Wi, beta, dt, mu, w, Phi0=P0)
    s = make_solver(dim, n, alpha, Wi, beta, dt, mu, w, precision)
    s.set_state(None if P0 is None else torch.as_tensor(P0, dtype=s.dtype, device=s.device))
    assert float(s.stress().abs().max()) == 0.0            # Psi before the first step
    for k in range(steps):
        kn, km = K(k), K(k - 1) if k > 0 else K(0)
        ref = pf.step(kn, km)
        kt = torch.as_tensor(kn, dtype=s.dtype, device=s.device).contiguous()
        kmt = torch.as_tensor(km, dtype=s.dtype, device=s.device).contiguous()
        s.step(kt, kmt if k > 0 else None)
    got = s.stress().double().cpu().numpy()
    assert not (s.status() & (tfs.TFS_FLAG_NONFINITE | tfs.TFS_FLAG_SINGULAR | tfs.TFS_FLAG_TIMEOUT))
    s.close()
    assert got.shape == (nc, N)
    assert np.max(np.abs(ref)) > 1e-2
    tol = {0: 1e-11, 1: 2e-5, 2: 1e-3}[precision]   # plain float sums: a precision-study mode
    assert np.all(rel_err_per_component(got, ref) < tol), rel_err_per_component(got, ref)


@pytest.mark.parametrize("dim,n,alpha,m,phi0", [(2, (37, 29), 0.5, 8, True), (3, (9, 7, 5), 0.35, 12, True),
                                                 (2, (20, 9), 0.7, 6, False)])
@pytest.mark.parametrize("precision", [0, 1])
def test_paper_form_sdirk2_start_matches_oracle(dim, n, alpha, m, phi0, precision):
    import torch
    from paper_2411_17294_gb300 import tfs
    steps, dt, Wi, beta = 5, 4e-3, 1.3, 0.4
    N = int(np.prod(n))
    mu, w = soe.soe_nnls(1 - alpha, dt, 50 * dt, m)
    K = kap_sequence(dim, n, 71, True)
    P0 = inputs.random_stress(dim, n, 72) if phi0 else None
    if precision != 0:
        cast = lambda a: np.asarray(a, np.float32).astype(np.float64)
        K0 = K
        K = lambda k: cast(K0(k))
        P0 = None if P0 is None else cast(P0)
    pf = PaperForm(dim, N, Wi, beta, dt, mu, w, Phi0=P0, start="sdirk2")
    pb = PaperForm(dim, N, Wi, beta, dt, mu, w, Phi0=P0)
    s = make_solver(dim, n, alpha, Wi, beta, dt, mu, w, precision, start="sdirk2")
    s.set_state(None if P0 is None else torch.as_tensor(P0, dtype=s.dtype, device=s.device))
    for k in range(steps):
        kn, km = K(k), K(k - 1) if k > 0 else K(0)
        ref = pf.step(kn, km)
        other = pb.step(kn, km)
        s.step(torch.as_tensor(kn, dtype=s.dtype, device=s.device).contiguous(),
               torch.as_tensor(km, dtype=s.dtype, device=s.device).contiguous() if k > 0 else None)
    got = s.stress().double().cpu().numpy()
    assert not (s.status() & (tfs.TFS_FLAG_NONFINITE | tfs.TFS_FLAG_SINGULAR))
    s.close()
    # the start matters, and the library follows the oracle's
    assert np.max(np.abs(ref - other)) > 1e3 * (1e-11 if precision == 0 else 2e-5) * np.max(np.abs(ref))
    assert np.all(rel_err_per_component(got, ref) < (1e-11 if precision == 0 else 2e-5))


def test_paper_form_sdirk2_checkpoint_restores_the_host_modes():
    import torch
    dim, n, alpha, m, dt = 2, (16, 8), 0.5, 8, 5e-3
    mu, w = soe.soe_nnls(1 - alpha, dt, 1.0, m)
    _, kap = inputs.spectral_velocity(dim, n, 2, seed=81)
    s = make_solver(dim, n, alpha, 1.1, 0.3, dt, mu, w, 0, start="sdirk2")
    s.set_state(torch.as_tensor(inputs.random_stress(dim, n, 82), device=s.device))
    kt = torch.as_tensor(0.5 * np.asarray(kap), device=s.device).contiguous()
    for _ in range(3):
        s.step(kt, kt)
    ck = s.new_checkpoint()
    s.save(ck)
    for _ in range(4):
        s.step(kt, kt)
    a = s.stress().clone()
    s.load(ck)
    for _ in range(4):
        s.step(kt, kt)
    assert torch.equal(s.stress(), a)
    s.close()


def test_paper_form_256_cubed_bench_configuration_sampled():
    import torch
    from paper_2411_17294_gb300 import tfs
    n, m, alpha, Wi, beta, dt, steps = (256, 256, 256), 32, 0.6, 2.0, 0.9, 2e-4, 3
    mu, w = soe.soe_nnls(1 - alpha, dt, 200 * dt, m)
    dev = torch.device("cuda", 0)
    _, kap = inputs.spectral_velocity(3, n, 24, 3, device=dev)
    s = make_solver(3, n, alpha, Wi, beta, dt, mu, w, tfs.TFS_FP32)
    kt = torch.as_tensor(kap, dtype=torch.float32, device=dev).contiguous()
    s.set_state(None)
    for _ in range(steps):
        s.step(kt, kt)
    out = s.stress().cpu().numpy().astype(np.float64)
    s.close()
    rng = np.random.default_rng(77)
    idx = np.concatenate([rng.integers(0, 256 ** 3, size=4000), [0, 256 ** 3 - 1]])
    k32 = kt[:, torch.as_tensor(idx, device=dev)].cpu().numpy().astype(np.float64)
    pf = PaperForm(3, len(idx), Wi, beta, dt, mu, w)
    for _ in range(steps):
        ref = pf.step(k32, k32)
    assert np.max(np.abs(ref)) > 0
    assert np.all(rel_err_per_component(out[:, idx], ref) < 2e-5)


def test_paper_form_with_transport_256_cubed_sampled():
    # The 256^3 m = 32 FP32 grid with explicit transport of Psi: after s steps a
    # point depends only on the points within 2 s cells (radius-2 stencil on the
    # extrapolated Psi), so the oracle runs on the periodic (4 s + 1)^3 block
    # around each sample and its centre value is exact.
    import torch
    from paper_2411_17294_gb300 import tfs
    n, m, alpha, Wi, beta, dt, steps = (256, 256, 256), 32, 0.6, 2.0, 0.9, 2e-4, 3
    mu, w = soe.soe_nnls(1 - alpha, dt, 200 * dt, m)
    dev = torch.device("cuda", 0)
    u, kap = inputs.spectral_velocity(3, n, 24, 3, device=dev)
    s = tfs.Solver(3, n, alpha, Wi, beta, dt, m=m, precision=tfs.TFS_FP32, mu=mu, w=w, transport=True,
                   form="paper")
    kt = torch.as_tensor(kap, dtype=torch.float32, device=dev).contiguous()
    ut = (0.1 * torch.as_tensor(u, dtype=torch.float32, device=dev)).contiguous()
    s.set_state(None)
    for _ in range(steps):
        s.step(kt, kt, ut)
    out = s.stress().cpu().numpy().astype(np.float64)
    assert not (s.status() & (tfs.TFS_FLAG_NONFINITE | tfs.TFS_FLAG_TIMEOUT))
    s.close()
    kap32 = kt.cpu().numpy().astype(np.float64)
    u32 = ut.cpu().numpy().astype(np.float64)
    rng = np.random.default_rng(2025)
    R = 2 * steps
    B = 2 * R + 1
    samples = [tuple(int(v) for v in rng.integers(0, 256, size=3)) for _ in range(6)] + [(0, 0, 0), (255, 255, 255)]
    got, ref = [], []
    for (x, y, z) in samples:
        xs, ys, zs = (np.arange(c - R, c + R + 1) % 256 for c in (x, y, z))
        idx = (xs[None, None, :] + 256 * (ys[None, :, None] + 256 * zs[:, None, None])).ravel()
        pf = PaperForm(3, B ** 3, Wi, beta, dt, mu, w, grid=(B, B, B), L=(2 * np.pi * B / 256,) * 3)
        kb, ub = np.ascontiguousarray(kap32[:, idx]), np.ascontiguousarray(u32[:, idx])
        for _ in range(steps):
            psi = pf.step(kb, kb, ub)
        centre = R + B * (R + B * R)
        ref.append(psi[:, centre])
        got.append(out[:, x + 256 * (y + 256 * z)])
    got, ref = np.array(got).T, np.array(ref).T
    assert np.max(np.abs(ref)) > 0
    assert np.all(rel_err_per_component(got, ref) < 2e-5), rel_err_per_component(got, ref)


def test_paper_form_checkpoint_round_trip():
    import torch
    dim, n, alpha, m, dt = 2, (40, 24), 0.5, 8, 5e-3
    mu, w = soe.soe_nnls(1 - alpha, dt, 1.0, m)
    _, kap = inputs.spectral_velocity(dim, n, 2, seed=61)
    s = make_solver(dim, n, alpha, 1.1, 0.3, dt, mu, w, 0)
    s.set_state(torch.as_tensor(inputs.random_stress(dim, n, 62), device=s.device))
    kt = torch.as_tensor(0.5 * np.asarray(kap), device=s.device).contiguous()
    for _ in range(4):
        s.step(kt, kt)
    ck = s.new_checkpoint()
    s.save(ck)
    psi_saved = s.stress().clone()
    for _ in range(5):
        s.step(kt, kt)
    a = s.stress().clone()
    s.load(ck)
    assert torch.equal(s.stress(), psi_saved)
    assert s.step_index() == 4
    for _ in range(5):
        s.step(kt, kt)
    assert torch.equal(s.stress(), a)
    s.close()


def test_paper_form_refusals():
    import torch
    from paper_2411_17294_gb300 import tfs
    n, dt = (8, 8), 1e-2
    mu, w = soe.soe_nnls(0.5, dt, 1.0, 4)
    with pytest.raises(tfs.TfsError):
        tfs.Solver(2, n, 1.0, 1.0, 0.5, dt, m=0, precision=tfs.TFS_FP64, transport=False, form="paper")
    # explicit transport and the SDIRK2 start together are refused at the first step
    for tr in (True,):
        s = tfs.Solver(2, n, 0.5, 1.0, 0.5, dt, m=4, precision=tfs.TFS_FP64, mu=mu, w=w, form="paper",
                       transport=tr, start="sdirk2")
        s.set_state(None)
        k = torch.zeros((4, 64), dtype=torch.float64, device=s.device)
        u = torch.zeros((2, 64), dtype=torch.float64, device=s.device)
        with pytest.raises(tfs.TfsError):
            s.step(k, k, u)
        assert s.step_index() == 0
        s.close()


TRANSPORT_CASES = [
    # dim, n, alpha, m, stencil, eps   (n0 % 32 == 0 and n1 % 8 == 0: the tiled pre-pass)
    (2, (37, 29), 0.5, 8, 0, 0.0),
    (2, (64, 16), 0.4, 8, 1, 0.005),   # inside this variable's explicit diffusion bound
    (3, (9, 7, 5), 0.6, 6, 1, 0.01),
    (3, (32, 8, 5), 0.3, 6, 0, 0.0),
]


@pytest.mark.parametrize("dim,n,alpha,m,stencil,eps", TRANSPORT_CASES)
@pytest.mark.parametrize("precision", [0, 1])
def test_paper_form_with_transport_matches_oracle(dim, n, alpha, m, stencil, eps, precision):
    import torch
    from paper_2411_17294_gb300 import tfs
    steps, dt, Wi, beta = 6, 4e-3, 1.3, 0.4
    N = int(np.prod(n))
    mu, w = soe.soe_nnls(1 - alpha, dt, 50 * dt, m)
    K = kap_sequence(dim, n, 91, True)
    u, _ = inputs.spectral_velocity(dim, n, 2, seed=92)
    u = 0.3 * np.asarray(u)
    P0 = inputs.random_stress(dim, n, 93)
    if precision != 0:
        cast = lambda a: np.asarray(a, np.float32).astype(np.float64)
        K0 = K
        K = lambda k: cast(K0(k))
        P0, u = cast(P0), cast(u)
    pf = PaperForm(dim, N, Wi, beta, dt, mu, w, Phi0=P0, grid=n, eps=eps, stencil=stencil)
    s = tfs.Solver(dim, n, alpha, Wi, beta, dt, m=m, precision=precision, mu=mu, w=w, transport=True,
                   form="paper", stencil=stencil, eps=eps)
    s.set_state(torch.as_tensor(P0, dtype=s.dtype, device=s.device))
    ut = torch.as_tensor(u, dtype=s.dtype, device=s.device).contiguous()
    for k in range(steps):
        kn, km = K(k), K(k - 1) if k > 0 else K(0)
        ref = pf.step(kn, km, u)
        s.step(torch.as_tensor(kn, dtype=s.dtype, device=s.device).contiguous(),
               torch.as_tensor(km, dtype=s.dtype, device=s.device).contiguous() if k > 0 else None, ut)
    got = s.stress().double().cpu().numpy()
    assert not (s.status() & (tfs.TFS_FLAG_NONFINITE | tfs.TFS_FLAG_SINGULAR | tfs.TFS_FLAG_TIMEOUT))
    s.close()
    # the transport changes the result, and the library follows the oracle's
    pb = PaperForm(dim, N, Wi, beta, dt, mu, w, Phi0=P0)
    for k in range(steps):
        other = pb.step(K(k), K(k - 1) if k > 0 else K(0))
    assert np.max(np.abs(ref - other)) > 1e-3 * np.max(np.abs(ref))
    assert np.all(rel_err_per_component(got, ref) < (1e-11 if precision == 0 else 2e-5))


IMPLICIT_CASES = [
    # dim, n, alpha, m, stencil, eps, dt max|u| / h
    (2, (16, 12), 0.5, 8, 0, 0.0, 0.5),
    (2, (12, 10), 0.3, 6, 1, 0.02, 0.08),   # xi ~ 100 at alpha = 0.3: dt xi |u|/h ~ 5x the diagonal
    (3, (6, 5, 4), 0.6, 6, 0, 0.01, 0.4),
]


@pytest.mark.parametrize("dim,n,alpha,m,stencil,eps,speed", IMPLICIT_CASES)
@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("start", ["bdf2", "sdirk2"])
def test_paper_form_implicit_transport_matches_oracle(dim, n, alpha, m, stencil, eps, speed, precision, start):
    import torch
    from paper_2411_17294_gb300 import tfs
    steps, dt, Wi, beta = 6, 2e-3, 1.3, 0.4
    N = int(np.prod(n))
    mu, w = soe.soe_nnls(1 - alpha, dt, 50 * dt, m)
    K = kap_sequence(dim, n, 95, True)
    u, _ = inputs.spectral_velocity(dim, n, 2, seed=96)
    h = 2 * np.pi / min(n)
    u = np.asarray(u) * (speed * h / dt / np.abs(np.asarray(u)).max())   # dt max|u| / h = speed
    # (the explicit transport of the stress variable is stable only to dt max|u| / h of about 0.01 here)
    P0 = inputs.random_stress(dim, n, 97)
    if precision != 0:
        cast = lambda a: np.asarray(a, np.float32).astype(np.float64)
        K0 = K
        K = lambda k: cast(K0(k))
        P0, u = cast(P0), cast(u)
    pf = PaperForm(dim, N, Wi, beta, dt, mu, w, Phi0=P0, grid=n, eps=eps, stencil=stencil, implicit=True,
                   start=start)
    s = tfs.Solver(dim, n, alpha, Wi, beta, dt, m=m, precision=precision, mu=mu, w=w, transport="implicit",
                   form="paper", stencil=stencil, eps=eps, start=start)
    s.set_state(torch.as_tensor(P0, dtype=s.dtype, device=s.device))
    s.set_krylov(maxit=2000)
    ut = torch.as_tensor(u, dtype=s.dtype, device=s.device).contiguous()
    for k in range(steps):
        kn, km = K(k), K(k - 1) if k > 0 else K(0)
        ref = pf.step(kn, km, u)
        s.step(torch.as_tensor(kn, dtype=s.dtype, device=s.device).contiguous(),
               torch.as_tensor(km, dtype=s.dtype, device=s.device).contiguous() if k > 0 else None, ut)
        it, rr = s.last_solve()
        assert 0 < it < 2000
    got = s.stress().double().cpu().numpy()
    assert not (s.status() & (tfs.TFS_FLAG_NONFINITE | tfs.TFS_FLAG_NOCONV | tfs.TFS_FLAG_TIMEOUT))
    s.close()
    assert np.max(np.abs(ref)) > 1e-2
    assert np.all(rel_err_per_component(got, ref) < (1e-10 if precision == 0 else 2e-5)), \
        rel_err_per_component(got, ref)
