"""Parity at the workload sizes, in the launch configuration the benchmark
times, on sampled outputs the oracle computes one by one.

3D 256^3 (m = 32, FP32 + compensated sum, alpha = 0.6, Wi = 2, beta = 0.9,
dt = 2e-4, spectral velocity |k| <= 24 at unit RMS, transport on): a few steps;
the stress at a sampled point after s steps depends only on the points within
2 s grid cells (radius-2 stencil), so the oracle runs on the periodic
(4 s + 1)^3 block centred on each sample and its centre value is exact.

2D 1024^2 (m = 32, FP32 and FP64, dt = 5e-4, alpha in {0.3, 0.5, 0.8}, 1000
steps): the explicit transport is outside its stability region at these sizes,
so these cases run the pointwise law (transport off); the oracle then runs on
the sampled points alone, FP32 storage is compared with the FP64 form over the
whole field, and the zero-flow case is compared with the Mittag-Leffler closed
form.
"""
import numpy as np
import pytest

from helpers import ensure_lib, rel_err_per_component
from oracle import orc, special
from oracle import soe as osoe
from paper_2411_17294_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_lib()


def test_3d_256_bench_configuration_sampled():
    import torch
    from paper_2411_17294_gb300 import tfs
    n, m, alpha, Wi, beta, dt, steps = (256, 256, 256), 32, 0.6, 2.0, 0.9, 2e-4, 3
    mu, w = osoe.soe_nnls(alpha, dt, 200 * dt, m)
    dev = torch.device("cuda", 0)
    u, kap = inputs.spectral_velocity(3, n, 24, 3, device=dev)
    s = tfs.Solver(3, n, alpha, Wi, beta, dt, m=m, precision=tfs.TFS_FP32, mu=mu, w=w, transport=True)
    kt = torch.as_tensor(kap, dtype=torch.float32, device=dev).contiguous()
    k2 = kt.clone()
    ut = torch.as_tensor(u, dtype=torch.float32, device=dev).contiguous()
    s.set_state(None)
    for _ in range(steps):
        s.step(kt, k2, ut)
    out = s.stress().cpu().numpy().astype(np.float64)
    s.close()
    # the oracle sees the same (float-rounded) inputs
    kap32 = kt.cpu().numpy().astype(np.float64)
    u32 = ut.cpu().numpy().astype(np.float64)
    rng = np.random.default_rng(2024)
    R = 2 * steps
    B = 2 * R + 1
    samples = [tuple(int(v) for v in rng.integers(0, 256, size=3)) for _ in range(12)] + [(0, 0, 0), (255, 255, 255)]
    got, ref = [], []
    L = 2 * np.pi
    for (x, y, z) in samples:
        xs = (np.arange(x - R, x + R + 1) % 256)
        ys = (np.arange(y - R, y + R + 1) % 256)
        zs = (np.arange(z - R, z + R + 1) % 256)
        idx = (xs[None, None, :] + 256 * (ys[None, :, None] + 256 * zs[:, None, None])).ravel()
        prob = orc.Problem(dim=3, n=(B, B, B), alpha=alpha, Wi=Wi, beta=beta, dt=dt, mu=mu, w=w, transport=True,
                           L=(L * B / 256,) * 3)
        o = orc.Oracle(prob)
        kb = np.ascontiguousarray(kap32[:, idx])
        ub = np.ascontiguousarray(u32[:, idx])
        o.run(steps, kb, ub)
        centre = R + B * (R + B * R)
        ref.append(o.sig_n[:, centre])
        got.append(out[:, x + 256 * (y + 256 * z)])
    got = np.array(got).T
    ref = np.array(ref).T
    assert np.max(np.abs(ref)) > 0
    assert np.all(rel_err_per_component(got, ref) < 2e-5)


@pytest.mark.parametrize("alpha", [0.3, 0.5, 0.8])
def test_2d_1024_pointwise_sampled(alpha):
    import torch
    from paper_2411_17294_gb300 import tfs
    n, m, Wi, beta, dt, steps = (1024, 1024), 32, 1.0, 0.5, 5e-4, 1000
    mu, w = osoe.soe_nnls(alpha, dt, 1000 * dt, m)
    dev = torch.device("cuda", 0)
    u, kap = inputs.spectral_velocity(2, n, 32, 2, device=dev)
    kap = 0.05 * kap      # keep the pointwise stress moderate over the run
    sig0 = inputs.random_stress(2, n, 5, amplitude=0.5)
    outs = {}
    for prec in (tfs.TFS_FP32, tfs.TFS_FP64):
        s = tfs.Solver(2, n, alpha, Wi, beta, dt, m=m, precision=prec, mu=mu, w=w, transport=False)
        kt = torch.as_tensor(kap, dtype=s.dtype, device=dev).contiguous()
        s.set_state(torch.as_tensor(sig0, dtype=s.dtype, device=dev))
        for _ in range(steps):
            s.step(kt, kt, None)
        outs[prec] = s.stress().cpu().numpy().astype(np.float64)
        s.close()
    rng = np.random.default_rng(7)
    pts = np.unique(np.concatenate([rng.integers(0, 1024 * 1024, size=64), [0, 1024 * 1024 - 1]]))
    kap64 = torch.as_tensor(kap, dtype=torch.float64).cpu().numpy()[:, pts]
    kap32 = kap64.astype(np.float32).astype(np.float64)
    sig032 = sig0.astype(np.float32).astype(np.float64)[:, pts]
    ref32 = orc.forward(orc.Problem(dim=2, n=(len(pts), 1), alpha=alpha, Wi=Wi, beta=beta, dt=dt, mu=mu, w=w),
                        sig032, np.ascontiguousarray(kap32), None, steps)
    ref64 = orc.forward(orc.Problem(dim=2, n=(len(pts), 1), alpha=alpha, Wi=Wi, beta=beta, dt=dt, mu=mu, w=w),
                        np.ascontiguousarray(sig0[:, pts]), np.ascontiguousarray(kap64), None, steps)
    assert np.all(rel_err_per_component(outs[tfs.TFS_FP32][:, pts], ref32) < 2e-5)
    assert np.all(rel_err_per_component(outs[tfs.TFS_FP64][:, pts], ref64) < 1e-11)
    # FP32 storage against the FP64 form over the whole field (inputs rounded once)
    assert np.all(rel_err_per_component(outs[tfs.TFS_FP32], outs[tfs.TFS_FP64]) < 2e-5)


@pytest.mark.parametrize("alpha", [0.3, 0.5, 0.8])
def test_2d_1024_zero_flow_mittag_leffler(alpha):
    # Zero flow on the full 1024^2 grid, 1000 steps of 5e-4: sigma(T) = sigma0
    # E_alpha(-T^alpha/Wi) at every point, up to the scheme's error, with the
    # mass-completed SOE and the SDIRK2 start (about 1e-6 on the oracle).
    import torch
    from paper_2411_17294_gb300 import tfs
    n, m, Wi, dt, steps = (1024, 1024), 32, 1.0, 5e-4, 1000
    T = dt * steps
    mu, w = osoe.soe_build(alpha, dt, T, m)
    exact = special.mittag_leffler(alpha, -T ** alpha / Wi)
    dev = torch.device("cuda", 0)
    sig0 = inputs.random_stress(2, n, 9, amplitude=1.0)
    for prec, tol in ((tfs.TFS_FP64, 5e-6), (tfs.TFS_FP32, 3e-5)):
        s = tfs.Solver(2, n, alpha, Wi, 0.5, dt, m=m, precision=prec, mu=mu, w=w, transport=False, start="sdirk2")
        s0 = torch.as_tensor(sig0, dtype=s.dtype, device=dev)
        k = torch.zeros((4, n[0] * n[1]), dtype=s.dtype, device=dev)
        s.set_state(s0)
        for _ in range(steps):
            s.step(k, k, None)
        out = s.stress().double()
        s.close()
        err = (out - exact * s0.double()).abs().amax(dim=1) / (exact * s0.double()).abs().amax(dim=1)
        assert float(err.max()) < tol, (prec, err)


W3D256 = dict(n=(256, 256, 256), m=32, alpha=0.6, Wi=2.0, beta=0.9, dt=2e-4, steps=200)


def _w3d256_fields(dev, scale=1.0):
    import torch
    u, kap = inputs.spectral_velocity(3, W3D256["n"], 24, 3, device=dev)
    u = torch.as_tensor(u, dtype=torch.float64, device=dev) * scale
    kap = torch.as_tensor(kap, dtype=torch.float64, device=dev) * scale
    return u, kap


def _courant_fraction_gpu(s, u, n):
    # max_p sum_a |u_a(p)| / h_a over U sum_a 1/h_a, U = tfs_transport_limit
    U = s.transport_limit()
    return float(u.abs().sum(dim=0).max()) / (3 * U)


def test_3d_256_workload_as_stated_200_steps_explicit():
    # The 3D workload as stated (spectral velocity at unit RMS, 200 steps of
    # 2e-4, explicit transport) uses about 2.5 times the explicit transport's
    # velocity limit: the library latches TFS_FLAG_COURANT on the first step.
    # The run is reported (max |sigma|, flags) but, being outside the scheme's
    # stability region, it has no reference to match; the two tests below check
    # this workload inside the stability region (pointwise law, and velocity
    # scaled to 0.9 of the limit).
    import torch
    from paper_2411_17294_gb300 import soe as psoe
    from paper_2411_17294_gb300 import tfs
    C = W3D256
    dev = torch.device("cuda", 0)
    mu, w = psoe.build(C["alpha"], C["dt"], C["steps"] * C["dt"], C["m"])
    u, kap = _w3d256_fields(dev)
    s = tfs.Solver(3, C["n"], C["alpha"], C["Wi"], C["beta"], C["dt"], m=C["m"], precision=tfs.TFS_FP32, mu=mu,
                   w=w, transport=True)
    cf = _courant_fraction_gpu(s, u, C["n"])
    kt = kap.float().contiguous()
    k2 = kt.clone()
    ut = u.float().contiguous()
    del u, kap
    s.set_state(None)
    maxs = []
    for k in range(C["steps"]):
        s.step(kt, k2, ut)
        if (k + 1) % 50 == 0:
            maxs.append(float(s.stress().abs().max()))
    flags = s.status()
    s.close()
    print(f"3D 256^3 m=32 workload as stated: Courant fraction {cf:.3f}, max |sigma| after 50/100/150/200 steps {maxs}, "
          f"flags {flags}")
    assert cf > 1.0
    assert flags & tfs.TFS_FLAG_COURANT
    assert not (flags & tfs.TFS_FLAG_TIMEOUT)


def test_3d_256_200_steps_pointwise_sampled():
    # The 3D 256^3 workload's grid, parameters and gradient field for the full 200 steps,
    # with the pointwise law (transport off): every point is independent, so
    # the oracle on the sampled points alone is exact; FP32 storage + the
    # compensated sum against the FP64 oracle fed the FP32-rounded gradient.
    import torch
    from paper_2411_17294_gb300 import tfs
    C = W3D256
    dev = torch.device("cuda", 0)
    mu, w = osoe.soe_build(C["alpha"], C["dt"], C["steps"] * C["dt"], C["m"])
    _, kap = _w3d256_fields(dev)
    s = tfs.Solver(3, C["n"], C["alpha"], C["Wi"], C["beta"], C["dt"], m=C["m"], precision=tfs.TFS_FP32, mu=mu,
                   w=w, transport=False)
    kt = kap.float().contiguous()
    del kap
    s.set_state(None)
    for _ in range(C["steps"]):
        s.step(kt, kt, None)
    out = s.stress()
    flags = s.status()
    s.close()
    assert not (flags & (tfs.TFS_FLAG_NONFINITE | tfs.TFS_FLAG_TIMEOUT))
    N = 256 ** 3
    rng = np.random.default_rng(31)
    pts = np.unique(np.concatenate([rng.integers(0, N, size=96), [0, N - 1]]))
    pts_t = torch.as_tensor(pts, device=dev)
    got = out[:, pts_t].double().cpu().numpy()
    kap_s = kt[:, pts_t].double().cpu().numpy()
    ref = orc.forward(orc.Problem(dim=3, n=(len(pts), 1, 1), alpha=C["alpha"], Wi=C["Wi"], beta=C["beta"],
                                  dt=C["dt"], mu=mu, w=w), None, np.ascontiguousarray(kap_s), None, C["steps"])
    assert np.max(np.abs(ref)) > 1e-3
    assert np.all(rel_err_per_component(got, ref) < 2e-5)


def test_3d_256_200_steps_stable_velocity_fp32_against_fp64():
    # The 3D 256^3 workload with transport for the full 200 steps, the velocity (and its
    # gradient) scaled to 0.9 of the explicit transport's limit so that the
    # scheme is stable: the FP32 storage form (the benchmark's) against the
    # FP64 form over the whole 256^3 field, per component within 2e-5.  The
    # FP64 form itself matches the oracle to 1e-11 on every grid the oracle can
    # run whole (test_gpu_parity.py); the first steps of this workload match it
    # on sampled dependence blocks (test_3d_256_bench_configuration_sampled).
    import torch
    from paper_2411_17294_gb300 import soe as psoe
    from paper_2411_17294_gb300 import tfs
    C = W3D256
    dev = torch.device("cuda", 0)
    mu, w = psoe.build(C["alpha"], C["dt"], C["steps"] * C["dt"], C["m"])
    u, kap = _w3d256_fields(dev)
    outs = {}
    for prec in (tfs.TFS_FP64, tfs.TFS_FP32):
        s = tfs.Solver(3, C["n"], C["alpha"], C["Wi"], C["beta"], C["dt"], m=C["m"], precision=prec, mu=mu, w=w,
                       transport=True)
        if prec == tfs.TFS_FP64:
            scale = 0.9 / _courant_fraction_gpu(s, u, C["n"])
            u, kap = u * scale, kap * scale
            # both forms see the same (FP32-representable) inputs
            u, kap = u.float().double(), kap.float().double()
        kt = kap.to(s.dtype).contiguous()
        ut = u.to(s.dtype).contiguous()
        s.set_state(None)
        for _ in range(C["steps"]):
            s.step(kt, kt, ut)
        outs[prec] = s.stress().double()
        flags = s.status()
        s.close()
        del kt, ut
        torch.cuda.empty_cache()
        assert flags == 0, (prec, flags)
    ref = outs[tfs.TFS_FP64]
    scale = ref.abs().amax(dim=1)
    assert float(scale.min()) > 0
    err = ((outs[tfs.TFS_FP32] - ref).abs().amax(dim=1) / scale).cpu().numpy()
    print(f"3D 256^3 workload, velocity at 0.9 of the explicit limit, 200 steps: FP32 vs FP64 per component {err}")
    assert np.all(err < 2e-5)
