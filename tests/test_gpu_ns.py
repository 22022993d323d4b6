"""The Navier-Stokes projection step (tfs_ns_*, Section 4.1) through the C ABI
against the NumPy oracle (oracle/ns.py), and the coupled run -- velocity step,
then the stress step with that velocity -- against the coupled oracle.

Tolerances (normwise per component): the NS step alone 1e-12 (both sides FP64;
the transforms differ only in rounding order); the coupled run 1e-10 in FP64
and 2e-5 with FP32 storage (the fields exchanged between the two steps are
rounded to float every step).
"""
import math

import numpy as np
import pytest

from helpers import ensure_lib, rel_err_per_component, stable_velocity
from oracle import orc, soe
from oracle.ns import NSOracle
from paper_2411_17294_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_lib()


def test_ns_step_matches_oracle():
    import torch
    from paper_2411_17294_gb300 import tfs
    n, L, beta, Re, dt = (64, 32), (2 * math.pi, 4 * math.pi), 0.6, 20.0, 5e-3
    rng = np.random.default_rng(61)
    u0 = rng.normal(size=(2, n[0] * n[1]))
    sigmas = [0.2 * rng.normal(size=(3, n[0] * n[1])) for _ in range(6)]
    o = NSOracle(n, L, beta, Re, dt)
    o.set_state(u0)
    s = tfs.NSSolver(n, L, beta, Re, dt, precision=tfs.TFS_FP64)
    s.set_state(u0)
    for sg in sigmas:
        u_ref, k_ref = o.step(sg)
        u, k = s.step(torch.as_tensor(sg, device="cuda"))
    s.close()
    assert np.all(rel_err_per_component(u.cpu().numpy(), u_ref) < 1e-12)
    assert np.all(rel_err_per_component(k.cpu().numpy(), k_ref) < 1e-12)


def test_taylor_green_second_order_on_gpu():
    from paper_2411_17294_gb300 import tfs
    n, beta, Re, T = 32, 0.5, 10.0, 1.0
    nu = beta / Re
    x = np.arange(n) * 2 * math.pi / n
    X, Y = np.meshgrid(x, x)

    def tg(t):
        return np.stack([np.sin(X) * np.cos(Y), -np.cos(X) * np.sin(Y)]).reshape(2, -1) * math.exp(-2 * nu * t)

    errs = []
    for steps in (20, 40):
        dt = T / steps
        s = tfs.NSSolver((n, n), (2 * math.pi, 2 * math.pi), beta, Re, dt)
        s.set_state(tg(0.0), tg(-dt))
        for _ in range(steps):
            u, _ = s.step()
        errs.append(float(np.max(np.abs(u.cpu().numpy() - tg(T)))))
        s.close()
    assert errs[0] < 1e-6 and 3.8 < errs[0] / errs[1] < 4.2, errs


@pytest.mark.parametrize("precision", [0, 1])
def test_coupled_velocity_and_stress_match_oracle(precision):
    # The paper's order within a step: the velocity from the stress at t_n,
    # then the stress with that velocity (kappa* = kappa^{n+1}), explicit
    # transport, alpha = 0.5, m = 8, a velocity inside the transport's limit.
    import torch
    from paper_2411_17294_gb300 import tfs
    n, L, beta, Re, dt, steps = (32, 32), (2 * math.pi, 2 * math.pi), 0.5, 5.0, 2e-3, 12
    alpha, Wi, m = 0.5, 0.8, 8
    mu, w = soe.soe_nnls(alpha, dt, steps * dt, m)
    case = dict(dim=2, n=n, alpha=alpha, dt=dt, mu=mu, w=w)
    u0, _ = inputs.spectral_velocity(2, n, 4, seed=62)
    u0 = 0.5 * np.asarray(stable_velocity(case, u0, target=0.3))
    sig0 = 0.1 * inputs.random_stress(2, n, 63)
    dtype = torch.float64 if precision == 0 else torch.float32
    if precision == 1:
        u0, sig0 = (np.asarray(a, np.float32).astype(np.float64) for a in (u0, sig0))
    # oracle
    ons = NSOracle(n, L, beta, Re, dt)
    ons.set_state(u0)
    ost = orc.Oracle(orc.Problem(dim=2, n=n, alpha=alpha, Wi=Wi, beta=beta, dt=dt, mu=mu, w=w, transport=True,
                                 L=L), sig0)
    for _ in range(steps):
        u, kap = ons.step(ost.sig_n)
        ost.step(kap, kap, u)
    ref_u, ref_s = u, ost.sig_n
    # library
    ns = tfs.NSSolver(n, L, beta, Re, dt, precision=precision)
    st = tfs.Solver(2, n, alpha, Wi, beta, dt, m=m, precision=precision, mu=mu, w=w, transport=True, L=L)
    ns.set_state(u0)
    st.set_state(torch.as_tensor(sig0, dtype=dtype, device="cuda"))
    for _ in range(steps):
        u_t, k_t = ns.step(st.stress())
        st.step(k_t, k_t, u_t)
    got_u, got_s = u_t.double().cpu().numpy(), st.stress().double().cpu().numpy()
    flags = st.status()
    ns.close()
    st.close()
    tol = 1e-10 if precision == 0 else 2e-5
    assert flags == 0
    assert np.max(np.abs(ref_s)) > 1e-3 and np.max(np.abs(ref_u)) > 1e-3
    assert np.all(rel_err_per_component(got_u, ref_u) < tol)
    assert np.all(rel_err_per_component(got_s, ref_s) < tol)


def test_coupled_1024_matches_oracle():
    # The coupled step at the 2D 1024^2 size of the benchmark record (alpha =
    # 0.5, m = 32, Wi = 2, beta = 0.9, Re = 100, dt = 5e-4, FP32 storage,
    # spectral velocity at 0.3 of the explicit transport's limit), six steps,
    # against the coupled oracle over the whole field.
    import torch
    from paper_2411_17294_gb300 import soe as psoe
    from paper_2411_17294_gb300 import tfs
    n, L, dt, steps = (1024, 1024), (2 * math.pi, 2 * math.pi), 5e-4, 6
    alpha, Wi, beta, Re, m = 0.5, 2.0, 0.9, 100.0, 32
    mu, w = psoe.build(alpha, dt, 200 * dt, m)
    st = tfs.Solver(2, n, alpha, Wi, beta, dt, m=m, precision=tfs.TFS_FP32, mu=mu, w=w, transport=True, L=L)
    U = st.transport_limit()
    u0, _ = inputs.spectral_velocity(2, n, 32, 2)
    u0 = np.asarray(u0) * (0.3 * U / np.max(np.abs(u0)))
    u0 = np.asarray(u0, np.float32).astype(np.float64)
    ns = tfs.NSSolver(n, L, beta, Re, dt, precision=tfs.TFS_FP32)
    ns.set_state(u0)
    st.set_state(None)
    for _ in range(steps):
        u_t, k_t = ns.step(st.stress())
        st.step(k_t, k_t, u_t)
    got_u, got_s, flags = u_t.double().cpu().numpy(), st.stress().double().cpu().numpy(), st.status()
    ns.close()
    st.close()
    ons = NSOracle(n, L, beta, Re, dt)
    ons.set_state(u0)
    ost = orc.Oracle(orc.Problem(dim=2, n=n, alpha=alpha, Wi=Wi, beta=beta, dt=dt, mu=mu, w=w, transport=True,
                                 L=L), None)
    for _ in range(steps):
        u, kap = ons.step(ost.sig_n)
        ost.step(kap, kap, u)
    assert flags == 0
    assert np.all(rel_err_per_component(got_u, u) < 2e-5)
    assert np.all(rel_err_per_component(got_s, ost.sig_n) < 2e-5)
