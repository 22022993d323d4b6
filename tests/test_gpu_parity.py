"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances (per stress component, max |GPU - oracle| / max |oracle|):
  FP64 mode   1e-11   (both sides FP64; differences are summation order and FMA
                       contraction, ~1e-16 per operation, grown over the steps)
  FP32 modes  2e-5    (float storage of stress and modes: ~6e-8 rounding per
                       step and value, accumulated over up to a few hundred steps)
"""
import math

import numpy as np
import pytest

from helpers import courant_fraction, ensure_lib, rel_err_per_component, run_gpu, run_oracle, stable_velocity
from oracle import soe
from paper_2411_17294_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL64 = 1e-11
TOL32 = 2e-5


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_lib()


def case_dict(dim, n, alpha, Wi, beta, dt, m, T, transport, eps=0.0, stencil=0, L=None):
    c = dict(dim=dim, n=n, alpha=alpha, Wi=Wi, beta=beta, dt=dt, transport=transport, eps=eps, stencil=stencil, L=L)
    if alpha < 1:
        # the NNLS builder reaches exactly m positive terms up to m = 48; beyond,
        # a trapezoidal table (positive, less accurate) serves parity just as well
        c["mu"], c["w"] = soe.soe_nnls(alpha, dt, T, m) if m <= 48 else soe.soe_expquad(alpha, dt, T, m)
    return c


def taylor_green_case():
    # 2D periodic 64 x 64, FP64, alpha = 0.5, Wi = 1, beta = 0.5, m = 16 on [1e-3, 1],
    # dt = 1e-3, 100 steps, Taylor-Green gradient plus N(0, 1e-3) noise, sigma0 = 0
    c = case_dict(2, (64, 64), 0.5, 1.0, 0.5, 1e-3, 16, 1.0, transport=True)
    u, kap = inputs.taylor_green((64, 64), seed=1)
    assert courant_fraction(c, u) < 1.0   # inside the explicit-transport stability region as given
    return c, u, kap


def test_taylor_green_64_fp64_full_grid():
    c, u, kap = taylor_green_case()
    ref = run_oracle(c, None, kap, u, 100)
    got = run_gpu(c, None, kap, u, 100, precision=0)
    assert np.max(np.abs(ref)) > 1e-3
    assert np.all(rel_err_per_component(got, ref) < TOL64)


@pytest.mark.parametrize("precision", [1, 2])
def test_taylor_green_64_fp32(precision):
    c, u, kap = taylor_green_case()
    ref = run_oracle(c, None, kap, u, 100)
    got = run_gpu(c, None, kap, u, 100, precision=precision)
    assert np.all(rel_err_per_component(got, ref) < TOL32)


RAGGED = [
    # dim, n, alpha, m, transport, eps, stencil
    (3, (7, 5, 9), 0.6, 8, True, 0.0, 0),
    (3, (33, 3, 2), 0.3, 12, True, 0.01, 0),
    (2, (37, 29), 0.8, 20, True, 0.02, 1),
    (2, (1, 1), 0.5, 5, False, 0.0, 0),
    (3, (1, 2, 1), 0.7, 3, True, 0.0, 0),
    (2, (2, 45), 1.0, 0, True, 0.01, 0),
    (3, (6, 6, 6), 1.0, 0, False, 0.0, 0),
    (2, (16, 16), 0.45, 64, True, 0.0, 0),
    (3, (4, 4, 4), 0.55, 48, True, 0.0, 0),
    (2, (10, 7), 0.5, 1, True, 0.0, 1),
    # sizes with n0 % 32 == 0 and n1 % 8 == 0 take the tiled transport pre-pass
    (3, (32, 16, 10), 0.6, 8, True, 0.01, 0),
    (3, (64, 8, 3), 0.4, 6, True, 0.0, 1),
    (3, (32, 8, 1), 0.5, 4, True, 0.0, 1),
    (2, (64, 24), 0.5, 8, True, 0.02, 0),
]


@pytest.mark.parametrize("dim,n,alpha,m,transport,eps,stencil", RAGGED)
@pytest.mark.parametrize("precision", [0, 1])
def test_ragged_and_degenerate_grids(dim, n, alpha, m, transport, eps, stencil, precision):
    steps = 15
    dt = 2e-3
    c = case_dict(dim, n, alpha, 1.3, 0.4, dt, max(m, 1), steps * dt, transport, eps, stencil)
    u, kap = inputs.spectral_velocity(dim, n, max(1, min(n) // 2), seed=4) if min(n) > 1 else (None, None)
    N = int(np.prod(n))
    rng = np.random.default_rng(3)
    if kap is None:
        kap = rng.normal(size=(dim * dim, N))
        u = rng.normal(size=(dim, N))
    u = stable_velocity(c, u)
    sigma0 = inputs.random_stress(dim, n, seed=8)
    ref = run_oracle(c, sigma0, kap, u if transport else None, steps)
    got = run_gpu(c, sigma0, kap, u if transport else None, steps, precision=precision)
    tol = TOL64 if precision == 0 else TOL32
    assert np.all(rel_err_per_component(got, ref) < tol)


@pytest.mark.parametrize("precision", [0, 1])
def test_time_dependent_gradient_and_first_step(precision):
    # kappa^n changes every step (extrapolation 2 kappa^n - kappa^{n-1} is exercised);
    # the first call passes no kappa^{n-1}
    dim, n, steps, dt = 3, (9, 8, 7), 25, 1e-3
    c = case_dict(dim, n, 0.4, 0.9, 0.2, dt, 10, steps * dt, transport=True, eps=0.01)
    u, k0 = inputs.spectral_velocity(dim, n, 3, seed=5)
    u = stable_velocity(c, u)

    def kap(nn):
        return k0 * (1.0 + 0.3 * math.sin(0.7 * nn)) + 0.1 * nn / steps

    ref = run_oracle(c, None, kap, u, steps)
    got = run_gpu(c, None, kap, u, steps, precision=precision)
    assert np.all(rel_err_per_component(got, ref) < (TOL64 if precision == 0 else TOL32))


def test_checkpoint_roundtrip_bitwise():
    import torch
    dim, n, dt = 2, (20, 18), 1e-3
    c = case_dict(dim, n, 0.5, 1.0, 0.5, dt, 8, 0.05, transport=True)
    u, kap = inputs.spectral_velocity(dim, n, 5, seed=6)
    out, s = run_gpu(c, inputs.random_stress(dim, n, 2), kap, u, 10, precision=1, return_solver=True)
    buf = s.new_checkpoint()
    s.save(buf)
    kt = torch.as_tensor(kap, dtype=s.dtype, device=s.device)
    ut = torch.as_tensor(u, dtype=s.dtype, device=s.device)
    for _ in range(5):
        s.step(kt, kt, ut)
    a = s.stress().cpu().numpy()
    s.load(buf)
    assert s.step_index() == 10
    for _ in range(5):
        s.step(kt, kt, ut)
    b = s.stress().cpu().numpy()
    assert np.array_equal(a, b)
    s.close()


def test_status_flags_nonfinite():
    import torch
    from paper_2411_17294_gb300 import tfs
    dim, n, dt = 2, (8, 8), 1e-3
    c = case_dict(dim, n, 0.5, 1.0, 0.5, dt, 4, 0.01, transport=False)
    s = tfs.Solver(dim, n, 0.5, 1.0, 0.5, dt, m=4, precision=0, mu=c["mu"], w=c["w"], transport=False)
    s.set_state(None)
    kap = torch.zeros((4, 64), dtype=torch.float64, device=s.device)
    s.step(kap, kap)
    assert s.status() == 0
    kap[1, 5] = float("nan")
    s.step(kap, kap)
    assert s.status() & tfs.TFS_FLAG_NONFINITE
    s.set_state(None)
    assert s.status() == 0
    s.close()


def test_homogeneous_fields_uniform_on_gpu():
    # P6 on the device: uniform kappa and constant u give the same value everywhere
    dim, n, dt = 3, (16, 8, 8), 2e-4
    c = case_dict(dim, n, 0.6, 2.0, 0.9, dt, 32, 0.04, transport=True)
    km = np.array([[0.2, 1.0, 0.0], [0.3, -0.1, 0.4], [0.0, 0.2, -0.1]])
    kap = inputs.uniform_kappa(3, n, km)
    u = inputs.uniform_velocity(3, n, [0.3, -1.2, 0.5])
    for precision in (0, 1):
        got = run_gpu(c, None, kap, u, 20, precision=precision)
        assert np.all(got == got[:, :1])


def _packed(dim):
    return [(0, 0), (0, 1), (1, 1)] if dim == 2 else [(0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1)]


def point_system_stats(dim, kap, a, dt):
    """Condition number and row diagonal dominance of every point system
    (a I - dt L(kappa)) in packed components, L(kappa) s = kappa s + s kappa^T;
    used only to show which regime the case below covers."""
    P = _packed(dim)
    nc, N = len(P), kap.shape[1]
    K = kap.T.reshape(N, dim, dim)
    M = np.zeros((N, nc, nc))
    for k, (i, j) in enumerate(P):
        S = np.zeros((dim, dim))
        S[i, j] = S[j, i] = 1.0
        L = K @ S + S @ np.swapaxes(K, 1, 2)
        for r, (p, q) in enumerate(P):
            M[:, r, k] = -dt * L[:, p, q]
        M[:, k, k] += a
    cond = np.linalg.cond(M)
    dominant = np.all(2 * np.abs(np.einsum("nii->ni", M)) > np.sum(np.abs(M), axis=2), axis=1)
    return cond, dominant


@pytest.mark.parametrize("dim,n,strength", [(2, (48, 40), 2.0), (3, (20, 12, 9), 1.0)])
@pytest.mark.parametrize("precision", [0, 1])
def test_ill_conditioned_point_solves(dim, n, strength, precision):
    # High Weissenberg number and a strong velocity gradient: dt |kappa| is
    # comparable to eta + dt/Wi, so most point systems are far from diagonally
    # dominant (the FP32 solve takes its pivoting path) and the worst reach
    # condition numbers of 1e3..1e5.  One step from a nonzero initial stress
    # (the mode history is still zero), with inputs exactly representable in
    # FP32 on both sides, isolates the point solve: the GPU result must match
    # the FP64 oracle at EVERY point (not only normwise); a plain FP32 LU
    # solve of the same systems misses that by about 5x (1e-4 per point).
    alpha, Wi, beta, dt, m = 0.5, 50.0, 0.3, 1e-3, 16
    c = case_dict(dim, n, alpha, Wi, beta, dt, m, 4 * dt, transport=False)
    mu, w = np.asarray(c["mu"]), np.asarray(c["w"])
    a = 1.5 * np.sum(w * dt / (1.5 + mu * dt)) + dt / Wi
    _, kap = inputs.spectral_velocity(dim, n, 3, seed=21)
    kap = (kap * (strength * a / (dt * np.max(np.abs(kap))))).astype(np.float32).astype(np.float64)
    cond, dominant = point_system_stats(dim, kap, a, dt)
    assert 1e3 < np.max(cond) < 1e5 and np.mean(~dominant) > 0.5
    sigma0 = inputs.random_stress(dim, n, seed=22).astype(np.float32).astype(np.float64)
    ref = run_oracle(c, sigma0, kap, None, 1)
    got = run_gpu(c, sigma0, kap, None, 1, precision=precision)
    per_point = np.max(np.abs(got - ref), axis=0) / np.max(np.abs(ref), axis=0)
    assert np.max(per_point) < (TOL64 if precision == 0 else TOL32), (np.max(per_point), np.max(cond))


@pytest.mark.parametrize("precision", [0, 1])
def test_alpha_near_one_with_completed_table(precision):
    # alpha = 0.999 with a mass-completed table (the kernel's mass sits almost
    # entirely in the completing Dirac term, the fitted tail carries ~1e-3 of
    # it): the library matches the oracle, and both lie within O(1 - alpha) of
    # the alpha = 1 (Oldroyd-B, BDF2) path, the limit the oracle pins
    dim, n, Wi, beta, dt, steps, m = 2, (48, 40), 1.1, 0.4, 2e-3, 40, 32
    alpha = 0.999
    c = dict(dim=dim, n=n, alpha=alpha, Wi=Wi, beta=beta, dt=dt, transport=True, eps=0.01, stencil=0)
    c["mu"], c["w"] = soe.soe_build(alpha, dt, steps * dt, m)
    u, kap = inputs.spectral_velocity(dim, n, 12, seed=5)
    u = stable_velocity(c, u)
    sigma0 = inputs.random_stress(dim, n, seed=6)
    ref = run_oracle(c, sigma0, kap, u, steps)
    got = run_gpu(c, sigma0, kap, u, steps, precision=precision)
    tol = TOL64 if precision == 0 else TOL32
    assert np.all(rel_err_per_component(got, ref) < tol)
    c1 = dict(c, alpha=1.0)
    c1.pop("mu"), c1.pop("w")
    got1 = run_gpu(c1, sigma0, kap, u, steps, precision=precision)
    assert np.all(rel_err_per_component(got, got1) < 10 * (1 - alpha))
