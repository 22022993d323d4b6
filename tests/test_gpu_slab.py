"""Slab decomposition on one GPU: the periodic domain cut along its slowest
axis (z in 3D, y in 2D) into slabs, one handle per slab, the neighbours'
boundary planes exchanged before every step (tfs_get_halo -> tfs_step_slab),
must give the whole-domain step's result exactly: every point's arithmetic
is the same, only where the stencil's neighbour values come from differs.

The grid spacing is a power of two (box length n/4 on every axis), so that a
slab's inverse spacing n_s / L_s is the whole domain's exactly.  Cases cover
the tiled transport pre-pass (n0 % 32 == 0, n1 % 8 == 0 on every slab) and
the per-point one, two and three slabs, uneven slabs, diffusion and both
stencils, FP64 and FP32 storage.
"""
import numpy as np
import pytest

from helpers import ensure_lib, stable_velocity
from oracle import soe
from paper_2411_17294_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_lib()


CASES = [
    # dim, whole grid, slab lengths along the slowest axis, eps, stencil
    (3, (64, 32, 20), (10, 10), 0.0, 0),
    (3, (64, 16, 12), (4, 5, 3), 0.02, 0),
    (3, (20, 12, 9), (5, 4), 0.0, 1),
    (2, (64, 48), (24, 24), 0.01, 0),
    (2, (37, 30), (12, 8, 10), 0.0, 0),
]


def _slice(field, dim, n, lo, hi):
    """The points of slab planes [lo, hi) of a [rows][N] field (the slowest axis
    is outermost, so a slab is one contiguous range of points)."""
    plane = n[0] * (n[1] if dim == 3 else 1)
    return np.ascontiguousarray(field[:, lo * plane:hi * plane])


@pytest.mark.parametrize("dim,n,slabs,eps,stencil", CASES)
@pytest.mark.parametrize("precision", [0, 1])
def test_slabs_equal_whole_domain(dim, n, slabs, eps, stencil, precision):
    import torch
    from paper_2411_17294_gb300 import slab, tfs
    assert sum(slabs) == n[-1]
    alpha, Wi, beta, dt, m, steps = 0.6, 1.3, 0.4, 2e-3, 8, 7
    L = [0.25 * k for k in n]
    mu, w = soe.soe_nnls(alpha, dt, steps * dt, m)
    u, kap = inputs.spectral_velocity(dim, n, max(1, min(n) // 3), seed=51)
    case = dict(dim=dim, n=n, alpha=alpha, dt=dt, mu=mu, w=w, eps=eps, stencil=stencil, L=L)
    u = stable_velocity(case, u)
    sig0 = inputs.random_stress(dim, n, 52)
    dev = torch.device("cuda", 0)
    dtype = torch.float64 if precision == 0 else torch.float32

    def solver(grid, lengths):
        return tfs.Solver(dim, grid, alpha, Wi, beta, dt, m=m, precision=precision, mu=mu, w=w, eps=eps,
                          stencil=stencil, transport=True, L=lengths)

    t = lambda a: torch.as_tensor(np.asarray(a), dtype=dtype, device=dev).contiguous()
    whole = solver(n, L)
    whole.set_state(t(sig0))
    kt, ut = t(kap), t(u)
    for _ in range(steps):
        whole.step(kt, kt, ut)
    ref = whole.stress().cpu().numpy()
    flags_whole = whole.status()
    whole.close()

    parts, k0 = [], 0
    for ns in slabs:
        grid = tuple(n[:-1]) + (ns,)
        lengths = L[:-1] + [0.25 * ns]
        s = solver(grid, lengths)
        s.set_state(t(_slice(sig0, dim, n, k0, k0 + ns)))
        parts.append((s, t(_slice(kap, dim, n, k0, k0 + ns)), t(_slice(u, dim, n, k0, k0 + ns))))
        k0 += ns
    for _ in range(steps):
        sends = []
        for s, _, _ in parts:
            lo, hi = s.halo_buffers()
            s.get_halo(lo, hi)
            sends.append((lo, hi))
        recvs = slab.exchange_local(sends)
        for (s, ks, us), (rlo, rhi) in zip(parts, recvs):
            s.step_slab(ks, ks, us, rlo, rhi)
    got = np.concatenate([s.stress().cpu().numpy() for s, _, _ in parts], axis=1)
    flags = [s.status() for s, _, _ in parts]
    for s, _, _ in parts:
        s.close()
    assert np.max(np.abs(ref)) > 0
    assert np.array_equal(got, ref)
    assert all(f == flags_whole for f in flags)


@pytest.mark.parametrize("precision", [0, 1])
def test_unaligned_velocity_and_halo_planes(precision):
    """The 3D tiled pre-pass stages whole rows in 16-byte pieces; a velocity or
    halo buffer that does not start on a 16-byte boundary is served by the
    pre-pass that loads value by value, with the same arithmetic.  Both paths,
    whole domain and two slabs, give the stress of the aligned whole-domain
    run."""
    import torch
    from paper_2411_17294_gb300 import slab, tfs
    dim, n, slabs = 3, (64, 16, 12), (6, 6)
    alpha, Wi, beta, dt, m, steps = 0.6, 1.3, 0.4, 2e-3, 8, 5
    L = [0.25 * k for k in n]
    mu, w = soe.soe_nnls(alpha, dt, steps * dt, m)
    u, kap = inputs.spectral_velocity(dim, n, 4, seed=53)
    case = dict(dim=dim, n=n, alpha=alpha, dt=dt, mu=mu, w=w, eps=0.01, stencil=0, L=L)
    u = stable_velocity(case, u)
    sig0 = inputs.random_stress(dim, n, 54)
    dev = torch.device("cuda", 0)
    dtype = torch.float64 if precision == 0 else torch.float32
    t = lambda a: torch.as_tensor(np.asarray(a), dtype=dtype, device=dev).contiguous()

    def shifted(x):
        """x in a buffer that starts one element past a 16-byte boundary"""
        buf = torch.zeros(x.numel() + 1, dtype=x.dtype, device=x.device)
        v = buf[1:].view(x.shape)
        v.copy_(x)
        assert v.data_ptr() % 16 != 0
        return v

    def solver(grid, lengths):
        return tfs.Solver(dim, grid, alpha, Wi, beta, dt, m=m, precision=precision, mu=mu, w=w, eps=0.01,
                          stencil=0, transport=True, L=lengths)

    def whole_run(ut):
        s = solver(n, L)
        s.set_state(t(sig0))
        kt = t(kap)
        for _ in range(steps):
            s.step(kt, kt, ut)
        out = s.stress().cpu().numpy()
        s.close()
        return out

    ref = whole_run(t(u))
    got_u = whole_run(shifted(t(u)))
    parts, k0 = [], 0
    for ns in slabs:
        s = solver(tuple(n[:-1]) + (ns,), L[:-1] + [0.25 * ns])
        s.set_state(t(_slice(sig0, dim, n, k0, k0 + ns)))
        parts.append((s, t(_slice(kap, dim, n, k0, k0 + ns)), t(_slice(u, dim, n, k0, k0 + ns))))
        k0 += ns
    for _ in range(steps):
        sends = []
        for s, _, _ in parts:
            lo, hi = s.halo_buffers()
            s.get_halo(lo, hi)
            sends.append((lo, hi))
        recvs = slab.exchange_local(sends)
        for (s, ks, us), (rlo, rhi) in zip(parts, recvs):
            s.step_slab(ks, ks, us, shifted(rlo), shifted(rhi))
    got_slab = np.concatenate([s.stress().cpu().numpy() for s, _, _ in parts], axis=1)
    for s, _, _ in parts:
        s.close()
    scale = np.max(np.abs(ref))
    assert scale > 0
    tol = 1e-13 if precision == 0 else 1e-6
    for got in (got_u, got_slab):
        assert np.max(np.abs(got - ref)) <= tol * scale


def test_slab_entry_points_refuse_what_they_do_not_serve():
    import torch
    from paper_2411_17294_gb300 import tfs
    n, m, dt = (32, 8, 6), 4, 1e-3
    mu, w = soe.soe_nnls(0.5, dt, 10 * dt, m)
    s = tfs.Solver(3, n, 0.5, 1.0, 0.5, dt, m=m, precision=1, mu=mu, w=w, transport="implicit")
    s.set_state(None)
    lo, hi = s.halo_buffers()
    k = torch.zeros((9, s.N), dtype=torch.float32, device="cuda")
    u = torch.zeros((3, s.N), dtype=torch.float32, device="cuda")
    with pytest.raises(tfs.TfsError) as ei:
        s.step_slab(k, k, u, lo, hi)
    assert ei.value.code == tfs.TFS_ERR_ARG
    s.close()
    thin = tfs.Solver(3, (32, 8, 1), 0.5, 1.0, 0.5, dt, m=m, precision=1, mu=mu, w=w, transport=True)
    thin.set_state(None)
    lo, hi = thin.halo_buffers()
    with pytest.raises(tfs.TfsError):
        thin.get_halo(lo, hi)
    thin.close()
