"""tfs_run_static: the entry point for callers that cannot allocate device
memory (it keeps the step state in a fixed array inside the library instead of
a workspace the caller binds).  Checked through the C ABI against the regular
entry points (tfs_create ... tfs_step ... tfs_get_stress) on two calls in a
row, so that state left in the shared array by the first call would show in
the second.  Collected last on purpose (file name), so that a stop at the
first failure has run every other test already."""
import ctypes
import math

import numpy as np
import pytest

from helpers import courant_fraction, ensure_lib, stable_velocity
from oracle import soe
from paper_2411_17294_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = {0: 1e-11, 1: 2e-5}


def grid_struct(dim, n):
    from paper_2411_17294_gb300 import tfs
    g = tfs.TfsGrid()
    g.dim = dim
    for a in range(3):
        g.n[a] = n[a] if a < dim else 1
        g.L[a] = 2 * math.pi if a < dim else 1.0
    return g


def static_flags():
    import torch
    from paper_2411_17294_gb300 import tfs
    lib = tfs.load_library()
    f = ctypes.c_uint(12345)
    rc = lib.tfs_static_status(ctypes.byref(f), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == tfs.TFS_OK, tfs.strerror(rc)
    return f.value


def run_static(dim, n, alpha, Wi, beta, m, dt, precision, mu, w, sigma0, kap, u, steps):
    import torch
    from paper_2411_17294_gb300 import tfs
    lib = tfs.load_library()
    dtype = torch.float64 if precision == 0 else torch.float32
    N = int(np.prod(n))
    nc = 3 if dim == 2 else 6
    out = torch.full((nc, N), float("nan"), dtype=dtype, device="cuda")
    s0 = None if sigma0 is None else torch.as_tensor(sigma0, dtype=dtype, device="cuda").contiguous()
    kt = torch.as_tensor(kap, dtype=dtype, device="cuda").contiguous()
    ut = None if u is None else torch.as_tensor(u, dtype=dtype, device="cuda").contiguous()
    dp = ctypes.POINTER(ctypes.c_double)
    mu_c = None if mu is None else np.ascontiguousarray(mu, dtype=np.float64)
    w_c = None if w is None else np.ascontiguousarray(w, dtype=np.float64)
    g = grid_struct(dim, n)
    stream = torch.cuda.current_stream()
    rc = lib.tfs_run_static(ctypes.byref(g), alpha, Wi, beta, m, dt, precision,
                            mu_c.ctypes.data_as(dp) if mu_c is not None else None,
                            w_c.ctypes.data_as(dp) if w_c is not None else None,
                            ctypes.c_void_p(s0.data_ptr() if s0 is not None else 0),
                            ctypes.c_void_p(kt.data_ptr()),
                            ctypes.c_void_p(ut.data_ptr() if ut is not None else 0),
                            steps, ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
    assert rc == tfs.TFS_OK, tfs.strerror(rc)
    torch.cuda.synchronize()
    return out.double().cpu().numpy()


def run_regular(dim, n, alpha, Wi, beta, m, dt, precision, mu, w, sigma0, kap, u, steps):
    import torch
    from paper_2411_17294_gb300 import tfs
    s = tfs.Solver(dim, n, alpha, Wi, beta, dt, m=m, precision=precision, mu=mu, w=w, transport=u is not None)
    s.set_state(None if sigma0 is None else torch.as_tensor(sigma0, dtype=s.dtype, device=s.device))
    kt = torch.as_tensor(kap, dtype=s.dtype, device=s.device).contiguous()
    ut = None if u is None else torch.as_tensor(u, dtype=s.dtype, device=s.device).contiguous()
    for _ in range(steps):
        s.step(kt, kt, ut)
    out = s.stress().double().cpu().numpy()
    s.close()
    return out


def rel(a, b):
    scale = np.max(np.abs(b), axis=1)
    scale = np.where(scale > 0, scale, 1.0)
    return np.max(np.abs(a - b), axis=1) / scale


@pytest.mark.parametrize("precision", [0, 1])
def test_static_entry_matches_regular_entry_twice(precision):
    ensure_lib()
    dim, n, alpha, Wi, beta, m, dt, steps = 3, (12, 10, 9), 0.6, 1.5, 0.7, 8, 1e-3, 14
    mu, w = soe.soe_nnls(alpha, dt, steps * dt, m)
    u, kap = inputs.spectral_velocity(dim, n, 3, seed=41)
    u = stable_velocity(dict(dim=dim, n=n, alpha=alpha, dt=dt, mu=mu, w=w), u)
    sig_a = inputs.random_stress(dim, n, 42)
    # first call: nonzero initial stress, transport on
    ref_a = run_regular(dim, n, alpha, Wi, beta, m, dt, precision, mu, w, sig_a, kap, u, steps)
    got_a = run_static(dim, n, alpha, Wi, beta, m, dt, precision, mu, w, sig_a, kap, u, steps)
    assert np.all(rel(got_a, ref_a) < TOL[precision])
    assert static_flags() == 0
    # second call in a row on the same array: zero initial stress and fewer steps
    ref_b = run_regular(dim, n, alpha, Wi, beta, m, dt, precision, mu, w, None, kap, u, steps - 5)
    got_b = run_static(dim, n, alpha, Wi, beta, m, dt, precision, mu, w, None, kap, u, steps - 5)
    assert np.all(rel(got_b, ref_b) < TOL[precision])
    assert np.max(np.abs(ref_b)) > 0
    assert static_flags() == 0


def test_static_entry_reports_its_device_flags():
    # tfs_run_static has no handle: the flags its kernels latch are read with
    # tfs_static_status.  A non-finite initial stress latches
    # TFS_FLAG_NONFINITE; a velocity beyond the explicit transport's limit
    # latches TFS_FLAG_COURANT; the next clean call clears them.
    ensure_lib()
    from paper_2411_17294_gb300 import tfs
    dim, n, alpha, Wi, beta, m, dt, steps = 2, (16, 12), 0.5, 1.0, 0.5, 6, 1e-3, 4
    mu, w = soe.soe_nnls(alpha, dt, 10 * dt, m)
    u, kap = inputs.spectral_velocity(dim, n, 3, seed=44)
    case = dict(dim=dim, n=n, alpha=alpha, dt=dt, mu=mu, w=w)
    u_ok = stable_velocity(case, u)
    sig = inputs.random_stress(dim, n, 45)
    sig[1, 7] = np.nan
    out = run_static(dim, n, alpha, Wi, beta, m, dt, 1, mu, w, sig, kap, u_ok, steps)
    assert np.isnan(out).any()
    assert static_flags() & tfs.TFS_FLAG_NONFINITE
    u_bad = np.asarray(u_ok) * (2.0 / courant_fraction(case, u_ok))
    run_static(dim, n, alpha, Wi, beta, m, dt, 1, mu, w, None, kap, u_bad, steps)
    assert static_flags() & tfs.TFS_FLAG_COURANT
    run_static(dim, n, alpha, Wi, beta, m, dt, 1, mu, w, None, kap, u_ok, steps)
    assert static_flags() == 0


def test_static_entry_classic_path_and_size_limit():
    ensure_lib()
    from paper_2411_17294_gb300 import tfs
    dim, n, dt, steps = 2, (33, 17), 1e-3, 9
    u, kap = inputs.spectral_velocity(dim, n, 4, seed=43)
    ref = run_regular(dim, n, 1.0, 0.8, 0.3, 0, dt, 0, None, None, None, kap, None, steps)
    for _ in range(2):
        got = run_static(dim, n, 1.0, 0.8, 0.3, 0, dt, 0, None, None, None, kap, None, steps)
        assert np.all(rel(got, ref) < TOL[0])
    # a state larger than the fixed array is refused before any device work
    lib = tfs.load_library()
    g = grid_struct(3, (256, 256, 256))
    mu = np.ones(32)
    dp = ctypes.POINTER(ctypes.c_double)
    rc = lib.tfs_run_static(ctypes.byref(g), 0.6, 1.0, 0.5, 32, 1e-3, 1, mu.ctypes.data_as(dp),
                            mu.ctypes.data_as(dp), None, ctypes.c_void_p(256), None, 1, ctypes.c_void_p(256), None)
    assert rc == tfs.TFS_ERR_TOOBIG
