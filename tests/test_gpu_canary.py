"""Guard bands around every device buffer the library writes (a stand-in for a
memory checker, which this pool does not offer): the workspace, the stress
output, the checkpoint buffer, the adjoint workspace and the gradient outputs
are each placed between two 64 KiB bands of a known byte pattern; after steps
in every variant (explicit, implicit and no transport; the stress form and the
paper's variable; BDF2 and SDIRK2 starts; FP64 and FP32 storage), a checkpoint
round trip and (where built: either variable with the BDF2 start with or without explicit
transport or the SDIRK2 start without; implicit transport with either
start) the adjoint, every band must be intact.  Odd and
tiny grids make the periodic wrap-around and the ragged last tile touch the
ends of each array.
"""
import ctypes

import numpy as np
import pytest

from helpers import ensure_lib
from oracle import soe
from paper_2411_17294_gb300 import inputs

pytestmark = pytest.mark.gpu

GUARD = 64 * 1024
PATTERN = 0xA5


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_lib()


class Guarded:
    """nbytes of device memory at a 256-byte aligned address between two guard bands."""

    def __init__(self, nbytes, device):
        import torch
        self.nbytes = int(nbytes)
        self.buf = torch.full((self.nbytes + 2 * GUARD + 256,), PATTERN, dtype=torch.uint8, device=device)
        base = self.buf.data_ptr()
        self.off = GUARD + (-(base + GUARD)) % 256
        self.ptr = base + self.off

    def intact(self):
        lo = self.buf[: self.off]
        hi = self.buf[self.off + self.nbytes:]
        return bool((lo == PATTERN).all()) and bool((hi == PATTERN).all())


CASES = [
    # dim, n, transport, form, start, precision
    (2, (7, 5), True, "stress", "bdf2", 0),
    (2, (7, 5), True, "stress", "bdf2", 1),
    (3, (3, 5, 7), True, "stress", "bdf2", 1),
    (2, (37, 29), False, "paper", "sdirk2", 1),
    (3, (5, 3, 4), False, "paper", "bdf2", 0),
    (3, (3, 5, 7), "implicit", "stress", "sdirk2", 0),
    (2, (33, 9), "implicit", "stress", "bdf2", 1),
    (2, (40, 1), False, "stress", "sdirk2", 1),
    (2, (32, 8), True, "paper", "bdf2", 1),
    (3, (3, 5, 7), True, "paper", "bdf2", 0),
    (2, (9, 7), "implicit", "paper", "bdf2", 1),
]


@pytest.mark.parametrize("dim,n,transport,form,start,precision", CASES)
def test_guard_bands_intact(dim, n, transport, form, start, precision):
    import torch
    from paper_2411_17294_gb300 import tfs
    alpha, m, dt, steps = 0.55, 6, 4e-3, 5
    N = int(np.prod(n))
    nc = 3 if dim == 2 else 6
    mu, w = soe.soe_build(1 - alpha if form == "paper" else alpha, dt, 100 * dt, m)
    s = tfs.Solver(dim, n, alpha, 1.2, 0.4, dt, m=m, precision=precision, mu=mu, w=w, eps=0.01,
                   transport=transport, start=start, form=form)
    lib, h, dev, tdt = s.lib, s.h, s.device, s.dtype
    es = 8 if precision == tfs.TFS_FP64 else 4
    need = lib.tfs_workspace_bytes(h)
    ws = Guarded(need, dev)
    assert lib.tfs_bind_workspace(h, ctypes.c_void_p(ws.ptr), need) == tfs.TFS_OK
    u, kap = inputs.spectral_velocity(dim, n, 2, seed=5)
    scale = 0.05 if transport is True else 1.0        # inside the explicit limit
    kt = torch.as_tensor(np.asarray(kap), dtype=tdt, device=dev).contiguous()
    ut = torch.as_tensor(scale * np.asarray(u), dtype=tdt, device=dev).contiguous()
    s.set_state(torch.as_tensor(inputs.random_stress(dim, n, 6), dtype=tdt, device=dev))
    for _ in range(steps):
        s.step(kt, kt, ut if transport else None)
    out = Guarded(nc * N * es, dev)
    assert lib.tfs_get_stress(h, ctypes.c_void_p(out.ptr), None) == tfs.TFS_OK
    ck = Guarded(lib.tfs_checkpoint_bytes(h), dev)
    assert lib.tfs_save(h, ctypes.c_void_p(ck.ptr), None) == tfs.TFS_OK
    s.step(kt, kt, ut if transport else None)
    assert lib.tfs_load(h, ctypes.c_void_p(ck.ptr), None) == tfs.TFS_OK
    s.step(kt, kt, ut if transport else None)
    guarded = [ws, out, ck]
    adjoint_built = ((transport in (False, True) and (start == "bdf2" or transport is False))
                     or transport == "implicit")
    if adjoint_built:
        K = 2
        ckpts = []
        s.set_state(None)
        for k in range(steps):
            if k % K == 0:
                c = s.new_checkpoint()
                s.save(c)
                ckpts.append(c)
            s.step(kt, kt, ut if transport else None)
        aneed = lib.tfs_adjoint_workspace_bytes(h, K)
        aws = Guarded(aneed, dev)
        assert lib.tfs_bind_adjoint_workspace(h, ctypes.c_void_p(aws.ptr), aneed) == tfs.TFS_OK
        dJ = torch.ones((nc, N), dtype=tdt, device=dev)
        g_s0 = Guarded(nc * N * 8, dev)
        g_k = Guarded(dim * dim * N * 8, dev)
        arr = (ctypes.c_void_p * len(ckpts))(*[ctypes.c_void_p(c.data_ptr()) for c in ckpts])
        gWi, gb = ctypes.c_double(0.0), ctypes.c_double(0.0)
        rc = lib.tfs_backward(h, ctypes.c_void_p(dJ.data_ptr()), arr, K, steps, ctypes.c_void_p(kt.data_ptr()),
                              ctypes.c_void_p(ut.data_ptr() if transport else 0), ctypes.c_void_p(g_s0.ptr),
                              ctypes.c_void_p(g_k.ptr), ctypes.byref(gWi), ctypes.byref(gb), None)
        assert rc == tfs.TFS_OK
        assert np.isfinite(gWi.value) and np.isfinite(gb.value)
        guarded += [aws, g_s0, g_k]
    torch.cuda.synchronize()
    flags = s.status()
    s.close()
    assert not (flags & (tfs.TFS_FLAG_TIMEOUT | tfs.TFS_FLAG_NONFINITE))
    assert all(g.intact() for g in guarded), [g.intact() for g in guarded]
