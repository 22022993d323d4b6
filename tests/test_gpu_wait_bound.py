"""The bounded device wait (failure detection without a GPU fault): a wait
that nothing satisfies gives up after about 2 s, latches TFS_FLAG_TIMEOUT, and
the GPU context stays usable -- the next step runs and matches the oracle."""
import ctypes

import numpy as np
import pytest

from helpers import ensure_lib, rel_err_per_component
from oracle import orc, soe
from paper_2411_17294_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_lib()


def test_wait_gives_up_and_the_context_stays_usable():
    import torch
    from paper_2411_17294_gb300 import tfs
    lib = tfs.load_library()
    torch.cuda.init()
    flags = ctypes.c_uint(0)
    secs = ctypes.c_double(0.0)
    assert lib.tfs_check_wait_bound(ctypes.byref(flags), ctypes.byref(secs), None) == tfs.TFS_OK
    assert flags.value & tfs.TFS_FLAG_TIMEOUT
    assert 0.5 < secs.value < 5.0, secs.value
    assert lib.tfs_check_wait_bound(None, ctypes.byref(secs), None) == tfs.TFS_ERR_ARG
    # the context is intact: a step afterwards matches the oracle
    dim, n, alpha, m, dt = 2, (12, 10), 0.5, 6, 2e-3
    mu, w = soe.soe_build(alpha, dt, 10 * dt, m)
    _, kap = inputs.spectral_velocity(dim, n, 2, seed=3)
    sigma0 = inputs.random_stress(dim, n, 4)
    s = tfs.Solver(dim, n, alpha, 1.2, 0.4, dt, m=m, precision=tfs.TFS_FP64, mu=mu, w=w, transport=False)
    s.set_state(torch.as_tensor(sigma0, device=s.device))
    kt = torch.as_tensor(np.asarray(kap), device=s.device).contiguous()
    for _ in range(3):
        s.step(kt, kt)
    got = s.stress().cpu().numpy()
    assert s.status() == 0
    s.close()
    ref = orc.forward(orc.Problem(dim=dim, n=n, alpha=alpha, Wi=1.2, beta=0.4, dt=dt, mu=mu, w=w), sigma0, kap,
                      None, 3)
    assert np.all(rel_err_per_component(got, ref) < 1e-11)
