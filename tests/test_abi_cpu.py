"""The C-ABI library loads on a machine without a GPU, exports every symbol
declared in include/tfs.h, and its host-side argument checks behave as
documented (no compute calls: no device is touched)."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

from helpers import ensure_lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    ensure_lib()
    from paper_2411_17294_gb300 import tfs
    return tfs.load_library()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "tfs.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(tfs_[a-z_0-9]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    from paper_2411_17294_gb300 import tfs
    names = declared_functions()
    assert len(names) >= 18
    for name in names:
        assert hasattr(lib, name), name
    assert sorted(tfs.EXPORTS) == sorted(n for n in names if n in tfs.EXPORTS)
    assert set(names) <= set(tfs.EXPORTS)


def make(lib, dim=3, n=(8, 8, 8), alpha=0.6, Wi=2.0, beta=0.9, m=4, dt=2e-4, precision=1, L=None):
    from paper_2411_17294_gb300 import tfs
    g = tfs.TfsGrid()
    g.dim = dim
    Ls = L or [2 * math.pi] * 3
    for a in range(3):
        g.n[a] = n[a] if a < len(n) else 1
        g.L[a] = Ls[a]
    h = ctypes.c_void_p()
    rc = lib.tfs_create(ctypes.byref(h), ctypes.byref(g), alpha, Wi, beta, m, dt, precision)
    return rc, h


def test_create_validation(lib):
    from paper_2411_17294_gb300 import tfs
    rc, h = make(lib)
    assert rc == tfs.TFS_OK and h.value
    assert lib.tfs_destroy(h) == tfs.TFS_OK
    bad = [
        dict(dim=4), dict(alpha=0.0), dict(alpha=1.2), dict(Wi=0.0), dict(beta=1.0), dict(beta=-0.1),
        dict(dt=0.0), dict(m=65), dict(m=0), dict(alpha=1.0, m=3), dict(precision=7), dict(n=(0, 4, 4)),
    ]
    for kw in bad:
        rc, h = make(lib, **kw)
        assert rc == tfs.TFS_ERR_ARG, kw
        assert not h.value
    rc, h = make(lib, alpha=1.0, m=0)
    assert rc == tfs.TFS_OK
    lib.tfs_destroy(h)


def test_soe_and_params_validation(lib):
    from paper_2411_17294_gb300 import tfs
    rc, h = make(lib, m=3)
    dp = ctypes.POINTER(ctypes.c_double)
    mu = np.array([1.0, 10.0, 100.0])
    w = np.array([0.5, 0.4, 0.3])
    assert lib.tfs_set_soe(h, mu.ctypes.data_as(dp), w.ctypes.data_as(dp), 2) == tfs.TFS_ERR_ARG
    wn = np.array([0.5, -0.4, 0.3])
    assert lib.tfs_set_soe(h, mu.ctypes.data_as(dp), wn.ctypes.data_as(dp), 3) == tfs.TFS_ERR_ARG
    mnan = np.array([1.0, np.nan, 100.0])
    assert lib.tfs_set_soe(h, mnan.ctypes.data_as(dp), w.ctypes.data_as(dp), 3) == tfs.TFS_ERR_ARG
    assert lib.tfs_set_soe(h, mu.ctypes.data_as(dp), w.ctypes.data_as(dp), 3) == tfs.TFS_OK
    assert lib.tfs_set_param(h, tfs.TFS_PARAM_RE, 0.0) == tfs.TFS_ERR_ARG
    assert lib.tfs_set_param(h, tfs.TFS_PARAM_EPS, -1.0) == tfs.TFS_ERR_ARG
    assert lib.tfs_set_param(h, tfs.TFS_PARAM_STENCIL, 5.0) == tfs.TFS_ERR_ARG
    assert lib.tfs_set_param(h, 99, 1.0) == tfs.TFS_ERR_ARG
    assert lib.tfs_set_param(h, tfs.TFS_PARAM_EPS, 0.01) == tfs.TFS_OK
    # velocity bound above the explicit-transport Courant limit is refused
    assert lib.tfs_set_param(h, tfs.TFS_PARAM_UMAX, 1e6) == tfs.TFS_ERR_UNSTABLE
    assert lib.tfs_set_param(h, tfs.TFS_PARAM_UMAX, 1e-3) == tfs.TFS_OK
    # with transport off any bound is accepted
    assert lib.tfs_set_param(h, tfs.TFS_PARAM_TRANSPORT, 0.0) == tfs.TFS_OK
    assert lib.tfs_set_param(h, tfs.TFS_PARAM_UMAX, 1e6) == tfs.TFS_OK
    # first-step method: BDF2 or SDIRK2 only; tfs_backward checks its pointers in any mode
    assert lib.tfs_set_param(h, tfs.TFS_PARAM_START, 2.0) == tfs.TFS_ERR_ARG
    assert lib.tfs_set_param(h, tfs.TFS_PARAM_START, 0.5) == tfs.TFS_ERR_ARG
    assert lib.tfs_set_param(h, tfs.TFS_PARAM_START, float(tfs.TFS_START_SDIRK2)) == tfs.TFS_OK
    assert lib.tfs_backward(h, None, None, 1, 1, None, None, None, None, None, None, None) == tfs.TFS_ERR_ARG
    assert lib.tfs_set_param(h, tfs.TFS_PARAM_START, float(tfs.TFS_START_BDF2)) == tfs.TFS_OK
    # variable carried: stress or the paper's Phi (null arguments to tfs_backward: TFS_ERR_ARG)
    assert lib.tfs_set_param(h, tfs.TFS_PARAM_FORM, 2.0) == tfs.TFS_ERR_ARG
    assert lib.tfs_set_param(h, tfs.TFS_PARAM_FORM, float(tfs.TFS_FORM_PAPER)) == tfs.TFS_OK
    assert lib.tfs_backward(h, None, None, 1, 1, None, None, None, None, None, None, None) == tfs.TFS_ERR_ARG
    assert lib.tfs_set_param(h, tfs.TFS_PARAM_FORM, float(tfs.TFS_FORM_STRESS)) == tfs.TFS_OK
    lib.tfs_destroy(h)
    rc, h = make(lib, alpha=1.0, m=0)
    assert lib.tfs_set_param(h, tfs.TFS_PARAM_START, float(tfs.TFS_START_SDIRK2)) == tfs.TFS_ERR_ARG
    assert lib.tfs_set_param(h, tfs.TFS_PARAM_FORM, float(tfs.TFS_FORM_PAPER)) == tfs.TFS_ERR_ARG
    lib.tfs_destroy(h)


def test_calls_out_of_order_and_workspace(lib):
    from paper_2411_17294_gb300 import tfs
    rc, h = make(lib, dim=2, n=(16, 16), m=4, precision=0)
    # no workspace bound yet: no device access happens
    assert lib.tfs_step(h, ctypes.c_void_p(16), None, ctypes.c_void_p(16), None) == tfs.TFS_ERR_NOWORKSPACE
    assert lib.tfs_set_state(h, None, None) == tfs.TFS_ERR_NOWORKSPACE
    need = lib.tfs_workspace_bytes(h)
    N, nc, m = 256, 3, 4
    field = nc * N * 8
    up = lambda b: (b + 255) // 256 * 256
    assert need == 256 + 5 * up(field) + 2 * up(m * field)
    assert lib.tfs_bind_workspace(h, ctypes.c_void_p(256 * 1000), need - 1) == tfs.TFS_ERR_NOWORKSPACE
    assert lib.tfs_bind_workspace(h, ctypes.c_void_p(256 * 1000 + 8), need) == tfs.TFS_ERR_ARG
    assert lib.tfs_bind_workspace(h, ctypes.c_void_p(256 * 1000), need) == tfs.TFS_OK
    # bound but no state: refused before any launch
    assert lib.tfs_step(h, ctypes.c_void_p(256), None, ctypes.c_void_p(256), None) == tfs.TFS_ERR_STATE
    assert lib.tfs_step_index(h) == 0
    assert lib.tfs_strerror(tfs.TFS_ERR_UNSTABLE).decode().startswith("velocity")
    lib.tfs_destroy(h)


def test_form_and_transport_resize_checks(lib):
    # The paper's variable adds two stress-sized buffers (Psi^n, Psi^{n-1}) and,
    # with implicit transport, one more FP64 vector; with a workspace bound, a
    # parameter change that needs more than it returns TFS_ERR_NOWORKSPACE and
    # changes nothing.  Host logic only: no device memory is touched.
    from paper_2411_17294_gb300 import tfs
    rc, h = make(lib, dim=2, n=(16, 16), m=4, precision=0)
    assert rc == tfs.TFS_OK
    stress = lib.tfs_workspace_bytes(h)
    assert lib.tfs_set_param(h, tfs.TFS_PARAM_FORM, float(tfs.TFS_FORM_PAPER)) == tfs.TFS_OK
    paper = lib.tfs_workspace_bytes(h)
    field = 3 * 256 * 8
    assert paper == stress + 2 * field
    assert lib.tfs_set_param(h, tfs.TFS_PARAM_TRANSPORT, 2.0) == tfs.TFS_OK
    paper_imp = lib.tfs_workspace_bytes(h)
    assert lib.tfs_set_param(h, tfs.TFS_PARAM_FORM, float(tfs.TFS_FORM_STRESS)) == tfs.TFS_OK
    stress_imp = lib.tfs_workspace_bytes(h)
    assert paper_imp == stress_imp + 2 * field + field      # Psi ring + h
    # bind the stress-form workspace (explicit transport), then ask for more
    assert lib.tfs_set_param(h, tfs.TFS_PARAM_TRANSPORT, 1.0) == tfs.TFS_OK
    assert lib.tfs_bind_workspace(h, ctypes.c_void_p(256 * 1000), stress) == tfs.TFS_OK
    assert lib.tfs_set_param(h, tfs.TFS_PARAM_FORM, float(tfs.TFS_FORM_PAPER)) == tfs.TFS_ERR_NOWORKSPACE
    assert lib.tfs_set_param(h, tfs.TFS_PARAM_TRANSPORT, 2.0) == tfs.TFS_ERR_NOWORKSPACE
    assert lib.tfs_workspace_bytes(h) == stress
    # a large enough workspace takes both
    assert lib.tfs_bind_workspace(h, ctypes.c_void_p(256 * 1000), paper_imp) == tfs.TFS_OK
    assert lib.tfs_set_param(h, tfs.TFS_PARAM_FORM, float(tfs.TFS_FORM_PAPER)) == tfs.TFS_OK
    assert lib.tfs_set_param(h, tfs.TFS_PARAM_TRANSPORT, 2.0) == tfs.TFS_OK
    assert lib.tfs_checkpoint_bytes(h) == 256 + 5 * field + 2 * 4 * field
    lib.tfs_destroy(h)


def test_adjoint_workspace_sizing(lib):
    # tfs_adjoint_workspace_bytes: two ping-pong pairs of FP64 adjoint fields and
    # lamR (5 fields), two mode-ring levels, the 32-point partials, the scalar
    # output slot and K segment levels; explicit transport in the paper's
    # variable adds the Psi ring (4 fields), implicit transport the transposed
    # tap coefficients (4 d N doubles), both together one more field.  A
    # workspace bound before a change of form is refused by tfs_backward before
    # any device access.  Host logic only.
    from paper_2411_17294_gb300 import tfs
    rc, h = make(lib, dim=2, n=(16, 16), m=4, precision=0)
    assert rc == tfs.TFS_OK
    N, nc, m, d = 256, 3, 4, 2
    up = lambda b: (b + 255) // 256 * 256
    dfield = nc * N * 8
    fixed = 2 * up(m * dfield) + up((N + 31) // 32 * 16) + 256
    cft = up(4 * d * N * 8)

    def expect(extra_fields, extra_bytes, K):
        return (5 + extra_fields) * up(dfield) + extra_bytes + fixed + K * up(dfield)

    cases = [
        (tfs.TFS_FORM_STRESS, 0, 0, 0), (tfs.TFS_FORM_STRESS, 1, 0, 0), (tfs.TFS_FORM_STRESS, 2, 0, cft),
        (tfs.TFS_FORM_PAPER, 0, 0, 0), (tfs.TFS_FORM_PAPER, 1, 4, 0), (tfs.TFS_FORM_PAPER, 2, 1, cft),
    ]
    for form, transport, fields, extra in cases:
        assert lib.tfs_set_param(h, tfs.TFS_PARAM_FORM, float(form)) == tfs.TFS_OK
        assert lib.tfs_set_param(h, tfs.TFS_PARAM_TRANSPORT, float(transport)) == tfs.TFS_OK
        for K in (1, 7):
            assert lib.tfs_adjoint_workspace_bytes(h, K) == expect(fields, extra, K), (form, transport, K)
    assert lib.tfs_adjoint_workspace_bytes(h, 0) == 0
    # bind for the stress form with explicit transport, then carry the paper's variable
    assert lib.tfs_set_param(h, tfs.TFS_PARAM_FORM, float(tfs.TFS_FORM_STRESS)) == tfs.TFS_OK
    assert lib.tfs_set_param(h, tfs.TFS_PARAM_TRANSPORT, 1.0) == tfs.TFS_OK
    big = 1 << 24
    assert lib.tfs_bind_workspace(h, ctypes.c_void_p(256 * 1000), big) == tfs.TFS_OK
    small = lib.tfs_adjoint_workspace_bytes(h, 1)
    assert lib.tfs_bind_adjoint_workspace(h, ctypes.c_void_p(256 * 4000), small - 1) == tfs.TFS_ERR_NOWORKSPACE
    assert lib.tfs_bind_adjoint_workspace(h, ctypes.c_void_p(256 * 4000 + 8), small) == tfs.TFS_ERR_ARG
    assert lib.tfs_bind_adjoint_workspace(h, ctypes.c_void_p(256 * 4000), small) == tfs.TFS_OK
    assert lib.tfs_set_param(h, tfs.TFS_PARAM_FORM, float(tfs.TFS_FORM_PAPER)) == tfs.TFS_OK
    p = ctypes.c_void_p(256)
    arr = (ctypes.c_void_p * 1)(p)
    gWi, gb = ctypes.c_double(0.0), ctypes.c_double(0.0)
    rc = lib.tfs_backward(h, p, arr, 1, 1, p, p, p, p, ctypes.byref(gWi), ctypes.byref(gb), None)
    assert rc == tfs.TFS_ERR_NOWORKSPACE
    lib.tfs_destroy(h)
