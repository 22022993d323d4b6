"""Shared helpers of the test-suite: building the library, running the CUDA
path through the C ABI, running the oracle on the same inputs, and the
per-component error measure (max |difference| / max |oracle|)."""
from __future__ import annotations

import numpy as np

from paper_2411_17294_gb300 import inputs


def ensure_lib():
    from paper_2411_17294_gb300 import build
    return build.build()


def rel_err_per_component(got: np.ndarray, ref: np.ndarray) -> np.ndarray:
    """Normwise relative error of each stress component."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    scale = np.max(np.abs(ref), axis=1)
    scale = np.where(scale > 0, scale, 1.0)
    return np.max(np.abs(got - ref), axis=1) / scale


def run_gpu(case: dict, sigma0, kap_seq, u, steps: int, precision: int, return_solver=False):
    """Run the CUDA path; kap_seq is a frozen array [d*d][N] or a callable n -> array."""
    import torch
    from paper_2411_17294_gb300 import tfs
    s = tfs.Solver(case["dim"], case["n"], case["alpha"], case["Wi"], case["beta"], case["dt"],
                   m=len(case.get("mu", [])) if case["alpha"] < 1 else 0, precision=precision,
                   mu=case.get("mu") if case["alpha"] < 1 else None, w=case.get("w"),
                   eps=case.get("eps", 0.0), stencil=case.get("stencil", 0),
                   transport=case.get("transport", False), L=case.get("L"))
    dt = s.dtype
    dev = s.device
    s.set_state(None if sigma0 is None else torch.as_tensor(sigma0, dtype=dt, device=dev))
    ut = None if u is None else torch.as_tensor(u, dtype=dt, device=dev).contiguous()
    if callable(kap_seq):
        cache = {}

        def K(n):
            if n not in cache:
                cache.clear() if len(cache) > 4 else None
                cache[n] = torch.as_tensor(kap_seq(n), dtype=dt, device=dev).contiguous()
            return cache[n]
        for n in range(steps):
            s.step(K(n), K(n - 1) if n > 0 else None, ut)
    else:
        kt = torch.as_tensor(kap_seq, dtype=dt, device=dev).contiguous()
        for n in range(steps):
            s.step(kt, kt, ut)
    out = s.stress().double().cpu().numpy()
    # no kernel gave up waiting for its own tile copies
    assert not (s.status() & tfs.TFS_FLAG_TIMEOUT)
    if return_solver:
        return out, s
    s.close()
    return out


def run_oracle(case: dict, sigma0, kap_seq, u, steps: int):
    from oracle import orc
    prob = orc.Problem(dim=case["dim"], n=case["n"], alpha=case["alpha"], Wi=case["Wi"], beta=case["beta"],
                       dt=case["dt"], mu=np.asarray(case.get("mu", np.zeros(0))),
                       w=np.asarray(case.get("w", np.zeros(0))), eps=case.get("eps", 0.0),
                       stencil=case.get("stencil", 0), transport=case.get("transport", False), L=case.get("L"))
    o = orc.Oracle(prob, sigma0)
    return o.run(steps, kap_seq, u)


def transport_limit(case: dict) -> float:
    """tfs_transport_limit for the case (host-only calls of the C ABI)."""
    import ctypes
    import math
    ensure_lib()
    from paper_2411_17294_gb300 import tfs
    lib = tfs.load_library()
    g = tfs.TfsGrid()
    g.dim = case["dim"]
    L = case.get("L") or [2 * math.pi] * case["dim"]
    for a in range(3):
        g.n[a] = case["n"][a] if a < case["dim"] else 1
        g.L[a] = L[a] if a < case["dim"] else 1.0
    h = ctypes.c_void_p()
    m = len(case.get("mu", [])) if case["alpha"] < 1 else 0
    tfs.check(lib.tfs_create(ctypes.byref(h), ctypes.byref(g), case["alpha"], 1.0, 0.5, m, case["dt"], 0), "create")
    tfs.check(lib.tfs_set_param(h, tfs.TFS_PARAM_STENCIL, float(case.get("stencil", 0))), "stencil")
    if m:
        dp = ctypes.POINTER(ctypes.c_double)
        mu = np.ascontiguousarray(case["mu"], dtype=np.float64)
        w = np.ascontiguousarray(case["w"], dtype=np.float64)
        tfs.check(lib.tfs_set_soe(h, mu.ctypes.data_as(dp), w.ctypes.data_as(dp), m), "soe")
    tfs.check(lib.tfs_set_param(h, tfs.TFS_PARAM_EPS, float(case.get("eps", 0.0))), "eps")
    U = ctypes.c_double(0.0)
    tfs.check(lib.tfs_transport_limit(h, ctypes.byref(U)), "limit")
    lib.tfs_destroy(h)
    return U.value


def courant_fraction(case: dict, u) -> float:
    """max_p sum_a |u_a(p)|/h_a over U sum_a 1/h_a: the fraction of the
    library's velocity limit that the field uses (flagged above 1)."""
    n = case["n"]
    L = case.get("L") or [2 * np.pi] * case["dim"]
    inv_h = np.array([n[a] / L[a] for a in range(case["dim"])])
    return float(np.max(np.abs(np.asarray(u)).T @ inv_h) / (transport_limit(case) * inv_h.sum()))


def stable_velocity(case: dict, u, target: float = 0.5):
    """Scale u to use at most `target` of the library's explicit-transport
    velocity limit (parity needs a stable recurrence: unstable modes amplify
    rounding differences exponentially)."""
    c = courant_fraction(case, u)
    return u if c <= target else np.asarray(u) * (target / c)


def spectral_case(dim, n, seed, kmax=None):
    kmax = kmax or max(1, min(n) // 3)
    u, kap = inputs.spectral_velocity(dim, n, kmax, seed)
    return u, kap
