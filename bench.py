"""Benchmark of the fractional polymer-stress step on GB300.

Workload (one step = one tfs_step over the whole grid: extrapolated velocity
gradient, upwind transport stencil, compensated mode history sum, FP64-accurate
per-point 6x6 solve, push-forward of all modes):
    3D periodic 256^3, 6 stress components, FP32 modes, alpha = 0.6, Wi = 2,
    beta = 0.9, m = 32, dt = 2e-4, seeded divergence-free k^-5/3 velocity
    |k| <= 24 at unit RMS, transport on.
Metric: G point-mode updates/s = N * m * steps / time, plus the fraction of
the HBM roofline of the step kernel.  The per-step working set (~41 GB) is far
larger than L2, so no L2 flush is needed between steps.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun (N > 1) the ranks share one periodic domain of 256 x 256 x
(256 N) points cut into z-slabs, one 256^3 slab per rank (weak scaling):
before every step each rank sends its two boundary planes of both stress
levels to its neighbours on the ring and steps its slab with theirs
(tfs_get_halo -> NCCL point-to-point -> tfs_step_slab); rank 0 prints one JSON
line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "G point-mode updates/s per fractional stress step and % of HBM peak; adjoint/forward ratio"
UNIT = "G point-mode updates/s"

WORKLOAD = dict(name="3D periodic 256^3 fractional stress step, m=32 SOE modes, FP32 modes + compensated sum",
                dim=3, n=(256, 256, 256), alpha=0.6, Wi=2.0, beta=0.9, m=32, dt=2e-4, horizon_steps=200,
                kmax=24, seed=3)


def algorithmic_bytes_per_point(dim: int, m: int, elem: int, sigma0_nonzero: bool = False) -> int:
    """3 words per (mode, component) + 3 nc stress words + (2 d^2 + d) input
    words (+ nc for a nonzero initial stress)."""
    nc = 3 if dim == 2 else 6
    b = 3 * m * nc * elem + 3 * nc * elem + (2 * dim * dim + dim) * elem
    if sigma0_nonzero:
        b += nc * elem
    return b


def step_kernel_bytes_per_point(dim: int, m: int, elem: int, transport: bool) -> int:
    """Algorithmic bytes of the step kernel alone: 3 words per (mode, component),
    both velocity-gradient levels, the stress written, and either the transport
    term (written by the pre-pass) or the two stress levels it reads."""
    nc = 3 if dim == 2 else 6
    b = 3 * m * nc * elem + 2 * dim * dim * elem + nc * elem
    b += nc * elem if transport else 2 * nc * elem
    return b


TRAFFIC_FILE = os.path.join(ROOT, "profiles", "fwd_kernel_3d256_fp32_traffic.md")
STEP_KERNEL_SOURCES = [os.path.join(ROOT, "paper_2411_17294_gb300", "csrc", f)
                       for f in ("tfs_forward.cu", "tfs_device.cuh", "tfs_internal.h", "tfs_util.cu")]


def step_kernel_source_hash() -> str:
    """SHA-256 of the step kernel's sources without their whole-line comments
    (an edit of a comment does not change the kernel)."""
    import hashlib
    h = hashlib.sha256()
    for f in STEP_KERNEL_SOURCES:
        with open(f, "rb") as fh:
            for ln in fh:
                if not ln.lstrip().startswith(b"//"):
                    h.update(ln)
    return h.hexdigest()


def read_traffic():
    """DRAM bytes per step-kernel launch from the committed ncu capture, or None
    when the step kernel's sources changed since that capture."""
    try:
        fields = {}
        with open(TRAFFIC_FILE) as f:
            for ln in f:
                if ":" in ln and ln.startswith("- "):
                    k, v = ln[2:].split(":", 1)
                    fields[k.strip()] = v.strip().strip("`")
        if fields.get("source_sha256") != step_kernel_source_hash():
            return None
        return float(fields["traffic_bytes_per_launch"])
    except Exception:
        return None


def read_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str | None):
        self.gpu_id = gpu_id
        self.proc = None
        self.file = None

    def start(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
            if self.gpu_id:
                cmd.insert(1, f"--id={self.gpu_id}")
            self.proc = subprocess.Popen(cmd, stdout=self.file, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.file.flush()
        self.file.seek(0)
        rows = [r.split(",") for r in self.file.read().strip().splitlines() if r.strip()]
        os.unlink(self.file.name)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
                for nm, v in zip(names, r[5:9]):
                    if v.strip() == "Active":
                        reasons.add(nm)
            except Exception:
                continue
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


ADJOINT = dict(name="adjoint 2D 512^2, m=32, alpha=0.5, checkpoint every 50", dim=2, n=(512, 512), alpha=0.5,
               Wi=1.0, beta=0.5, m=32, dt=1e-3, steps=100, K=50, seed=2)


def adjoint_ratio(dev, precision, form="stress"):
    """Time of tfs_backward (segment recompute + reverse sweep) over the time of
    the forward run with checkpoints, on the adjoint workload (frozen gradient,
    transport off as in that workload); form "paper" runs it in the paper's
    variable (the SOE of order 1 - alpha).  Returns a dict for the JSON line."""
    import numpy as np
    import torch

    from paper_2411_17294_gb300 import inputs, soe, tfs

    A = ADJOINT
    order = 1.0 - A["alpha"] if form == "paper" else A["alpha"]
    mu, w = soe.build(order, A["dt"], A["steps"] * A["dt"], A["m"])
    s = tfs.Solver(A["dim"], A["n"], A["alpha"], A["Wi"], A["beta"], A["dt"], m=A["m"], precision=precision,
                   mu=mu, w=w, transport=False, device=dev, form=form)
    _, kap = inputs.spectral_velocity(A["dim"], A["n"], 32, A["seed"], device=dev)
    kt = torch.as_tensor(kap, dtype=s.dtype, device=dev).contiguous()
    sig0 = torch.as_tensor(inputs.random_stress(A["dim"], A["n"], 5, 0.1), dtype=s.dtype, device=dev)
    nck = (A["steps"] + A["K"] - 1) // A["K"]
    ckpts = [s.new_checkpoint() for _ in range(nck)]
    s.ensure_adjoint_workspace(A["K"])
    stream = torch.cuda.Stream(device=dev)

    def forward():
        s.set_state(sig0, stream=stream)
        for k in range(A["steps"]):
            if k % A["K"] == 0:
                s.save(ckpts[k // A["K"]], stream=stream)
            s.step(kt, kt, None, stream=stream)

    with torch.cuda.stream(stream):
        forward()                                   # warm-up (also builds the stability cache)
        torch.cuda.synchronize()
        dJ = s.stress(stream=stream)
        s.backward(dJ, ckpts, A["K"], A["steps"], kt, None, stream=stream)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        forward()
        e1.record(stream)
        torch.cuda.synchronize()
        t_fwd = e0.elapsed_time(e1)
        dJ = s.stress(stream=stream)
        t0 = time.perf_counter()
        e0.record(stream)
        s.backward(dJ, ckpts, A["K"], A["steps"], kt, None, stream=stream)   # synchronises at its end
        e1.record(stream)
        torch.cuda.synchronize()
        t_bwd = e0.elapsed_time(e1)
        wall_bwd = (time.perf_counter() - t0) * 1e3
    s.close()
    return {"workload": A["name"] + (", the paper's variable" if form == "paper" else ""),
            "precision": {0: "fp64", 1: "fp32", 2: "fp32plain"}[precision],
            "steps": A["steps"], "forward_ms": t_fwd, "backward_ms": max(t_bwd, wall_bwd),
            "ratio": max(t_bwd, wall_bwd) / t_fwd}


def cpu_baseline(steps_hint: int = 3, budget_s: float = 15.0):
    """The FP64 C oracle, as it stands, on a bounded sample of the workload:
    a 64^3 periodic sub-problem with the same parameters and velocity recipe."""
    import numpy as np

    from oracle import orc
    from oracle import soe as osoe
    from paper_2411_17294_gb300 import inputs

    W = WORKLOAD
    n = (64, 64, 64)
    dt = W["dt"]
    mu, w = osoe.soe_build(W["alpha"], dt, W["horizon_steps"] * dt, W["m"])
    u, kap = inputs.spectral_velocity(3, n, W["kmax"], W["seed"])
    prob = orc.Problem(dim=3, n=n, alpha=W["alpha"], Wi=W["Wi"], beta=W["beta"], dt=dt, mu=mu, w=w,
                       transport=True)
    o = orc.Oracle(prob)
    o.step(kap, kap, u)                       # warm-up
    t0 = time.perf_counter()
    o.step(kap, kap, u)
    one = time.perf_counter() - t0
    steps = max(steps_hint, int(budget_s / max(one, 1e-3)))
    t0 = time.perf_counter()
    for _ in range(steps):
        o.step(kap, kap, u)
    el = time.perf_counter() - t0
    N = int(np.prod(n))
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": N * W["m"] * steps / el / 1e9, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"64^3 sub-problem, same parameters and velocity recipe, {steps} steps after 1 warm-up, "
                      f"FP64 C oracle with OpenMP", "seconds": el}


def make_stepper(s, world: int, rank: int, stream):
    """One step of this rank's problem: tfs_step on one GPU; with several ranks,
    the slab step of the shared domain (boundary planes exchanged on the ring
    first, on `stream`'s order)."""
    if world == 1:
        return lambda kn, km, u: s.step(kn, km, u, stream=stream)
    from paper_2411_17294_gb300 import slab
    lo, hi = s.halo_buffers()
    rlo, rhi = s.halo_buffers()

    def step(kn, km, u):
        s.get_halo(lo, hi, stream=stream)
        slab.exchange(lo, hi, rlo, rhi, rank, world)
        s.step_slab(kn, km, u, rlo, rhi, stream=stream)
    return step


def end_to_end(s, kap, u, steps: int, stream, dev, stepper=None):
    """Steps fed from pinned host memory as a time-dependent run would be: per
    step the host-to-device copy of that step's velocity gradient kappa^n and
    velocity u, and the device-to-host read of the new stress through
    tfs_get_stress.  kappa^{n-1} is the previous step's kappa^n, already on the
    device.  The copies run on two copy streams, double-buffered, so that the
    inputs of step k+1 and the result of step k-1 move while step k computes.
    Returns (ms, host-to-device bytes per step, device-to-host bytes per step)."""
    import torch
    N = s.N
    tdt = kap.dtype
    h_k = torch.empty(kap.shape, dtype=tdt, pin_memory=True)
    h_u = torch.empty(u.shape, dtype=tdt, pin_memory=True)
    h_k.copy_(kap.cpu())
    h_u.copy_(u.cpu())
    h_sig = [torch.empty((s.nc, N), dtype=tdt, pin_memory=True) for _ in range(2)]
    d_k = [torch.empty_like(kap) for _ in range(3)]      # kappa^n, kappa^{n-1} and the one being loaded
    d_u = [torch.empty_like(u) for _ in range(2)]
    d_sig = [torch.empty((s.nc, N), dtype=tdt, device=dev) for _ in range(2)]
    s_in, s_out = torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)
    ev = lambda: torch.cuda.Event()
    loaded = [ev() for _ in range(steps)]
    stepped = [ev() for _ in range(steps)]
    read = [ev() for _ in range(steps)]
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    s_in.wait_event(e0)
    s_out.wait_event(e0)

    def load(k):
        if k >= 2:
            s_in.wait_event(stepped[k - 2])          # buffers k % 3 and k % 2 were last read by step k - 2
        with torch.cuda.stream(s_in):
            d_k[k % 3].copy_(h_k, non_blocking=True)
            d_u[k % 2].copy_(h_u, non_blocking=True)
        loaded[k].record(s_in)

    load(0)
    for k in range(steps):
        if k + 1 < steps:
            load(k + 1)
        stream.wait_event(loaded[k])
        if k >= 2:
            stream.wait_event(read[k - 2])           # d_sig[k % 2] was read out after step k - 2
        (stepper or (lambda a, b, c: s.step(a, b, c, stream=stream)))(
            d_k[k % 3], d_k[(k - 1) % 3] if k > 0 else d_k[0], d_u[k % 2])
        if s.lib.tfs_get_stress(s.h, d_sig[k % 2].data_ptr(), stream.cuda_stream) != 0:
            raise RuntimeError("tfs_get_stress failed")
        stepped[k].record(stream)
        s_out.wait_event(stepped[k])
        with torch.cuda.stream(s_out):
            h_sig[k % 2].copy_(d_sig[k % 2], non_blocking=True)
        read[k].record(s_out)
    stream.wait_event(read[steps - 1])
    e1.record(stream)
    torch.cuda.synchronize()
    elem = kap.element_size()
    return e0.elapsed_time(e1), (h_k.numel() + h_u.numel()) * elem, h_sig[0].numel() * elem


IMPLICIT = dict(name="implicit transport, 2D periodic 1024^2, m=32 SOE modes, alpha=0.5, dt=5e-4, FP32 storage",
                dim=2, n=(1024, 1024), alpha=0.5, Wi=1.0, beta=0.5, m=32, dt=5e-4, steps=10, warmup=2, kmax=32,
                seed=2)


def implicit_transport_record(dev):
    """The 2D 1024^2 alpha = 0.5 workload with transport at unit-RMS velocity,
    where the explicit transport is unstable, run with implicit transport:
    time per step, BiCGStab iterations per step and the explicit Courant
    fraction (> 1: explicit unstable)."""
    import numpy as np
    import torch

    from paper_2411_17294_gb300 import inputs, soe, tfs
    I = IMPLICIT
    mu, w = soe.build(I["alpha"], I["dt"], 200 * I["dt"], I["m"])
    u, kap = inputs.spectral_velocity(2, I["n"], I["kmax"], I["seed"], device=dev)
    s = tfs.Solver(2, I["n"], I["alpha"], I["Wi"], I["beta"], I["dt"], m=I["m"], precision=tfs.TFS_FP32, mu=mu,
                   w=w, transport="implicit", device=dev)
    kt = torch.as_tensor(kap, dtype=torch.float32, device=dev).contiguous()
    ut = torch.as_tensor(u, dtype=torch.float32, device=dev).contiguous()
    U = s.transport_limit()
    courant = float(torch.max(torch.abs(ut).sum(dim=0)).item()) / (2 * U) if U > 0 else float("inf")
    stream = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(stream):
        s.set_state(None, stream=stream)
        for _ in range(I["warmup"]):
            s.step(kt, kt, ut, stream=stream)
        torch.cuda.synchronize()
        its = []
        t0 = time.perf_counter()
        for _ in range(I["steps"]):
            s.step(kt, kt, ut, stream=stream)      # synchronises its stream (convergence checks)
            its.append(s.last_solve())
        torch.cuda.synchronize()
        ms = (time.perf_counter() - t0) * 1e3 / I["steps"]
    flags = s.status()
    s.close()
    return {"workload": I["name"], "ms_per_step": ms,
            "G_point_mode_updates_per_s": I["n"][0] * I["n"][1] * I["m"] / (ms * 1e-3) / 1e9,
            "krylov_iterations": [it for it, _ in its], "max_relative_residual": max(r for _, r in its),
            "explicit_courant_fraction": courant, "device_flags": flags}


def paper_form_bytes_per_point(dim: int, m: int, elem: int) -> int:
    """Algorithmic bytes of the step kernel in the paper's variable: 3 words per
    (mode, component), both velocity-gradient levels, Phi^n and Phi^{n-1} read,
    Phi^{n+1} and the stress Psi^{n+1} written."""
    nc = 3 if dim == 2 else 6
    return 3 * m * nc * elem + 2 * dim * dim * elem + 4 * nc * elem


def paper_form_record(dev, steps: int, warmup: int, grid: int | None = None):
    """The step in the paper's own variable (Phi, Psi = D^{1-alpha} Phi; the SOE
    approximates g_alpha) on the 3D 256^3 m = 32 FP32 grid of the main workload,
    pointwise (this form carries no transport): time per step and the HBM
    roofline fraction of its step kernel, timed with events around the kernel."""
    import torch

    from paper_2411_17294_gb300 import inputs, soe, tfs
    W = dict(WORKLOAD)
    if grid:
        W["n"] = (grid,) * 3
    dt = W["dt"]
    mu, w = soe.build(1.0 - W["alpha"], dt, W["horizon_steps"] * dt, W["m"])
    _, kap = inputs.spectral_velocity(3, W["n"], W["kmax"], W["seed"], device=dev)
    s = tfs.Solver(3, W["n"], W["alpha"], W["Wi"], W["beta"], dt, m=W["m"], precision=tfs.TFS_FP32, mu=mu, w=w,
                   transport=False, form="paper", device=dev)
    kn = torch.as_tensor(kap, dtype=torch.float32, device=dev).contiguous()
    km = kn.clone()
    del kap
    stream = torch.cuda.Stream(device=dev)
    kb = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ka = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        s.set_state(None, stream=stream)
        for _ in range(warmup):
            s.step(kn, km, stream=stream)
        for e in kb + ka:
            e.record(stream)
        torch.cuda.synchronize()
        e0.record(stream)
        for k in range(steps):
            s.set_step_events(kb[k], ka[k])
            s.step(kn, km, stream=stream)
        e1.record(stream)
    torch.cuda.synchronize()
    s.set_step_events(None, None)
    flags = s.status()
    N = s.N
    s.close()
    launch_ms = statistics.mean(kb[k].elapsed_time(ka[k]) for k in range(steps))
    bpp = paper_form_bytes_per_point(3, W["m"], 4)
    peak, peak_kind = read_peaks()
    achieved = bpp * N / (launch_ms * 1e-3) / 1e9
    return {"workload": f"paper's variable Phi, Psi = D^{{1-alpha}} Phi (Section 3.4), 3D {W['n'][0]}^3, m=32, "
                        "FP32, pointwise (no transport), alpha=0.6, SOE of g_alpha",
            "ms_per_step": e0.elapsed_time(e1) / steps, "avg_launch_ms": launch_ms,
            "G_point_mode_updates_per_s": N * W["m"] / (launch_ms * 1e-3) / 1e9,
            "algorithmic_bytes_per_point": bpp, "achieved_gbs": achieved, "peak": peak, "peak_kind": peak_kind,
            "frac": achieved / peak, "device_flags": flags}


def fp64_record(dev, steps: int, warmup: int, grid: int | None = None):
    """The main workload in the FP64 storage form (everything in double): time
    per step and the HBM roofline fraction of its step kernel against the FP64
    byte count, beside the FP32 headline (the FP32 form is the faster one)."""
    import torch

    from paper_2411_17294_gb300 import inputs, soe, tfs
    W = dict(WORKLOAD)
    if grid:
        W["n"] = (grid,) * 3
    dt = W["dt"]
    mu, w = soe.build(W["alpha"], dt, W["horizon_steps"] * dt, W["m"])
    u, kap = inputs.spectral_velocity(3, W["n"], W["kmax"], W["seed"], device=dev)
    s = tfs.Solver(3, W["n"], W["alpha"], W["Wi"], W["beta"], dt, m=W["m"], precision=tfs.TFS_FP64, mu=mu, w=w,
                   transport=True, device=dev)
    kn = torch.as_tensor(kap, dtype=torch.float64, device=dev).contiguous()
    km = kn.clone()
    ut = torch.as_tensor(u, dtype=torch.float64, device=dev).contiguous()
    del kap, u
    stream = torch.cuda.Stream(device=dev)
    kb = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ka = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        s.set_state(None, stream=stream)
        for _ in range(warmup):
            s.step(kn, km, ut, stream=stream)
        for e in kb + ka:
            e.record(stream)
        torch.cuda.synchronize()
        e0.record(stream)
        for k in range(steps):
            s.set_step_events(kb[k], ka[k])
            s.step(kn, km, ut, stream=stream)
        e1.record(stream)
    torch.cuda.synchronize()
    s.set_step_events(None, None)
    N = s.N
    s.close()
    launch_ms = statistics.mean(kb[k].elapsed_time(ka[k]) for k in range(steps))
    ms = e0.elapsed_time(e1) / steps
    bpp = step_kernel_bytes_per_point(3, W["m"], 8, transport=True)
    peak, peak_kind = read_peaks()
    achieved = bpp * N / (launch_ms * 1e-3) / 1e9
    return {"workload": W["name"].replace("FP32 modes + compensated sum", "FP64 storage and arithmetic"),
            "ms_per_step": ms, "avg_launch_ms": launch_ms,
            "G_point_mode_updates_per_s": N * W["m"] / (ms * 1e-3) / 1e9,
            "algorithmic_bytes_per_point": bpp, "achieved_gbs": achieved, "peak": peak, "peak_kind": peak_kind,
            "frac": achieved / peak, "bound": "fp64 pipe (1/64 of the FP32 rate on this GPU)"}


# beta = 0.9, Wi = 2 (a dilute solution, as the 3D workload): the explicit
# stress divergence of the momentum equation makes the coupled step unstable
# at the highest wavenumbers of this grid when (1 - beta)/(beta Wi) is of order
# one (beta = 0.5, Wi = 1: perturbations grow 16x per step)
NS_COUPLED = dict(name="coupled Navier-Stokes projection + stress step, 2D periodic 1024^2, m=32 SOE modes, alpha=0.5, "
                       "Wi=2, beta=0.9, Re=100, FP32 storage, explicit transport", n=(1024, 1024), alpha=0.5, Wi=2.0,
                  beta=0.9, Re=100.0, m=32, dt=5e-4, kmax=32, seed=2)


def ns_coupled_record(dev, steps: int = 10, warmup: int = 3):
    """The coupled step in the paper's order (Section 4.1): the velocity from the
    stress at t_n by the projection step (tfs_ns_step: 11 FFTs of 1024^2 and the
    per-mode Poisson and Helmholtz solves), then the stress step with that
    velocity.  The initial velocity is the spectral field scaled to 0.3 of the
    explicit transport's limit.  Times per step of both parts (CUDA events)."""
    import torch

    from paper_2411_17294_gb300 import inputs, soe, tfs
    C = NS_COUPLED
    n, dt = C["n"], C["dt"]
    mu, w = soe.build(C["alpha"], dt, 200 * dt, C["m"])
    L = (2 * math.pi, 2 * math.pi)
    st = tfs.Solver(2, n, C["alpha"], C["Wi"], C["beta"], dt, m=C["m"], precision=tfs.TFS_FP32, mu=mu, w=w,
                    transport=True, device=dev, L=L)
    U = st.transport_limit()
    u0, _ = inputs.spectral_velocity(2, n, C["kmax"], C["seed"], device=dev)
    u0 = torch.as_tensor(u0, dtype=torch.float64, device=dev)
    u0 = u0 * (0.3 * U / float(u0.abs().max()))
    ns = tfs.NSSolver(n, L, C["beta"], C["Re"], dt, precision=tfs.TFS_FP32, device=dev)
    stream = torch.cuda.Stream(device=dev)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3 * steps)]
    with torch.cuda.stream(stream):
        ns.set_state(u0.float(), stream=stream)
        st.set_state(None, stream=stream)
        sig = torch.empty((3, st.N), dtype=torch.float32, device=dev)
        u_t = torch.empty((2, st.N), dtype=torch.float32, device=dev)
        k_t = torch.empty((4, st.N), dtype=torch.float32, device=dev)

        def coupled(k=None):
            if k is not None:
                ev[3 * k].record(stream)
            st.lib.tfs_get_stress(st.h, sig.data_ptr(), stream.cuda_stream)
            ns.step(sig, u_t, k_t, stream=stream)
            if k is not None:
                ev[3 * k + 1].record(stream)
            st.step(k_t, k_t, u_t, stream=stream)
            if k is not None:
                ev[3 * k + 2].record(stream)
        for _ in range(warmup):
            coupled()
        torch.cuda.synchronize()
        for k in range(steps):
            coupled(k)
    torch.cuda.synchronize()
    ns_ms = statistics.mean(ev[3 * k].elapsed_time(ev[3 * k + 1]) for k in range(steps))
    st_ms = statistics.mean(ev[3 * k + 1].elapsed_time(ev[3 * k + 2]) for k in range(steps))
    flags = st.status()
    N = st.N
    ns.close()
    st.close()
    return {"workload": C["name"], "ns_ms_per_step": ns_ms, "stress_ms_per_step": st_ms,
            "coupled_ms_per_step": ns_ms + st_ms,
            "G_point_mode_updates_per_s": N * C["m"] / ((ns_ms + st_ms) * 1e-3) / 1e9, "device_flags": flags}


def prepass_record(total_ms: float, launch_ms, steps: int, N: int, elem: int, peak: float) -> dict:
    """The transport pre-pass of the 3D step on one GPU: its time per step is
    the step's time less the step kernel's (the two kernels are the only
    launches of a step and run back to back on one stream; with slabs the step
    also exchanges halos, so no figure is given there); algorithmic bytes per
    point: two stress levels and u read, the transport term written, 84 B in
    FP32."""
    ms = max(total_ms - sum(launch_ms), 0.0) / steps
    bpp = (2 * 6 + 3 + 6) * elem
    gbs = bpp * N / (ms * 1e-3) / 1e9 if ms > 0 else None
    return {"kernel": "transport pre-pass (staged 3D tile, cp.async)", "ms_per_step": ms,
            "algorithmic_bytes_per_point": bpp, "achieved_gbs": gbs,
            "frac": gbs / peak if gbs else None}


def max_over_ranks(local_ms: float, dist, device) -> float:
    """The slowest rank's time (all ranks get it); local_ms itself on one process."""
    if dist is None:
        return local_ms
    import torch
    t = torch.tensor([local_ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, t_max_ms: float) -> float:
    """G units per second for the whole job: every rank processes units_per_rank
    (weak scaling), the job takes as long as its slowest rank."""
    return world * units_per_rank / (t_max_ms * 1e-3) / 1e9


def run_reference(args, rank):
    if rank != 0:
        return
    res = cpu_baseline(steps_hint=max(args.steps, 1), budget_s=20.0)
    line = {"impl": "reference", "metric": METRIC, "value": res["value"], "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD["name"], "sample": res["sample"]},
            "cpu_baseline": {"value": res["value"], "unit": UNIT, "cores": res["cores"], "kind": "oracle",
                             "sample": res["sample"]},
            "e2e": {"value": res["value"], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--adjoint-only", default=None, choices=["fp32", "fp64", "fp32-paper", "fp64-paper"],
                    help="time only the adjoint workload in one precision and print its record (profiling)")
    ap.add_argument("--paper-only", action="store_true",
                    help="time only the step in the paper's variable and print its record (profiling)")
    ap.add_argument("--implicit-only", action="store_true",
                    help="time only the implicit-transport step and print its record (profiling)")
    ap.add_argument("--coupled-only", action="store_true",
                    help="time only the coupled Navier-Stokes + stress step and print its record (profiling)")
    ap.add_argument("--fp64-only", action="store_true",
                    help="time only the FP64 storage form of the step and print its record (profiling)")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64", "fp32plain"])
    ap.add_argument("--grid", type=int, default=WORKLOAD["n"][0],
                    help="cube side of the step workload (default 256; smaller sides are for profiling)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        run_reference(args, rank)
        return
    if args.adjoint_only:
        import torch
        from paper_2411_17294_gb300 import build as tbuild
        from paper_2411_17294_gb300 import tfs
        tbuild.build()
        torch.cuda.set_device(0)
        prec = tfs.TFS_FP32 if args.adjoint_only.startswith("fp32") else tfs.TFS_FP64
        form = "paper" if args.adjoint_only.endswith("paper") else "stress"
        print(json.dumps(adjoint_ratio(torch.device("cuda", 0), prec, form)), flush=True)
        return

    if args.implicit_only:
        import torch
        from paper_2411_17294_gb300 import build as tbuild
        tbuild.build()
        torch.cuda.set_device(0)
        print(json.dumps(implicit_transport_record(torch.device("cuda", 0))), flush=True)
        return
    if args.coupled_only:
        import torch
        from paper_2411_17294_gb300 import build as tbuild
        tbuild.build()
        torch.cuda.set_device(0)
        print(json.dumps(ns_coupled_record(torch.device("cuda", 0))), flush=True)
        return
    if args.fp64_only:
        import torch
        from paper_2411_17294_gb300 import build as tbuild
        tbuild.build()
        torch.cuda.set_device(0)
        print(json.dumps(fp64_record(torch.device("cuda", 0), steps=args.steps, warmup=args.warmup,
                                     grid=args.grid)), flush=True)
        return
    if args.paper_only:
        import torch
        from paper_2411_17294_gb300 import build as tbuild
        tbuild.build()
        torch.cuda.set_device(0)
        print(json.dumps(paper_form_record(torch.device("cuda", 0), steps=args.steps, warmup=args.warmup,
                                           grid=args.grid)), flush=True)
        return

    import numpy as np
    import torch

    from paper_2411_17294_gb300 import build as tbuild
    from paper_2411_17294_gb300 import inputs, soe, tfs

    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    else:
        dist = None
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    if rank == 0:
        tbuild.build()
    if dist is not None:
        dist.barrier()

    W = dict(WORKLOAD)
    if args.grid != WORKLOAD["n"][0]:
        W["n"] = (args.grid,) * 3
        W["name"] = W["name"].replace("256^3", f"{args.grid}^3")
    prec = {"fp32": tfs.TFS_FP32, "fp64": tfs.TFS_FP64, "fp32plain": tfs.TFS_FP32_PLAIN}[args.precision]
    dt = W["dt"]
    mu, w = soe.build(W["alpha"], dt, W["horizon_steps"] * dt, W["m"])
    u64, kap64 = inputs.spectral_velocity(3, W["n"], W["kmax"], W["seed"] + rank, device=dev)
    s = tfs.Solver(3, W["n"], W["alpha"], W["Wi"], W["beta"], dt, m=W["m"], precision=prec, mu=mu, w=w,
                   transport=True, device=dev)
    tdt = s.dtype
    kap_n = torch.as_tensor(kap64, dtype=tdt, device=dev).contiguous()
    kap_nm1 = kap_n.clone()          # frozen velocity, but a distinct buffer: both levels are read
    u = torch.as_tensor(u64, dtype=tdt, device=dev).contiguous()
    del u64, kap64
    U_lim = s.transport_limit()
    courant = float(u.double().abs().sum(dim=0).max()) / (3 * U_lim) if U_lim > 0 else float("inf")
    stream = torch.cuda.Stream(device=dev)
    N = s.N
    elem = 8 if prec == tfs.TFS_FP64 else 4
    bytes_pp = step_kernel_bytes_per_point(3, W["m"], elem, transport=True)
    bytes_launch = bytes_pp * N

    stepper = make_stepper(s, world, rank, stream)
    with torch.cuda.stream(stream):
        s.set_state(None, stream=stream)
        for _ in range(args.warmup):
            stepper(kap_n, kap_nm1, u)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()

    gpu_uuid = None
    try:
        gpu_uuid = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        pass
    sampler = ClockSampler(gpu_uuid)
    sampler.start()
    time.sleep(0.3)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    kb = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ka = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    for e in kb + ka:
        e.record(stream)                        # creates the event handles
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        ev[0].record(stream)
        for k in range(args.steps):
            s.set_step_events(kb[k], ka[k])     # recorded on `stream` around the step kernel only
            stepper(kap_n, kap_nm1, u)
        ev[1].record(stream)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    s.set_step_events(None, None)
    clocks = sampler.stop()
    launch_ms = [kb[k].elapsed_time(ka[k]) for k in range(args.steps)]
    total_ms = ev[0].elapsed_time(ev[1])
    flags = s.status()
    t_max = max_over_ranks(total_ms, dist, dev)
    ms_per_step = t_max / args.steps
    value = whole_job_rate(N * W["m"] * args.steps, world, t_max)
    avg_launch_s = statistics.mean(launch_ms) * 1e-3
    achieved = bytes_launch / avg_launch_s / 1e9
    peak, peak_kind = read_peaks()
    traffic = read_traffic() if prec == tfs.TFS_FP32 else None
    launches_per_step = 2         # transport pre-pass + step kernel (slabs: plus the halo copies)

    # ---- end to end through the C ABI with host buffers ----------------------
    e2e = None
    if args.e2e_steps > 0:
        if dist is not None:
            dist.barrier()
        with torch.cuda.stream(stream):
            e2e_ms, bi, bo = end_to_end(s, kap_n, u, args.e2e_steps, stream, dev, stepper)
        e2e_ms = max_over_ranks(e2e_ms, dist, dev)
        e2e = {"value": whole_job_rate(N * W["m"] * args.e2e_steps, world, e2e_ms), "unit": UNIT,
               "h2d_bytes_per_step": bi, "d2h_bytes_per_step": bo,
               "overlap": "inputs of step k+1 and the result of step k-1 copied on two copy streams during step k"}

    adj = None
    if not args.no_adjoint:
        try:
            adj = [adjoint_ratio(dev, tfs.TFS_FP64), adjoint_ratio(dev, tfs.TFS_FP32),
                   adjoint_ratio(dev, tfs.TFS_FP32, "paper")]
        except Exception as exc:  # pragma: no cover - reported, not fatal
            adj = {"error": str(exc)}

    imp = None
    if not args.no_adjoint:
        try:
            imp = implicit_transport_record(dev)
        except Exception as exc:  # pragma: no cover - reported, not fatal
            imp = {"error": str(exc)}

    paper = None
    if not args.no_adjoint:
        try:
            paper = paper_form_record(dev, steps=10, warmup=3)
        except Exception as exc:  # pragma: no cover - reported, not fatal
            paper = {"error": str(exc)}

    coupled = None
    if not args.no_adjoint:
        try:
            coupled = ns_coupled_record(dev)
        except Exception as exc:  # pragma: no cover - reported, not fatal
            coupled = {"error": str(exc)}

    fp64 = None
    if not args.no_adjoint and prec != tfs.TFS_FP64:
        try:
            fp64 = fp64_record(dev, steps=5, warmup=3, grid=args.grid)
        except Exception as exc:  # pragma: no cover - reported, not fatal
            fp64 = {"error": str(exc)}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        try:
            cpu = cpu_baseline()
            cpu.pop("seconds", None)
        except Exception as exc:  # pragma: no cover - reported, not fatal
            cpu = {"error": str(exc)}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": {tfs.TFS_FP64: "f64", tfs.TFS_FP32: "f32", tfs.TFS_FP32_PLAIN: "f32"}[prec],
            "data": "synthetic",
            "config": {"workload": W["name"], "grid": list(W["n"]), "m": W["m"], "alpha": W["alpha"],
                       "Wi": W["Wi"], "beta": W["beta"], "dt": W["dt"], "transport": True,
                       "precision": args.precision, "l2": f"per-step working set {algorithmic_bytes_per_point(3, W['m'], elem) * N / 1e9:.1f} GB "
                             f">> 129 MB L2, no flush",
                       "points_per_gpu": N,
                       "parallelism": "one GPU" if world == 1 else
                       f"{world} z-slabs of one periodic 256 x 256 x {256 * world} domain, ring halo exchange "
                       "(NCCL point-to-point, 2 planes x 2 levels x 6 components per side per step)"},
            "roofline": {"bound": "hbm", "kernel": "fwd_kernel<float,3> (step kernel)", "achieved": achieved,
                         "peak": peak, "unit": "GB/s", "frac": achieved / peak, "traffic": traffic,
                         "traffic_source": "ncu dram__bytes of the committed capture, used only while the "
                                           "step kernel's sources hash to the captured ones (else null)",
                         "peak_kind": peak_kind, "algorithmic_bytes_per_point": bytes_pp,
                         "algorithmic_bytes_per_launch": bytes_launch, "avg_launch_ms": avg_launch_s * 1e3,
                         "step_share": sum(launch_ms) / total_ms,
                         "whole_step_gbs": algorithmic_bytes_per_point(3, W["m"], elem) * N / (ms_per_step * 1e-3) / 1e9,
                         "prepass": prepass_record(total_ms, launch_ms, args.steps, N, elem, peak) if world == 1
                         else None},
            "gpu_launches": launches_per_step * args.steps,
            "device_flags": flags,
            "stability": {
                "explicit_courant_fraction": courant,
                "note": ("inside the explicit transport's stability region" if courant <= 1.0 else
                         "the velocity exceeds the explicit transport's stability limit (TFS_FLAG_COURANT, "
                         "device_flags & 4): bytes and work per step do not depend on it, but a long run of "
                         "this workload needs the implicit transport (transport=2); the test-suite checks the "
                         "200-step workload pointwise and at a velocity inside the limit")},
            "clocks": clocks,
            "e2e": e2e,
            "adjoint_forward": adj,
            "implicit_transport": imp,
            "paper_form": paper,
            "fp64_form": fp64,
            "ns_coupled": coupled,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    s.close()
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
