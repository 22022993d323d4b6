"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle runs.

This module holds none of the stress scheme's arithmetic: it only draws
reproducible velocity fields, velocity gradients and initial stresses on a
periodic grid.  The paper's own workloads are finite-element meshes that are
not available; these periodic fields stand in for them.

Layouts (x fastest, point index p = x + nx (y + ny z)):
    u      [d][N]      velocity
    kappa  [d*d][N]    velocity gradient, component i*d + j = d u_i / d x_j
    sigma  [nc][N]     packed symmetric stress, 2D (xx, xy, yy),
                       3D (xx, yy, zz, yz, xz, xy)

All generators return FP64 NumPy arrays.
"""
from __future__ import annotations

import numpy as np


def grid_points(n) -> int:
    return int(np.prod(n))


def ncomp(dim: int) -> int:
    return 3 if dim == 2 else 6


def _coords(n, L):
    axes = [np.arange(k) * (Lk / k) for k, Lk in zip(n, L)]
    # index order (z, y, x) so that x is fastest after ravel
    mesh = np.meshgrid(*axes[::-1], indexing="ij")
    return [m.ravel() for m in mesh[::-1]]          # x, y(, z)


def taylor_green(n, seed: int = 1, noise: float = 1e-3):
    """2D Taylor-Green velocity u = (sin x cos y, -cos x sin y) on [0, 2pi)^2
    with its analytic gradient plus seeded N(0, noise^2) noise on the gradient.
    Returns (u [2][N], kappa [4][N])."""
    n = tuple(int(k) for k in n)
    x, y = _coords(n, (2 * np.pi, 2 * np.pi))
    u = np.stack([np.sin(x) * np.cos(y), -np.cos(x) * np.sin(y)])
    kap = np.stack([
        np.cos(x) * np.cos(y),          # du/dx
        -np.sin(x) * np.sin(y),         # du/dy
        np.sin(x) * np.sin(y),          # dv/dx
        -np.cos(x) * np.cos(y),         # dv/dy
    ])
    rng = np.random.default_rng(seed)
    kap = kap + rng.normal(0.0, noise, size=kap.shape)
    return np.ascontiguousarray(u), np.ascontiguousarray(kap)


def spectral_velocity(dim: int, n, kmax: int, seed: int, device=None):
    """Divergence-free random Fourier velocity on [0, 2pi)^dim.

    Modes with 0 < |k| <= kmax get energy |k|^(-5/3) divided by the number of
    integer wavevectors in their shell (so each shell carries a k^(-5/3)
    spectrum), uniform random phases (NumPy default_rng(seed)), and are projected
    onto divergence-free vectors (I - k k^T/|k|^2).  The real part of the
    inverse transform is the field, rescaled to unit RMS of |u|.  The gradient
    is the exact spectral derivative of that field.
    Returns (u [d][N], kappa [d*d][N]) as FP64 NumPy arrays.  With `device`
    (a torch device) the inverse transforms run there with torch.fft."""
    n = tuple(int(k) for k in n)
    assert len(n) == dim
    rng = np.random.default_rng(seed)
    kint = [np.fft.fftfreq(nk, d=1.0 / nk) for nk in n]
    # wavevector components as arrays over the (z, y, x) index order
    grids = np.meshgrid(*kint[::-1], indexing="ij")
    kvec = grids[::-1]                                  # kx, ky(, kz)
    kk = np.sqrt(sum(k * k for k in kvec))
    shell = np.rint(kk).astype(np.int64)
    active = (kk > 0) & (kk <= kmax)
    mult = np.bincount(shell[active], minlength=kmax + 2).astype(np.float64)
    energy = np.zeros(kk.shape)
    energy[active] = kk[active] ** (-5.0 / 3.0) / mult[shell[active]]
    amp = np.sqrt(energy)
    coeffs = []
    for _ in range(dim):
        phase = rng.uniform(0.0, 2 * np.pi, size=kk.shape)
        gauss = rng.normal(size=kk.shape)
        coeffs.append(amp * gauss * np.exp(1j * phase))
    # projection onto divergence-free fields
    kk_safe = np.where(kk > 0, kk, 1.0)
    kdotc = sum(kvec[a] * coeffs[a] for a in range(dim)) / (kk_safe ** 2)
    uhat = [np.where(active, coeffs[a] - kvec[a] * kdotc, 0.0) for a in range(dim)]

    if device is None:
        def ifft(a):
            return np.real(np.fft.ifftn(a))
        def to_np(a):
            return a
    else:
        import torch

        def ifft(a):
            t = torch.from_numpy(np.ascontiguousarray(a)).to(device)
            return torch.fft.ifftn(t).real

        def to_np(a):
            return a.cpu().numpy()

    u = [ifft(uhat[a]) for a in range(dim)]
    rms = float(np.sqrt(sum(float((to_np(ua) ** 2).mean()) for ua in u)))
    scale = 1.0 / rms
    u_out = np.stack([to_np(ua).ravel() * scale for ua in u])
    kap = []
    for i in range(dim):
        for j in range(dim):
            kap.append(to_np(ifft(1j * kvec[j] * uhat[i])).ravel() * scale)
    return np.ascontiguousarray(u_out), np.ascontiguousarray(np.stack(kap))


def random_stress(dim: int, n, seed: int, amplitude: float = 1.0):
    """Smooth seeded symmetric stress field: a few low Fourier modes per
    component.  Returns sigma [nc][N]."""
    n = tuple(int(k) for k in n)
    rng = np.random.default_rng(seed)
    coords = _coords(n, (2 * np.pi,) * dim)
    nc = ncomp(dim)
    out = np.zeros((nc, grid_points(n)))
    for c in range(nc):
        out[c] += amplitude * rng.normal()
        for _ in range(3):
            k = rng.integers(-2, 3, size=dim)
            ph = rng.uniform(0, 2 * np.pi)
            out[c] += 0.3 * amplitude * rng.normal() * np.cos(sum(k[a] * coords[a] for a in range(dim)) + ph)
    return out


def uniform_kappa(dim: int, n, kappa_matrix):
    """The same velocity gradient (d x d matrix) at every point: [d*d][N]."""
    km = np.asarray(kappa_matrix, dtype=np.float64).reshape(dim * dim)
    return np.ascontiguousarray(np.repeat(km[:, None], grid_points(n), axis=1))


def uniform_velocity(dim: int, n, u_vec):
    uv = np.asarray(u_vec, dtype=np.float64).reshape(dim)
    return np.ascontiguousarray(np.repeat(uv[:, None], grid_points(n), axis=1))


def ramp(t: float) -> float:
    """Smooth start from rest: sin^2(pi/2 min(max(0, 4t - 1), 1)), the forcing
    ramp of the coupled convergence study (Section 5.1)."""
    s = min(max(0.0, 4.0 * t - 1.0), 1.0)
    return float(np.sin(0.5 * np.pi * s) ** 2)
