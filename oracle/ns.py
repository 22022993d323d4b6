"""FP64 oracle of the Navier-Stokes projection step the stress is coupled to
(Section 4.1), on the periodic square, with Fourier spectral derivatives.

TEST INFRASTRUCTURE ONLY (see the package docstring): a plain NumPy restatement
of the scheme, checked against the Taylor-Green closed form; the library's
GPU step (its own FFT and spectral kernels) is compared with it.

Scheme, one step t_n -> t_{n+1} with the BDF2 coefficients b0 = 3/2, b1 = -2,
b2 = 1/2 and the extrapolation E(f) = 2 f^n - f^{n-1} of eq.
BDF_and_extrapolation (nu = beta/Re; sigma is the polymer extra stress whose
divergence drives the momentum equation, eq. Navier_Stokes):
  Xi = (b1 u^n + b2 u^{n-1})/dt + E(nu curl curl u + (u.grad)u - div sigma)
      (eq. time_discretization_NS, with the viscous term in the rotational form
      of eq. velocity_correction)
  Lap p = -div Xi, mean(p) = 0                      (eq. NS_Poisson, div u^{n+1} = 0)
  (b0/dt) u^{n+1} - nu Lap u^{n+1}
      = -grad p - (b1 u^n + b2 u^{n-1})/dt + E(-(u.grad)u + div sigma)   (eq. NS_Helmholtz)
The first step takes an empty past (u^{-1} = u^0, f^{-1} = f^0), as the stress
step does, unless the level u^{-1} is given (then f^{-1} is formed from it
with no stress).  Derivatives are spectral: d/dx_a multiplies mode k by i k_a,
zero at the Nyquist wavenumber of that axis, and the Laplacian is the square
of that derivative, -(k_x^2 + k_y^2) with the same zeroing, so that div curl
curl = 0 and the projection leave exactly divergence-free fields; products are
formed on the grid (no dealiasing).  The initial velocity is projected onto
divergence-free fields.  Fields are [component][N] with x fastest, N = n0 n1;
the velocity gradient is kappa_ij = du_i/dx_j, row-major [4][N].
"""
from __future__ import annotations

import numpy as np

B0, B1, B2 = 1.5, -2.0, 0.5


class NSOracle:
    def __init__(self, n, L, beta: float, Re: float, dt: float):
        self.n0, self.n1 = int(n[0]), int(n[1])
        self.L = (float(L[0]), float(L[1]))
        self.nu = beta / Re
        self.dt = dt
        kx = np.fft.fftfreq(self.n0, d=1.0 / self.n0) * (2 * np.pi / self.L[0])
        ky = np.fft.fftfreq(self.n1, d=1.0 / self.n1) * (2 * np.pi / self.L[1])
        # grids [y][x] (x fastest in memory)
        dx, dy = kx.copy(), ky.copy()
        if self.n0 % 2 == 0:
            dx[self.n0 // 2] = 0.0
        if self.n1 % 2 == 0:
            dy[self.n1 // 2] = 0.0
        self.DX, self.DY = np.meshgrid(1j * dx, 1j * dy)     # first-derivative multipliers
        self.K2 = -(self.DX ** 2 + self.DY ** 2).real         # -Laplacian
        self.step_index = 0

    # ---- helpers on [y][x] arrays
    def _hat(self, f):
        return np.fft.fft2(np.asarray(f, dtype=np.float64).reshape(self.n1, self.n0))

    def _real(self, fh):
        return np.real(np.fft.ifft2(fh)).reshape(-1)

    def _project(self, u):
        """Spectral components of the divergence-free part of u (mode 0 kept)."""
        u = np.asarray(u, dtype=np.float64).reshape(2, -1)
        uh = [self._hat(u[0]), self._hat(u[1])]
        div = self.DX * uh[0] + self.DY * uh[1]
        with np.errstate(divide="ignore", invalid="ignore"):
            phi = np.where(self.K2 > 0, div / -self.K2, 0.0)
        return [uh[0] - self.DX * phi, uh[1] - self.DY * phi]

    def set_state(self, u0, u_prev=None):
        self.uh = self._project(u0)
        if u_prev is None:
            self.uh_prev = [self.uh[0].copy(), self.uh[1].copy()]
            self.f_prev = None      # explicit terms of the previous level: the current ones (empty past)
        else:
            self.uh_prev = self._project(u_prev)
            self.f_prev = self._explicit_terms(None, self.uh_prev)
        self.step_index = 0

    def velocity(self, uh=None):
        u = self.uh if uh is None else uh
        return np.stack([self._real(u[0]), self._real(u[1])])

    def gradient(self, uh=None):
        """kappa_ij = du_i/dx_j, [4][N]: (dux/dx, dux/dy, duy/dx, duy/dy)."""
        u = self.uh if uh is None else uh
        return np.stack([self._real(self.DX * u[0]), self._real(self.DY * u[0]),
                         self._real(self.DX * u[1]), self._real(self.DY * u[1])])

    def _explicit_terms(self, sigma, uh=None):
        """Spectral curl curl u, (u.grad)u and div sigma of a level (the current one by default)."""
        u = self.uh if uh is None else uh
        # curl curl u = grad(div u) - Lap u
        div = self.DX * u[0] + self.DY * u[1]
        cc = [self.DX * div + self.K2 * u[0], self.DY * div + self.K2 * u[1]]
        vel = self.velocity(u)
        g = self.gradient(u)
        conv = [self._hat(vel[0] * g[0] + vel[1] * g[1]), self._hat(vel[0] * g[2] + vel[1] * g[3])]
        if sigma is None:
            ds = [np.zeros_like(u[0]), np.zeros_like(u[0])]
        else:
            s = np.asarray(sigma, dtype=np.float64).reshape(3, -1)      # xx, xy, yy
            sh = [self._hat(s[0]), self._hat(s[1]), self._hat(s[2])]
            ds = [self.DX * sh[0] + self.DY * sh[1], self.DX * sh[1] + self.DY * sh[2]]
        return cc, conv, ds

    def step(self, sigma=None):
        """Advance the velocity by one step with the stress sigma at t_n
        ([3][N] packed xx, xy, yy, or None); returns u^{n+1}, kappa^{n+1}."""
        dt, nu = self.dt, self.nu
        cc, conv, ds = self._explicit_terms(sigma)
        cur = (cc, conv, ds)
        prev = cur if self.f_prev is None else self.f_prev
        ext = lambda a, b: 2.0 * a - b
        hist = [(B1 * self.uh[a] + B2 * self.uh_prev[a]) / dt for a in range(2)]
        xi = [hist[a] + ext(nu * cc[a] + conv[a] - ds[a], nu * prev[0][a] + prev[1][a] - prev[2][a])
              for a in range(2)]
        # Lap p = -div Xi, mean zero
        rhs = -(self.DX * xi[0] + self.DY * xi[1])
        with np.errstate(divide="ignore", invalid="ignore"):
            ph = np.where(self.K2 > 0, rhs / -self.K2, 0.0)
        grad_p = [self.DX * ph, self.DY * ph]
        new = []
        for a in range(2):
            r = -grad_p[a] - hist[a] + ext(-conv[a] + ds[a], -prev[1][a] + prev[2][a])
            new.append(r / (B0 / dt + nu * self.K2))
        self.f_prev = cur
        self.uh_prev = self.uh
        self.uh = new
        self.step_index += 1
        return self.velocity(), self.gradient()
