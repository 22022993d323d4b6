"""The scheme in the paper's own variable (oracle side), pointwise law.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Section 3.4 (eq. macroscopic_fokker_planck) advances the Hermite coefficients
Phi with a time derivative on Phi and the fractional operator on the right:

    d Phi/dt = (A(grad u) - (u.grad - eps Lap)) Psi,      Psi := D^{1-alpha} Phi,

D^{1-alpha} f = d/dt (g_alpha * f) with g_alpha(t) = t^(alpha-1)/Gamma(alpha)
(Section 1).  For the degree-2 block, in the stress units of the oracle's
stress form (the coupling of eq. mm_coupling_order2 with relaxation rate 1/Wi,
Wi the relaxation time, and the Oldroyd-B source sqrt2 kappa_ii on the
diagonal entries of eq. conf_op_tested, which is kappa + kappa^T in stress
units),

    d Phi2/dt = L(kappa) Psi2 - Psi2/Wi + G (kappa + kappa^T) Psi0,   L(k) s = k s + s k^T,

and the stress is Psi2; Phi0 == 1, so Psi0 = D^{1-alpha} 1 (= g_alpha(t)
exactly).  Kernel compression (Section 2.2) replaces g_alpha by sum_j w_j
exp(-mu_j t), i.e. Psi = sum_j w_j (-mu_j phi_j + Phi) with the mode ODEs
d phi_j/dt = -mu_j phi_j + Phi (phi_j(0) = 0), and every ODE is advanced by
BDF2 (Section 4.1):

    phi_j^{n+1} = c_j (-b1 phi_j^n - b2 phi_j^{n-1} + dt Phi^{n+1}),   c_j = 1/(b0 + mu_j dt)
    Psi^{n+1}   = xi Phi^{n+1} + h^n,   xi = b0 sum_j w_j c_j,
                  h^n = sum_j w_j mu_j c_j (b1 phi_j^n + b2 phi_j^{n-1})
    (b0 I - dt xi (L(kappa*) - I/Wi)) Phi2^{n+1}
        = -b1 Phi2^n - b2 Phi2^{n-1} + dt (L(kappa*) - I/Wi) h2^n + dt G (kappa* + kappa*^T) Psi0^{n+1}

(kappa* = 2 kappa^n - kappa^{n-1}, eq. BDF_and_extrapolation); Psi0 comes from
the same recurrence with Phi0 = 1.  The SOE of g_alpha is that of the Caputo
kernel of order 1 - alpha (t^(alpha-1)/Gamma(alpha) = t^-(1-alpha)/Gamma(alpha)),
so the tables of oracle.soe with order 1 - alpha serve.  Zero past: Phi^{-1} =
Phi^0, phi_j^0 = phi_j^{-1} = 0, Psi^0 = Psi^{-1} = 0.

Transport (optional, on a periodic grid): the operator (u.grad - eps Lap) acts
on Psi; taken explicitly on the extrapolation E = 2 Psi^n - Psi^{n-1} (the
choice the stress form makes for sigma), it adds -dt (sum_a u_a D_a E - eps Lap E)
to the right-hand side, with D_a the upwind-biased third-order difference
(radius 2, biased by the sign of u_a at the point) or the central second-order
one, and Lap the three-point Laplacian per axis, periodic (numpy.roll).
Implicit transport (the form of eq. FP_discrete): the operator acts on
Psi^{n+1} = xi Phi^{n+1} + h^n inside the solve,
    (b0 I - dt xi (L(kappa*) - I/Wi)) Phi + dt xi T(Phi)
        = -b1 Phi^n - b2 Phi^{n-1} + dt (L(kappa*) - I/Wi) h + dt G (kappa* + kappa*^T) Psi0 - dt T(h),
T = u.grad - eps Lap with the same stencils; the global system is assembled
densely from unit vectors (small grids only) and solved with numpy.linalg.solve.
The per-point systems are assembled column by column from unit vectors and
solved with numpy.linalg.solve.
"""
from __future__ import annotations

import numpy as np

B0, B1, B2 = 1.5, -2.0, 0.5


def packed_pairs(dim):
    return [(0, 0), (0, 1), (1, 1)] if dim == 2 else [(0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1)]


def upper_convected(dim, K, s):
    """L(K) s for packed symmetric s, K [N, d, d], s [nc, N] -> [nc, N]."""
    P = packed_pairs(dim)
    N = s.shape[1]
    S = np.zeros((N, dim, dim))
    for c, (i, j) in enumerate(P):
        S[:, i, j] = s[c]
        S[:, j, i] = s[c]
    T = K @ S + S @ np.swapaxes(K, 1, 2)
    return np.stack([T[:, i, j] for (i, j) in P])


def transport_op(dim, grid, L, eps, stencil, E, u):
    """sum_a u_a D_a E - eps Lap E for E [nc][N], u [d][N] on the periodic grid
    (x fastest), box lengths L: D_a upwind-biased third order (radius 2, biased
    by the sign of u_a at the point; stencil 0) or central second order
    (stencil 1), Lap the three-point Laplacian per axis (numpy.roll)."""
    d = dim
    nc = E.shape[0]
    shp = (nc,) + tuple(reversed(grid))                          # [nc][(z)][y][x]
    F = E.reshape(shp)
    U = np.asarray(u, float).reshape((d,) + tuple(reversed(grid)))
    out = np.zeros(shp)
    for a in range(d):
        ax = F.ndim - 1 - a                                      # x is the last array axis
        h = L[a] / grid[a]
        at = lambda k: np.roll(F, -k, axis=ax)                   # F at offset k along axis a
        ua = U[a][None]
        if stencil == 1:
            D = (at(1) - at(-1)) / (2 * h)
        else:
            fw = (at(-2) - 6 * at(-1) + 3 * F + 2 * at(1)) / (6 * h)
            bw = (-2 * at(-1) - 3 * F + 6 * at(1) - at(2)) / (6 * h)
            D = np.where(ua >= 0, fw, bw)
        out += ua * D
        if eps != 0.0:
            out -= eps * (at(-1) - 2 * F + at(1)) / h ** 2
    return out.reshape(nc, -1)


class PaperForm:
    """State of the paper-variable scheme on a set of independent points."""

    def __init__(self, dim, N, Wi, beta, dt, mu, w, Phi0=None, Re=1.0, start="bdf2", grid=None, L=None,
                 eps=0.0, stencil=0, implicit=False):
        self.dim, self.N = dim, N
        # transport: grid shape (x fastest), box lengths, eps, stencil (0 upwind3, 1 central2)
        self.grid = tuple(grid) if grid is not None else None
        if self.grid is not None and int(np.prod(self.grid)) != N:
            raise ValueError("grid does not match N")
        self.L = tuple(L) if L is not None else (2 * np.pi,) * dim
        self.eps, self.stencil = eps, stencil
        self.implicit = implicit
        self.nc = 3 if dim == 2 else 6
        self.Wi, self.dt = Wi, dt
        self.G = (1.0 - beta) / (Wi * Re)
        self.mu = np.asarray(mu, float)
        self.w = np.asarray(w, float)
        self.c = 1.0 / (B0 + self.mu * dt)
        self.xi = B0 * np.sum(self.w * self.c)
        m = len(self.mu)
        z = np.zeros((self.nc, N)) if Phi0 is None else np.asarray(Phi0, float).reshape(self.nc, N).copy()
        self.Phi_n, self.Phi_nm1 = z.copy(), z.copy()
        self.phi_n = np.zeros((m, self.nc, N))
        self.phi_nm1 = np.zeros((m, self.nc, N))
        self.phi0_n = np.zeros(m)        # modes of Phi0 == 1
        self.phi0_nm1 = np.zeros(m)
        self.kap_prev = None
        self.Psi = None
        self.Psi_n = np.zeros((self.nc, N))
        self.Psi_nm1 = np.zeros((self.nc, N))
        self.start = start       # first step: "bdf2" (empty past) or "sdirk2" (Section 5.1)
        self.n = 0

    def _h(self, phi_n, phi_nm1):
        wmc = self.w * self.mu * self.c
        return np.tensordot(wmc, B1 * phi_n + B2 * phi_nm1, axes=(0, 0))

    def _solve(self, K, scale, rhs):
        """Solve (I - scale (L(K) - I/Wi)) X = rhs per point (unit-vector assembly)."""
        d, N, nc = self.dim, self.N, self.nc
        M = np.zeros((N, nc, nc))
        for k in range(nc):
            e = np.zeros((nc, N))
            e[k] = 1.0
            M[:, :, k] = (e - scale * (upper_convected(d, K, e) - e / self.Wi)).T
        return np.linalg.solve(M, rhs.T[..., None])[..., 0].T

    def _sdirk2_first_step(self, K, u=None):
        """Two-stage SDIRK2 (gamma = 1 - 1/sqrt2, stiffly accurate) on the ODE system
        d Phi/dt = (L - I/Wi) Psi + G (K + K^T) Psi0,  d phi_j/dt = -mu_j phi_j + Phi,
        Psi = sum_j w_j (-mu_j phi_j + Phi).  At a stage with explicit parts ZPhi,
        Zphi_j: phi_j = (Zphi_j + g dt Phi)/(1 + g mu_j dt), so Psi = xi' Phi - h',
        xi' = sum_j w_j/(1 + g mu_j dt), h' = sum_j w_j mu_j Zphi_j/(1 + g mu_j dt), and
        (I - g dt xi' (L - I/Wi)) Phi = ZPhi - g dt (L - I/Wi) h' + g dt G (K + K^T) Psi0;
        with implicit transport T = u.grad - eps Lap acting on Psi = xi' Phi - h' the
        left side gains g dt xi' T(Phi) and the right side g dt T(h') (global solve)."""
        d, dt = self.dim, self.dt
        g = 1.0 - np.sqrt(0.5)
        den = 1.0 + g * self.mu * dt
        xi1 = np.sum(self.w / den)
        P = packed_pairs(d)
        KS = K + np.swapaxes(K, 1, 2)
        src = np.stack([KS[:, i, j] for (i, j) in P])
        ZPhi, Zphi, Zphi0 = self.Phi_n.copy(), self.phi_n.copy(), self.phi0_n.copy()
        for stage in (1, 2):
            h1 = np.tensordot(self.w * self.mu / den, Zphi, axes=(0, 0))
            psi0 = xi1 - float(np.sum(self.w * self.mu * Zphi0 / den))
            Lh = upper_convected(d, K, h1) - h1 / self.Wi
            rhs = ZPhi - g * dt * Lh + g * dt * self.G * src * psi0
            if u is not None:
                Phi = self._solve_implicit(K, rhs + g * dt * self._transport_op(h1, u), u, 1.0, g * dt * xi1)
            else:
                Phi = self._solve(K, g * dt * xi1, rhs)
            phi = (Zphi + g * dt * Phi[None]) / den[:, None, None]
            phi0 = (Zphi0 + g * dt * 1.0) / den
            if stage == 1:
                KPhi = (Phi - ZPhi) / (g * dt)
                Kphi = -self.mu[:, None, None] * phi + Phi[None]
                Kphi0 = -self.mu * phi0 + 1.0
                ZPhi = self.Phi_n + dt * (1.0 - g) * KPhi
                Zphi = self.phi_n + dt * (1.0 - g) * Kphi
                Zphi0 = self.phi0_n + dt * (1.0 - g) * Kphi0
        Psi = xi1 * Phi - h1
        return Phi, phi, phi0, Psi

    def _transport(self, E, u):
        """dt (sum_a u_a D_a E - eps Lap E) for E [nc][N], u [d][N], periodic."""
        return self.dt * self._transport_op(E, u)

    def _transport_op(self, E, u):
        """sum_a u_a D_a E - eps Lap E for E [nc][N], u [d][N], periodic."""
        return transport_op(self.dim, self.grid, self.L, self.eps, self.stencil, E, u)

    def _solve_implicit(self, K, rhs, u, diag=B0, scale=None):
        """Solve (diag I - scale (L(K) - I/Wi)) Phi + scale T(Phi) = rhs over the grid (dense);
        scale defaults to dt xi (the BDF2 step)."""
        d, N, nc, dt = self.dim, self.N, self.nc, self.dt
        if scale is None:
            scale = dt * self.xi
        n = nc * N
        A = np.zeros((n, n))
        for k in range(n):
            e = np.zeros((nc, N))
            e.flat[k] = 1.0
            img = diag * e - scale * (upper_convected(d, K, e) - e / self.Wi)
            img = img + scale * self._transport_op(e, u)
            A[:, k] = img.ravel()
        return np.linalg.solve(A, rhs.ravel()).reshape(nc, N)

    def step(self, kap_n, kap_nm1=None, u=None):
        """Advance one step; returns the stress Psi2^{n+1} [nc][N].  u [d][N]
        turns the transport on (grid required)."""
        d, N, nc, dt = self.dim, self.N, self.nc, self.dt
        if u is not None and self.grid is None:
            raise ValueError("transport needs the grid")
        if self.start == "sdirk2" and self.n == 0:
            if u is not None and not self.implicit:
                raise ValueError("the SDIRK2 start takes the transport implicitly only")
            kap0 = np.asarray(kap_n, float).reshape(d * d, N)
            Phi, phi, phi0, Psi = self._sdirk2_first_step(kap0.T.reshape(N, d, d), u)
            self.Psi = Psi
            self.Psi_nm1, self.Psi_n = self.Psi_n, Psi
            self.Phi_nm1, self.Phi_n = self.Phi_n, Phi
            self.phi_nm1, self.phi_n = self.phi_n, phi
            self.phi0_nm1, self.phi0_n = self.phi0_n, phi0
            self.kap_prev = kap0
            self.n += 1
            return Psi.copy()
        kap_n = np.asarray(kap_n, float).reshape(d * d, N)
        if kap_nm1 is None:
            kap_nm1 = self.kap_prev if self.kap_prev is not None else kap_n
        kap_nm1 = np.asarray(kap_nm1, float).reshape(d * d, N)
        K = (2.0 * kap_n - kap_nm1).T.reshape(N, d, d)
        # degree 0: Phi0 = 1, Psi0^{n+1} = xi + h0^n
        h0 = float(np.sum(self.w * self.mu * self.c * (B1 * self.phi0_n + B2 * self.phi0_nm1)))
        psi0 = self.xi * 1.0 + h0
        # degree 2
        h = self._h(self.phi_n, self.phi_nm1)
        Lh = upper_convected(d, K, h) - h / self.Wi
        P = packed_pairs(d)
        KS = K + np.swapaxes(K, 1, 2)
        src = np.stack([KS[:, i, j] for (i, j) in P])
        rhs = -B1 * self.Phi_n - B2 * self.Phi_nm1 + dt * Lh + dt * self.G * src * psi0
        if u is not None and self.implicit:
            Phi = self._solve_implicit(K, rhs - self._transport(h, u), u)
        elif u is not None:
            rhs = rhs - self._transport(2.0 * self.Psi_n - self.Psi_nm1, u)
        # system matrix per point: b0 I - dt xi (L(K) - I/Wi), column k = image of unit vector k
        if not (u is not None and self.implicit):
            M = np.zeros((N, nc, nc))
            for k in range(nc):
                e = np.zeros((nc, N))
                e[k] = 1.0
                img = B0 * e - dt * self.xi * (upper_convected(d, K, e) - e / self.Wi)
                M[:, :, k] = img.T
            Phi = np.linalg.solve(M, rhs.T[..., None])[..., 0].T
        phi_new = self.c[:, None, None] * (-B1 * self.phi_n - B2 * self.phi_nm1 + dt * Phi[None])
        phi0_new = self.c * (-B1 * self.phi0_n - B2 * self.phi0_nm1 + dt * 1.0)
        self.Psi = self.xi * Phi + h
        self.Psi_nm1, self.Psi_n = self.Psi_n, self.Psi
        self.Phi_nm1, self.Phi_n = self.Phi_n, Phi
        self.phi_nm1, self.phi_n = self.phi_n, phi_new
        self.phi0_nm1, self.phi0_n = self.phi0_n, phi0_new
        self.kap_prev = kap_n
        self.n += 1
        return self.Psi.copy()


def paper_gradients(dim, N, Wi, beta, dt, mu, w, Phi0, kap, steps, dJ, Re=1.0, u=None, grid=None, L=None, eps=0.0,
                    stencil=0, implicit=False):
    """Reverse-mode derivatives of J = <dJ, Psi^steps> for the BDF2 start and a
    frozen velocity gradient kap [d*d][N] (kappa* = kappa), pointwise or with
    transport (u, grid as for PaperForm; explicit on 2 Psi^n - Psi^{n-1}, or
    implicit): returns dict(Psi_T, Phi0, kappa, Wi, beta).  Plain reverse sweep
    of the step above, one linear operation at a time (no combination of terms):

        h      = sum_j w_j mu_j c_j (b1 phi_j^n + b2 phi_j^{n-1})
        rhs    = -b1 Phi^n - b2 Phi^{n-1} + dt (L h - h/Wi) + dt G k Psi0^{n+1}
        Phi^{n+1} = M^-1 rhs,  M = b0 I - dt xi (L - I/Wi)
        phi_j^{n+1} = c_j (-b1 phi_j^n - b2 phi_j^{n-1} + dt Phi^{n+1})
        Psi^{n+1} = xi Phi^{n+1} + h

    (k = kappa + kappa^T, G = (1 - beta)/(Wi Re)); Phi^{-1} = Phi^0 = Phi0 and
    the modes start at zero.  Explicit transport subtracts dt T(2 Psi^n -
    Psi^{n-1}) from rhs; implicit transport adds dt xi T to M and subtracts
    dt T(h) from rhs (T = u.grad - eps Lap, assembled densely from unit
    vectors: small grids only).  The kappa derivative of L(kappa) X is taken by
    unit perturbations of kappa, one entry at a time."""
    d = dim
    nc = 3 if d == 2 else 6
    mu = np.asarray(mu, float)
    w = np.asarray(w, float)
    c = 1.0 / (B0 + mu * dt)
    xi = B0 * np.sum(w * c)
    G = (1.0 - beta) / (Wi * Re)
    kap = np.asarray(kap, float).reshape(d * d, N)
    K = kap.T.reshape(N, d, d)
    P = packed_pairs(d)
    KS = K + np.swapaxes(K, 1, 2)
    ks = np.stack([KS[:, i, j] for (i, j) in P])
    # forward, keeping what the reverse sweep reads
    pf = PaperForm(dim, N, Wi, beta, dt, mu, w, Phi0=Phi0, Re=Re, grid=grid, L=L, eps=eps, stencil=stencil,
                   implicit=implicit)
    hist = []
    for _ in range(steps):
        h0 = float(np.sum(w * mu * c * (B1 * pf.phi0_n + B2 * pf.phi0_nm1)))
        psi0 = xi + h0
        h = np.tensordot(w * mu * c, B1 * pf.phi_n + B2 * pf.phi_nm1, axes=(0, 0))
        psi = pf.step(kap, kap, u)
        hist.append((pf.Phi_n.copy(), h, psi0))
    nn = nc * N
    Tm = None
    if u is not None:
        Tm = np.zeros((nn, nn))        # column k = T applied to unit vector k
        for k in range(nn):
            e = np.zeros((nc, N))
            e.flat[k] = 1.0
            Tm[:, k] = pf._transport_op(e, u).ravel()
    TT = lambda v: (Tm.T @ v.ravel()).reshape(nc, N)
    # per-point matrix M and its transpose
    M = np.zeros((N, nc, nc))
    for k in range(nc):
        e = np.zeros((nc, N))
        e[k] = 1.0
        M[:, :, k] = (B0 * e - dt * xi * (upper_convected(d, K, e) - e / Wi)).T
    Mt = np.swapaxes(M, 1, 2)
    AT = None
    if u is not None and implicit:
        A = np.zeros((nn, nn))
        for k in range(nn):
            e = np.zeros((nc, N))
            e.flat[k] = 1.0
            A[:, k] = (B0 * e - dt * xi * (upper_convected(d, K, e) - e / Wi)).ravel()
        A += dt * xi * Tm
        AT = A.T

    def L_T(v):
        """L(kappa)^T v per point: column k of L is L(kappa) e_k."""
        out = np.zeros((nc, N))
        for k in range(nc):
            e = np.zeros((nc, N))
            e[k] = 1.0
            out[k] = np.sum(upper_convected(d, K, e) * v, axis=0)
        return out

    def dL_dot(v, X):
        """[d*d][N]: entry (a, b) = v . (d/dkappa_ab) L(kappa) X = v . L(E_ab) X."""
        out = np.zeros((d * d, N))
        for a in range(d):
            for b in range(d):
                E = np.zeros((N, d, d))
                E[:, a, b] = 1.0
                out[a * d + b] = np.sum(v * upper_convected(d, E, X), axis=0)
        return out

    m = len(mu)
    aPhi1 = np.zeros((nc, N))          # adjoint of Phi^{n+1}
    aPhi0 = np.zeros((nc, N))          # partial adjoint of Phi^n (from step n+1)
    aphi1 = np.zeros((m, nc, N))       # adjoint of phi_j^{n+1}
    aphi0 = np.zeros((m, nc, N))       # partial adjoint of phi_j^n
    aPsi1 = np.zeros((nc, N))          # explicit transport: adjoint of Psi^{n+1} from later steps
    aPsi0 = np.zeros((nc, N))          # and the partial one of Psi^n
    g_kap = np.zeros((d * d, N))
    gWi = gbeta = 0.0
    for n in range(steps - 1, -1, -1):
        Phi_new, h, psi0 = hist[n]
        aPsi = aPsi1 + (np.asarray(dJ, float).reshape(nc, N) if n == steps - 1 else 0.0)
        # Psi^{n+1} = xi Phi^{n+1} + h;  phi_j^{n+1} = c_j (... + dt Phi^{n+1})
        aPhi_new = aPhi1 + xi * aPsi + dt * np.tensordot(c, aphi1, axes=(0, 0))
        ah = aPsi.copy()
        # Phi^{n+1} = M^-1 rhs (implicit transport: the dense operator)
        if AT is not None:
            arhs = np.linalg.solve(AT, aPhi_new.ravel()).reshape(nc, N)
        else:
            arhs = np.linalg.solve(Mt, aPhi_new.T[..., None])[..., 0].T
        # rhs = -b1 Phi^n - b2 Phi^{n-1} + dt (L h - h/Wi) + dt G k psi0 [- dt T(h) | - dt T(2 Psi^n - Psi^{n-1})]
        ah += dt * (L_T(arhs) - arhs / Wi)
        if AT is not None:
            ah -= dt * TT(arhs)
        if u is not None and not implicit:
            aPsi1, aPsi0 = aPsi0 - 2.0 * dt * TT(arhs), dt * TT(arhs)
        new_aPhi1 = aPhi0 - B1 * arhs
        new_aPhi0 = -B2 * arhs
        # h = sum_j w_j mu_j c_j (b1 phi_j^n + b2 phi_j^{n-1}); phi_j^{n+1} = c_j (-b1 phi_j^n - b2 phi_j^{n-1} + ...)
        wmc = (w * mu * c)[:, None, None]
        new_aphi1 = aphi0 + B1 * wmc * ah[None] - B1 * c[:, None, None] * aphi1
        new_aphi0 = B2 * wmc * ah[None] - B2 * c[:, None, None] * aphi1
        # parameters: M (through kappa and Wi), L h, G and k
        g_kap += dt * dL_dot(arhs, h) + dt * xi * dL_dot(arhs, Phi_new)
        for a in range(d):
            for b in range(d):
                dks = np.zeros((nc, N))
                for cc, (i, j) in enumerate(P):
                    dks[cc] = (1.0 if (i, j) == (a, b) else 0.0) + (1.0 if (j, i) == (a, b) else 0.0)
                g_kap[a * d + b] += dt * G * psi0 * np.sum(arhs * dks, axis=0)
        gWi += dt * xi / Wi ** 2 * np.sum(arhs * Phi_new) + dt / Wi ** 2 * np.sum(arhs * h) \
            - dt * (G / Wi) * psi0 * np.sum(arhs * ks)
        gbeta += -dt * psi0 * np.sum(arhs * ks) / (Wi * Re)
        aPhi1, aPhi0, aphi1, aphi0 = new_aPhi1, new_aPhi0, new_aphi1, new_aphi0
    return dict(Psi_T=psi, Phi0=aPhi1 + aPhi0, kappa=g_kap, Wi=gWi, beta=gbeta)
