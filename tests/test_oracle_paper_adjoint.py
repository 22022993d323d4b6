"""The oracle's reference adjoint in the paper's variable
(oracle.paper_form.paper_gradients: a plain reverse sweep of the step of
Section 3.4, BDF2 start, frozen velocity gradient; pointwise, explicit or
implicit transport) pinned to
central differences of the oracle's own forward, every entry of every
gradient field: exactly along Phi(0) (Psi(T) is affine in it), to the
differences' O(h^2) truncation in kappa, Wi and beta."""
import numpy as np
import pytest

from oracle import soe
from oracle.paper_form import PaperForm, paper_gradients
from paper_2411_17294_gb300 import inputs


CASES = [
    # dim, n, alpha, m, steps, transport (None, "explicit", "implicit"), stencil, eps, velocity scale
    (2, (4, 3), 0.5, 5, 6, None, 0, 0.0, 0.0),
    (3, (2, 2, 3), 0.3, 4, 5, None, 0, 0.0, 0.0),
    (2, (3, 3), 0.7, 8, 1, None, 0, 0.0, 0.0),
    (2, (4, 3), 0.5, 5, 5, "explicit", 0, 0.0, 0.3),
    (3, (2, 3, 2), 0.5, 5, 5, "explicit", 1, 0.01, 0.3),
    (2, (4, 3), 0.5, 5, 5, "implicit", 1, 0.01, 2.0),
    (3, (2, 3, 2), 0.4, 4, 4, "implicit", 0, 0.0, 3.0),
]


@pytest.mark.parametrize("dim,n,alpha,m,steps,transport,stencil,eps,speed", CASES)
def test_paper_gradients_against_central_differences(dim, n, alpha, m, steps, transport, stencil, eps, speed):
    N = int(np.prod(n))
    dt, Wi, beta, Re = 4e-3, 1.3, 0.4, 1.7
    mu, w = soe.soe_nnls(1 - alpha, dt, 50 * dt, m)
    u, kap = inputs.spectral_velocity(dim, n, 1, seed=3)
    kap = 0.6 * np.asarray(kap)
    u = speed * np.asarray(u) if transport else None
    P0 = inputs.random_stress(dim, n, 4)
    dJ = np.random.default_rng(5).normal(size=P0.shape)
    tk = dict(grid=n, eps=eps, stencil=stencil, implicit=transport == "implicit")
    g = paper_gradients(dim, N, Wi, beta, dt, mu, w, P0, kap, steps, dJ, Re=Re, u=u, **tk)

    def J(P, k, Wi_, b_):
        pf = PaperForm(dim, N, Wi_, b_, dt, mu, w, Phi0=P, Re=Re, **tk)
        for _ in range(steps):
            psi = pf.step(k, k, u)
        return float(np.sum(dJ * psi))

    assert np.isclose(J(P0, kap, Wi, beta), float(np.sum(dJ * g["Psi_T"])), rtol=1e-14)
    fdP = np.zeros_like(P0)
    for idx in np.ndindex(P0.shape):
        d = np.zeros_like(P0)
        d[idx] = 1.0
        fdP[idx] = (J(P0 + d, kap, Wi, beta) - J(P0 - d, kap, Wi, beta)) / 2.0
    assert np.max(np.abs(g["Phi0"] - fdP)) <= 1e-12 * np.max(np.abs(fdP))
    h = 1e-5
    fdK = np.zeros_like(kap)
    for idx in np.ndindex(kap.shape):
        d = np.zeros_like(kap)
        d[idx] = h
        fdK[idx] = (J(P0, kap + d, Wi, beta) - J(P0, kap - d, Wi, beta)) / (2 * h)
    assert np.max(np.abs(g["kappa"] - fdK)) <= 1e-7 * np.max(np.abs(fdK))
    fdW = (J(P0, kap, Wi + h, beta) - J(P0, kap, Wi - h, beta)) / (2 * h)
    fdB = (J(P0, kap, Wi, beta + h) - J(P0, kap, Wi, beta - h)) / (2 * h)
    assert abs(g["Wi"] - fdW) <= 1e-7 * abs(fdW)
    assert abs(g["beta"] - fdB) <= 1e-7 * abs(fdB)
    if transport:
        # the transport changes the gradient, so its adjoint is what the pins see
        g0 = paper_gradients(dim, N, Wi, beta, dt, mu, w, P0, kap, steps, dJ, Re=Re)
        assert np.max(np.abs(g0["Phi0"] - g["Phi0"])) > 1e-3 * np.max(np.abs(g["Phi0"]))

