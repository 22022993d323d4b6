"""The oracle's reference adjoint of the implicit-transport step in the stress
form (oracle.orc.gradients_implicit: a numpy reverse sweep with the dense
global operator), pinned entry by entry to central differences of the C
oracle's implicit forward (orc_step_implicit): exactly along sigma0 (sigma(T)
is affine in it), to the differences' O(h^2) truncation in kappa, Wi and beta;
alpha < 1 and alpha = 1, both stencils, with diffusion, 2D and 3D."""
import numpy as np
import pytest

from oracle import orc, soe
from paper_2411_17294_gb300 import inputs


@pytest.mark.parametrize("dim,n,alpha,stencil,eps,speed", [(2, (4, 3), 0.5, 0, 0.0, 2.0),
                                                           (2, (4, 3), 1.0, 1, 0.01, 20.0),
                                                           (3, (2, 3, 2), 0.4, 1, 0.01, 3.0)])
def test_implicit_gradients_against_central_differences(dim, n, alpha, stencil, eps, speed):
    dt, Wi, beta, steps = 2e-3, 1.3, 0.4, 5
    m = 5 if alpha < 1 else 0
    mu, w = soe.soe_nnls(alpha, dt, 20 * dt, m) if alpha < 1 else (np.zeros(0), np.zeros(0))
    u, kap = inputs.spectral_velocity(dim, n, 1, seed=3)
    kap = 0.5 * np.asarray(kap)
    u = speed * np.asarray(u)
    s0 = inputs.random_stress(dim, n, 4)
    dJ = np.random.default_rng(5).normal(size=s0.shape)

    def prob(Wi_, b_, implicit=True):
        return orc.Problem(dim=dim, n=n, alpha=alpha, Wi=Wi_, beta=b_, dt=dt, mu=mu, w=w, eps=eps, stencil=stencil,
                           transport=implicit, implicit=implicit)

    g = orc.gradients_implicit(prob(Wi, beta), s0, kap, u, steps, dJ)

    def J(S, k, Wi_, b_):
        return float(np.sum(dJ * orc.forward(prob(Wi_, b_), S, k, u, steps)))

    assert np.isclose(J(s0, kap, Wi, beta), float(np.sum(dJ * g["sigma_T"])), rtol=1e-14)
    fdS = np.zeros_like(s0)
    for idx in np.ndindex(s0.shape):
        dd = np.zeros_like(s0)
        dd[idx] = 1.0
        fdS[idx] = (J(s0 + dd, kap, Wi, beta) - J(s0 - dd, kap, Wi, beta)) / 2.0
    assert np.max(np.abs(g["sigma0"] - fdS)) <= 1e-12 * np.max(np.abs(fdS))
    h = 1e-5
    fdK = np.zeros_like(kap)
    for idx in np.ndindex(kap.shape):
        dd = np.zeros_like(kap)
        dd[idx] = h
        fdK[idx] = (J(s0, kap + dd, Wi, beta) - J(s0, kap - dd, Wi, beta)) / (2 * h)
    assert np.max(np.abs(g["kappa"] - fdK)) <= 1e-7 * np.max(np.abs(fdK))
    fdW = (J(s0, kap, Wi + h, beta) - J(s0, kap, Wi - h, beta)) / (2 * h)
    fdB = (J(s0, kap, Wi, beta + h) - J(s0, kap, Wi, beta - h)) / (2 * h)
    assert abs(g["Wi"] - fdW) <= 1e-7 * abs(fdW)
    assert abs(g["beta"] - fdB) <= 1e-7 * abs(fdB)
    # the transport changes the gradient: the pointwise law's differs
    p0 = prob(Wi, beta, implicit=False)
    d = np.random.default_rng(6).normal(size=s0.shape)
    fd0 = float(np.sum(dJ * (orc.forward(p0, s0 + d, kap, None, steps) - orc.forward(p0, s0 - d, kap, None, steps)))) / 2
    assert abs(fd0 - float(np.sum(g["sigma0"] * d))) > 1e-3 * float(np.sum(np.abs(g["sigma0"] * d)))
