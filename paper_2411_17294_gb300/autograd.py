"""torch.autograd.Function around the fractional stress run and its adjoint.

``fractional_stress(sigma0, grad_u, Wi, beta, ...)`` advances the stress
``steps`` steps with a frozen velocity gradient and returns sigma(T).  Its
backward is the library's hand-written adjoint (tfs_backward): the forward
keeps a full-state checkpoint every K steps (the mode history is m times the
stress and is not stored); the backward recomputes each K-step segment from its
checkpoint and sweeps it in reverse.  Gradients flow to sigma0, grad_u, Wi and
beta.
"""
from __future__ import annotations

import torch

from . import tfs


class TFSFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, sigma0, grad_u, Wi, beta, u, cfg):
        dim, n = cfg["dim"], cfg["n"]
        alpha, dt, steps, K = cfg["alpha"], cfg["dt"], cfg["steps"], cfg["K"]
        mu, w = cfg.get("mu"), cfg.get("w")
        precision = cfg.get("precision", tfs.TFS_FP64)
        transport = cfg.get("transport", u is not None)
        s = tfs.Solver(dim, n, alpha, float(Wi), float(beta), dt, m=0 if alpha == 1.0 else len(mu),
                       precision=precision, mu=mu, w=w, transport=transport, eps=cfg.get("eps", 0.0),
                       stencil=cfg.get("stencil", tfs.TFS_STENCIL_UPWIND3), L=cfg.get("L"), Re=cfg.get("Re", 1.0),
                       device=grad_u.device, start=cfg.get("start", "bdf2"), form=cfg.get("form", "stress"))
        kt = grad_u.detach().to(s.dtype).reshape(dim * dim, -1).contiguous()
        ut = u.detach().to(s.dtype).reshape(dim, -1).contiguous() if transport else None
        s.set_state(sigma0.detach())
        ckpts = []
        for k in range(steps):
            if k % K == 0:
                buf = s.new_checkpoint()
                s.save(buf)
                ckpts.append(buf)
            s.step(kt, kt, ut)
        out = s.stress().to(sigma0.dtype).reshape(sigma0.shape)
        ctx.solver = s
        ctx.ckpts = ckpts
        ctx.kt, ctx.ut = kt, ut
        ctx.meta = (steps, K, sigma0.dtype, sigma0.shape, grad_u.dtype, grad_u.shape, Wi, beta)
        return out

    @staticmethod
    def backward(ctx, g_out):
        steps, K, s_dtype, s_shape, k_dtype, k_shape, Wi, beta = ctx.meta
        s = ctx.solver
        g_s0, g_k, gWi, gb = s.backward(g_out.detach().reshape(s.nc, -1), ctx.ckpts, K, steps, ctx.kt, ctx.ut)
        s.close()
        ctx.solver = None
        ctx.ckpts = None
        dWi = torch.tensor(gWi, dtype=Wi.dtype, device=Wi.device) if isinstance(Wi, torch.Tensor) else None
        db = torch.tensor(gb, dtype=beta.dtype, device=beta.device) if isinstance(beta, torch.Tensor) else None
        return (g_s0.to(s_dtype).reshape(s_shape), g_k.to(k_dtype).reshape(k_shape), dWi, db, None, None)


def fractional_stress(sigma0, grad_u, Wi, beta, *, dim, n, alpha, dt, steps, K=50, mu=None, w=None, u=None,
                      precision=tfs.TFS_FP64, transport=None, eps=0.0, stencil=tfs.TFS_STENCIL_UPWIND3, L=None,
                      Re=1.0, start="bdf2", form="stress"):
    """sigma(T) after `steps` steps from sigma0 [nc, N] with the frozen velocity
    gradient grad_u [d*d, N] (and velocity u [d, N] when transport is on);
    differentiable in sigma0, grad_u, Wi and beta (0-d tensors).
    transport: False (pointwise law), True or "explicit", or "implicit" (u.grad
    and eps Lap inside the global solve; the reverse sweep solves the
    transposed system).  start: "bdf2" (empty past) or "sdirk2" (the paper's
    first step), which takes the pointwise law or implicit transport (the
    library refuses it with explicit transport).  form="paper": the paper's
    variable (Section 3.4; sigma0 is Phi(0), the result Psi(T), mu/w the SOE of
    the kernel of order 1 - alpha), with every transport mode and start that
    the stress form takes."""
    cfg = dict(dim=dim, n=tuple(n), alpha=alpha, dt=dt, steps=int(steps), K=int(K), mu=mu, w=w,
               precision=precision, transport=(u is not None) if transport is None else transport, eps=eps,
               stencil=stencil, L=L, Re=Re, start=start, form=form)
    return TFSFunction.apply(sigma0, grad_u, Wi, beta, u, cfg)
