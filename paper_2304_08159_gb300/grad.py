"""Drag gradients with respect to the body: the hand-written adjoint of the time step
(wl_grad_forward / wl_grad_backward in libwl.so) behind a torch.autograd.Function.

    theta = torch.tensor([R, cx, cy], dtype=torch.float64, requires_grad=True)
    F = rollout_forces(theta, dims=(256, 128), nu=0.12, U=(1.0, 0.0), nsteps=50, dt=0.1)
    J = F[:, 0].mean() / (0.5 * 1.0**2 * 2 * theta[0])   # mean drag coefficient
    J.backward()                                         # theta.grad = dJ/d(R, cx, cy)

The forward pass creates a simulation of a circle (2-D) / sphere (3-D) of radius theta[0]
centred at theta[1:] (or a torus, theta = (R, r, c_x, c_y, c_z)), runs nsteps steps at the fixed dt from the uniform inflow and
returns the pressure force after each step (nsteps x D, float64).  The backward pass
recomputes each segment of `every` steps from its checkpoint and runs the adjoint
kernels backwards, so memory grows with nsteps/every checkpoints plus one segment.
Every step of both passes runs in the library's CUDA kernels; this module only
marshals arguments.
"""
from __future__ import annotations

import warnings

import torch

from . import wl


class _Rollout(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, cfg):
        th = theta.detach().double().cpu().tolist()
        D = len(cfg["dims"])
        if cfg.get("torus"):
            assert D == 3 and len(th) == 5, "torus theta = (R, r, c_x, c_y, c_z)"
            body = dict(kind=wl.WL_BODY_TORUS, center=th[2:], radius=th[0], radius2=th[1])
        else:
            assert len(th) == D + 1, "theta = (R, c_0, .., c_{D-1})"
            body = dict(kind=wl.WL_BODY_SPHERE, center=th[1:], radius=th[0])
        sim = wl.Sim(cfg["dims"], cfg["nu"], cfg["U"], body=body,
                     periodic=cfg.get("periodic", 0), tol=cfg.get("tol", 1e-6), dt_fixed=cfg["dt"],
                     max_vcycles=cfg.get("max_vcycles", 32), precision=1)
        F = sim.grad_forward(cfg["nsteps"], cfg.get("every", 10))
        ctx.sim = sim
        return torch.as_tensor(F, dtype=torch.float64, device=theta.device)

    @staticmethod
    def backward(ctx, gF):
        sim = ctx.sim
        g = gF.detach().double().cpu().numpy()
        tb, rc = sim.grad_backward(g, return_status=True)
        if rc == wl.WL_WNOTCONV:
            warnings.warn("an adjoint Poisson solve hit max_vcycles: the gradient is less accurate")
        sim.close()
        ctx.sim = None
        return torch.as_tensor(tb, dtype=gF.dtype, device=gF.device), None


def rollout_forces(theta, dims, nu, U, nsteps, dt, every=10, periodic=0, tol=1e-6, max_vcycles=32, torus=False):
    """Pressure force after each of nsteps steps (nsteps x D) as a differentiable function
    of theta = (R, c_0, .., c_{D-1}) of a circle/sphere body, or with torus=True (3-D) of
    theta = (R, r, c_x, c_y, c_z) of a torus (ring radius R in the y-z plane, tube radius
    r); dt is fixed."""
    cfg = dict(dims=tuple(int(d) for d in dims), nu=float(nu), U=tuple(float(u) for u in U), nsteps=int(nsteps),
               dt=float(dt), every=int(every), periodic=int(periodic), tol=float(tol), max_vcycles=int(max_vcycles),
               torus=bool(torus))
    return _Rollout.apply(theta, cfg)
