"""Differentiable Stillinger-Weber energy over the libnefe kernels.

``sw_energy(x, theta, box)`` returns the SW energy (Sec. 2, the interatomic model the
switching Hamiltonians are built on) as a torch scalar whose backward gives
dE/dx = -F and dE/dtheta for theta = (A, B, p, q, a, lambda3, gamma); eps, sigma and cos0
stay fixed.  Both passes run in one ``nefe_sw_energy_grad`` call (neighbour list from
``nefe_neighbor_build``); this module only marshals tensors and applies the chain rule to
the incoming scalar gradient.
"""
from __future__ import annotations

import torch

from . import nefe as N

THETA_NAMES = ("A", "B", "p", "q", "a", "lambda3", "gamma")
SILICON_THETA = (7.049556277, 0.6022245584, 4.0, 0.0, 1.80, 21.0, 1.20)
SILICON_FIXED = (2.1683, 2.0951, -1.0 / 3.0)     # eps (eV), sigma (A), cos0


def _params(theta, fixed):
    eps, sigma, cos0 = (float(v) for v in fixed)
    A, B, p, q, a, lam, gam = (float(v) for v in theta)
    return N.nefe_sw_params(eps, sigma, A, B, p, q, a, lam, gam, cos0)


class SWEnergy(torch.autograd.Function):
    """Forward: E(x; theta).  Backward: (-F g, dE/dtheta g).  Not twice differentiable."""

    @staticmethod
    def forward(ctx, x, theta, box, fixed, rcs, cap, precision):
        if x.device.type != "cuda" or x.dtype != torch.float64 or x.dim() != 2 or x.shape[0] != 3:
            raise ValueError("x must be a (3, n) float64 CUDA tensor (structure of arrays)")
        n = x.shape[1]
        xs = x.contiguous()
        prm = _params(theta.detach().cpu().tolist(), fixed)
        nbr = torch.empty(max(n, 1) * cap, dtype=torch.int32, device=x.device)
        cnt = torch.empty(max(n, 1), dtype=torch.int32, device=x.device)
        f = torch.empty(3 * max(n, 1), dtype=torch.float64, device=x.device)
        eg = torch.empty(8, dtype=torch.float64, device=x.device)
        stream = torch.cuda.current_stream(x.device)
        N.nefe_neighbor_build(xs, n, box, rcs, cap, nbr, cnt, stream=stream)
        N.nefe_sw_energy_grad(xs, n, box, rcs, nbr, cnt, cap, prm, precision, f, eg, stream=stream)
        ctx.n = n
        ctx.theta_device = theta.device
        ctx.save_for_backward(f, eg)
        return eg[0].clone()

    @staticmethod
    @torch.autograd.function.once_differentiable
    def backward(ctx, g):
        f, eg = ctx.saved_tensors
        gx = gth = None
        if ctx.needs_input_grad[0]:
            gx = f[: 3 * ctx.n].view(3, ctx.n) * (-g)
        if ctx.needs_input_grad[1]:
            gth = (eg[1:] * g).to(ctx.theta_device)
        return gx, gth, None, None, None, None, None


def sw_energy(x, theta=None, box=None, fixed=SILICON_FIXED, skin=0.5, cap=48, precision=N.NEFE_FP64):
    """SW energy of the (3, n) FP64 CUDA positions ``x`` in the orthorhombic periodic ``box``
    (three lengths, A).  ``theta`` (7,) float64 tensor of (A, B, p, q, a, lambda3, gamma)
    defaults to silicon; the list radius is a*sigma + skin."""
    if box is None:
        raise ValueError("box is required")
    if theta is None:
        theta = torch.tensor(SILICON_THETA, dtype=torch.float64)
    rcs = float(theta.detach()[4]) * float(fixed[1]) + skin
    return SWEnergy.apply(x, theta, [float(b) for b in box], tuple(fixed), rcs, int(cap), int(precision))


class SwitchingWork(torch.autograd.Function):
    """W(theta) of one switching run of an ``nefe.Adjoint`` context; backward by the adjoint
    sweep (noise and initial state fixed)."""

    @staticmethod
    def forward(ctx, theta, adj, nsteps, fixed):
        th = theta.detach().cpu().tolist()
        adj.set_params(_params(th, fixed))
        W = adj.forward(int(nsteps))
        ctx.adj = adj
        ctx.theta_device = theta.device
        return torch.tensor(W, dtype=torch.float64, device=theta.device)

    @staticmethod
    @torch.autograd.function.once_differentiable
    def backward(ctx, g):
        gth = torch.tensor(ctx.adj.backward(), dtype=torch.float64, device=ctx.theta_device)
        return gth * g, None, None, None


def switching_work(theta, adj, nsteps, fixed=SILICON_FIXED):
    """Switching work of ``adj`` over ``nsteps`` as a differentiable function of theta."""
    return SwitchingWork.apply(theta, adj, int(nsteps), tuple(fixed))
