"""torch.autograd wrappers of the GPW path.

* :func:`rho` — the finest-grid density rho(D, R) (Eq. rho_wrap plus Fourier
  interpolation).  Its backward is hand-written with the two integration directions:
  for an upstream gradient g on the grid (with respect to the raw array),
  dL/dD = (N/Omega) eval_mat(g) and dL/dR = (N/Omega) eval_mat_ip1(D, g), because
  sum_r g(r) rho(r) = (N/Omega) <g, rho> and <v, rho(D)> = tr(D eval_mat(v)).
* :func:`tau` — the finest-grid kinetic energy density tau(D, R) (meta-GGA), the same way
  with the tau integration directions: dL/dD = (N/Omega) eval_mat_tau(g) and
  dL/dR = (N/Omega) eval_mat_tau_ip1(D, g) (the plan needs tau=True).
* :func:`energy` — E_H + E_x of one Fock build (the plan's exchange functional, LDA or
  PBE).  Forward is gpw_fock_grad (one pass); backward returns dE/dD = V and dE/dR = the
  Hxc gradient contraction (Algorithm 3).

D is treated as symmetric: the gradient with respect to D is the gradient of
E((D + D^T)/2).  Atom positions R move the Gaussians with the plan's pair set and boxes
frozen (gpw_plan_update_coords), so E(R) is smooth for small displacements; rebuild the
plan after large moves.  A plan holds one geometry at a time: run a backward before the
next forward on the same plan.
"""
from __future__ import annotations

import numpy as np
import torch

__all__ = ["rho", "tau", "energy"]


def _set_coords(plan, coords):
    if coords is None:
        return
    c = coords.detach().to("cpu", torch.float64).numpy()
    if getattr(plan, "_coords", None) is None or not np.array_equal(plan._coords, c):
        plan.update_coords(c)
        plan._coords = c.copy()


def _scale(plan):
    """N_fine / Omega: the inverse of the finest level's grid weight, as the plan
    reports it (Omega = |det lattice| for any cell)."""
    return 1.0 / plan.stats()["weight"][0]


class _Rho(torch.autograd.Function):
    @staticmethod
    def forward(ctx, D, coords, plan):
        _set_coords(plan, coords)
        Dd = D.detach().to("cuda", torch.float64).contiguous()
        out = plan.eval_rho(Dd)
        ctx.plan = plan
        ctx.save_for_backward(Dd)
        return out

    @staticmethod
    def backward(ctx, g):
        plan = ctx.plan
        (D,) = ctx.saved_tensors
        g = g.detach().to("cuda", torch.float64).contiguous()
        s = _scale(plan)
        gD = plan.eval_mat(g) * s if ctx.needs_input_grad[0] else None
        gR = plan.eval_mat_ip1(D, g) * s if ctx.needs_input_grad[1] else None
        return gD, gR, None


class _Tau(torch.autograd.Function):
    @staticmethod
    def forward(ctx, D, coords, plan):
        _set_coords(plan, coords)
        Dd = D.detach().to("cuda", torch.float64).contiguous()
        out = plan.eval_tau(Dd)
        ctx.plan = plan
        ctx.save_for_backward(Dd)
        return out

    @staticmethod
    def backward(ctx, g):
        plan = ctx.plan
        (D,) = ctx.saved_tensors
        g = g.detach().to("cuda", torch.float64).contiguous()
        s = _scale(plan)
        gD = plan.eval_mat_tau(g) * s if ctx.needs_input_grad[0] else None
        gR = plan.eval_mat_tau_ip1(D, g) * s if ctx.needs_input_grad[1] else None
        return gD, gR, None


class _Energy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, D, coords, plan):
        _set_coords(plan, coords)
        Dd = D.detach().to("cuda", torch.float64).contiguous()
        out = plan.fock_grad(Dd)
        ctx.save_for_backward(out["V"], out["grad"])
        return torch.tensor(out["EH"] + out["Ex"], dtype=torch.float64, device="cuda")

    @staticmethod
    def backward(ctx, gE):
        V, grad = ctx.saved_tensors
        gD = gE * V if ctx.needs_input_grad[0] else None
        gR = gE * grad if ctx.needs_input_grad[1] else None
        return gD, gR, None


def rho(D, coords, plan):
    """Finest-grid density of D with the atoms at coords (natm x 3, or None to keep the
    plan's geometry); differentiable in both."""
    return _Rho.apply(D, coords, plan)


def tau(D, coords, plan):
    """Finest-grid kinetic energy density (1/2) sum D grad phi . grad phi of D with the
    atoms at coords (or None); differentiable in both.  The plan needs tau=True."""
    return _Tau.apply(D, coords, plan)


def energy(D, coords, plan):
    """E_H + E_x (Hartree) of one Fock build; differentiable in D and coords."""
    return _Energy.apply(D, coords, plan)
