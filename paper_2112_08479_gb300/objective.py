"""Differentiable lock-exchange objectives of the initial scalar field and C_s.

``LBMObjective.apply(chi0, cs, params, nsteps, K, kind)`` runs the
lock-exchange forward (BGK-Smagorinsky or cumulant fluid, D3Q7 scalar, FP32)
on the GPU and returns J (FP64):

- kind "friction": the time-integrated bottom friction J = sum_{n=1..N}
  F_w(s_n) (Eq. 62-64), accumulated on the device;
- kind "front": the front position after N steps, J = (x_f + 1/2 - x0) / H
  (Sec. 3.1), whose threshold crossing is interpolated between columns so
  that J is a continuous, piecewise smooth function of chi0 (lbm_front_adjoint).

Its backward returns dJ/dchi0 and dJ/dC_s (0 for the cumulant model, which
has no Smagorinsky closure) from the library's discrete adjoint: the forward keeps a checkpoint of the state every K steps, and the
reverse sweep recomputes each K-step segment from its checkpoint before
stepping the adjoint back through it (lbm_adjoint_segment).  Device memory:
N/K + 1 checkpoints plus one K-state segment buffer.
"""
from __future__ import annotations

from dataclasses import replace

import torch

from . import lbm


class LBMObjective(torch.autograd.Function):

    @staticmethod
    def forward(ctx, chi0, cs, params: lbm.Params, nsteps: int, K: int = 100,
                kind: str = "friction"):
        if params.storage != lbm.LBM_FP32 or params.scalar != lbm.LBM_SCALAR_Q7:
            raise ValueError("the adjoint exists for the D3Q7 scalar and FP32 storage "
                             "(BGK-Smagorinsky or cumulant fluid)")
        if nsteps < 1 or K < 1:
            raise ValueError("nsteps and K must be >= 1")
        if kind not in ("friction", "front"):
            raise ValueError(f"unknown objective {kind!r}")
        p = replace(params, cs_smag=float(cs))
        lat = lbm.Lattice(p, device=chi0.device)
        lat.set_scalar(chi0.detach().to(torch.float32).contiguous())
        acc = torch.zeros(1, dtype=torch.float64, device=chi0.device)
        nck = (nsteps + K - 1) // K
        ckpts = torch.empty(nck, lat.Q + lat.NS, lat.N, device=chi0.device)
        lat.objective_forward(nsteps, K, ckpts, acc if kind == "friction" else None)
        ctx.lat = lat
        ctx.ckpts = ckpts
        ctx.final = lat.get_state()
        ctx.kind = kind
        if kind == "front":
            lat.front_adjoint(ctx.final, None, acc)
        ctx.nsteps, ctx.K = nsteps, K
        ctx.chi_dtype = chi0.dtype
        ctx.cs_dtype = cs.dtype if torch.is_tensor(cs) else torch.float64
        return acc[0]

    @staticmethod
    def backward(ctx, gJ):
        lat, K, nsteps = ctx.lat, ctx.K, ctx.nsteps
        dev = ctx.final.device
        N, S = lat.N, lat.Q + lat.NS
        lam = torch.empty(S, N, device=dev)
        tmp = torch.empty(S, N, device=dev)
        dcs = torch.zeros(1, dtype=torch.float64, device=dev)
        w_fw = 1.0 if ctx.kind == "friction" else 0.0
        if ctx.kind == "friction":
            lat.adjoint_step(ctx.final, None, lam, None, 1.0)   # lam_N = dF_w(s_N)/ds_N
        else:
            lat.front_adjoint(ctx.final, lam, None)             # lam_N = d front(s_N)/ds_N
        seg_buf = torch.empty(min(K, nsteps), S, N, device=dev)
        for seg in range(ctx.ckpts.shape[0] - 1, -1, -1):
            n0 = seg * K
            lat.adjoint_segment(ctx.ckpts[seg], n0, min(K, nsteps - n0), seg_buf, lam, tmp, dcs,
                                w_fw)
        grad = torch.empty(N, device=dev)
        lat.adjoint_chi0(lam, grad)
        g = gJ.to(torch.float64)
        return ((g * grad.to(torch.float64)).to(ctx.chi_dtype),
                (g * dcs[0]).to(ctx.cs_dtype), None, None, None, None)


def _cs(cs, chi0):
    if not torch.is_tensor(cs):
        cs = torch.tensor(float(cs), dtype=torch.float64, device=chi0.device)
    return cs


def friction_objective(chi0, cs, params: lbm.Params, nsteps: int, K: int = 100):
    """J(chi0, C_s) = sum_{n=1..N} F_w(s_n) with autograd support (see LBMObjective)."""
    return LBMObjective.apply(chi0, _cs(cs, chi0), params, nsteps, K, "friction")


def front_objective(chi0, cs, params: lbm.Params, nsteps: int, K: int = 100):
    """J(chi0, C_s) = front position after nsteps, with autograd support."""
    return LBMObjective.apply(chi0, _cs(cs, chi0), params, nsteps, K, "front")
