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
stepping the adjoint back through it (lbm_recompute_segment,
lbm_adjoint_sweep), the recompute of the next segment overlapping the sweep
of the current one on a second stream.  Device memory: N/K + 1 checkpoints
plus two K-state segment buffers.
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
        reverse_sweep(lat, ctx.ckpts, nsteps, K, lam, tmp, dcs, w_fw)
        grad = torch.empty(N, device=dev)
        lat.adjoint_chi0(lam, grad)
        g = gJ.to(torch.float64)
        return ((g * grad.to(torch.float64)).to(ctx.chi_dtype),
                (g * dcs[0]).to(ctx.cs_dtype), None, None, None, None)


def reverse_sweep(lat, ckpts, nsteps: int, K: int, lam, tmp, dcs, w_fw: float,
                  overlap: bool = True):
    """lam_N -> lam_0 through all segments of checkpoints `ckpts` (state n0 =
    s K of segment s).  With `overlap` the recompute of segment s - 1 runs on
    a second stream while segment s is swept on the lattice's stream (two
    segment buffers); the two phases have different bottlenecks (the sweep is
    issue-bound, the recompute streams memory), so they share the GPU."""
    nseg = ckpts.shape[0]
    dev = lam.device
    S, N = lam.shape
    kmax = min(K, nsteps)
    main = lat.stream
    ks = [min(K, nsteps - s * K) for s in range(nseg)]
    if not overlap or nseg == 1:
        buf = torch.empty(kmax, S, N, device=dev)
        for s in range(nseg - 1, -1, -1):
            lat.recompute_segment(ckpts[s], ks[s], buf)
            lat.adjoint_sweep(ckpts[s], buf, s * K, ks[s], lam, tmp, dcs, w_fw)
        return
    side = torch.cuda.Stream(device=dev)
    bufs = [torch.empty(kmax, S, N, device=dev) for _ in range(2)]
    for b in bufs:
        b.record_stream(side)
    side.wait_stream(main)                    # checkpoints and lam_N are ready
    rec_done, sweep_done = {}, {}

    def recompute(s):
        if s + 2 in sweep_done:               # its buffer was swept by segment s + 2
            side.wait_event(sweep_done[s + 2])
        lat.recompute_segment(ckpts[s], ks[s], bufs[s % 2], stream=side)
        rec_done[s] = side.record_event()

    recompute(nseg - 1)
    for s in range(nseg - 1, -1, -1):
        if s >= 1:
            recompute(s - 1)
        main.wait_event(rec_done[s])
        lat.adjoint_sweep(ckpts[s], bufs[s % 2], s * K, ks[s], lam, tmp, dcs, w_fw)
        sweep_done[s] = main.record_event()
    main.wait_stream(side)


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
