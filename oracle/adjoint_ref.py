"""FP64 reference gradients of two lock-exchange objectives.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Objectives, with s_n the state after n steps of the BGK-Smagorinsky + D3Q7
scalar + Boussinesq step:
- "friction" (Sec. 3.2, Eq. 62-64): J = sum_{n=1..N} F_w(s_n),
  F_w = sum_{x,y} nu (9 u_x(z=0) - u_x(z=1)) / 3;
- "front" (Sec. 3.1, reading R11): J = (x_f(s_N) + 1/2 - x0) / H, x_f the
  threshold crossing of m(x) = max_z mean_y chi, linearly interpolated
  between the last column at or above the threshold and the next one.
Gradients with respect to the initial scalar field chi0 (s_0: f = w,
Phi_k = w_k chi0) and the Smagorinsky constant C_s.

The step is restated here with torch float64 tensor operations, vectorised
over nodes, directly from the equations (Eq. 11, 17, 19-30, 32-35 with the
readings R1-R5 of the C oracle); it is checked against the C oracle to round
off.  The gradient is plain reverse accumulation: the states s_0..s_N are
kept, and for n = N-1..0 the vector-Jacobian product of one step is taken by
torch.autograd.  The norm |Pi| uses torch.linalg.vector_norm, whose gradient
at 0 is 0 (the subgradient).
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import oracle as O

DT = torch.float64


class BGKStep:
    """One time step on a (nz, ny, nx) box with x and z walls, periodic y."""

    def __init__(self, p: O.OracleParams):
        assert p.model == 0
        self.p = p
        c, w = O.velocities(0)
        c7, w7 = O.velocities_q7()
        self.c = torch.tensor(c, dtype=DT)
        self.w = torch.tensor(w, dtype=DT)
        self.c7 = torch.tensor(c7, dtype=DT)
        self.w7 = torch.tensor(w7, dtype=DT)
        self.eg = torch.tensor(p.eg, dtype=DT)
        self.src_f = torch.tensor(self._pull_index(c), dtype=torch.long)
        self.src_p = torch.tensor(self._pull_index(c7), dtype=torch.long)

    def _pull_index(self, c):
        """Flat index into the post-collision array that each population is
        pulled from: (x - c_i, slot i), or (x, slot opp(i)) across a wall."""
        p = self.p
        q = len(c)
        opp = [int(np.where((c == -c[i]).all(1))[0][0]) for i in range(q)]
        z, y, x = np.meshgrid(np.arange(p.nz), np.arange(p.ny), np.arange(p.nx), indexing="ij")
        idx = np.zeros((p.nz, p.ny, p.nx, q), dtype=np.int64)
        for i in range(q):
            xs, ys, zs = x - c[i][0], (y - c[i][1]) % p.ny, z - c[i][2]
            if p.periodic_x:
                xs = xs % p.nx
            if p.periodic_z:
                zs = zs % p.nz
            inside = (xs >= 0) & (xs < p.nx) & (zs >= 0) & (zs < p.nz)
            node = (z * p.ny + y) * p.nx + x
            src = (np.clip(zs, 0, p.nz - 1) * p.ny + ys) * p.nx + np.clip(xs, 0, p.nx - 1)
            idx[..., i] = np.where(inside, src * q + i, node * q + opp[i])
        return idx

    def macros(self, f, phi):
        chi = phi.sum(-1)
        F = self.p.gprime * chi[..., None] * self.eg
        rho = f.sum(-1)
        u = (f @ self.c + 0.5 * F) / rho[..., None]
        return rho, u, chi, F

    def collide(self, f, phi, cs):
        p = self.p
        rho, u, chi, F = self.macros(f, phi)
        cu = u @ self.c.T
        usq = (u * u).sum(-1, keepdim=True)
        feq = self.w * rho[..., None] * (1 + 3 * cu + 4.5 * cu * cu - 1.5 * usq)
        Pi = torch.einsum("...i,ia,ib->...ab", f - feq, self.c, self.c)
        q = torch.linalg.vector_norm(Pi, dim=(-2, -1))
        tau0 = 3 * p.nu + 0.5
        tau = 0.5 * (tau0 + torch.sqrt(tau0 * tau0 + 18 * math.sqrt(2) * cs * cs * q / rho))
        cF = F @ self.c.T
        uF = (u * F).sum(-1, keepdim=True)
        S = (1 - 0.5 / tau[..., None]) * self.w * (3 * cF - 3 * uF + 9 * cu * cF)
        fo = f - (f - feq) / tau[..., None] + S
        nu_t = (tau - tau0) / 3
        taup = 0.5 + 4 * (p.D + nu_t / p.sc_t)
        phieq = self.w7 * chi[..., None] * (1 + 4 * (u @ self.c7.T))
        po = phi - (phi - phieq) / taup[..., None]
        return fo, po

    def __call__(self, f, phi, cs):
        fo, po = self.collide(f, phi, cs)
        return fo.reshape(-1)[self.src_f], po.reshape(-1)[self.src_p]

    def friction(self, f, phi):
        _, u, _, _ = self.macros(f, phi)
        ux = u[..., 0]
        return (self.p.nu * (9 * ux[0] - ux[1]) / 3).sum()

    def front(self, f, phi, x0: int, H: float, thr: float = 0.02):
        """Front position (x_f + 1/2 - x0) / H; differentiable where the
        crossing column and the maximising z do not change (torch.max passes
        the gradient to the maximising element).  Columns x < xlim are searched
        (all with x walls, the half ahead of the lock with periodic ends)."""
        chi = phi.sum(-1)                       # (nz, ny, nx)
        m = chi.mean(1).max(0).values           # (nx,)
        nx = m.shape[0]
        xlim = O.front_xlim(nx, x0, self.p.periodic_x)
        above = torch.nonzero(m[:xlim] >= thr)
        if above.numel() == 0:
            xn = m.new_tensor(-1.0)
        else:
            xf = int(above.max())
            if xf == xlim - 1:
                xn = m.new_tensor(float(xf))
            else:
                xn = xf + (m[xf] - thr) / (m[xf] - m[xf + 1])
        return (xn + 0.5 - x0) / H


def initial_state(step: BGKStep, chi0):
    p = step.p
    chi0 = torch.as_tensor(np.asarray(chi0).reshape(p.nz, p.ny, p.nx), dtype=DT)
    f = step.w.expand(p.nz, p.ny, p.nx, 19).clone()
    phi = step.w7 * chi0[..., None]
    return f, phi


def objective(p: O.OracleParams, chi0, cs: float, nsteps: int) -> float:
    """J = sum_{n=1..N} F_w(s_n) with the torch restatement (FP64)."""
    st = BGKStep(p)
    f, phi = initial_state(st, chi0)
    J = 0.0
    cs_t = torch.tensor(cs, dtype=DT)
    with torch.no_grad():
        for _ in range(nsteps):
            f, phi = st(f, phi, cs_t)
            J += float(st.friction(f, phi))
    return J


def gradient(p: O.OracleParams, chi0, cs: float, nsteps: int, objective: str = "friction",
             x0: int = 0, H: float = 1.0, thr: float = 0.02):
    """Returns (J, dJ/dchi0 with the shape of chi0, dJ/dC_s) in FP64 for the
    objective "friction" or "front" (the latter with x0, H, thr)."""
    st = BGKStep(p)
    f, phi = initial_state(st, chi0)
    cs_t = torch.tensor(cs, dtype=DT)
    traj = [(f, phi)]
    J = 0.0
    with torch.no_grad():
        for _ in range(nsteps):
            f, phi = st(f, phi, cs_t)
            traj.append((f, phi))
            if objective == "friction":
                J += float(st.friction(f, phi))
    # lam_N = dJ/ds_N of the final state's term
    fN, pN = (t.clone().requires_grad_(True) for t in traj[-1])
    if objective == "friction":
        final = st.friction(fN, pN)
    else:
        final = st.front(fN, pN, x0, H, thr)
        J = float(final.detach())
    if final.requires_grad:
        lf, lp = torch.autograd.grad(final, (fN, pN), allow_unused=True)
        lf = torch.zeros_like(fN) if lf is None else lf
        lp = torch.zeros_like(pN) if lp is None else lp
    else:                                       # a front that does not move
        lf, lp = torch.zeros_like(fN), torch.zeros_like(pN)
    gcs = 0.0
    for n in range(nsteps - 1, -1, -1):
        fn, pn = (t.clone().requires_grad_(True) for t in traj[n])
        c = cs_t.clone().requires_grad_(True)
        f1, p1 = st(fn, pn, c)
        inner = (f1 * lf).sum() + (p1 * lp).sum()
        if n >= 1 and objective == "friction":
            inner = inner + st.friction(fn, pn)
        lf, lp, gc = torch.autograd.grad(inner, (fn, pn, c))
        gcs += float(gc)
    gchi = (lp * st.w7).sum(-1)        # Phi_k = w_k chi0 at t = 0
    return J, gchi.numpy(), gcs
