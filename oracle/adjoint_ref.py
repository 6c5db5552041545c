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
    """One time step of the BGK-Smagorinsky D3Q19 fluid with the D3Q7 scalar
    on a (nz, ny, nx) box with x and z walls (or periodic), periodic y."""

    MODEL = 0

    def __init__(self, p: O.OracleParams):
        assert p.model == self.MODEL and p.scalar == 0
        self.p = p
        c, w = O.velocities(p.model)
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


class CumulantStep(BGKStep):
    """One time step of the D3Q27 cumulant fluid (Eq. 54-58, reading R7) with
    the D3Q7 scalar (molecular D only, no eddy diffusivity).

    The cumulants are the coefficients of ln G, G(Xi) = sum_i f_i exp(Xi.c_i)
    (Eq. 54), computed in the ring of Taylor coefficients truncated at degree
    2 per axis (exact for those coefficients; the series of ln(1 + H) and
    exp(K) stop at degree 6).  Relaxation as Eq. 55-58: rho kept, first order
    to (j + F)/rho, off-diagonal second order and the deviators with omega1 =
    1/(3 nu + 1/2), the trace with omega_bulk to 1, orders >= 3 with
    omega_high to 0.  Populations from the moments by the per-axis inverse of
    the Vandermonde map {f(-1), f(0), f(1)} -> {m0, m1, m2}."""

    MODEL = 1

    def __init__(self, p: O.OracleParams):
        super().__init__(p)
        idx = [(a, b, c) for a in range(3) for b in range(3) for c in range(3)]
        i1, i2, o = [], [], []
        for n1, (a1, b1, c1) in enumerate(idx):
            for n2, (a2, b2, c2) in enumerate(idx):
                if a1 + a2 < 3 and b1 + b2 < 3 and c1 + c2 < 3:
                    i1.append(n1)
                    i2.append(n2)
                    o.append(idx.index((a1 + a2, b1 + b2, c1 + c2)))
        self.i1, self.i2, self.o = (torch.tensor(v, dtype=torch.long) for v in (i1, i2, o))
        fact = [1.0, 1.0, 2.0]
        self.fact = torch.tensor([fact[a] * fact[b] * fact[c] for a, b, c in idx], dtype=DT)
        c = self.c.numpy()
        self.mom = torch.tensor([[c[i][0] ** a * c[i][1] ** b * c[i][2] ** cc for i in range(27)]
                                 for a, b, cc in idx], dtype=DT)          # m = mom @ f

        def coef(cv, n):
            if cv == 0:
                return {0: 1.0, 1: 0.0, 2: -1.0}[n]
            return {0: 0.0, 1: 0.5 * cv, 2: 0.5}[n]
        self.inv = torch.tensor([[coef(c[i][0], a) * coef(c[i][1], b) * coef(c[i][2], cc)
                                  for a, b, cc in idx] for i in range(27)], dtype=DT)
        self.n_of = [a + b + cc for a, b, cc in idx]
        self.pos = {t: n for n, t in enumerate(idx)}

    def _mul(self, A, B):
        out = torch.zeros_like(A)
        return out.index_add(-1, self.o, A[..., self.i1] * B[..., self.i2])

    def _log1p(self, H):
        P, S = H, H
        for k in range(2, 7):
            P = self._mul(P, H)
            S = S + ((1.0 if k % 2 else -1.0) / k) * P
        return S

    def _exp(self, K):
        S = torch.zeros_like(K)
        S = S.index_fill(-1, torch.tensor([0]), 1.0)
        P, fk = K, 1.0
        for k in range(1, 7):
            if k > 1:
                P = self._mul(P, K)
            fk *= k
            S = S + P / fk
        return S

    def collide(self, f, phi, cs):
        p = self.p
        rho, u, chi, F = self.macros(f, phi)
        m = f @ self.mom.T
        g = m / self.fact
        H = g / rho[..., None]
        H = H * (torch.arange(27) != 0).to(DT)              # G / rho = 1 + H
        C = self._log1p(H) * self.fact                       # C_abc, C_000 replaced below
        om1 = 1.0 / (3.0 * p.nu + 0.5)
        om2, omh = p.omega_bulk, p.omega_high
        P = self.pos
        cxx, cyy, czz = C[..., P[2, 0, 0]], C[..., P[0, 2, 0]], C[..., P[0, 0, 2]]
        d1 = (1 - om1) * (cxx - cyy)
        d2 = (1 - om1) * (cxx - czz)
        tr = (1 - om2) * (cxx + cyy + czz) + om2
        nxx = (tr + d1 + d2) / 3
        new = {(2, 0, 0): nxx, (0, 2, 0): nxx - d1, (0, 0, 2): nxx - d2,
               (1, 1, 0): (1 - om1) * C[..., P[1, 1, 0]], (1, 0, 1): (1 - om1) * C[..., P[1, 0, 1]],
               (0, 1, 1): (1 - om1) * C[..., P[0, 1, 1]],
               (1, 0, 0): C[..., P[1, 0, 0]] + F[..., 0] / rho,
               (0, 1, 0): C[..., P[0, 1, 0]] + F[..., 1] / rho,
               (0, 0, 1): C[..., P[0, 0, 1]] + F[..., 2] / rho,
               (0, 0, 0): torch.zeros_like(rho)}
        cols = []
        for n, t in enumerate(P):
            cols.append(new[t] if t in new else (1 - omh) * C[..., n])
        K = torch.stack(cols, -1) / self.fact
        ms = rho[..., None] * self._exp(K) * self.fact       # exp(C_000) = rho
        fo = ms @ self.inv.T
        taup = 0.5 + 4 * p.D
        phieq = self.w7 * chi[..., None] * (1 + 4 * (u @ self.c7.T))
        po = phi - (phi - phieq) / taup
        return fo, po


def make_step(p: O.OracleParams):
    return CumulantStep(p) if p.model == 1 else BGKStep(p)


def initial_state(step: BGKStep, chi0):
    p = step.p
    chi0 = torch.as_tensor(np.asarray(chi0).reshape(p.nz, p.ny, p.nx), dtype=DT)
    f = step.w.expand(p.nz, p.ny, p.nx, len(step.w)).clone()
    phi = step.w7 * chi0[..., None]
    return f, phi


def objective(p: O.OracleParams, chi0, cs: float, nsteps: int) -> float:
    """J = sum_{n=1..N} F_w(s_n) with the torch restatement (FP64)."""
    st = make_step(p)
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
    objective "friction" or "front" (the latter with x0, H, thr).  BGK or
    cumulant fluid (p.model) with the D3Q7 scalar; for the cumulant model
    dJ/dC_s is 0 (no Smagorinsky closure)."""
    st = make_step(p)
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
        lf, lp, gc = torch.autograd.grad(inner, (fn, pn, c), allow_unused=True)
        gcs += 0.0 if gc is None else float(gc)     # the cumulant step does not use C_s
    gchi = (lp * st.w7).sum(-1)        # Phi_k = w_k chi0 at t = 0
    return J, gchi.numpy(), gcs
