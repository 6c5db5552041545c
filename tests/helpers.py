"""Shared test helpers: parameter mapping between the library and the oracle,
conversion between the library's canonical state layout ([Q+7][nz][ny][nx],
f - w and Phi) and the oracle's node-major arrays, and a light-cone window
that lets the oracle reproduce single nodes of a full-size run."""
from __future__ import annotations

import numpy as np

import oracle as O
from paper_2112_08479_gb300 import lbm


def oracle_params(p: lbm.Params, **kw) -> O.OracleParams:
    op = O.OracleParams(p.nx, p.ny, p.nz, model=p.model, nu=p.nu, D=p.D, cs_smag=p.cs_smag,
                        sc_t=p.sc_t, gprime=p.gprime, eg=tuple(p.eg), omega_bulk=p.omega_bulk,
                        omega_high=1.0,
                        periodic_x=bool(p.flags & lbm.LBM_FLAG_PERIODIC_X),
                        periodic_z=bool(p.flags & lbm.LBM_FLAG_PERIODIC_Z),
                        no_collide=bool(p.flags & lbm.LBM_FLAG_NO_COLLIDE),
                        scalar=p.scalar, omega_phi_high=1.0)
    for k, v in kw.items():
        setattr(op, k, v)
    return op


def weights(model: int) -> np.ndarray:
    return O.velocities(model)[1]


def w7() -> np.ndarray:
    return O.velocities_q7()[1]


def wscalar(p: lbm.Params) -> np.ndarray:
    """Weights of the scalar lattice of p (D3Q7, D3Q6 or D3Q27)."""
    return O.velocities_scalar(p.scalar)[1]


def stored_phi(phi, p: lbm.Params, k0: int = 0) -> np.ndarray:
    """Magnitude, in canonical units, of what 16-bit storage holds for the
    canonical scalar rows phi (Phi - w, rows k0, k0 + 1, ... of the scalar
    lattice): |Phi - LBM_SCALAR_CHI16 w|, the magnitude its rounding scales
    with.  FP32 storage holds Phi - w itself."""
    phi = np.asarray(phi, dtype=np.float64)
    if p.storage == lbm.LBM_FP32:
        return np.abs(phi)
    w = wscalar(p)[k0:k0 + phi.shape[0]]
    w = w.reshape((-1,) + (1,) * (phi.ndim - 1))
    return np.abs(phi + (1.0 - lbm.LBM_SCALAR_CHI16) * w)


def canonical_to_oracle(state: np.ndarray, p: lbm.Params, shifted: bool = True):
    """[Q+7, N] float32 (f - w, Phi - w) -> oracle (f, phi) float64 arrays.
    shifted=False takes the rows as they are (streaming tests, adjoints)."""
    Q = p.Q
    s = np.asarray(state, dtype=np.float64).reshape(Q + p.NS, *p.shape)
    f = np.moveaxis(s[:Q], 0, -1).copy()
    phi = np.moveaxis(s[Q:], 0, -1).copy()
    if shifted:
        f += weights(p.model)
        phi += wscalar(p)
    return f, phi


def oracle_to_canonical(f: np.ndarray, phi: np.ndarray, p: lbm.Params, shifted: bool = True):
    """oracle (f, phi) -> [Q+7, N] float64 in the library layout."""
    ff = f - weights(p.model) if shifted else f
    pp = phi - wscalar(p) if shifted else phi
    return np.concatenate([np.moveaxis(ff, -1, 0), np.moveaxis(pp, -1, 0)]).reshape(p.Q + p.NS, -1)


def lock_state_oracle(p: lbm.Params):
    op = oracle_params(p)
    chi0 = O.lock_chi0(p.nx, p.ny, p.nz, p.x0, p.noise_amp, p.seed)
    return op, O.init(op, chi0)


def rel_inf(a, b) -> float:
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    den = np.abs(b).max()
    return float(np.abs(a - b).max() / den) if den > 0 else float(np.abs(a - b).max())


def window_oracle(p: lbm.Params, state0: np.ndarray, node, steps: int):
    """Oracle value of every population at `node` after `steps` steps of a
    full-size run, from a (2 steps + 1)-wide window of the initial canonical
    state `state0` ([Q+NS, nz, ny, nx] float32, numpy or torch).  Window edges inside the
    domain are given walls (x, z) or a wrap (y); their wrong values travel one
    node per step and do not reach the centre within `steps` steps."""
    Q = p.Q
    x, y, z = node
    k = steps
    xs = np.arange(max(0, x - k), min(p.nx, x + k + 1))
    zs = np.arange(max(0, z - k), min(p.nz, z + k + 1))
    if p.ny >= 2 * k + 1:
        ys = (np.arange(y - k, y + k + 1)) % p.ny
        cy = k
    else:
        ys = np.arange(p.ny)
        cy = y
    sub = state0[:, zs][:, :, ys][:, :, :, xs]
    if not isinstance(sub, np.ndarray):          # a torch tensor (possibly on the GPU)
        sub = sub.cpu().numpy()
    sub = sub.astype(np.float64)
    f = np.moveaxis(sub[:Q], 0, -1) + weights(p.model)
    phi = np.moveaxis(sub[Q:], 0, -1) + wscalar(p)
    op = oracle_params(p)
    op.nx, op.ny, op.nz = len(xs), len(ys), len(zs)
    op.periodic_x = False
    op.periodic_z = False
    f, phi = O.run(op, steps, f, phi)
    cx = int(np.where(xs == x)[0][0])
    cz = int(np.where(zs == z)[0][0])
    return f[cz, cy, cx] - weights(p.model), phi[cz, cy, cx] - wscalar(p)


def rest_row_tol(p, pre, rel):
    """Bound on the error of the scalar's rest population after one step
    under 16-bit storage, where it is held in FP32 and receives the storage
    roundings of the node's post-collision moving populations: at most one
    half-ulp (rel = 2^-11 FP16, 2^-8 BF16) of each of them.  The rest
    population never moves, so the populations whose roundings it receives
    are those the node's own collision produced (they stream away
    afterwards).  pre: canonical columns [Q + NS, M] of the nodes before the
    step; returns the bound for each of the M nodes (FP64 oracle collision)."""
    import numpy as np
    op = oracle_params(p)
    pre = np.asarray(pre, dtype=np.float64)
    w, ws = weights(p.model), wscalar(p)
    out = np.zeros(pre.shape[1])
    for m in range(pre.shape[1]):
        _, po = O.collide_node(op, pre[: p.Q, m] + w, pre[p.Q:, m] + ws)
        out[m] = rel * stored_phi(po[1:] - ws[1:], p, 1).sum() * 1.01
    return out
