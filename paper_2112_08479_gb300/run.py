"""Lock-exchange runs with logged diagnostics.

    python -m paper_2112_08479_gb300.run --nx 1024 --ny 64 --nz 128 --H 128 \\
        --x0 128 --ub 0.04 --Re 5000 --model cumulant --steps 20000 \\
        --every 100 --out run.jsonl

Every `--every` steps one JSON line with the step, the dimensionless time
t = step u_b / H, the front position (Sec. 3.1), the bottom friction F_w
(Eq. 62-64, lattice units and F_w / (u_b^2 H^2)), and the FP64 budgets is
appended to `--out` (the paper writes results files at N_t output times,
Sec. 3.2).  At the end the Froude number of Eq. 59 is fitted over the
requested window.  All time stepping and diagnostics run in the CUDA library.
"""
from __future__ import annotations

import argparse
import json
import sys
import time

import numpy as np

from . import lbm


def froude(t, front, t0: float = 2.5, t1: float = 10.0):
    """Eq. 59: slope of the front position against time over t0 <= t <= t1
    (least squares).  None when fewer than two samples fall in the window."""
    t = np.asarray(t, dtype=np.float64)
    front = np.asarray(front, dtype=np.float64)
    m = (t >= t0) & (t <= t1)
    if m.sum() < 2:
        return None
    A = np.vstack([t[m], np.ones(m.sum())]).T
    slope, _ = np.linalg.lstsq(A, front[m], rcond=None)[0]
    return float(slope)


def run(p: lbm.Params, u_b: float, steps: int, every: int, out=None, device="cuda"):
    """Advances `steps` steps, logging every `every`; returns the records."""
    import torch
    lat = lbm.Lattice(p, device=device)
    recs = []
    fh = open(out, "w") if out else None

    def log():
        d = lat.diag()
        r = {"step": int(d["step"]), "t": d["step"] * u_b / p.H, "front": d["front"],
             "front_node": d["front_node"], "Fw": d["Fw"],
             "Fw_nd": d["Fw"] / (u_b * u_b * p.H * p.H), "mass_delta": d["mass_delta"],
             "scalar_mass": d["scalar_mass"], "flags": d["flags"]}
        recs.append(r)
        if fh:
            fh.write(json.dumps(r) + "\n")
            fh.flush()

    log()
    t0 = time.perf_counter()
    done = 0
    while done < steps:
        k = min(every, steps - done)
        lat.step(k)
        done += k
        log()
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    if fh:
        fh.close()
    return recs, wall


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--nx", type=int, required=True)
    ap.add_argument("--ny", type=int, required=True)
    ap.add_argument("--nz", type=int, required=True)
    ap.add_argument("--H", type=int, required=True)
    ap.add_argument("--x0", type=int, required=True)
    ap.add_argument("--ub", type=float, default=0.03)
    ap.add_argument("--Re", type=float, required=True)
    ap.add_argument("--Sc", type=float, default=1.0)
    ap.add_argument("--model", default="bgk", choices=sorted(lbm.MODELS))
    ap.add_argument("--storage", default="fp32", choices=sorted(lbm.STORAGES))
    ap.add_argument("--scalar", default="q7", choices=sorted(lbm.SCALARS),
                    help="scalar lattice: q7 (both models), q6 (BGK, Eq. 29-31), "
                         "q27 (cumulant, factorized central moments, Eq. 37-51)")
    ap.add_argument("--geometry", default="walls", choices=lbm.GEOMETRIES,
                    help="walls: Fig. 4a (Cases 2, 4, 6, 8); periodic: Fig. 4b, periodic "
                         "ends (Cases 1, 3, 5, 7)")
    ap.add_argument("--sc-t", default="1.0",
                    help="turbulent Schmidt number (Eq. 35) or 'paper' for Sc_T = C_s^2")
    ap.add_argument("--cs", type=float, default=0.17)
    ap.add_argument("--seed", type=int, default=2112)
    ap.add_argument("--steps", type=int, default=None)
    ap.add_argument("--t-end", type=float, default=None, help="dimensionless end time")
    ap.add_argument("--every", type=int, default=100)
    ap.add_argument("--out", default=None)
    ap.add_argument("--fr-window", type=float, nargs=2, default=(2.5, 10.0))
    a = ap.parse_args(argv)
    p = lbm.lock_exchange(a.nx, a.ny, a.nz, H=a.H, x0=a.x0, u_b=a.ub, Re=a.Re, Sc=a.Sc,
                          model=a.model, storage=a.storage, cs_smag=a.cs, seed=a.seed,
                          scalar=a.scalar, geometry=a.geometry,
                          sc_t=a.sc_t if a.sc_t == "paper" else float(a.sc_t))
    steps = a.steps if a.steps is not None else int(round(a.t_end * a.H / a.ub))
    recs, wall = run(p, a.ub, steps, a.every, a.out)
    fr = froude([r["t"] for r in recs], [r["front"] for r in recs], *a.fr_window)
    summary = {"steps": steps, "wall_s": wall, "mnups_incl_diag": p.N * steps / wall / 1e6,
               "froude": fr, "fr_window": list(a.fr_window), "final": recs[-1]}
    print(json.dumps(summary))
    return summary


if __name__ == "__main__":
    sys.exit(0 if main() else 1)
