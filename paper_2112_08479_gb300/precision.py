"""Storage-precision comparison: the same lock-exchange run with FP32 and with
16-bit shifted storage (FP16 / BF16 of scale (f - w), FP32 collisions), from
the same initial condition, diagnostics logged side by side.

    python -m paper_2112_08479_gb300.precision --nx 2048 --ny 128 --nz 256 \\
        --H 256 --x0 256 --ub 0.03 --Re 30000 --model cumulant \\
        --t-end 20 --every 100 --out prec.jsonl

Reported per 16-bit storage, against the FP32 run (error measures of the
front, scalar mass and friction as relative differences: |x_f - x_f32| /
x_f32 with x the dimensionless front (x_f + 1/2 - x0) / H of Sec. 3.1,
|sum chi - sum chi_32| / sum chi_32, |F_w - F_w32| / max_t |F_w32|):
  - the front error at the requested times (--at, default t = 10 and 20);
  - the largest front error over fr_t0 <= t < t_wall, t_wall the first
    logged time at which the FP32 front stands within two nodes of the end
    wall (a front at the wall is pinned there whatever the precision, so
    later samples do not discriminate);
  - scalar-mass and friction errors at the last logged time.
All stepping and diagnostics run in the CUDA library (run.run).
"""
from __future__ import annotations

import argparse
import json
import sys

import numpy as np

from . import lbm
from .run import run


def wall_time(recs, nx: int, margin: float = 2.0):
    """First logged t at which the front node is within `margin` nodes of
    the end wall (x = nx - 1), None if never."""
    for r in recs:
        if r["front_node"] >= nx - 1 - margin:
            return r["t"]
    return None


def compare(ref, other, nx: int, at=(10.0, 20.0), t0: float = 2.5) -> dict:
    """Errors of `other` against `ref` (lists of run.run records logged at the
    same steps)."""
    assert len(ref) == len(other)
    t = np.array([r["t"] for r in ref])
    fr = np.array([r["front"] for r in ref])
    fo = np.array([r["front"] for r in other])
    err = np.abs(fo - fr) / np.maximum(np.abs(fr), 1e-300)
    tw = wall_time(ref, nx)
    win = (t >= t0) & (t < (tw if tw is not None else np.inf))
    out = {"t_wall": tw, "window": [t0, tw]}
    out["front_err_max_before_wall"] = float(err[win].max()) if win.any() else None
    out["t_of_max"] = float(t[win][np.argmax(err[win])]) if win.any() else None
    for ta in at:
        k = int(np.argmin(np.abs(t - ta)))
        out[f"front_err_t{ta:g}"] = float(err[k]) if abs(t[k] - ta) < 0.5 else None
    fw = np.array([r["Fw"] for r in ref])
    fwo = np.array([r["Fw"] for r in other])
    out["Fw_err_last_of_max"] = float(abs(fwo[-1] - fw[-1]) / max(np.abs(fw).max(), 1e-300))
    out["scalar_mass_err_last"] = float(abs(other[-1]["scalar_mass"] - ref[-1]["scalar_mass"]) /
                                        abs(ref[-1]["scalar_mass"]))
    out["t_last"] = float(t[-1])
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__,
                                 formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--nx", type=int, required=True)
    ap.add_argument("--ny", type=int, required=True)
    ap.add_argument("--nz", type=int, required=True)
    ap.add_argument("--H", type=int, required=True)
    ap.add_argument("--x0", type=int, required=True)
    ap.add_argument("--ub", type=float, default=0.03)
    ap.add_argument("--Re", type=float, required=True)
    ap.add_argument("--model", default="cumulant", choices=sorted(lbm.MODELS))
    ap.add_argument("--storages", default="fp16s,bf16s")
    ap.add_argument("--seed", type=int, default=2112)
    ap.add_argument("--t-end", type=float, required=True)
    ap.add_argument("--every", type=int, default=100)
    ap.add_argument("--at", type=float, nargs="*", default=[10.0, 20.0])
    ap.add_argument("--t0", type=float, default=2.5)
    ap.add_argument("--out", default=None, help="JSON lines: every logged record of every run")
    a = ap.parse_args(argv)
    steps = int(round(a.t_end * a.H / a.ub))
    runs = {}
    walls = {}
    for storage in ["fp32"] + [s for s in a.storages.split(",") if s]:
        p = lbm.lock_exchange(a.nx, a.ny, a.nz, H=a.H, x0=a.x0, u_b=a.ub, Re=a.Re,
                              model=a.model, storage=storage, seed=a.seed)
        recs, wall = run(p, a.ub, steps, a.every)
        runs[storage] = recs
        walls[storage] = wall
        print(json.dumps({"storage": storage, "wall_s": wall,
                          "mnups_incl_diag": p.N * steps / wall / 1e6, "final": recs[-1]}),
              flush=True)
    if a.out:
        with open(a.out, "w") as fh:
            for s, recs in runs.items():
                for r in recs:
                    fh.write(json.dumps(dict(r, storage=s)) + "\n")
    summary = {"box": [a.nx, a.ny, a.nz], "H": a.H, "x0": a.x0, "u_b": a.ub, "Re": a.Re,
               "model": a.model, "steps": steps, "every": a.every}
    for s, recs in runs.items():
        if s != "fp32":
            summary[s] = compare(runs["fp32"], recs, a.nx, a.at, a.t0)
    print(json.dumps(summary), flush=True)
    return summary


if __name__ == "__main__":
    sys.exit(0 if main() else 1)
