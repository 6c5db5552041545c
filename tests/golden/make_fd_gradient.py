"""Writes fd_gradient_32x4x8.txt: the central finite-difference gradient of
the time-integrated bottom friction J = sum_{n=1..2000} F_w(s_n) (Eq. 62-64)
with respect to every value of the initial scalar field chi0 and to C_s, on
the 32 x 4 x 8 differentiation sub-case (the lattice parameters of the
256 x 32 x 64 box: nu = D = 9.6e-4, g' = 1.40625e-5, C_s = 0.17, lock at
x0 = 8, walls in x and z, periodic y), computed with the FP64 C oracle only.

Central differences with step eps = 1e-4 on each chi0 value (truncation
O(eps^2) ~ 1e-8 relative; the oracle's FP64 round-off in J, ~1e-15 relative,
enters as ~1e-11 / eps) and h = 1e-4 on C_s.

    python tests/golden/make_fd_gradient.py      # about 10 minutes on 8 cores
"""
import multiprocessing as mp
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

NX, NY, NZ, X0, STEPS = 32, 4, 8, 8, 2000
NU, GP, CS, EPS, H = 9.6e-4, 1.40625e-5, 0.17, 1e-4, 1e-4


def _params(cs=CS):
    import oracle as O
    return O.OracleParams(NX, NY, NZ, model=0, nu=NU, D=NU, cs_smag=cs, sc_t=1.0, gprime=GP)


def _chi0():
    import oracle as O
    return O.lock_chi0(NX, NY, NZ, X0, 1e-3, 2112)


def _J(chi0, cs=CS):
    import oracle as O
    p = _params(cs)
    f, phi = O.init(p, chi0)
    _, _, fw = O.run(p, STEPS, f, phi, record_fw=True)
    return float(fw.sum())


def _fd(k):
    chi0 = _chi0()
    idx = np.unravel_index(k, chi0.shape)
    a, b = chi0.copy(), chi0.copy()
    a[idx] += EPS
    b[idx] -= EPS
    return k, (_J(a) - _J(b)) / (2 * EPS)


def main():
    chi0 = _chi0()
    n = chi0.size
    g = np.zeros(n)
    with mp.get_context("spawn").Pool(os.cpu_count()) as pool:
        for k, v in pool.imap_unordered(_fd, range(n)):
            g[k] = v
    gcs = (_J(chi0, CS + H) - _J(chi0, CS - H)) / (2 * H)
    J = _J(chi0)
    out = os.path.join(HERE, "fd_gradient_32x4x8.txt")
    with open(out, "w") as fh:
        fh.write("# Central finite-difference gradient of J = sum_{n=1..2000} F_w(s_n) (Eq. 62-64)\n")
        fh.write("# on the 32x4x8 sub-case, FP64 C oracle, written by make_fd_gradient.py.\n")
        fh.write(f"# J {J:.17e}\n# dJ/dC_s {gcs:.17e}\n")
        fh.write("# dJ/dchi0, node index n = x + 32 (y + 4 z):\n")
        for v in g:
            fh.write(f"{v:.17e}\n")
    print("wrote", out, "J", J, "|g|", np.linalg.norm(g), "dJ/dCs", gcs)


if __name__ == "__main__":
    main()
