"""Pins of the FP64 reference gradient (oracle/adjoint_ref.py).

Its forward step is a second, independent restatement of the BGK step and must
agree with the C oracle to round-off; its gradient must agree with central
finite differences of the objective computed by the C oracle."""
import numpy as np
import pytest

import oracle as O
from oracle import adjoint_ref as A
from paper_2112_08479_gb300 import inputs

torch = pytest.importorskip("torch")


def _params(nx=16, ny=4, nz=6, **kw):
    base = dict(nx=nx, ny=ny, nz=nz, model=0, nu=9.6e-4 * 4, D=9.6e-4 * 4, cs_smag=0.17,
                sc_t=1.0, gprime=1.40625e-5 * 40)
    base.update(kw)
    return O.OracleParams(**base)


def _J_c_oracle(p, chi0, nsteps):
    f, phi = O.init(p, chi0)
    _, _, fw = O.run(p, nsteps, f, phi, record_fw=True)
    return float(fw.sum())


def test_torch_step_matches_c_oracle():
    p = _params(periodic_x=False)
    chi0 = O.lock_chi0(p.nx, p.ny, p.nz, 5, 1e-2, 3)
    f, phi = O.init(p, chi0)
    st = A.BGKStep(p)
    ft, pt = A.initial_state(st, chi0)
    cs = torch.tensor(p.cs_smag, dtype=torch.float64)
    with torch.no_grad():
        for _ in range(25):
            ft, pt = st(ft, pt, cs)
    f, phi = O.run(p, 25, f, phi)
    assert np.abs(ft.numpy() - f).max() < 1e-14
    assert np.abs(pt.numpy() - phi).max() < 1e-14
    assert A.objective(p, chi0, p.cs_smag, 25) == pytest.approx(_J_c_oracle(p, chi0, 25), rel=1e-12)


@pytest.mark.parametrize("flags", [{}, {"periodic_x": True}])
def test_gradient_matches_central_differences(flags):
    p = _params(**flags)
    n = 60
    chi0 = O.lock_chi0(p.nx, p.ny, p.nz, 5, 1e-2, 3)
    J, g, gcs = A.gradient(p, chi0, p.cs_smag, n)
    assert J == pytest.approx(_J_c_oracle(p, chi0, n), rel=1e-12)
    # eps = 1e-3 balances the O(eps^2) truncation against the FP64 round-off of
    # J (measured agreement ~3e-8 there, ~6e-7 at eps = 1e-4)
    eps = 1e-3
    for seed in (1, 2, 3):
        d = inputs.unit_direction(chi0.shape, seed)
        fd = (_J_c_oracle(p, chi0 + eps * d, n) - _J_c_oracle(p, chi0 - eps * d, n)) / (2 * eps)
        assert np.sum(g * d) == pytest.approx(fd, rel=1e-5)
    h = 1e-4
    pp, pm = _params(**flags), _params(**flags)
    pp.cs_smag += h
    pm.cs_smag -= h
    fd = (_J_c_oracle(pp, chi0, n) - _J_c_oracle(pm, chi0, n)) / (2 * h)
    assert gcs == pytest.approx(fd, rel=1e-5)
