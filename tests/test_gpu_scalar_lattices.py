"""GPU parity of the alternative scalar lattices: D3Q6 BGK with the BGK fluid
(Eq. 29-31, RAFSINE) and D3Q27 factorized central moments with the cumulant
fluid (Eq. 37-51, VirtualFluids), against the FP64 oracle."""
import numpy as np
import pytest

import oracle as O
from paper_2112_08479_gb300 import inputs, lbm

from helpers import (canonical_to_oracle, lock_state_oracle, oracle_params, oracle_to_canonical,
                     rel_inf, rest_row_tol, stored_phi, weights, wscalar)

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

PAIRS = [(lbm.LBM_BGK_SMAG_Q19, lbm.LBM_SCALAR_Q6), (lbm.LBM_CUMULANT_Q27, lbm.LBM_SCALAR_Q27)]


def _random_state(p, seed, amp=0.05):
    w = weights(p.model)
    ws = wscalar(p)
    fdev = w[:, None] * inputs.uniform((p.Q, p.N), seed, amp)
    chi = 0.5 * (1.0 + inputs.uniform(p.N, seed + 1, 1.0))
    phi = ws[:, None] * (chi[None, :] * (1.0 + inputs.uniform((p.NS, p.N), seed + 2, amp)) - 1.0)
    return np.concatenate([fdev, phi]).astype(np.float32)


@pytest.mark.parametrize("model,scalar", PAIRS)
@pytest.mark.parametrize("shape", [(5, 3, 4), (66, 3, 2), (2, 2, 3)])
@pytest.mark.parametrize("flags", [0, lbm.LBM_FLAG_PERIODIC_X | lbm.LBM_FLAG_PERIODIC_Z])
def test_streaming_permutation_bit_exact(model, scalar, shape, flags):
    nx, ny, nz = shape
    p = lbm.Params(nx, ny, nz, model=model, scalar=scalar,
                   flags=lbm.LBM_FLAG_NO_COLLIDE | flags, x0=1, H=nz)
    lat = lbm.Lattice(p, device="cuda")
    s0 = inputs.distinct_values((p.Q + p.NS, p.N), 5).astype(np.float32)
    lat.set_state(torch.from_numpy(s0).cuda())
    op = oracle_params(p)
    f, phi = canonical_to_oracle(s0, p, shifted=False)
    for n in range(1, 5):
        lat.step(1)
        f, phi = O.step(op, f, phi)
        got = lat.get_state().cpu().numpy()
        assert np.array_equal(got, oracle_to_canonical(f, phi, p, shifted=False).astype(np.float32)), n


@pytest.mark.parametrize("model,scalar", PAIRS)
@pytest.mark.parametrize("shape", [(33, 5, 6), (66, 3, 4)])
def test_random_state_two_steps(model, scalar, shape):
    nx, ny, nz = shape
    p = lbm.Params(nx, ny, nz, model=model, scalar=scalar, nu=0.01, D=0.012, cs_smag=0.3,
                   sc_t=0.7, gprime=2e-3, eg=(0.48, 0.6, -0.64), x0=1, H=nz)
    lat = lbm.Lattice(p, device="cuda")
    s0 = _random_state(p, 13)
    lat.set_state(torch.from_numpy(s0).cuda())
    op = oracle_params(p)
    f, phi = canonical_to_oracle(s0, p)
    scale = np.abs(s0[: p.Q]).max()
    for n in (1, 2):
        lat.step(1)
        f, phi = O.step(op, f, phi)
        got = lat.get_state().cpu().numpy().astype(np.float64)
        want = oracle_to_canonical(f, phi, p)
        assert np.abs(got[: p.Q] - want[: p.Q]).max() < 1e-5 * scale, n
        assert np.abs(got[p.Q:] - want[p.Q:]).max() < 1e-6, n


@pytest.mark.parametrize("model,scalar,steps", [(0, 1, 500), (1, 2, 60)])
def test_lock_exchange_runs(model, scalar, steps):
    p = lbm.lock_exchange(64, 4, 16, H=16, x0=16, u_b=0.05, Re=1000.0,
                          model="bgk" if model == 0 else "cumulant",
                          scalar="q6" if scalar == 1 else "q27")
    lat = lbm.Lattice(p, device="cuda")
    op, (f, phi) = lock_state_oracle(p)
    lat.step(steps)
    f, phi = O.run(op, steps, f, phi)
    rho, u, chi = (t.cpu().numpy() for t in lat.macros())
    rho_o, u_o, chi_o = O.macros(op, f, phi)
    assert np.abs(rho - rho_o).max() < 1e-5
    assert rel_inf(np.moveaxis(u, 0, -1), u_o) < 1e-4
    # FP32 against FP64: at most one unit roundoff of chi per step, accumulated
    # linearly over the run (measured 1.2e-5 after 500 BGK + D3Q6 steps)
    assert rel_inf(chi, chi_o) < max(1e-5, steps * 2.0**-24)
    d = lat.diag()
    do = O.diag(op, f, phi, p.x0, float(p.H))
    assert abs(d["front"] - do["front"]) < 1e-4
    assert d["scalar_mass"] == pytest.approx(do["scalar_mass"], rel=1e-6)


@pytest.mark.parametrize("model,scalar", [("bgk", "q6"), ("cumulant", "q27")])
def test_scalar_mass_conserved(model, scalar):
    p = lbm.lock_exchange(256, 32, 64, H=64, x0=64, u_b=0.04, Re=5000.0, model=model, scalar=scalar)
    lat = lbm.Lattice(p, device="cuda")
    d0 = lat.diag()
    steps = 2000
    lat.step(steps)
    d1 = lat.diag()
    # round-off bound as in the D3Q7 long-run test: one unit roundoff of each
    # stored |Phi - w| (summing to at most 1.5 per node) per node and step, x2
    assert abs(d1["scalar_mass"] - d0["scalar_mass"]) < 2 * 2.0**-24 * 1.5 * p.N * steps
    assert d1["front"] > d0["front"] and d1["flags"] == 0


@pytest.mark.parametrize("storage", [lbm.LBM_FP16S, lbm.LBM_BF16S])
@pytest.mark.parametrize("model,scalar", PAIRS)
def test_16bit_one_step_within_rounding(storage, model, scalar):
    p = lbm.Params(33, 4, 6, model=model, scalar=scalar, storage=storage, nu=0.01, D=0.012,
                   cs_smag=0.3, gprime=2e-3, eg=(0.48, 0.6, -0.64), x0=1, H=6)
    lat = lbm.Lattice(p, device="cuda")
    lat.set_state(torch.from_numpy(_random_state(p, 6)).cuda())
    s0 = lat.get_state().cpu().numpy()
    op = oracle_params(p)
    f, phi = canonical_to_oracle(s0, p)
    f, phi = O.step(op, f, phi)
    lat.step(1)
    got = lat.get_state().cpu().numpy().astype(np.float64)
    want = oracle_to_canonical(f, phi, p)
    rel = 2.0**-11 if storage == lbm.LBM_FP16S else 2.0**-8
    scale = np.abs(s0[: p.Q]).max()
    mag = np.concatenate([np.abs(want[: p.Q]), stored_phi(want[p.Q:], p)])   # what is stored
    tol = rel * mag * 1.01 + 1e-5 * np.r_[[scale] * p.Q, [1e-1] * p.NS][:, None]
    if scalar == lbm.LBM_SCALAR_Q27:   # FP32 rest population with rounding feedback
        tol[p.Q] = rest_row_tol(p, s0, rel) + 1e-6
    assert np.all(np.abs(got - want) <= tol)


def test_adjoint_rejects_other_scalar_lattices():
    """The adjoint exists for the D3Q7 scalar only (either fluid)."""
    p = lbm.Params(8, 2, 4, scalar=lbm.LBM_SCALAR_Q6, x0=1, H=4)
    lat = lbm.Lattice(p, device="cuda")
    st = lat.get_state()
    with pytest.raises(lbm.LBMError) as e:
        lat.adjoint_step(st, None, torch.empty_like(st), None, 1.0)
    assert e.value.status == lbm.LBM_ERR_STATE
