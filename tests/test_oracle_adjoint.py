"""Pins of the FP64 reference gradient (oracle/adjoint_ref.py).

Its forward step is a second, independent restatement of the BGK step and must
agree with the C oracle to round-off; its gradient must agree with central
finite differences of the objective computed by the C oracle."""
import os

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


# ---------------------------------------------------------------------------
# Front objective (Sec. 3.1, reading R11)

def _front_field(seed, nx=12, ny=3, nz=4, xc=6.4):
    """A distinct-valued scalar field that falls from ~1 to ~0 around x = xc,
    so that the threshold crossing lies between two interior columns."""
    x = np.arange(nx)[None, None, :]
    base = 1.0 / (1.0 + np.exp(3.0 * (x - xc)))
    noise = 0.05 * inputs.uniform((nz, ny, nx), seed, 1.0)
    return np.clip(base + noise * base, 0.0, None) + 1e-3 * inputs.uniform((nz, ny, nx), seed + 1, 1.0)


def _torch_front(chi, x0, H, thr=0.02):
    st = A.BGKStep(_params(nx=chi.shape[2], ny=chi.shape[1], nz=chi.shape[0]))
    c = torch.tensor(chi, dtype=torch.float64, requires_grad=True)
    phi = c[..., None] * st.w7
    f = st.w.expand(*chi.shape, 19)
    return st.front(f, phi, x0, H, thr), c


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_torch_front_matches_c_front(seed):
    chi = _front_field(seed)
    for thr in (0.02, 0.3, 0.9):
        J, _ = _torch_front(chi, 5, 4.0, thr)
        want = (O.front_node(chi, thr) + 0.5 - 5) / 4.0
        assert float(J.detach()) == pytest.approx(want, abs=1e-14)
    # no column reaches the threshold; the last column does
    J, _ = _torch_front(np.zeros((4, 3, 12)), 5, 4.0)
    assert float(J) == pytest.approx((-1 + 0.5 - 5) / 4.0)
    J, _ = _torch_front(np.ones((4, 3, 12)), 5, 4.0)
    assert float(J) == pytest.approx((11 + 0.5 - 5) / 4.0)


@pytest.mark.parametrize("seed", [1, 2])
def test_front_gradient_matches_central_differences_of_c_front(seed):
    """The interpolated front is smooth away from a change of crossing column
    or maximising z; node by node, the torch gradient equals central
    differences of the C oracle's front."""
    chi = _front_field(seed)
    x0, H, thr = 5, 4.0, 0.3
    J, c = _torch_front(chi, x0, H, thr)
    (g,) = torch.autograd.grad(J, c)
    g = g.numpy()
    eps = 1e-6
    fd = np.zeros_like(chi)
    for idx in np.ndindex(chi.shape):
        a, b = chi.copy(), chi.copy()
        a[idx] += eps
        b[idx] -= eps
        fd[idx] = ((O.front_node(a, thr) - O.front_node(b, thr)) / (2 * eps)) / H
    assert np.count_nonzero(fd) == 2 * chi.shape[1]      # (x_f, ., z0) and (x_f + 1, ., z1)
    assert np.abs(g - fd).max() < 1e-7 * np.abs(fd).max()


def _front_c_oracle(p, chi0, nsteps, x0, H):
    f, phi = O.init(p, chi0)
    f, phi = O.run(p, nsteps, f, phi)
    return O.diag(p, f, phi, x0, H)["front"]


def test_front_objective_gradient_matches_central_differences():
    """Adjoint of the front after n steps of the lock exchange against central
    differences of the C oracle, in random directions and in C_s."""
    p = _params()
    x0, H, n = 5, 6.0, 60
    chi0 = O.lock_chi0(p.nx, p.ny, p.nz, x0, 1e-2, 3)
    J, g, gcs = A.gradient(p, chi0, p.cs_smag, n, objective="front", x0=x0, H=H)
    assert J == pytest.approx(_front_c_oracle(p, chi0, n, x0, H), abs=1e-12)
    assert np.abs(g).max() > 0
    eps = 1e-3
    for seed in (1, 2, 3):
        d = inputs.unit_direction(chi0.shape, seed)
        fd = (_front_c_oracle(p, chi0 + eps * d, n, x0, H)
              - _front_c_oracle(p, chi0 - eps * d, n, x0, H)) / (2 * eps)
        assert np.sum(g * d) == pytest.approx(fd, rel=1e-4, abs=1e-9)
    h = 1e-3
    pp, pm = _params(), _params()
    pp.cs_smag += h
    pm.cs_smag -= h
    fd = (_front_c_oracle(pp, chi0, n, x0, H) - _front_c_oracle(pm, chi0, n, x0, H)) / (2 * h)
    assert gcs == pytest.approx(fd, rel=1e-4, abs=1e-9)


# ---------------------------------------------------------------------------
# Cumulant fluid (Eq. 54-58): torch restatement and its gradients

def test_torch_cumulant_step_matches_c_oracle():
    p = _params(model=1, omega_bulk=0.8, eg=(0.48, 0.6, -0.64))
    chi0 = O.lock_chi0(p.nx, p.ny, p.nz, 5, 1e-2, 3)
    f, phi = O.init(p, chi0)
    st = A.make_step(p)
    assert isinstance(st, A.CumulantStep)
    ft, pt = A.initial_state(st, chi0)
    cs = torch.tensor(p.cs_smag, dtype=torch.float64)
    with torch.no_grad():
        for _ in range(25):
            ft, pt = st(ft, pt, cs)
    f, phi = O.run(p, 25, f, phi)
    assert np.abs(ft.numpy() - f).max() < 1e-14
    assert np.abs(pt.numpy() - phi).max() < 1e-14
    assert A.objective(p, chi0, p.cs_smag, 25) == pytest.approx(_J_c_oracle(p, chi0, 25), rel=1e-12)


@pytest.mark.parametrize("objective", ["friction", "front"])
def test_cumulant_gradient_matches_central_differences(objective):
    p = _params(model=1)
    x0, H, n = 5, 6.0, 60
    chi0 = O.lock_chi0(p.nx, p.ny, p.nz, x0, 1e-2, 3)
    J, g, gcs = A.gradient(p, chi0, p.cs_smag, n, objective=objective, x0=x0, H=H)
    Jc = (_J_c_oracle if objective == "friction" else
          (lambda pp, c, nn: _front_c_oracle(pp, c, nn, x0, H)))
    assert J == pytest.approx(Jc(p, chi0, n), rel=1e-12)
    assert gcs == 0.0                     # no Smagorinsky closure in the cumulant model
    eps = 1e-3
    for seed in (1, 2, 3):
        d = inputs.unit_direction(chi0.shape, seed)
        fd = (Jc(p, chi0 + eps * d, n) - Jc(p, chi0 - eps * d, n)) / (2 * eps)
        assert np.sum(g * d) == pytest.approx(fd, rel=1e-4, abs=1e-9)


def _load_fd_golden():
    path = os.path.join(os.path.dirname(__file__), "golden", "fd_gradient_32x4x8.txt")
    head = {}
    vals = []
    for line in open(path):
        if line.startswith("# J "):
            head["J"] = float(line.split()[2])
        elif line.startswith("# dJ/dC_s "):
            head["cs"] = float(line.split()[2])
        elif not line.startswith("#"):
            vals.append(float(line))
    return head["J"], np.array(vals), head["cs"]


def test_reference_gradient_matches_full_fd_golden():
    """The FP64 reference gradient over 2,000 steps of the 32 x 4 x 8
    sub-case against the full central-difference gradient (all 1,024 chi0
    values and C_s) that tests/golden/make_fd_gradient.py computed with the C
    oracle."""
    J_fd, g_fd, cs_fd = _load_fd_golden()
    p = O.OracleParams(32, 4, 8, model=0, nu=9.6e-4, D=9.6e-4, cs_smag=0.17, sc_t=1.0,
                       gprime=1.40625e-5)
    chi0 = O.lock_chi0(32, 4, 8, 8, 1e-3, 2112)
    J, g, gcs = A.gradient(p, chi0, 0.17, 2000)
    assert J == pytest.approx(J_fd, rel=1e-12)
    g = g.ravel()
    assert np.linalg.norm(g - g_fd) < 1e-7 * np.linalg.norm(g_fd)
    assert np.abs(g - g_fd).max() < 1e-6 * np.abs(g_fd).max()
    assert gcs == pytest.approx(cs_fd, rel=1e-6)
