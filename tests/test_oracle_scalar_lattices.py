"""Pins of the oracle's alternative scalar lattices: D3Q6 BGK (Eq. 29-31 as
printed, RAFSINE) and D3Q27 with factorized central moments (Eq. 37-51,
VirtualFluids).  Expected values are closed forms of the moments, the printed
velocity table, an equilibrium fixed point and the exact diffusion-moment
recurrence."""
import os

import numpy as np
import pytest

import oracle as O
from paper_2112_08479_gb300 import inputs

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _params(scalar, **kw):
    base = dict(nx=1, ny=1, nz=1, model=1 if scalar == 2 else 0, nu=0.02, D=0.015,
                cs_smag=0.0, sc_t=1.0, gprime=2e-3, eg=(0.3, -0.4, -0.866), scalar=scalar)
    base.update(kw)
    return O.OracleParams(**base)


def test_d3q6_matches_eq31():
    c, w = O.velocities_scalar(1)
    rows = [ln.split() for ln in open(os.path.join(GOLD, "d3q6_eq31.txt"))
            if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 6
    for k, r in enumerate(rows):
        assert tuple(c[k]) == tuple(int(v) for v in r[:3])
        assert w[k] == pytest.approx(int(r[3]) / int(r[4]), abs=1e-16)
    assert np.allclose(np.einsum("k,ka,kb->ab", w, c, c), np.eye(3) / 3)   # c_s^2 = 1/3


def test_phieq_q6_moments():
    c, _ = O.velocities_scalar(1)
    u = np.array([0.03, -0.02, 0.05])
    pe = O.phieq_q6(0.7, u)
    assert pe.sum() == pytest.approx(0.7, rel=1e-15)
    assert np.allclose(c.T @ pe, 0.7 * u, atol=1e-16)


def _node(scalar, seed, amp=0.1):
    c, w = O.velocities_scalar(scalar)
    chi = 0.6
    phi = w * chi * (1.0 + inputs.uniform(len(w), seed, amp))
    f = O.velocities(0 if scalar != 2 else 1)[1] * (1 + inputs.uniform(27 if scalar == 2 else 19, seed + 1, 0.02))
    return f, phi, c.astype(float)


@pytest.mark.parametrize("scalar", [1, 2])
@pytest.mark.parametrize("seed", [1, 2])
def test_scalar_conservation_and_first_moment(scalar, seed):
    p = _params(scalar)
    f, phi, c = _node(scalar, seed)
    _, po = O.collide_node(p, f, phi)
    chi = phi.sum()
    cq = O.velocities(p.model)[0].astype(float)
    F = p.gprime * chi * np.array(p.eg)
    u = (cq.T @ f + F / 2) / f.sum()
    assert po.sum() == pytest.approx(chi, rel=1e-14)
    if scalar == 1:
        om = 1 / (0.5 + 3 * p.D)                       # Eq. 30 with c_s^2 = 1/3
        expect = (1 - om) * (c.T @ phi) + om * chi * u
    else:
        om = 1 / (3 * p.D + 0.5)                       # Eq. 51
        expect = chi * u + (1 - om) * (c.T @ phi - chi * u)
    assert np.allclose(c.T @ po, expect, atol=1e-16)


@pytest.mark.parametrize("omh", [1.0, 0.6])
def test_fcm_second_central_moments(omh):
    """Eq. 44 and 50: M_200 = kappa_200 - chi/3 and M_110 = kappa_110 relax by
    (1 - omega) towards 0."""
    p = _params(2, omega_phi_high=omh)
    f, phi, c = _node(2, 7)
    _, po = O.collide_node(p, f, phi)
    cq = O.velocities(1)[0].astype(float)
    chi = phi.sum()
    u = (cq.T @ f + p.gprime * chi * np.array(p.eg) / 2) / f.sum()
    d0 = c - u
    k0 = np.einsum("k,ka,kb->ab", phi, d0, d0)
    k1 = np.einsum("k,ka,kb->ab", po, d0, d0)
    expect = (1 - omh) * (k0 - chi * np.eye(3) / 3) + chi * np.eye(3) / 3
    assert np.allclose(k1, expect, atol=1e-15)


def test_fcm_fourth_and_sixth_order_moments():
    """Eq. 46 and 49 with the equilibrium shares chi/9 and chi/27:
    kappa*_220 = (1 - w)(kappa_220 - chi/9) + chi/9, same for 222 with 1/27."""
    omh = 0.6
    p = _params(2, omega_phi_high=omh)
    f, phi, c = _node(2, 9, amp=0.3)
    _, po = O.collide_node(p, f, phi)
    cq = O.velocities(1)[0].astype(float)
    chi = phi.sum()
    u = (cq.T @ f + p.gprime * chi * np.array(p.eg) / 2) / f.sum()
    d0 = c - u
    for (a, b, cc), share in (((2, 2, 0), 1 / 9), ((0, 2, 2), 1 / 9), ((2, 2, 2), 1 / 27)):
        mono = d0[:, 0] ** a * d0[:, 1] ** b * d0[:, 2] ** cc
        k0, k1 = np.sum(phi * mono), np.sum(po * mono)
        assert k1 == pytest.approx((1 - omh) * (k0 - share * chi) + share * chi, abs=1e-15)


@pytest.mark.parametrize("omh", [1.0, 0.6])
def test_fcm_equilibrium_is_fixed_point(omh):
    """The D3Q27 equilibrium chi prod_a E(c_a), E(0) = 2/3 - u_a^2,
    E(+-1) = (1/3 + u_a^2 +- u_a)/2, has M = 0 for every order >= 1, so it
    is a fixed point whatever the rates."""
    p = _params(2, gprime=0.0, omega_phi_high=omh)
    c27, w27 = O.velocities(1)
    u = np.array([0.04, -0.03, 0.02])
    f = np.array([np.prod([2/3 - u[a]**2 if ci[a] == 0 else (1/3 + u[a]**2 + ci[a] * u[a]) / 2
                           for a in range(3)]) for ci in c27])
    chi = 0.8
    phi = chi * f
    _, po = O.collide_node(p, f, phi)
    assert np.allclose(po, phi, atol=1e-16)


@pytest.mark.parametrize("scalar", [1, 2])
def test_diffusion_moment_recurrence_cs2_third(scalar):
    """As for D3Q7 but with c_s^2 = 1/3: A(t) = c^2 N (1 - (1-w)^t) / w,
    M2(t+1) - M2(t) = c^2 N + 2 (1-w) A(t), w = 1/(1/2 + 3 D); the increment
    tends to 2 D N."""
    L, T, D = 27, 10, 0.03
    p = O.OracleParams(L, L, L, model=1 if scalar == 2 else 0, nu=0.1, D=D, cs_smag=0.0,
                       periodic_x=True, periodic_z=True, scalar=scalar)
    chi0 = np.zeros((L, L, L))
    chi0[L // 2, L // 2, L // 2] = 1.0
    chi0[L // 2, L // 2 - 1, L // 2 + 1] = 0.25
    f, phi = O.init(p, chi0)
    N = chi0.sum()
    x = np.arange(L) - L // 2
    w = 1 / (0.5 + 3 * D)

    def M2(phi):
        return np.sum(phi.sum(-1) * x[None, None, :] ** 2)

    m_prev = M2(phi)
    for t in range(T):
        A = N / 3 * (1 - (1 - w) ** t) / w
        f, phi = O.run(p, 1, f, phi)
        m = M2(phi)
        assert m - m_prev == pytest.approx(N / 3 + 2 * (1 - w) * A, rel=1e-12)
        m_prev = m


@pytest.mark.parametrize("scalar", [1, 2])
def test_single_particle_scalar_streaming(scalar):
    nx, ny, nz = 4, 3, 3
    p = O.OracleParams(nx, ny, nz, model=0, scalar=scalar)
    c, _ = O.velocities_scalar(scalar)
    S = len(c)
    opp = [int(np.where((c == -c[k]).all(1))[0][0]) for k in range(S)]
    for (x, y, z) in [(0, 0, 0), (3, 2, 2), (1, 1, 1)]:
        for k in range(S):
            post = np.zeros((nz, ny, nx, S))
            post[z, y, x, k] = 1.0
            _, ph = O.stream(p, np.zeros((nz, ny, nx, 19)), post)
            xd, yd, zd = x + c[k][0], (y + c[k][1]) % ny, z + c[k][2]
            where = (zd, yd, xd, k) if (0 <= xd < nx and 0 <= zd < nz) else (z, y, x, opp[k])
            assert ph[where] == 1.0 and ph.sum() == 1.0


@pytest.mark.parametrize("scalar,model", [(1, 0), (2, 1)])
def test_lock_exchange_conserves_scalar(scalar, model):
    p = O.OracleParams(24, 4, 8, model=model, nu=2e-3, D=2e-3, gprime=4e-4, scalar=scalar)
    f, phi = O.init(p, O.lock_chi0(24, 4, 8, 8))
    d0 = O.diag(p, f, phi, 8, 8.0)
    f, phi = O.run(p, 40, f, phi)
    d1 = O.diag(p, f, phi, 8, 8.0)
    assert d1["scalar_mass"] == pytest.approx(d0["scalar_mass"], rel=1e-13)
    assert d1["front"] > d0["front"]
