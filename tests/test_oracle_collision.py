"""Pins of the oracle's single-node collisions.

BGK-Smagorinsky + Guo (Eq. 21-26, 32-34), scalar BGK on D3Q7 (Eq. 28-30, 35)
and the cumulant operator (Eq. 54-58).  Expected values come from moment
identities computed here with numpy, from a quadratic solved by numpy, and
from the textbook partition formula for joint cumulants - never from the
oracle's own formulas.
"""
import itertools
import math

import numpy as np
import pytest

import oracle as O
from paper_2112_08479_gb300 import inputs

C19, W19 = O.velocities(0)
C27, W27 = O.velocities(1)
C7, W7 = O.velocities_q7()


def _state(model, seed, amp=0.02, chi=0.6):
    c, w = (C27, W27) if model == 1 else (C19, W19)
    f = w * (1.0 + inputs.uniform(len(w), seed, amp))
    phi = W7 * chi * (1.0 + inputs.uniform(7, seed + 1, amp))
    return f, phi


def _params(model, **kw):
    base = dict(nx=1, ny=1, nz=1, model=model, nu=0.02, D=0.015, cs_smag=0.17, sc_t=0.8,
                gprime=3e-3, eg=(0.3, -0.4, -0.8660254037844386))
    base.update(kw)
    return O.OracleParams(**base)


@pytest.mark.parametrize("model", [0, 1])
@pytest.mark.parametrize("seed", [1, 2, 3])
def test_mass_and_momentum_with_force(model, seed):
    """Collision conserves mass and adds exactly the impulse F (Eq. 17, 20, 26)."""
    p = _params(model)
    c = (C27 if model == 1 else C19).astype(float)
    f, phi = _state(model, seed)
    fo, po = O.collide_node(p, f, phi)
    chi = phi.sum()
    F = p.gprime * chi * np.array(p.eg)
    assert fo.sum() == pytest.approx(f.sum(), rel=1e-14)
    assert np.allclose(c.T @ fo, c.T @ f + F, atol=1e-15)
    assert po.sum() == pytest.approx(chi, rel=1e-14)


def _pi_and_tau(p, f, rho, u):
    """Pi = sum cc f - rho (I/3 + uu) and the positive root of the quadratic
    tau^2 - tau0 tau - (9/sqrt2) C_s^2 q / rho = 0 (reading R3)."""
    c = C19.astype(float)
    Pi = np.einsum("i,ia,ib->ab", f, c, c) - rho * (np.eye(3) / 3 + np.outer(u, u))
    q = np.linalg.norm(Pi)
    tau0 = 3 * p.nu + 0.5
    roots = np.roots([1.0, -tau0, -(9 / math.sqrt(2)) * p.cs_smag**2 * q / rho])
    return Pi, q, float(max(roots.real)), tau0


@pytest.mark.parametrize("cs", [0.0, 0.17, 0.5])
@pytest.mark.parametrize("seed", [5, 6])
def test_bgk_second_moment_and_guo(cs, seed):
    """sum cc f_out = (1 - 1/tau) sum cc f + rho (I/3 + uu)/tau + (1 - 1/2tau)(uF + Fu)."""
    p = _params(0, cs_smag=cs)
    c = C19.astype(float)
    f, phi = _state(0, seed, amp=0.05)
    fo, _ = O.collide_node(p, f, phi)
    rho = f.sum()
    F = p.gprime * phi.sum() * np.array(p.eg)
    u = (c.T @ f + F / 2) / rho
    _, _, tau, tau0 = _pi_and_tau(p, f, rho, u)
    if cs == 0.0:
        assert tau == pytest.approx(tau0, rel=1e-15)
    m2 = np.einsum("i,ia,ib->ab", f, c, c)
    expect = (1 - 1 / tau) * m2 + rho * (np.eye(3) / 3 + np.outer(u, u)) / tau \
        + (1 - 0.5 / tau) * (np.outer(u, F) + np.outer(F, u))
    assert np.allclose(np.einsum("i,ia,ib->ab", fo, c, c), expect, atol=2e-15)


def test_tau_eff_closed_form_solves_quadratic():
    rng = np.random.default_rng(9)
    for _ in range(50):
        tau0 = rng.uniform(0.5, 1.5)
        cs = rng.uniform(0, 0.5)
        q = rng.uniform(0, 1e-2)
        rho = rng.uniform(0.9, 1.1)
        t = O.tau_eff(tau0, cs, q, rho)
        assert t * t - tau0 * t - 9 / math.sqrt(2) * cs * cs * q / rho == pytest.approx(0, abs=1e-15)
        assert t >= tau0
    assert O.tau_eff(0.7, 0.0, 1.0, 1.0) == 0.7


@pytest.mark.parametrize("model", [0, 1])
def test_scalar_collision_first_moment(model):
    """Eq. 28-30 on D3Q7: the first moment relaxes to chi u at rate 1/tau_Phi,
    with tau_Phi = 1/2 + D_eff / c_sPhi^2 and D_eff = D + nu_T / Sc_T (Eq. 35, R4)."""
    p = _params(model)
    f, phi = _state(model, 11, amp=0.05)
    _, po = O.collide_node(p, f, phi)
    c = (C27 if model == 1 else C19).astype(float)
    chi = phi.sum()
    F = p.gprime * chi * np.array(p.eg)
    rho = f.sum()
    u = (c.T @ f + F / 2) / rho
    if model == 0:
        _, _, tau, tau0 = _pi_and_tau(p, f, rho, u)
        Deff = p.D + (tau - tau0) / 3 / p.sc_t
        assert O.bgk_nu_t(p, f, phi) == pytest.approx((tau - tau0) / 3, rel=1e-12)
    else:
        Deff = p.D
    tp = 0.5 + 4 * Deff
    c7 = C7.astype(float)
    assert np.allclose(c7.T @ po, (1 - 1 / tp) * (c7.T @ phi) + chi * u / tp, atol=1e-16)
    # second moment of each axis relaxes towards chi c_sPhi^2 = chi / 4
    assert np.allclose(np.einsum("k,ka,ka->a", po, c7, c7),
                       (1 - 1 / tp) * np.einsum("k,ka,ka->a", phi, c7, c7) + chi / 4 / tp, atol=1e-16)


# --- cumulants -----------------------------------------------------------------


def _set_partitions(seq):
    if not seq:
        yield []
        return
    first, rest = seq[0], seq[1:]
    for part in _set_partitions(rest):
        for k in range(len(part)):
            yield part[:k] + [[first] + part[k]] + part[k + 1:]
        yield [[first]] + part


def _joint_cumulant(f, idx):
    """Textbook partition formula: kappa(X_1..X_n) = sum over set partitions pi
    of (|pi|-1)! (-1)^(|pi|-1) prod_B E[prod_{j in B} X_j], E = sum f c / rho."""
    c = C27.astype(float)
    rho = f.sum()
    total = 0.0
    for part in _set_partitions(list(range(len(idx)))):
        prod = 1.0
        for block in part:
            prod *= np.sum(f * np.prod([c[:, idx[j]] for j in block], axis=0)) / rho
        k = len(part)
        total += math.factorial(k - 1) * (-1) ** (k - 1) * prod
    return total


def test_cumulants_match_partition_formula():
    f, _ = _state(1, 21, amp=0.3)
    Cs = O.cumulants27(f)
    assert Cs[0] == pytest.approx(math.log(f.sum()), rel=1e-14)
    for a, b, c in itertools.product(range(3), repeat=3):
        if a + b + c == 0:
            continue
        idx = [0] * a + [1] * b + [2] * c
        assert Cs[(a * 3 + b) * 3 + c] == pytest.approx(_joint_cumulant(f, idx), abs=1e-14), (a, b, c)


def test_cumulant_round_trip():
    for seed in range(5):
        f, _ = _state(1, 30 + seed, amp=0.3)
        assert np.allclose(O.f_from_cumulants27(O.cumulants27(f)), f, atol=1e-15)


@pytest.mark.parametrize("gprime", [0.0, 3e-3])
def test_cumulant_rate_one_gives_product_equilibrium(gprime):
    """omega1 = omega_bulk = 1 (tau = 1, nu = 1/6): f_out = rho phi(ux) phi(uy) phi(uz)
    with phi_0 = 2/3 - u^2, phi_+-1 = (1/3 + u^2 +- u)/2 and u = (j + F)/rho."""
    p = _params(1, nu=1.0 / 6.0, gprime=gprime)
    f, phi = _state(1, 40, amp=0.2)
    fo, _ = O.collide_node(p, f, phi)
    c = C27.astype(float)
    rho = f.sum()
    us = (c.T @ f + p.gprime * phi.sum() * np.array(p.eg)) / rho

    def ph(v, u):
        return 2 / 3 - u * u if v == 0 else (1 / 3 + u * u + v * u) / 2

    expect = np.array([rho * ph(ci[0], us[0]) * ph(ci[1], us[1]) * ph(ci[2], us[2]) for ci in C27])
    assert np.allclose(fo, expect, atol=1e-16)


def test_cumulant_relaxation_rates():
    """Eq. 55 on the post-collision cumulants: shear parts * (1 - omega1),
    trace -> (1 - omega_bulk) tr + omega_bulk, order >= 3 -> (1 - omega_high) C."""
    p = _params(1, nu=0.04, omega_bulk=0.7, omega_high=0.35, gprime=0.0)
    f, phi = _state(1, 50, amp=0.2)
    fo, _ = O.collide_node(p, f, phi)
    C0, C1 = O.cumulants27(f), O.cumulants27(fo)
    om1 = 1 / (3 * p.nu + 0.5)
    I = lambda a, b, c: (a * 3 + b) * 3 + c  # noqa: E731
    assert C1[0] == pytest.approx(C0[0], abs=1e-15)
    for k in (I(1, 0, 0), I(0, 1, 0), I(0, 0, 1)):
        assert C1[k] == pytest.approx(C0[k], abs=1e-15)
    for k in (I(1, 1, 0), I(1, 0, 1), I(0, 1, 1)):
        assert C1[k] == pytest.approx((1 - om1) * C0[k], abs=1e-15)
    d = lambda C: (C[I(2, 0, 0)] - C[I(0, 2, 0)], C[I(2, 0, 0)] - C[I(0, 0, 2)])  # noqa: E731
    tr = lambda C: C[I(2, 0, 0)] + C[I(0, 2, 0)] + C[I(0, 0, 2)]  # noqa: E731
    assert np.allclose(d(C1), (1 - om1) * np.array(d(C0)), atol=1e-15)
    assert tr(C1) == pytest.approx((1 - 0.7) * tr(C0) + 0.7, abs=1e-15)
    for a, b, c in itertools.product(range(3), repeat=3):
        if a + b + c >= 3:
            assert C1[I(a, b, c)] == pytest.approx((1 - 0.35) * C0[I(a, b, c)], abs=1e-14)


def test_no_collide_is_identity():
    p = _params(0, no_collide=True)
    f, phi = _state(0, 60)
    fo, po = O.collide_node(p, f, phi)
    assert np.array_equal(fo, f) and np.array_equal(po, phi)
