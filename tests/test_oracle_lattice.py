"""Pins of the oracle's lattice tables, equilibria and random-number generator.

Each test checks the oracle against something other than itself: the vectors
printed in Eq. 23, 24 and 36, textbook lattice isotropy identities, the moment
identities the equilibria must satisfy, and the published splitmix64 outputs.
"""
import itertools
import os

import numpy as np
import pytest

import oracle as O

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    with open(os.path.join(GOLD, name)) as fh:
        return [ln.split() for ln in fh if ln.strip() and not ln.startswith("#")]


def test_d3q19_matches_eq23_eq24():
    c, w = O.velocities(0)
    rows = _rows("d3q19_eq23.txt")
    assert len(rows) == 19
    for r in rows:
        i = int(r[0])
        assert tuple(c[i]) == (int(r[1]), int(r[2]), int(r[3]))
        assert w[i] == pytest.approx(int(r[4]) / int(r[5]), abs=1e-16)


def test_d3q27_contains_eq36_and_is_complete():
    c, w = O.velocities(1)
    printed = [tuple(int(v) for v in r) for r in _rows("d3q27_eq36.txt")]
    # the first 19 follow Eq. 36 (identical to Eq. 23) in order
    assert [tuple(v) for v in c[:19]] == printed[:19]
    # all printed vectors are present and the set is all of {-1,0,1}^3
    assert set(printed) <= set(map(tuple, c))
    assert set(map(tuple, c)) == set(itertools.product((-1, 0, 1), repeat=3))
    # product weights (2/3, 1/6, 1/6) per axis
    for ci, wi in zip(c, w):
        n = int(np.sum(ci != 0))
        assert wi == pytest.approx((2 / 3) ** (3 - n) * (1 / 6) ** n, abs=1e-16)


@pytest.mark.parametrize("model", [0, 1])
def test_lattice_isotropy(model):
    """sum w = 1, sum w c_a c_b = delta/3, fourth-order tensor = (dd+dd+dd)/9."""
    c, w = O.velocities(model)
    c = c.astype(float)
    assert w.sum() == pytest.approx(1.0, abs=1e-15)
    assert np.allclose(np.einsum("i,ia->a", w, c), 0, atol=1e-16)
    assert np.allclose(np.einsum("i,ia,ib->ab", w, c, c), np.eye(3) / 3, atol=1e-15)
    assert np.allclose(np.einsum("i,ia,ib,ic->abc", w, c, c, c), 0, atol=1e-16)
    d = np.eye(3)
    iso = (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
           + np.einsum("ad,bc->abcd", d, d)) / 9
    assert np.allclose(np.einsum("i,ia,ib,ic,id->abcd", w, c, c, c, c), iso, atol=1e-15)


def test_d3q7_reading_r1():
    c, w = O.velocities_q7()
    assert set(map(tuple, c)) == {(0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0),
                                  (0, 0, 1), (0, 0, -1)}
    assert w.sum() == pytest.approx(1.0, abs=1e-16)
    # c_sPhi^2 = 1/4 on this lattice
    assert np.allclose(np.einsum("k,ka,kb->ab", w, c, c), np.eye(3) / 4, atol=1e-16)


def test_feq_moment_identities():
    """Eq. 22: sum feq = rho, sum c feq = rho u, sum cc feq = rho (I/3 + uu)."""
    c, _ = O.velocities(0)
    c = c.astype(float)
    rng = np.random.default_rng(3)
    for _ in range(20):
        rho = 1 + rng.uniform(-0.05, 0.05)
        u = rng.uniform(-0.1, 0.1, 3)
        feq = O.feq_q19(rho, u)
        assert feq.sum() == pytest.approx(rho, rel=1e-15)
        assert np.allclose(c.T @ feq, rho * u, atol=1e-16)
        assert np.allclose(np.einsum("i,ia,ib->ab", feq, c, c),
                           rho * (np.eye(3) / 3 + np.outer(u, u)), atol=1e-15)


def test_phieq_moment_identities():
    """Eq. 29 on D3Q7 (R1): sum Phi_eq = chi, sum c Phi_eq = chi u."""
    c, _ = O.velocities_q7()
    rng = np.random.default_rng(4)
    for _ in range(20):
        chi = rng.uniform(0, 1)
        u = rng.uniform(-0.1, 0.1, 3)
        pe = O.phieq_q7(chi, u)
        assert pe.sum() == pytest.approx(chi, rel=1e-15)
        assert np.allclose(c.T.astype(float) @ pe, chi * u, atol=1e-16)


def test_splitmix64_published_outputs():
    gamma = 0x9E3779B97F4A7C15
    for k, h in _rows("splitmix64.txt"):
        assert O.splitmix64((int(k) * gamma) & (2**64 - 1)) == int(h, 16)


def test_lock_initial_condition():
    """Table 1 / Sec. 2.5: chi0 = 1 in the lock x < x0, 0 outside; the gate
    column x0 - 1 carries a bounded zero-mean perturbation (R10)."""
    nx, ny, nz, x0, amp = 32, 8, 6, 10, 1e-3
    chi = O.lock_chi0(nx, ny, nz, x0, amp, 2112)
    assert np.all(chi[:, :, : x0 - 1] == 1.0)
    assert np.all(chi[:, :, x0:] == 0.0)
    col = chi[:, :, x0 - 1] - 1.0
    assert np.all(np.abs(col) <= amp) and np.std(col) > 0.3 * amp
    assert abs(col.mean()) < 4 * amp / np.sqrt(col.size)
    # the draw for node n is (splitmix64(seed ^ n) >> 11) * 2^-53
    n = (2 * ny + 3) * nx + (x0 - 1)
    r = (O.splitmix64(2112 ^ n) >> 11) * 2.0**-53
    assert chi[2, 3, x0 - 1] == 1.0 + amp * (2 * r - 1)
    # a different seed gives a different perturbation
    assert not np.array_equal(chi, O.lock_chi0(nx, ny, nz, x0, amp, 7))
