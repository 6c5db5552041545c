"""Pins of the oracle's streaming, whole time step and diagnostics.

Closed forms and invariants: single-particle transport (Eq. 17 read as a
push), time reversal of streaming with bounce-back, conservation, the exact
momentum gain under a uniform force, plane Poiseuille flow, Taylor-Green
decay, an exact recurrence for the second moment of a diffusing scalar,
exact advective drift of the scalar, the Smagorinsky closure against a
finite-difference shear rate, and the diagnostics on fields with known
answers.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2112_08479_gb300 import inputs

C19, W19 = O.velocities(0)
C27, W27 = O.velocities(1)
C7, W7 = O.velocities_q7()


def _opp(c, i):
    return [j for j in range(len(c)) if tuple(c[j]) == tuple(-c[i])][0]


@pytest.mark.parametrize("model", [0, 1])
def test_single_particle_streaming(model):
    """A lone post-collision population at x moves to x + c_i (y periodic); if
    x + c_i is beyond an x or z wall it returns to x in the opposite direction
    (half-way bounce-back, Sec. 2.5)."""
    nx, ny, nz = 4, 3, 3
    p = O.OracleParams(nx, ny, nz, model=model)
    c = C27 if model == 1 else C19
    Q = len(c)
    for (x, y, z) in [(0, 0, 0), (3, 2, 2), (1, 1, 1), (0, 2, 1), (3, 0, 2)]:
        for i in range(Q):
            post = np.zeros((nz, ny, nx, Q))
            post[z, y, x, i] = 1.0
            f, _ = O.stream(p, post, np.zeros((nz, ny, nx, 7)))
            xd, yd, zd = x + c[i][0], (y + c[i][1]) % ny, z + c[i][2]
            if 0 <= xd < nx and 0 <= zd < nz:
                where = (zd, yd, xd, i)
            else:
                where = (z, y, x, _opp(c, i))
            assert f[where] == 1.0 and f.sum() == 1.0, (x, y, z, i)
    for (x, y, z) in [(0, 0, 0), (3, 2, 2), (2, 1, 1)]:
        for k in range(7):
            post = np.zeros((nz, ny, nx, 7))
            post[z, y, x, k] = 1.0
            _, ph = O.stream(p, np.zeros((nz, ny, nx, Q)), post)
            xd, yd, zd = x + C7[k][0], (y + C7[k][1]) % ny, z + C7[k][2]
            where = (zd, yd, xd, k) if (0 <= xd < nx and 0 <= zd < nz) else (z, y, x, _opp(C7, k))
            assert ph[where] == 1.0 and ph.sum() == 1.0


@pytest.mark.parametrize("model", [0, 1])
def test_streaming_time_reversal(model):
    """Streaming with bounce-back is reversible: stream, flip every direction,
    stream, flip again gives back the start exactly."""
    p = O.OracleParams(5, 3, 4, model=model)
    c = C27 if model == 1 else C19
    Q = len(c)
    opp = [_opp(c, i) for i in range(Q)]
    opp7 = [_opp(C7, k) for k in range(7)]
    f0 = inputs.distinct_values((4, 3, 5, Q), 1)
    p0 = inputs.distinct_values((4, 3, 5, 7), 2)
    f1, p1 = O.stream(p, f0, p0)
    f2, p2 = O.stream(p, f1[..., opp], p1[..., opp7])
    assert np.array_equal(f2[..., opp], f0) and np.array_equal(p2[..., opp7], p0)
    # and it is a permutation
    assert np.array_equal(np.sort(f1.ravel()), np.sort(f0.ravel()))


@pytest.mark.parametrize("model", [0, 1])
def test_lock_exchange_conserves_mass_and_scalar(model):
    p = O.OracleParams(24, 4, 8, model=model, nu=2e-3, D=2e-3, gprime=4e-4)
    chi0 = O.lock_chi0(24, 4, 8, 8)
    f, phi = O.init(p, chi0)
    d0 = O.diag(p, f, phi, 8, 8.0)
    f, phi = O.run(p, 60, f, phi)
    d1 = O.diag(p, f, phi, 8, 8.0)
    # FP64 round-off only: 1e-14 per node
    assert abs(d1["mass_delta"] - d0["mass_delta"]) < 1e-14 * 24 * 4 * 8
    assert d1["scalar_mass"] == pytest.approx(d0["scalar_mass"], rel=1e-13)
    # the current moves: the front advanced and the bottom friction is nonzero
    assert d1["front"] > d0["front"] and abs(d1["Fw"]) > 0


@pytest.mark.parametrize("model", [0, 1])
def test_uniform_force_periodic_momentum(model):
    """Fully periodic, uniform chi: total momentum grows by exactly N F per step,
    and u (with the half-force shift) = (n + 1/2) F / rho."""
    nx, ny, nz = 3, 2, 4
    p = O.OracleParams(nx, ny, nz, model=model, gprime=1e-3, eg=(0.6, 0.0, -0.8),
                       periodic_x=True, periodic_z=True, nu=0.05, D=0.05)
    f, phi = O.init(p, np.full((nz, ny, nx), 0.5))
    F = 1e-3 * 0.5 * np.array([0.6, 0.0, -0.8])
    c = (C27 if model == 1 else C19).astype(float)
    N = nx * ny * nz
    for n in range(1, 6):
        f, phi = O.run(p, 1, f, phi)
        j = np.einsum("zyxi,ia->a", f, c)
        assert np.allclose(j, n * N * F, atol=1e-15)
        _, u, _ = O.macros(p, f, phi)
        assert np.allclose(u, (n + 0.5) * F, atol=1e-15)


def _poiseuille(nz, tau, steps, F=1e-5, model=0):
    nu = (tau - 0.5) / 3
    p = O.OracleParams(1, 1, nz, model=model, nu=nu, D=nu, cs_smag=0.0, gprime=F,
                       eg=(1.0, 0.0, 0.0), periodic_x=True)
    f, phi = O.init(p, np.ones((nz, 1, 1)))
    f, phi = O.run(p, steps, f, phi)
    _, u, _ = O.macros(p, f, phi)
    z = np.arange(nz)
    exact = F / (2 * nu) * (z + 0.5) * (nz - 0.5 - z)
    return p, f, phi, u[:, 0, 0, 0], exact


def test_poiseuille_magic_tau_exact():
    """BGK + half-way bounce-back + Guo forcing is exact for plane Poiseuille
    flow at (tau - 1/2)^2 = 3/16; F_w = F nx ny nz / 2 exactly (Eq. 62-64)."""
    tau = 0.5 + math.sqrt(3 / 16)
    p, f, phi, u, exact = _poiseuille(12, tau, 6000)
    assert np.max(np.abs(u - exact)) / exact.max() < 1e-11
    d = O.diag(p, f, phi, 0, 1.0)
    assert d["Fw"] == pytest.approx(1e-5 * 12 / 2, rel=1e-10)


def test_poiseuille_second_order_convergence():
    errs = []
    for nz in (8, 16, 32):
        _, _, _, u, exact = _poiseuille(nz, 0.8, int(40 * nz * nz))
        errs.append(np.max(np.abs(u - exact)) / exact.max())
    assert errs[2] < 1e-3
    assert errs[0] / errs[1] == pytest.approx(4, rel=0.1)
    assert errs[1] / errs[2] == pytest.approx(4, rel=0.1)


def _taylor_green_rate(model, L, nu, steps=(200, 600), U=0.01):
    p = O.OracleParams(L, L, 1, model=model, nu=nu, D=nu, cs_smag=0.0, periodic_x=True,
                       periodic_z=True)
    k = 2 * math.pi / L
    x = np.arange(L)
    X, Y = np.meshgrid(x, x, indexing="xy")
    ux = U * np.sin(k * X) * np.cos(k * Y)
    uy = -U * np.cos(k * X) * np.sin(k * Y)
    f = np.zeros((1, L, L, p.Q))
    for yy in range(L):
        for xx in range(L):
            u = np.array([ux[yy, xx], uy[yy, xx], 0.0])
            if model == 0:
                f[0, yy, xx] = O.feq_q19(1.0, u)
            else:
                Cs = np.zeros(27)
                Cs[9], Cs[3], Cs[1] = u
                Cs[18] = Cs[6] = Cs[2] = 1 / 3
                f[0, yy, xx] = O.f_from_cumulants27(Cs)
    phi = np.zeros((1, L, L, 7))
    E = []
    f1, phi1 = O.run(p, steps[0], f, phi)
    _, u1, _ = O.macros(p, f1, phi1)
    f2, phi2 = O.run(p, steps[1] - steps[0], f1, phi1)
    _, u2, _ = O.macros(p, f2, phi2)
    E = [np.sum(u1**2), np.sum(u2**2)]
    rate = -math.log(E[1] / E[0]) / (steps[1] - steps[0])
    return rate / (4 * nu * k * k)


@pytest.mark.parametrize("model", [0, 1])
def test_taylor_green_decay(model):
    """Kinetic energy of the Taylor-Green vortex decays as exp(-4 nu k^2 t)
    (Eq. 25 / Eq. 58 viscosity), with second-order convergence in k."""
    nu = 0.05 if model == 0 else 0.02
    r16 = _taylor_green_rate(model, 16, nu, steps=(25, 100))
    r32 = _taylor_green_rate(model, 32, nu, steps=(100, 400))
    assert abs(r32 - 1) < 1e-3
    assert abs(r16 - 1) / abs(r32 - 1) == pytest.approx(4, rel=0.15)


@pytest.mark.parametrize("model", [0, 1])
def test_scalar_diffusion_moment_recurrence(model):
    """Zero velocity, point release.  With A(t) = sum x sum_k c_kx Phi_k and
    N = sum chi, the D3Q7 BGK scheme from equilibrium obeys exactly
    A(t) = c^2 N (1 - (1-w)^t) / w and M2(t+1) - M2(t) = c^2 N + 2 (1-w) A(t),
    c^2 = 1/4, w = 1/tau_Phi; the increment tends to 2 D N (Eq. 30, R1)."""
    L, T, D = 31, 12, 0.03
    p = O.OracleParams(L, L, L, model=model, nu=0.1, D=D, cs_smag=0.0, periodic_x=True,
                       periodic_z=True)
    chi0 = np.zeros((L, L, L))
    chi0[L // 2, L // 2, L // 2] = 1.0
    chi0[L // 2 + 1, L // 2, L // 2 - 1] = 0.5
    f, phi = O.init(p, chi0)
    N = chi0.sum()
    x = np.arange(L) - L // 2
    w = 1 / (0.5 + 4 * D)

    def M2(phi):
        chi = phi.sum(-1)
        return np.sum(chi * x[None, None, :] ** 2)

    m_prev = M2(phi)
    for t in range(T):
        A = 0.25 * N * (1 - (1 - w) ** t) / w
        f, phi = O.run(p, 1, f, phi)
        m = M2(phi)
        assert m - m_prev == pytest.approx(0.25 * N + 2 * (1 - w) * A, rel=1e-12)
        m_prev = m
    A_inf = 0.25 * N / w
    assert 0.25 * N + 2 * (1 - w) * A_inf == pytest.approx(2 * D * N, rel=1e-12)


@pytest.mark.parametrize("model", [0, 1])
def test_uniform_flow_fixed_point_and_scalar_drift(model):
    """Uniform flow is a fixed point of the fluid step; the scalar's first
    moment moves by exactly u N per step from equilibrium (Eq. 29 with R1)."""
    L = 12
    u = np.array([0.05, -0.03, 0.02])
    p = O.OracleParams(L, L, L, model=model, nu=0.03, D=0.02, cs_smag=0.17, periodic_x=True,
                       periodic_z=True)
    if model == 0:
        fe = O.feq_q19(1.0, u)
    else:
        Cs = np.zeros(27)
        Cs[9], Cs[3], Cs[1] = u
        Cs[18] = Cs[6] = Cs[2] = 1 / 3
        fe = O.f_from_cumulants27(Cs)
    f = np.broadcast_to(fe, (L, L, L, p.Q)).copy()
    chi0 = np.zeros((L, L, L))
    chi0[5:7, 4:6, 6] = 1.0
    phi = chi0[..., None] * np.array([O.phieq_q7(1.0, u)])[0]
    x = np.arange(L).astype(float)
    N = chi0.sum()

    def M1(phi):
        chi = phi.sum(-1)
        return np.array([np.sum(chi * x[None, None, :]), np.sum(chi * x[None, :, None]),
                         np.sum(chi * x[:, None, None])])

    m0 = M1(phi)
    for n in range(1, 4):
        f, phi = O.run(p, 1, f, phi)
        assert np.allclose(f, fe, atol=1e-16)
        assert np.allclose(M1(phi) - m0, n * N * u, atol=1e-12)


def test_smagorinsky_closure_matches_fd_shear():
    """nu_T at each node equals (C_s Delta)^2 sqrt(2 S:S) with S from central
    differences of the simulated shear wave u_x = U sin(2 pi y / L) (Eq. 32-34,
    reading R2/R3), to the O(k^2) accuracy of the differences."""
    L, U = 64, 0.05
    p = O.OracleParams(1, L, 1, model=0, nu=0.01, D=0.01, cs_smag=0.17, periodic_x=True,
                       periodic_z=True)
    k = 2 * math.pi / L
    y = np.arange(L)
    f = np.zeros((1, L, 1, 19))
    for yy in y:
        f[0, yy, 0] = O.feq_q19(1.0, [U * math.sin(k * yy), 0, 0])
    phi = np.zeros((1, L, 1, 7))
    f, phi = O.run(p, 30, f, phi)
    _, u, _ = O.macros(p, f, phi)
    ux = u[0, :, 0, 0]
    dudy = (np.roll(ux, -1) - np.roll(ux, 1)) / 2
    nut_fd = 0.17**2 * np.abs(dudy)
    nut = np.array([O.bgk_nu_t(p, f[0, yy, 0], phi[0, yy, 0]) for yy in y])
    big = np.abs(dudy) > 0.5 * np.abs(dudy).max()
    assert np.max(np.abs(nut[big] / nut_fd[big] - 1)) < 0.03


def test_wall_friction_quadratic_profile():
    """tau_w = nu du/dz at the wall (Eq. 62) is exact for a quadratic profile
    vanishing at the wall z = -1/2: u = a (z + 1/2)(b - z) -> du/dz = a (b + 1/2)."""
    nx, ny, nz, nu = 5, 3, 6, 0.02
    a = np.linspace(0.001, 0.002, nx)[None, :]
    b = 7.0
    u = np.zeros((nz, ny, nx, 3))
    for z in range(nz):
        u[z, :, :, 0] = a * (z + 0.5) * (b - z)
    u[..., 1] = 0.3
    assert O.wall_friction(nu, u) == pytest.approx(nu * ny * np.sum(a) * (b + 0.5), rel=1e-14)


def test_front_on_synthetic_fields():
    """Sec. 3.1 with reading R11: span average, column max over z, last column
    reaching the threshold, linear crossing."""
    nx, ny, nz = 20, 4, 5
    chi = np.zeros((nz, ny, nx))
    chi[:, :, :9] = 1.0                     # step: m = 1 up to x = 8, then 0
    assert O.front_node(chi, 0.02) == pytest.approx(8 + 0.98, abs=1e-14)
    chi2 = np.zeros((nz, ny, nx))
    chi2[3, :2, :13] = 0.05                 # only z = 3, half the span -> mean 0.025
    chi2[1, :, :6] = 0.5
    assert O.front_node(chi2, 0.02) == pytest.approx(12 + (0.025 - 0.02) / 0.025, abs=1e-14)
    ramp = np.broadcast_to(np.linspace(1.0, 0.0, nx)[None, None, :], (nz, ny, nx)).copy()
    xc = (1.0 - 0.02) * (nx - 1)            # exact crossing of a linear ramp
    assert O.front_node(ramp, 0.02) == pytest.approx(xc, abs=1e-12)
    tail = np.broadcast_to((0.1 - 0.0095 * np.arange(nx))[None, None, :], (nz, ny, nx)).copy()
    assert O.front_node(tail, 0.02) == pytest.approx(8 + 0.004 / 0.0095, abs=1e-12)
    assert O.front_node(np.zeros((nz, ny, nx)), 0.02) == -1.0
    full = np.ones((nz, ny, nx))
    assert O.front_node(full, 0.02) == nx - 1


def test_front_window_with_periodic_ends():
    """Periodic ends (Fig. 4b): the current leaving the lock [0, x0) to the
    left re-enters at x = nx - 1; the front is searched in x < (nx + x0) / 2,
    the half of the ring ahead of the lock (reading of Sec. 3.1 for Cases 1,
    3, 5, 7)."""
    nx, ny, nz, x0 = 40, 3, 4, 8
    chi = np.zeros((nz, ny, nx))
    chi[:, :, :14] = 1.0                    # lock and the right-going current
    chi[0, :, 33:] = 0.6                    # the left-going current, wrapped
    xlim = O.front_xlim(nx, x0, True)
    assert xlim == (nx + x0) // 2 == 24 and O.front_xlim(nx, x0, False) == nx
    assert O.front_node(chi, 0.02) == nx - 1          # walls: the whole box
    assert O.front_node(chi, 0.02, xlim) == pytest.approx(13 + 0.98, abs=1e-14)
    # through the diagnostics: the window follows the periodic_x flag
    for periodic, want in ((False, nx - 1), (True, 13 + 0.98)):
        p = O.OracleParams(nx, ny, nz, model=0, periodic_x=periodic)
        f = np.broadcast_to(np.asarray(O.velocities(0)[1]), (nz, ny, nx, 19)).copy()
        phi = chi[..., None] * np.asarray(O.velocities_q7()[1])
        d = O.diag(p, f, phi, x0, 8.0)
        assert d["front_node"] == pytest.approx(want, abs=1e-12)
    # a front on the last searched column is not interpolated
    edge = np.zeros((nz, ny, nx))
    edge[:, :, :xlim] = 1.0
    edge[:, :, xlim:] = 0.5
    assert O.front_node(edge, 0.02, xlim) == xlim - 1


@pytest.mark.parametrize("model,scalar", [(0, 0), (1, 0), (0, 1), (1, 2)])
def test_threads_do_not_change_results(model, scalar):
    """The node loops of the oracle run on several threads; every node is
    computed on its own from the previous arrays, so a run on one thread and
    on several is bit for bit the same (collision, streaming, macros)."""
    p = O.OracleParams(13, 5, 6, model=model, scalar=scalar, nu=0.01, D=0.01, gprime=1e-3)
    chi0 = O.lock_chi0(13, 5, 6, 5, 0.1, 3)
    f0, phi0 = O.init(p, chi0)
    old = O.threads()
    try:
        out = []
        for t in (1, 4):
            O.set_threads(t)
            f, phi = O.run(p, 6, f0.copy(), phi0.copy())
            out.append((f, phi, O.macros(p, f, phi)))
    finally:
        O.set_threads(old)
    (fa, pa, ma), (fb, pb, mb) = out
    assert np.array_equal(fa, fb) and np.array_equal(pa, pb)
    for a, b in zip(ma, mb):
        assert np.array_equal(a, b)
