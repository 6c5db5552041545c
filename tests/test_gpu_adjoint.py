"""GPU discrete adjoint (lbm_adjoint_step, LBMObjective) against the FP64
reference gradient and against central finite differences.

Bar: 1e-3 relative (FP32 arithmetic on the GPU)."""
import numpy as np
import pytest

import oracle as O
from oracle import adjoint_ref as A
from paper_2112_08479_gb300 import inputs, lbm
from paper_2112_08479_gb300.objective import friction_objective, front_objective

from helpers import canonical_to_oracle, oracle_params, weights

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _sub_case(nx=32, ny=4, nz=8, **kw):
    # the 32 x 4 x 8 sub-case with the lattice parameters of the 256 x 32 x 64
    # differentiation box (H = 64, u_b = 0.03, Re = 2000): nu = 9.6e-4,
    # g' = 1.40625e-5, C_s = 0.17; lock at x = H of the sub-case
    base = dict(nx=nx, ny=ny, nz=nz, nu=9.6e-4, D=9.6e-4, cs_smag=0.17, sc_t=1.0,
                gprime=1.40625e-5, x0=nz, H=nz)
    base.update(kw)
    return lbm.Params(**base)


def _random_state(p, seed, amp=0.05):
    w = weights(p.model)
    fdev = w[:, None] * inputs.uniform((p.Q, p.N), seed, amp)
    chi = 0.5 * (1 + inputs.uniform(p.N, seed + 1, 1.0))
    w7 = O.velocities_q7()[1]
    phi = w7[:, None] * (chi[None, :] * (1 + inputs.uniform((7, p.N), seed + 2, amp)) - 1.0)
    return np.concatenate([fdev, phi]).astype(np.float32)


@pytest.mark.parametrize("flags", [0, lbm.LBM_FLAG_PERIODIC_X | lbm.LBM_FLAG_PERIODIC_Z])
@pytest.mark.parametrize("w_fw", [0.0, 1.0])
def test_adjoint_step_matches_autograd_vjp(flags, w_fw):
    """One reverse step: lam_n = C^T P^T lam + w dF_w/ds and the C_s term, vs
    torch.autograd on the FP64 restatement of the step."""
    p = _sub_case(nx=20, ny=5, nz=6, flags=flags, gprime=3e-3, eg=(0.3, -0.4, -0.866),
                  cs_smag=0.4, sc_t=0.7, nu=0.01, D=0.02)
    lat = lbm.Lattice(p, device="cuda")
    s0 = _random_state(p, 3)
    lam_next = inputs.normal((26, p.N), 8).astype(np.float32)
    st = torch.from_numpy(s0).cuda()
    ln = torch.from_numpy(lam_next).cuda()
    out = torch.empty(26, p.N, device="cuda")
    dcs = torch.zeros(1, dtype=torch.float64, device="cuda")
    lat.adjoint_step(st, ln, out, dcs, w_fw)
    got = out.cpu().numpy().astype(np.float64)

    op = oracle_params(p)
    step = A.BGKStep(op)
    f, phi = canonical_to_oracle(s0, p)
    ft = torch.tensor(f, requires_grad=True)
    pt = torch.tensor(phi, requires_grad=True)
    cs = torch.tensor(p.cs_smag, dtype=torch.float64, requires_grad=True)
    f1, p1 = step(ft, pt, cs)
    lf, lp = canonical_to_oracle(lam_next, p, shifted=False)
    inner = (f1 * torch.tensor(lf)).sum() + (p1 * torch.tensor(lp)).sum() + w_fw * step.friction(ft, pt)
    gf, gp, gc = torch.autograd.grad(inner, (ft, pt, cs))
    want = np.concatenate([np.moveaxis(gf.numpy(), -1, 0), np.moveaxis(gp.numpy(), -1, 0)]).reshape(26, -1)
    err = np.abs(got - want).max() / np.abs(want).max()
    assert err < 1e-4, err
    assert dcs.item() == pytest.approx(float(gc), rel=1e-3, abs=1e-6 * abs(float(gc)) + 1e-12)


def test_gradient_vs_fp64_reference_sub_case():
    """Full gradient over 2000 steps on the 32 x 4 x 8 sub-case with
    checkpoints every 100 steps, vs the FP64 reference gradient."""
    p = _sub_case()
    nsteps = 2000
    chi0 = O.lock_chi0(p.nx, p.ny, p.nz, p.x0, p.noise_amp, p.seed)
    J_ref, g_ref, gcs_ref = A.gradient(oracle_params(p), chi0, p.cs_smag, nsteps)
    x = torch.tensor(chi0.ravel(), dtype=torch.float32, device="cuda", requires_grad=True)
    cs = torch.tensor(p.cs_smag, dtype=torch.float64, device="cuda", requires_grad=True)
    J = friction_objective(x, cs, p, nsteps, K=100)
    J.backward()
    assert J.item() == pytest.approx(J_ref, rel=1e-4)
    g = x.grad.cpu().numpy().astype(np.float64)
    rel = np.linalg.norm(g - g_ref.ravel()) / np.linalg.norm(g_ref)
    assert rel < 1e-3, rel
    assert cs.grad.item() == pytest.approx(gcs_ref, rel=1e-3)
    # and against the full central-difference gradient of the C oracle
    # (tests/golden/fd_gradient_32x4x8.txt, same sub-case and steps)
    from test_oracle_adjoint import _load_fd_golden
    J_fd, g_fd, cs_fd = _load_fd_golden()
    assert J.item() == pytest.approx(J_fd, rel=1e-4)
    assert np.linalg.norm(g - g_fd) / np.linalg.norm(g_fd) < 1e-3
    assert cs.grad.item() == pytest.approx(cs_fd, rel=1e-3)


@pytest.mark.parametrize("model", [lbm.LBM_BGK_SMAG_Q19, lbm.LBM_CUMULANT_Q27])
def test_checkpoint_interval_does_not_change_gradient(model):
    """K = 300 is one segment (no overlap); K = 7 and 100 overlap the
    recompute of each segment with the sweep of the next on a second stream.
    The adjoint arithmetic is the same; the checkpoints come from the in-place
    forward kernel and the recomputed states from the out-of-place one, which
    for BGK agree bit for bit (so do the gradients), for the cumulant to
    FP32 rounding."""
    p = _sub_case(model=model)
    chi0 = torch.tensor(O.lock_chi0(p.nx, p.ny, p.nz, p.x0, p.noise_amp, p.seed).ravel(),
                        dtype=torch.float32, device="cuda")
    grads = []
    for K in (7, 100, 300):
        x = chi0.clone().requires_grad_(True)
        friction_objective(x, p.cs_smag, p, 300, K=K).backward()
        grads.append(x.grad.clone())
    if model == lbm.LBM_BGK_SMAG_Q19:
        assert torch.equal(grads[0], grads[1]) and torch.equal(grads[1], grads[2])
    else:
        scale = grads[2].abs().max()
        for g in grads[:2]:
            assert (g - grads[2]).abs().max() <= 1e-5 * scale


def test_gradient_vs_central_differences_full_box():
    """256 x 32 x 64, 2000 steps, K = 100: the adjoint's directional
    derivatives on 32 seeded unit directions against central differences of
    the FP32 forward (J accumulated in FP64), and dJ/dC_s.

    The FP32 forward carries round-off noise of a few 1e-8 relative in J; a
    step of 1.6e-2 per node (eps = 1.6e-2 sqrt(N) along a unit direction)
    keeps its effect on the difference quotient below 1e-4 of the projected
    gradient.  Bar: the 32-vector of directional derivatives within 1e-3
    (relative 2-norm); each direction within 1e-2 of its own value."""
    p = lbm.lock_exchange(256, 32, 64, H=64, x0=64, u_b=0.03, Re=2000.0)
    nsteps = 2000
    lat = lbm.Lattice(p, device="cuda")
    chi0 = lat.macros()[2].reshape(-1).clone()
    del lat
    x = chi0.clone().requires_grad_(True)
    cs = torch.tensor(p.cs_smag, dtype=torch.float64, device="cuda", requires_grad=True)
    friction_objective(x, cs, p, nsteps, K=100).backward()
    g = x.grad.double()

    def J(c, csv=p.cs_smag):
        with torch.no_grad():
            return friction_objective(c, csv, p, nsteps, K=100).item()

    eps = 1.6e-2 * np.sqrt(p.N)
    ad, fd = [], []
    for seed in range(1, 33):
        d = torch.tensor(inputs.unit_direction(p.N, seed), dtype=torch.float32, device="cuda")
        ad.append(float((g * d.double()).sum()))
        fd.append((J(chi0 + eps * d) - J(chi0 - eps * d)) / (2 * eps))
    ad, fd = np.array(ad), np.array(fd)
    rel = np.linalg.norm(ad - fd) / np.linalg.norm(fd)
    per = np.abs(ad - fd) / np.abs(fd)
    print(f"32 directions: relative 2-norm error {rel:.2e}, median per-direction {np.median(per):.2e}, "
          f"max {per.max():.2e}")
    assert rel < 1e-3
    assert per.max() < 1e-2
    h = 1e-3
    fd_cs = (J(chi0, p.cs_smag + h) - J(chi0, p.cs_smag - h)) / (2 * h)
    assert cs.grad.item() == pytest.approx(fd_cs, rel=1e-4)


def test_segment_matches_per_step_adjoint():
    """lbm_adjoint_segment (out-of-place recompute + k reverse steps) equals
    stepping lbm_adjoint_step by hand over the trajectory recorded with
    lbm_step_save."""
    p = _sub_case(nx=24, ny=4, nz=8, gprime=1e-3)
    lat = lbm.Lattice(p, device="cuda")
    lat.step(5)
    k = 9
    ck = lat.get_state()
    traj = torch.empty(k, 26, p.N, device="cuda")
    for j in range(k):
        lat.step_save(traj[j])
    lam0 = torch.tensor(inputs.normal((26, p.N), 4).astype(np.float32), device="cuda")
    # by hand
    a, b = lam0.clone(), torch.empty_like(lam0)
    dcs_a = torch.zeros(1, dtype=torch.float64, device="cuda")
    for j in range(k - 1, -1, -1):
        lat.adjoint_step(traj[j], a, b, dcs_a, 1.0)
        a, b = b, a
    # segment
    lam = lam0.clone()
    tmp = torch.empty_like(lam0)
    seg = torch.empty(k, 26, p.N, device="cuda")
    dcs_b = torch.zeros(1, dtype=torch.float64, device="cuda")
    lat.adjoint_segment(ck, 5, k, seg, lam, tmp, dcs_b)
    assert torch.allclose(lam, a, rtol=1e-5, atol=1e-6 * a.abs().max().item())
    assert dcs_b.item() == pytest.approx(dcs_a.item(), rel=1e-5)
    # the recomputed trajectory is the recorded one
    for j in range(1, k):
        assert torch.allclose(seg[j], traj[j], rtol=0, atol=1e-7)


# ---------------------------------------------------------------------------
# Front objective (Sec. 3.1, reading R11): lbm_front_adjoint and the adjoint
# sweep with the friction weight 0.

def _front_state(p, seed):
    """Canonical state whose scalar falls from ~1 to ~0 around x = nx / 2
    (distinct values, so the crossing column and the maximising z are
    unique), with a random fluid part."""
    w = weights(p.model)
    fdev = w[:, None] * inputs.uniform((p.Q, p.N), seed, 0.05)
    x = np.tile(np.arange(p.nx), p.ny * p.nz)
    chi = 1.0 / (1.0 + np.exp(2.0 * (x - p.nx / 2 - 0.37)))
    chi = chi * (1 + 0.05 * inputs.uniform(p.N, seed + 1, 1.0)) + 1e-3 * inputs.uniform(p.N, seed + 2, 1.0)
    w7 = O.velocities_q7()[1]
    phi = w7[:, None] * (chi[None, :] * (1 + inputs.uniform((7, p.N), seed + 3, 0.05)) - 1.0)
    return np.concatenate([fdev, phi]).astype(np.float32)


@pytest.mark.parametrize("model", [0, 1])
@pytest.mark.parametrize("thr", [0.02, 0.5])
def test_front_adjoint_of_a_state(model, thr):
    p = _sub_case(nx=40, ny=5, nz=6, model=model, front_threshold=thr)
    lat = lbm.Lattice(p, device="cuda")
    s0 = _front_state(p, 4)
    st = torch.from_numpy(s0).cuda()
    lam = torch.full((p.Q + 7, p.N), 7.0, device="cuda")
    val = torch.zeros(1, dtype=torch.float64, device="cuda")
    lat.front_adjoint(st, lam, val)
    got = lam.cpu().numpy().astype(np.float64)
    # oracle: chi from the stored values in FP64, front and its gradient
    chi = (1.0 + s0[p.Q:].astype(np.float64).sum(0)).reshape(p.nz, p.ny, p.nx)
    want_val = (O.front_node(chi, thr) + 0.5 - p.x0) / p.H
    assert val.item() == pytest.approx(want_val, abs=1e-5 / p.H)
    step = A.BGKStep(oracle_params(lbm.Params(nx=p.nx, ny=p.ny, nz=p.nz, x0=p.x0, H=p.H)))
    c = torch.tensor(chi, dtype=torch.float64, requires_grad=True)
    J = step.front(step.w.expand(*chi.shape, 19), c[..., None] * step.w7, p.x0, p.H, thr)
    (g,) = torch.autograd.grad(J, c)
    g = g.numpy().reshape(-1)
    assert np.all(got[: p.Q] == 0.0)
    for k in range(7):
        row = got[p.Q + k]
        assert np.array_equal(row != 0.0, g != 0.0)
        assert np.abs(row - g).max() < 1e-5 * np.abs(g).max()


def test_front_adjoint_degenerate_fronts():
    """No column at or above the threshold, and a front at the last column:
    the front does not move with the state, the derivative is zero."""
    p = _sub_case(nx=12, ny=3, nz=4)
    lat = lbm.Lattice(p, device="cuda")
    for chi_val, node in ((0.0, -1.0), (1.0, p.nx - 1.0)):
        s = np.zeros((26, p.N), dtype=np.float32)
        w7 = O.velocities_q7()[1]
        s[19:] = (w7 * (chi_val - 1.0))[:, None]
        lam = torch.full((26, p.N), 7.0, device="cuda")
        val = torch.zeros(1, dtype=torch.float64, device="cuda")
        lat.front_adjoint(torch.from_numpy(s).cuda(), lam, val)
        assert val.item() == pytest.approx((node + 0.5 - p.x0) / p.H)
        assert torch.count_nonzero(lam).item() == 0


def test_front_gradient_vs_fp64_reference_sub_case():
    """Front after 800 steps of the 32 x 4 x 8 sub-case (mid-domain, the
    crossing column and maximising z separated by >= 9e-4 in chibar), with
    checkpoints every 100 steps, vs the FP64 reference gradient."""
    p = _sub_case()
    nsteps = 800
    chi0 = O.lock_chi0(p.nx, p.ny, p.nz, p.x0, p.noise_amp, p.seed)
    J_ref, g_ref, gcs_ref = A.gradient(oracle_params(p), chi0, p.cs_smag, nsteps,
                                       objective="front", x0=p.x0, H=p.H)
    x = torch.tensor(chi0.ravel(), dtype=torch.float32, device="cuda", requires_grad=True)
    cs = torch.tensor(p.cs_smag, dtype=torch.float64, device="cuda", requires_grad=True)
    J = front_objective(x, cs, p, nsteps, K=100)
    J.backward()
    assert J.item() == pytest.approx(J_ref, abs=1e-4)
    g = x.grad.cpu().numpy().astype(np.float64)
    rel = np.linalg.norm(g - g_ref.ravel()) / np.linalg.norm(g_ref)
    assert rel < 1e-3, rel
    assert cs.grad.item() == pytest.approx(gcs_ref, rel=1e-3)


# ---------------------------------------------------------------------------
# Adjoint of the cumulant step (Eq. 54-58 with the D3Q7 scalar)

@pytest.mark.parametrize("flags", [0, lbm.LBM_FLAG_PERIODIC_X | lbm.LBM_FLAG_PERIODIC_Z])
@pytest.mark.parametrize("w_fw", [0.0, 1.0])
@pytest.mark.parametrize("nx", [20, 260])
def test_cumulant_adjoint_step_matches_autograd_vjp(flags, w_fw, nx):
    """One reverse step of the cumulant model against torch.autograd on the
    FP64 restatement (truncated ln / exp of the moment generating function).
    nx = 260 spans three blocks per row (the middle ones away from every
    wall)."""
    p = _sub_case(nx=nx, ny=5, nz=6, model=lbm.LBM_CUMULANT_Q27, flags=flags, gprime=3e-3,
                  eg=(0.3, -0.4, -0.866), nu=0.01, D=0.02, omega_bulk=0.8)
    lat = lbm.Lattice(p, device="cuda")
    s0 = _random_state(p, 3)
    lam_next = inputs.normal((p.Q + 7, p.N), 8).astype(np.float32)
    st = torch.from_numpy(s0).cuda()
    out = torch.empty(p.Q + 7, p.N, device="cuda")
    dcs = torch.zeros(1, dtype=torch.float64, device="cuda")
    lat.adjoint_step(st, torch.from_numpy(lam_next).cuda(), out, dcs, w_fw)
    got = out.cpu().numpy().astype(np.float64)
    assert dcs.item() == 0.0

    op = oracle_params(p)
    step = A.make_step(op)
    f, phi = canonical_to_oracle(s0, p)
    ft = torch.tensor(f, requires_grad=True)
    pt = torch.tensor(phi, requires_grad=True)
    f1, p1 = step(ft, pt, torch.tensor(0.0, dtype=torch.float64))
    lf, lp = canonical_to_oracle(lam_next, p, shifted=False)
    inner = (f1 * torch.tensor(lf)).sum() + (p1 * torch.tensor(lp)).sum() + w_fw * step.friction(ft, pt)
    gf, gp = torch.autograd.grad(inner, (ft, pt))
    want = np.concatenate([np.moveaxis(gf.numpy(), -1, 0),
                           np.moveaxis(gp.numpy(), -1, 0)]).reshape(p.Q + 7, -1)
    err = np.abs(got - want).max() / np.abs(want).max()
    assert err < 1e-4, err


@pytest.mark.parametrize("kind", ["friction", "front"])
def test_cumulant_gradient_vs_fp64_reference_sub_case(kind):
    """Both objectives through 800 cumulant steps of the 32 x 4 x 8 sub-case,
    checkpoints every 100 steps, against the FP64 reference gradient."""
    p = _sub_case(model=lbm.LBM_CUMULANT_Q27)
    nsteps = 800
    chi0 = O.lock_chi0(p.nx, p.ny, p.nz, p.x0, p.noise_amp, p.seed)
    J_ref, g_ref, _ = A.gradient(oracle_params(p), chi0, p.cs_smag, nsteps, objective=kind,
                                 x0=p.x0, H=p.H)
    x = torch.tensor(chi0.ravel(), dtype=torch.float32, device="cuda", requires_grad=True)
    fn = friction_objective if kind == "friction" else front_objective
    J = fn(x, p.cs_smag, p, nsteps, K=100)
    J.backward()
    if kind == "friction":
        assert J.item() == pytest.approx(J_ref, rel=1e-4)
    else:
        assert J.item() == pytest.approx(J_ref, abs=1e-4)
    g = x.grad.cpu().numpy().astype(np.float64)
    rel = np.linalg.norm(g - g_ref.ravel()) / np.linalg.norm(g_ref)
    assert rel < 1e-3, rel
