"""Parity at the full 2048 x 128 x 256 size, in the launch configuration the
benchmark times: two steps (one even, one odd AA parity) from a random
near-equilibrium state, checked node by node on a sample of nodes (corners,
edges, faces, interior) against the FP64 oracle run on each node's light cone;
plus conservation over a longer run."""
import numpy as np
import pytest

import oracle as O
from paper_2112_08479_gb300 import inputs, lbm

from helpers import rest_row_tol, stored_phi, weights, window_oracle

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

NX, NY, NZ = 2048, 128, 256


def _sample_nodes(seed=5, n_random=12):
    xs, ys, zs = [0, 1, NX - 2, NX - 1], [0, NY - 1], [0, 1, NZ - 2, NZ - 1]
    nodes = [(x, y, z) for x in (0, NX - 1) for y in (0, NY - 1) for z in (0, NZ - 1)]
    nodes += [(x, 64, 128) for x in xs] + [(1000, y, 128) for y in ys] + [(1000, 64, z) for z in zs]
    rng = np.random.default_rng(seed)
    nodes += [(int(rng.integers(NX)), int(rng.integers(NY)), int(rng.integers(NZ))) for _ in range(n_random)]
    return nodes


def _random_full_state(p, seed, amp=0.05):
    w = torch.tensor(weights(p.model), dtype=torch.float32, device="cuda")
    w7 = torch.tensor(O.velocities_q7()[1], dtype=torch.float32, device="cuda")
    s = torch.empty(p.Q + 7, p.N, dtype=torch.float32, device="cuda")
    s[: p.Q] = inputs.torch_uniform((p.Q, p.N), seed, amp) * w[:, None]
    chi = 0.5 * (1 + inputs.torch_uniform((p.N,), seed + 1, 1.0))
    s[p.Q:] = w7[:, None] * (chi[None, :] * (1 + inputs.torch_uniform((7, p.N), seed + 2, amp)) - 1.0)
    return s


@pytest.mark.parametrize("model,storage", [("bgk", "fp32"), ("cumulant", "fp32"), ("bgk", "fp16s"),
                                           ("cumulant", "bf16s")])
def test_full_size_sampled_nodes(model, storage):
    """One even and one odd step; each is checked against the oracle started
    from the state the storage actually holds before that step."""
    p = lbm.lock_exchange(NX, NY, NZ, H=256, x0=256, u_b=0.03, Re=30000.0, model=model,
                          storage=storage)
    # a stronger force so the force terms are visible in single steps
    p.gprime = 1e-3
    lat = lbm.Lattice(p, device="cuda")
    lat.set_state(_random_full_state(p, 17))
    rel = {"fp32": 0.0, "fp16s": 2.0**-11, "bf16s": 2.0**-8}[storage]
    for parity in ("even", "odd"):
        s0 = lat.get_state()        # what the storage holds (rounded for 16-bit)
        lat.step(1)                 # the kernel and grid the benchmark launches
        s1 = lat.get_state()
        s0v = s0.view(p.Q + 7, NZ, NY, NX)
        s1v = s1.view(p.Q + 7, NZ, NY, NX)
        scale = float(s0[: p.Q].abs().max())
        for node in _sample_nodes():
            x, y, z = node
            f_o, phi_o = window_oracle(p, s0v, node, 1)
            got = s1v[:, z, y, x].cpu().numpy().astype(np.float64)
            # FP32 arithmetic, then round-to-nearest into the storage type
            tol_f = rel * np.abs(f_o) * 1.001 + 1e-5 * scale
            tol_p = rel * stored_phi(phi_o, p) * 1.001 + 1e-6
            if rel:   # FP32 rest population with rounding feedback
                col = s0v[:, z, y, x].cpu().numpy().astype(np.float64)[:, None]
                tol_p[0] = rest_row_tol(p, col, rel)[0] + 1e-6
            assert np.all(np.abs(got[: p.Q] - f_o) <= tol_f), (parity, node)
            assert np.all(np.abs(got[p.Q:] - phi_o) <= tol_p), (parity, node)
        del s0, s1


def test_full_size_budgets_conserved():
    p = lbm.lock_exchange(NX, NY, NZ, H=256, x0=256, u_b=0.03, Re=30000.0)
    lat = lbm.Lattice(p, device="cuda")
    d0 = lat.diag()
    lat.step(200)
    d1 = lat.diag()
    assert d1["flags"] == 0
    assert abs(d1["scalar_mass"] - d0["scalar_mass"]) < 1e-7 * d0["scalar_mass"]
    assert abs(d1["mass_delta"] - d0["mass_delta"]) < 1e-7 * p.N
    # the gate column starts at x0 - 1 = 255: the front has moved forward
    assert d1["front"] > d0["front"]


@pytest.mark.parametrize("model,storage", [("cumulant", "fp16s"), ("bgk", "bf16s")])
def test_wide_box_sampled_nodes(model, storage):
    """A box past 32-bit element offsets: 2048 x 256 x 320 = 167.8 M nodes,
    (Q + 7) N >= 2^32 (the cumulant's fluid rows alone reach 27 N = 4.5e9), so
    the step kernels run with 64-bit offsets and the canonical state (22.8 GB
    for the cumulant) is read and written with them too.  One even and one odd
    step, sampled nodes against the oracle as above."""
    nx, ny, nz = 2048, 256, 320
    p = lbm.lock_exchange(nx, ny, nz, H=nz, x0=nz, u_b=0.03, Re=30000.0, model=model,
                          storage=storage)
    p.gprime = 1e-3
    assert (p.Q + p.NS) * p.N >= 2**32
    lat = lbm.Lattice(p, device="cuda")
    lat.set_state(_random_full_state(p, 23))
    rel = {"fp16s": 2.0**-11, "bf16s": 2.0**-8}[storage]
    rng = np.random.default_rng(7)
    nodes = [(0, 0, 0), (nx - 1, ny - 1, nz - 1), (nx - 1, 0, nz - 1), (1000, 200, 300)]
    nodes += [(int(rng.integers(nx)), int(rng.integers(ny)), int(rng.integers(nz)))
              for _ in range(8)]
    for parity in ("even", "odd"):
        s0 = lat.get_state()
        lat.step(1)
        s1 = lat.get_state()
        s0v = s0.view(p.Q + 7, nz, ny, nx)
        s1v = s1.view(p.Q + 7, nz, ny, nx)
        scale = float(s0[: p.Q, :: 997].abs().max())
        for node in nodes:
            x, y, z = node
            f_o, phi_o = window_oracle(p, s0v, node, 1)
            got = s1v[:, z, y, x].cpu().numpy().astype(np.float64)
            tol_f = rel * np.abs(f_o) * 1.001 + 1e-5 * scale
            tol_p = rel * stored_phi(phi_o, p) * 1.001 + 1e-6
            col = s0v[:, z, y, x].cpu().numpy().astype(np.float64)[:, None]
            tol_p[0] = rest_row_tol(p, col, rel)[0] + 1e-6
            assert np.all(np.abs(got[: p.Q] - f_o) <= tol_f), (parity, node)
            assert np.all(np.abs(got[p.Q:] - phi_o) <= tol_p), (parity, node)
        del s0, s1, s0v, s1v
        torch.cuda.empty_cache()
    assert lat.diag()["flags"] == 0
    # saved steps and the adjoint keep 32-bit canonical offsets
    with pytest.raises(lbm.LBMError) as e:
        lat.step_save(torch.empty(1, device="cuda"))
    assert e.value.status == lbm.LBM_ERR_STATE
