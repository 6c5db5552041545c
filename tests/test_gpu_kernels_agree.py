"""The two-node and TMA-staged step kernels against the one-node kernels.

With nx even the BGK step runs two x-adjacent nodes per thread, with paired
FP32 accesses and, on odd steps, the block-uniform wall-free and interior
bodies; with 16-bit storage and nx a multiple of 4 its even steps run four
nodes per thread on packed 8-byte words (nx = 34 and 770 take the two-node
form), and so do the cumulant model's even steps (D3Q7 scalar).
LBM_FLAG_ONE_NODE selects the one-node kernel.  Cases: x and z walls,
periodic ends, warp and block edges (nx = 770, 1028: three blocks, the
middle one wholly interior), both scalar lattices of the BGK fluid.

Pure streaming (collisions off) moves stored values only, so the two must
agree bit for bit: this checks every index, wall and edge path.  With
collisions the per-node arithmetic is the same source, but the compiler may
fuse multiply-adds differently where it inlines two collisions, so FP32
results can differ in the last bit; stored as FP32 they agree exactly in
every case here, and where such a difference decides a rounding to 16 bits
the stored values differ by one ulp of the storage type, at a few elements.
Each collision step therefore starts both kernels from the same state.

With LBM_FLAG_TMA_STAGED the cumulant model with the D3Q7 scalar and 16-bit
storage runs the TMA-staged kernel (tiles of 256 nodes whose population rows
move by bulk copies through shared memory); nx = 512, 1024 and 2560 give two,
four and ten tiles per row, so the first and last tiles meet the x ends
(clamped load windows, bounce-back or periodic wrap by direct loads and
stores), the others take the widened windows on both sides, and z = 0 and
nz - 1 take the wall body.  It must agree with the one-node kernel bit for
bit, with collisions too: the collision is the same inlined function."""
import numpy as np
import pytest

from paper_2112_08479_gb300 import inputs, lbm

from helpers import stored_phi, weights, wscalar

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

GEOMETRIES = {"walls": 0, "periodic_x": lbm.LBM_FLAG_PERIODIC_X,
              "periodic_z": lbm.LBM_FLAG_PERIODIC_Z,
              "periodic_xz": lbm.LBM_FLAG_PERIODIC_X | lbm.LBM_FLAG_PERIODIC_Z}


def _state(p, seed, amp=0.05):
    """Populations near equilibrium with noise, chi in (0, 1) varying in x
    (a smoothed lock) and at random."""
    w = weights(p.model)
    fdev = w[:, None] * inputs.uniform((p.Q, p.N), seed, amp)
    x = np.arange(p.N) % p.nx
    chi = 0.5 * (1 + np.tanh((p.nx / 3 - x) / 4.0)) * (1 + 0.2 * inputs.uniform(p.N, seed + 1, 1.0))
    chi = np.clip(chi, 0.0, 1.0)
    ws = wscalar(p)
    phi = ws[:, None] * (chi[None, :] * (1 + inputs.uniform((p.NS, p.N), seed + 2, amp)) - 1.0)
    return np.concatenate([fdev, phi]).astype(np.float32)


def _lat(p, s, step):
    lat = lbm.Lattice(p, device="cuda")
    lat.set_state(torch.from_numpy(s).cuda(), step)
    return lat


CASES = [("bgk", "fp32", "q7"), ("bgk", "fp16s", "q7"), ("bgk", "bf16s", "q7"),
         ("bgk", "fp32", "q6"), ("bgk", "fp16s", "q6"),
         # the cumulant's four-node even step (16-bit storage, nx a multiple of 4)
         ("cumulant", "fp16s", "q7"), ("cumulant", "bf16s", "q7")]
ULP = {"fp16s": 2.0**-10, "bf16s": 2.0**-7}


def _params(model, storage, scalar, geometry, nx, extra=0):
    kw = dict(model=lbm.MODELS[model], storage=lbm.STORAGES[storage], scalar=lbm.SCALARS[scalar],
              nu=0.01, D=0.012, cs_smag=0.3, gprime=2e-3, eg=(0.48, 0.6, -0.64), x0=1, H=5)
    return (lbm.Params(nx, 3, 5, flags=GEOMETRIES[geometry] | extra, **kw),
            lbm.Params(nx, 3, 5, flags=GEOMETRIES[geometry] | extra | lbm.LBM_FLAG_ONE_NODE, **kw))


@pytest.mark.parametrize("geometry", sorted(GEOMETRIES))
@pytest.mark.parametrize("model,storage,scalar", CASES)
@pytest.mark.parametrize("nx", [34, 36, 770, 1028])
def test_streaming_matches_one_node_exactly(model, storage, scalar, geometry, nx):
    p2, p1 = _params(model, storage, scalar, geometry, nx, lbm.LBM_FLAG_NO_COLLIDE)
    s0 = _state(p2, 11)
    a, b = _lat(p2, s0, 0), _lat(p1, s0, 0)
    for n in range(1, 5):
        a.step(1)
        b.step(1)
        x, y = a.get_state().cpu().numpy(), b.get_state().cpu().numpy()
        bad = np.argwhere(x != y)
        assert bad.size == 0, (n, bad[:5].tolist())
    assert not np.array_equal(x, s0)          # values moved


@pytest.mark.parametrize("geometry", sorted(GEOMETRIES))
@pytest.mark.parametrize("model,storage,scalar", CASES)
@pytest.mark.parametrize("nx", [34, 36, 770, 1028])
def test_collision_steps_match_one_node(model, storage, scalar, geometry, nx):
    p2, p1 = _params(model, storage, scalar, geometry, nx)
    s = _state(p2, 11)
    Q = p2.Q
    scale = np.r_[[p2.scale_f] * Q, [p2.scale_phi] * p2.NS][:, None]
    for n in range(4):                      # two even and two odd steps
        a, b = _lat(p2, s, n), _lat(p1, s, n)
        a.step(1)
        b.step(1)
        x, y = a.get_state().cpu().numpy(), b.get_state().cpu().numpy()
        assert not np.array_equal(y, s)
        if storage == "fp32":
            bad = np.argwhere(x != y)
            assert bad.size == 0, (n, bad[:5].tolist())
        else:
            d = np.abs(x.astype(np.float64) - y)
            # one ulp of the stored 16-bit value (normal or subnormal range);
            # the scalar is stored as Phi - chi_s w
            mag = np.maximum(np.abs(x), np.abs(y)).astype(np.float64)
            mag[Q:] = np.maximum(stored_phi(x[Q:], p2), stored_phi(y[Q:], p2))
            tol = np.maximum(mag * scale * ULP[storage], 2.0**-24) / scale
            # the FP32 rest population of the scalar takes the roundings of
            # the node's moving scalar populations: one ulp each
            if p2.scalar != lbm.LBM_SCALAR_Q6:
                tol[Q] = (stored_phi(y[Q + 1:], p2, 1).sum(axis=0) * ULP[storage] + 2.0**-24 * 8
                          + np.abs(y[Q]) * 2.0**-22)
            bad = np.argwhere(d > tol * 1.0001)
            assert bad.size == 0, (n, bad[:5].tolist(), [(float(x[r, c]), float(y[r, c]))
                                                         for r, c in bad[:5]])
            assert np.count_nonzero(d) <= max(8, 1e-3 * d.size), (n, np.count_nonzero(d))
        s = y


STAGED = [("cumulant", "fp16s", "q7"), ("cumulant", "bf16s", "q7")]


def _pair(model, storage, scalar, geometry, nx, extra=0):
    staged, one = _params(model, storage, scalar, geometry, nx, extra | lbm.LBM_FLAG_TMA_STAGED)
    return staged, one


@pytest.mark.parametrize("geometry", sorted(GEOMETRIES))
@pytest.mark.parametrize("model,storage,scalar", STAGED)
@pytest.mark.parametrize("nx", [512, 1024, 2560])
def test_staged_streaming_matches_one_node_exactly(model, storage, scalar, geometry, nx):
    p2, p1 = _pair(model, storage, scalar, geometry, nx, lbm.LBM_FLAG_NO_COLLIDE)
    s0 = _state(p2, 11)
    a, b = _lat(p2, s0, 0), _lat(p1, s0, 0)
    for n in range(1, 5):
        a.step(1)
        b.step(1)
        x, y = a.get_state().cpu().numpy(), b.get_state().cpu().numpy()
        bad = np.argwhere(x != y)
        assert bad.size == 0, (n, bad[:5].tolist())
    assert not np.array_equal(x, s0)
    assert a.diag()["flags"] == 0


@pytest.mark.parametrize("geometry", sorted(GEOMETRIES))
@pytest.mark.parametrize("model,storage,scalar", STAGED)
@pytest.mark.parametrize("nx", [512, 1024, 2560])
def test_staged_collision_steps_match_one_node_exactly(model, storage, scalar, geometry, nx):
    p2, p1 = _pair(model, storage, scalar, geometry, nx)
    s = _state(p2, 11)
    a, b = _lat(p2, s, 0), _lat(p1, s, 0)
    for n in range(4):                      # two even and two odd steps, one run each
        a.step(1)
        b.step(1)
        x, y = a.get_state().cpu().numpy(), b.get_state().cpu().numpy()
        bad = np.argwhere(x != y)
        assert bad.size == 0, (n, bad[:5].tolist())
    assert a.diag()["flags"] == 0
