"""Allocation-free diagnostics through the C ABI (lbm_diag_static).

Callers that cannot allocate device memory use lbm_diag_static, which keeps
its scratch in a fixed device array inside the library.  It must give the
same diagnostics as lbm_diag (which uses the caller's workspace) for the same
state, on consecutive calls: the second call has to start from a clean
scratch even though the array still holds the first call's contents.
"""
import ctypes as C

import pytest

from paper_2112_08479_gb300 import lbm

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _static_diag(lat, state, step, expect=lbm.LBM_OK, stream=None):
    d = lbm.lbm_diagnostics()
    st = (stream or lat.stream).cuda_stream
    s = lbm.load().lbm_diag_static(C.byref(lat._p), state.data_ptr(), step, st, C.byref(d))
    assert s == expect, lbm.lbm_status_string(s)
    return d.as_dict()


def _same(got, ref, p):
    assert got["front"] == pytest.approx(ref["front"], abs=1e-6)
    assert got["front_node"] == pytest.approx(ref["front_node"], abs=1e-6)
    assert got["Fw"] == pytest.approx(ref["Fw"], rel=1e-6)
    assert got["scalar_mass"] == pytest.approx(ref["scalar_mass"], rel=1e-6)
    assert got["mass_delta"] == pytest.approx(ref["mass_delta"], abs=1e-6 * p.N)
    assert got["step"] == ref["step"] and got["flags"] == 0


@pytest.mark.parametrize("model,geometry", [("bgk", "walls"), ("cumulant", "walls"),
                                            ("bgk", "periodic")])
def test_static_diag_matches_workspace_diag_on_consecutive_calls(model, geometry):
    p = lbm.lock_exchange(128, 8, 16, H=16, x0=16, u_b=0.05, Re=1000.0, model=model,
                          geometry=geometry)
    lat = lbm.Lattice(p, device="cuda")
    for steps in (37, 64):
        lat.step(steps)
        ref = lat.diag()
        got = _static_diag(lat, lat.get_state(), lat.step_count)
        _same(got, ref, p)


@pytest.mark.parametrize("model,scalar", [("bgk", "q6"), ("cumulant", "q27")])
def test_static_diag_other_scalar_lattices(model, scalar):
    """The D3Q6 (six scalar rows) and D3Q27 (27 rows) instantiations of the
    column kernel, on consecutive calls."""
    p = lbm.lock_exchange(130, 6, 12, H=12, x0=12, u_b=0.05, Re=800.0, model=model,
                          scalar=scalar)
    lat = lbm.Lattice(p, device="cuda")
    for steps in (41, 30):
        lat.step(steps)
        ref = lat.diag()
        _same(_static_diag(lat, lat.get_state(), lat.step_count), ref, p)


def test_static_diag_reports_a_planted_nan():
    """A state with one non-finite population: the call returns
    LBM_ERR_UNSTABLE with the same flag as lbm_diag (no device fault), and the
    next call on a clean state starts from cleared flags."""
    p = lbm.lock_exchange(128, 8, 16, H=16, x0=16, u_b=0.05, Re=1000.0)
    lat = lbm.Lattice(p, device="cuda")
    lat.step(10)
    clean = lat.get_state()
    bad = clean.clone()
    bad[3, 1000] = float("nan")
    got = _static_diag(lat, bad, 10, expect=lbm.LBM_ERR_UNSTABLE)
    lat2 = lbm.Lattice(p, device="cuda")
    lat2.set_state(bad, 10)
    ref = lat2.diag(raise_unstable=False)
    assert got["flags"] == ref["flags"] and got["flags"] & lbm.LBM_DEVFLAG_NONFINITE
    _same(_static_diag(lat, clean, 10), lat.diag(), p)


def test_static_diag_refuses_a_capturing_stream():
    """Every call synchronises its stream, which is not allowed under stream
    capture: the call returns LBM_ERR_ARG before enqueueing anything."""
    p = lbm.lock_exchange(64, 4, 8, H=8, x0=8, u_b=0.05, Re=500.0)
    lat = lbm.Lattice(p, device="cuda")
    state = lat.get_state()
    x = torch.zeros(16, device="cuda")
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    with torch.cuda.graph(g, stream=s):
        x.add_(1.0)
        _static_diag(lat, state, 0, expect=lbm.LBM_ERR_ARG, stream=s)
    assert "captured" in lbm.load().lbm_last_error(None).decode()
    g.replay()
    torch.cuda.synchronize()
    assert float(x.sum()) == 16.0


def test_static_diag_rejects_host_memory():
    p = lbm.lock_exchange(64, 4, 8, H=8, x0=8, u_b=0.05, Re=500.0)
    lat = lbm.Lattice(p, device="cuda")
    host = lat.get_state().cpu()
    _static_diag(lat, host, 0, expect=lbm.LBM_ERR_ARG)
    assert "current device" in lbm.load().lbm_last_error(None).decode()


def test_static_diag_rejects_sizes_beyond_its_scratch():
    lbm.load()
    p = lbm.Params(20000, 1, 2, x0=1, H=2).c()
    d = lbm.lbm_diagnostics()
    s = lbm.load().lbm_diag_static(C.byref(p), 256, 0, None, C.byref(d))
    assert s == lbm.LBM_ERR_ARG
    assert "lbm_diag_static" in lbm.load().lbm_last_error(None).decode()
