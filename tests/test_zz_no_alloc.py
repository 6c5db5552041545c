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


def _static_diag(lat, state, step):
    d = lbm.lbm_diagnostics()
    s = lbm.load().lbm_diag_static(C.byref(lat._p), state.data_ptr(), step,
                                   lat.stream.cuda_stream, C.byref(d))
    assert s == lbm.LBM_OK, lbm.lbm_status_string(s)
    return d.as_dict()


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
        assert got["front"] == pytest.approx(ref["front"], abs=1e-6)
        assert got["front_node"] == pytest.approx(ref["front_node"], abs=1e-6)
        assert got["Fw"] == pytest.approx(ref["Fw"], rel=1e-6)
        assert got["scalar_mass"] == pytest.approx(ref["scalar_mass"], rel=1e-6)
        assert got["mass_delta"] == pytest.approx(ref["mass_delta"], abs=1e-6 * p.N)
        assert got["step"] == ref["step"] and got["flags"] == 0


def test_static_diag_rejects_sizes_beyond_its_scratch():
    lbm.load()
    p = lbm.Params(20000, 1, 2, x0=1, H=2).c()
    d = lbm.lbm_diagnostics()
    s = lbm.load().lbm_diag_static(C.byref(p), 256, 0, None, C.byref(d))
    assert s == lbm.LBM_ERR_ARG
    assert "lbm_diag_static" in lbm.load().lbm_last_error(None).decode()
