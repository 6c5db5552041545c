"""The C ABI boundary without a GPU: the library loads, exports every entry
point that include/lbm.h declares, the Python binding declares the same set,
the ctypes structures match the C layouts, and argument checking (which runs
on the host before anything is enqueued) rejects bad parameters."""
import ctypes as C
import os
import re

import pytest

from paper_2112_08479_gb300 import _build
from paper_2112_08479_gb300 import lbm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lbm.h")


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return lbm.load()


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z0-9_]+)\s*\(", src)))


def test_header_symbols_exported(lib):
    names = _declared()
    assert len(names) >= 18
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(n for n, _, _ in lbm.SIGNATURES) == names


def test_debug_build_exports_the_same_entry_points(lib):
    """The index-checked debug build (built beside the release library by
    __graft_entry__.build) exports the same entry points and says so."""
    if not os.path.exists(_build.DEBUG_LIB) or not _build.up_to_date(_build.DEBUG_LIB):
        pytest.skip("liblbm_debug.so not built")
    dbg = C.CDLL(_build.DEBUG_LIB)
    for n in _declared():
        assert hasattr(dbg, n), n
    dbg.lbm_debug_build.restype = C.c_int32
    assert dbg.lbm_debug_build() == 1
    assert lbm.lbm_debug_build() is False


def test_release_build_rejects_the_index_check_hook(lib):
    s = lbm.lbm_validate(_good(flags=lbm.LBM_FLAG_TEST_BOUNDS))
    assert s == lbm.LBM_ERR_ARG
    assert b"debug build" in lbm.load().lbm_last_error(None)


def test_storage_constants_match_the_header():
    src = open(HEADER).read()
    m = re.search(r"#define LBM_SCALAR_CHI16 ([0-9.]+)", src)
    assert m and float(m.group(1)) == lbm.LBM_SCALAR_CHI16
    for name in ("LBM_FLAG_TEST_BOUNDS", "LBM_FLAG_TEST_STALL", "LBM_FLAG_TMA_STAGED",
                 "LBM_DEVFLAG_BOUNDS", "LBM_DEVFLAG_TIMEOUT"):
        m = re.search(rf"#define {name} (\d+)", src)
        assert m and int(m.group(1)) == getattr(lbm, name), name


def test_struct_layouts():
    # sizes computed from the C declarations with natural alignment
    assert C.sizeof(lbm.lbm_params) == 6 * 4 + 5 * 8 + 3 * 8 + 8 + 2 * 4 + 8 + 8 + 3 * 8 + 4 * 4
    assert C.sizeof(lbm.lbm_diagnostics) == 5 * 8 + 8 + 4 + 4


def _good(**kw):
    p = lbm.Params(nx=16, ny=4, nz=8, x0=4, H=8, gprime=1e-4)
    for k, v in kw.items():
        setattr(p, k, v)
    return p.c()


def test_validate_accepts_defaults(lib):
    assert lbm.lbm_validate(_good()) == lbm.LBM_OK
    assert lbm.lbm_workspace_bytes(_good()) > (19 + 7) * 16 * 4 * 8 * 4


@pytest.mark.parametrize("field,value", [
    ("nx", 0), ("ny", 70000), ("nz", -1), ("model", 5), ("storage", 9), ("flags", 128),
    ("nu", 0.0), ("nu", float("nan")), ("D", -1.0), ("cs_smag", -0.1), ("sc_t", 0.0),
    ("gprime", float("inf")), ("x0", 17), ("x0", -1), ("H", 0), ("noise_amp", -1.0),
    ("scale_f", 0.0), ("front_threshold", float("nan")), ("nx_global", 8), ("x_offset", -1),
    ("x_offset", 1),
])
def test_validate_rejects(lib, field, value):
    p = _good(**{field: value})
    assert lbm.lbm_validate(p) == lbm.LBM_ERR_ARG
    assert lbm.lbm_workspace_bytes(p) == 0


def test_one_node_flag_accepted(lib):
    """LBM_FLAG_ONE_NODE (a test hook selecting the one-node step kernels)
    combines with the geometry flags."""
    flags = lbm.LBM_FLAG_ONE_NODE | lbm.LBM_FLAG_PERIODIC_X | lbm.LBM_FLAG_PERIODIC_Z
    assert lbm.lbm_validate(_good(flags=flags)) == lbm.LBM_OK


def test_scalar_lattice_pairs(lib):
    """BGK runs with D3Q7 or D3Q6, the cumulant model with D3Q7 or D3Q27."""
    assert lbm.lbm_validate(_good(scalar=lbm.LBM_SCALAR_Q6)) == lbm.LBM_OK
    assert lbm.lbm_validate(_good(scalar=lbm.LBM_SCALAR_Q27)) == lbm.LBM_ERR_ARG
    assert lbm.lbm_validate(_good(model=lbm.LBM_CUMULANT_Q27, scalar=lbm.LBM_SCALAR_Q27)) == lbm.LBM_OK
    assert lbm.lbm_validate(_good(model=lbm.LBM_CUMULANT_Q27, scalar=lbm.LBM_SCALAR_Q6)) == lbm.LBM_ERR_ARG
    assert lbm.lbm_validate(_good(scalar=5)) == lbm.LBM_ERR_ARG
    N = 16 * 4 * 8
    b7 = lbm.lbm_workspace_bytes(_good())
    b6 = lbm.lbm_workspace_bytes(_good(scalar=lbm.LBM_SCALAR_Q6))
    assert b7 - b6 == pytest.approx(N * 4, abs=512)


def test_cumulant_bulk_rate_range(lib):
    assert lbm.lbm_validate(_good(model=lbm.LBM_CUMULANT_Q27, omega_bulk=2.5)) == lbm.LBM_ERR_ARG
    assert lbm.lbm_validate(_good(model=lbm.LBM_CUMULANT_Q27, omega_bulk=1.0)) == lbm.LBM_OK


def test_too_many_nodes(lib):
    assert lbm.lbm_validate(_good(nx=65536, ny=1024, nz=32)) == lbm.LBM_ERR_ARG


def test_workspace_scales_with_storage(lib):
    b32 = lbm.lbm_workspace_bytes(_good(nx=256, ny=32, nz=64))
    b16 = lbm.lbm_workspace_bytes(_good(nx=256, ny=32, nz=64, storage=lbm.LBM_FP16S))
    N = 256 * 32 * 64
    # 26 rows at half the width, plus the FP32 row of the scalar's rest
    # population that 16-bit storage adds
    assert b32 - b16 == pytest.approx(26 * N * 2 - N * 4, abs=4096)
    b16q6 = lbm.lbm_workspace_bytes(_good(nx=256, ny=32, nz=64, storage=lbm.LBM_FP16S,
                                          scalar=lbm.LBM_SCALAR_Q6))
    b32q6 = lbm.lbm_workspace_bytes(_good(nx=256, ny=32, nz=64, scalar=lbm.LBM_SCALAR_Q6))
    assert b32q6 - b16q6 == pytest.approx(25 * N * 2, abs=4096)   # D3Q6 has no rest population


def test_init_checks_before_touching_the_device(lib):
    # invalid parameters, null workspace, small workspace and misalignment are
    # all rejected on the host, so no device is needed
    with pytest.raises(lbm.LBMError) as e:
        lbm.lbm_init(_good(nu=-1.0), 256, 1 << 20, 0)
    assert e.value.status == lbm.LBM_ERR_ARG
    with pytest.raises(lbm.LBMError) as e:
        lbm.lbm_init(_good(), 0, 1 << 20, 0)
    assert e.value.status == lbm.LBM_ERR_ARG
    with pytest.raises(lbm.LBMError) as e:
        lbm.lbm_init(_good(), 4096 + 8, 1 << 30, 0)
    assert e.value.status == lbm.LBM_ERR_ARG
    with pytest.raises(lbm.LBMError) as e:
        lbm.lbm_init(_good(), 4096, 1024, 0)
    assert e.value.status == lbm.LBM_ERR_NOMEM


def test_status_strings(lib):
    for s in range(7):
        assert lbm.lbm_status_string(s)
    assert lbm.lbm_status_string(99) == "unknown status"


def test_null_context_is_rejected(lib):
    assert lib.lbm_step(None, 1) == lbm.LBM_ERR_ARG
    assert lib.lbm_sync(None) == lbm.LBM_ERR_ARG
    assert lib.lbm_front_adjoint(None, None, None, None) == lbm.LBM_ERR_ARG
    assert lib.lbm_adjoint_segment(None, None, 0, 1, None, None, None, None, 1.0) == lbm.LBM_ERR_ARG
    assert lib.lbm_adjoint_step(None, None, None, None, None, 1.0) == lbm.LBM_ERR_ARG
    assert lib.lbm_objective_forward(None, 1, 1, None, None) == lbm.LBM_ERR_ARG
    assert lib.lbm_get_step(None) == -1
    lib.lbm_destroy(None)


def test_lock_exchange_parameters():
    """Sec. 2.5 / Eq. 12-14 in lattice units: u_b = sqrt(g' H), nu = u_b H / Re."""
    p = lbm.lock_exchange(2048, 128, 256, H=256, x0=256, u_b=0.03, Re=30000.0)
    assert p.gprime == pytest.approx(0.03**2 / 256)
    assert p.nu == pytest.approx(2.56e-4)
    assert p.D == p.nu
    assert 3 * p.nu + 0.5 == pytest.approx(0.500768)
    assert p.flags == 0 and p.sc_t == 1.0
    q = lbm.lock_exchange(2500, 150, 100, H=100, x0=100, u_b=0.03, Re=895.0, geometry="periodic",
                          sc_t="paper")
    assert q.flags == lbm.LBM_FLAG_PERIODIC_X            # Fig. 4b: periodic ends
    assert q.sc_t == pytest.approx(0.17**2)               # literal Sc_T = C_s^2
    with pytest.raises(ValueError):
        lbm.lock_exchange(8, 2, 4, H=4, x0=2, u_b=0.03, Re=100.0, geometry="open")


def test_slab_fields_checked(lib):
    """An x-slab: x_offset + nx within nx_global, x0 within the whole box, no
    periodic flag on the slab itself; the face buffer size."""
    assert lbm.lbm_validate(_good(nx_global=64, x_offset=48, x0=40)) == lbm.LBM_OK
    assert lbm.lbm_validate(_good(nx_global=64, x_offset=49)) == lbm.LBM_ERR_ARG
    assert lbm.lbm_validate(_good(nx_global=64, x_offset=0, x0=65)) == lbm.LBM_ERR_ARG
    assert lbm.lbm_validate(_good(nx_global=64, flags=lbm.LBM_FLAG_PERIODIC_X)) == lbm.LBM_ERR_ARG
    # D3Q19 + D3Q7: 5 + 1 populations with c_x = +1, ny nz elements each
    assert lbm.lbm_halo_bytes(_good()) == (5 + 1) * 4 * 8 * 4
    assert lbm.lbm_halo_bytes(_good(model=1)) == (9 + 1) * 4 * 8 * 4
    assert lbm.lbm_halo_bytes(_good(model=1, scalar=2)) == (9 + 9) * 4 * 8 * 4
    assert lbm.lbm_halo_bytes(_good(scalar=1, storage=1)) == (5 + 1) * 4 * 8 * 2
