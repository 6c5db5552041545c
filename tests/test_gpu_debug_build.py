"""The debug build of the library (liblbm_debug.so, compiled with LBM_DEBUG):
every population access of the step, halo, adjoint and state-transfer
kernels is index-checked, a failed check is recorded and its access skipped
(include/lbm.h).  It stands in for a memory checker: no access may fail a
check anywhere in the GPU suite.

test_gpu_suite_under_index_checks reruns the GPU suite in a child process on
the debug build (tests/conftest.py fails any test whose lattices recorded a
failed check).  The planted tests run only there: LBM_FLAG_TEST_BOUNDS makes
each check use half its array's extent, so in-bounds accesses to the upper
half of every array fail the check; the status comes back as LBM_ERR_BOUNDS
with the first failure recorded, nothing leaves its array, and the device
stays usable."""
import ctypes
import os
import subprocess
import sys

import pytest

from paper_2112_08479_gb300 import _build, lbm

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _debug_only():
    if not lbm.lbm_debug_build():
        pytest.skip("runs under the debug build (LBM_LIBRARY=debug)")


def test_release_build_rejects_the_test_hook():
    if lbm.lbm_debug_build():
        pytest.skip("release build only")
    p = lbm.lock_exchange(64, 2, 8, H=8, x0=8, u_b=0.05, Re=500.0,
                          flags=lbm.LBM_FLAG_TEST_BOUNDS)
    with pytest.raises(lbm.LBMError) as e:
        lbm.Lattice(p)
    assert e.value.status == lbm.LBM_ERR_ARG


def _run_debug(args, timeout):
    _build.build(debug=True)
    env = dict(os.environ, LBM_LIBRARY="debug")
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                        "-m", "gpu", *args], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=timeout)
    return r.returncode, r.stdout[-3000:] + r.stderr[-2000:]


def test_gpu_suite_under_index_checks():
    if lbm.lbm_debug_build():
        pytest.skip("the parent run starts this one")
    here = os.path.basename(__file__)
    rc, out = _run_debug(["tests", "--deselect", f"tests/{here}::test_gpu_suite_under_index_checks",
                          "-k", "not planted"], 1800)
    assert rc == 0, out
    print("debug build, GPU suite:", out.strip().splitlines()[-1])
    rc, out = _run_debug([f"tests/{here}", "-k", "planted", "-rs"], 600)
    assert rc == 0, out
    assert "4 passed" in out and "skipped" not in out, out
    print("debug build, planted failures:", out.strip().splitlines()[-1])


def _planted(p, steps):
    lat = lbm.Lattice(p)
    lat.step(steps)
    d = lbm.lbm_diagnostics()
    assert lbm.load().lbm_diag(lat.ctx, ctypes.byref(d)) == lbm.LBM_ERR_BOUNDS
    assert d.flags & lbm.LBM_DEVFLAG_BOUNDS
    count, site, off, extent = lat.debug_record()
    lat.sync()                                   # no asynchronous CUDA error
    return count, site, off, extent


@pytest.mark.planted_bounds
@pytest.mark.parametrize("model,storage,nx,flags", [
    ("bgk", "fp32", 64, 0), ("bgk", "fp16s", 64, 0), ("cumulant", "bf16s", 64, 0),
    # TMA-staged: a bulk copy that fails its check is neither issued nor
    # announced on its barrier, so the waits still end
    ("cumulant", "fp16s", 512, lbm.LBM_FLAG_TMA_STAGED)])
def test_planted_failures_are_recorded(model, storage, nx, flags):
    _debug_only()
    p = lbm.lock_exchange(nx, 4, 8, H=8, x0=8, u_b=0.05, Re=500.0, model=model, storage=storage,
                          flags=flags)
    p.flags |= lbm.LBM_FLAG_TEST_BOUNDS
    count, site, off, extent = _planted(p, 2)
    assert count > 0 and site in lbm.SITES
    assert extent > 0 and not (0 <= off < extent)     # beyond the halved extent
    # the device goes on: an unchecked-hook lattice steps and reads cleanly
    p.flags &= ~lbm.LBM_FLAG_TEST_BOUNDS
    lat = lbm.Lattice(p)
    lat.step(4)
    assert lat.diag()["flags"] == 0 and lat.debug_record()[0] == 0
