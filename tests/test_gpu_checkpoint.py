"""Checkpoint and resume through the boundary: a run stopped after some steps,
saved in the FP32 form (lbm_get_state) with its step counter and restarted on
a fresh context (lbm_set_state) continues as the uninterrupted run.

The saved form is the AA layout's canonical state, so a context restarted
from it takes its next step as an even one.  Split at an even step count the
restarted run launches the same kernels in the same order as the
uninterrupted one and must agree bit for bit (16-bit storage too: the FP32
form of a stored value converts back to the same bits).  Split at an odd
count it takes the even kernel where the uninterrupted run takes the odd
one: the same arithmetic per node from the same populations, so the states
agree to the rounding of the collision (FP32, or one storage ulp where that
decides a 16-bit rounding), carried through the remaining steps."""
import numpy as np
import pytest

from paper_2112_08479_gb300 import lbm

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOTAL = 24
ULP = {"fp32": 2.0**-23, "fp16s": 2.0**-10, "bf16s": 2.0**-7}


@pytest.mark.parametrize("model,storage", [("bgk", "fp32"), ("cumulant", "fp32"),
                                           ("bgk", "fp16s"), ("cumulant", "bf16s")])
@pytest.mark.parametrize("split", [10, 11])
def test_resume_continues_the_run(model, storage, split):
    p = lbm.lock_exchange(64, 8, 16, H=16, x0=16, u_b=0.05, Re=1000.0, model=model,
                          storage=storage)
    whole = lbm.Lattice(p)
    whole.step(TOTAL)
    want = whole.get_state().cpu().numpy()
    dw = whole.diag()

    first = lbm.Lattice(p)
    first.step(split)
    saved = first.get_state().clone()
    n = first.step_count
    del first

    resumed = lbm.Lattice(p)
    resumed.set_state(saved, step=n)
    resumed.step(TOTAL - split)
    assert resumed.step_count == TOTAL
    got = resumed.get_state().cpu().numpy()
    d = resumed.diag()
    assert d["step"] == dw["step"] == TOTAL
    if split % 2 == 0:
        assert np.array_equal(got, want)
        assert d["front"] == dw["front"] and d["Fw"] == dw["Fw"]
        return
    # roundings of the first differing step, carried through the remaining
    # 13 steps: a few ulps of the stored values
    diff = np.abs(got.astype(np.float64) - want)
    scale = np.abs(want).max(axis=1, keepdims=True)
    tol = ULP[storage] * (np.abs(want) + 1e-3 * scale) * 16
    assert np.all(diff <= tol), float((diff / np.maximum(tol, 1e-30)).max())
    assert d["front"] == pytest.approx(dw["front"], abs=1e-4)
