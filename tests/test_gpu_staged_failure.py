"""Failure path of the TMA-staged step kernel (LBM_FLAG_TMA_STAGED): every
wait of its producer and consumer warps on a shared-memory mbarrier is
bounded.  LBM_FLAG_TEST_STALL announces each block's first tile on its
barrier but issues none of its copies (the barrier's phase never completes:
a flag nothing sets) and sets a 0.1 s limit: the waits run out, the kernel records
LBM_DEVFLAG_TIMEOUT and returns, lbm_diag reports LBM_ERR_TIMEOUT, and the
device stays usable.  No fault, no trap, no hang is provoked."""
import ctypes

import pytest

from paper_2112_08479_gb300 import lbm

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _params(flags):
    return lbm.lock_exchange(512, 4, 8, H=8, x0=8, u_b=0.05, Re=500.0, model="cumulant",
                             storage="fp16s", flags=flags)


def test_stalled_wait_gives_up_and_reports_timeout():
    lat = lbm.Lattice(_params(lbm.LBM_FLAG_TMA_STAGED | lbm.LBM_FLAG_TEST_STALL))
    lat.step(1)
    d = lbm.lbm_diagnostics()
    assert lbm.load().lbm_diag(lat.ctx, ctypes.byref(d)) == lbm.LBM_ERR_TIMEOUT
    assert d.flags & lbm.LBM_DEVFLAG_TIMEOUT
    with pytest.raises(lbm.LBMError):
        lat.diag()
    lat.sync()                                   # no asynchronous CUDA error
    # the device goes on: the staged and the one-node kernels still agree
    a = lbm.Lattice(_params(lbm.LBM_FLAG_TMA_STAGED))
    b = lbm.Lattice(_params(lbm.LBM_FLAG_ONE_NODE))
    a.step(3)
    b.step(3)
    assert torch.equal(a.get_state(), b.get_state())
    assert a.diag()["flags"] == 0
