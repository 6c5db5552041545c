import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: long-running CPU test")
    config.addinivalue_line("markers", "planted_bounds: makes the debug build's index checks "
                            "fail on purpose (LBM_FLAG_TEST_BOUNDS)")


@pytest.fixture(autouse=True, scope="session")
def _oracle_threads():
    """The oracle's node loops on every host core (results do not depend on
    the thread count, tests/test_oracle_flows.py checks that)."""
    import oracle as O
    O.set_threads(os.cpu_count() or 1)
    yield


@pytest.fixture(autouse=True)
def _index_checks(request):
    """Under the debug build of the library (LBM_LIBRARY=debug), no index
    check may fail in a test, except where a test plants the failures."""
    yield
    lbm = sys.modules.get("paper_2112_08479_gb300.lbm")
    if lbm is None or lbm._lib is None or not lbm._lib.lbm_debug_build():
        return
    import gc
    gc.collect()                       # destroy the test's lattices: their records count
    total = list(lbm.DEBUG_TOTAL)
    lbm.DEBUG_TOTAL[:] = [0, 0, 0, 0]
    if "planted_bounds" in request.keywords:
        return
    assert total[0] == 0, (f"{total[0]} failed index checks, first at site "
                           f"{lbm.SITES.get(total[1], total[1])}: offset {total[2]} of {total[3]}")


def pytest_collection_modifyitems(config, items):
    try:
        import torch
        have_gpu = torch.cuda.is_available()
    except Exception:  # pragma: no cover
        have_gpu = False
    if have_gpu:
        return
    skip = pytest.mark.skip(reason="no CUDA device")
    for item in items:
        if "gpu" in item.keywords:
            item.add_marker(skip)
