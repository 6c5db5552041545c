"""x-slab decomposition through the library's kernels: two ranks (gloo, host
staged face buffers), each running one half of a lock-exchange box on the
same GPU, against the whole box run on that GPU.

The ranks' kernels never wait on one another: every exchange goes through
the host (pack, copy, gloo send / receive, copy, unpack), so two processes
may share the one GPU.  Each odd AA step is bracketed by the halo exchange
(include/lbm.h); after even and odd steps the gathered slab states must
equal the whole box bit for bit (FP32; with 16-bit storage within one storage
ulp at a few elements, where the compiler's multiply-add fusion in the
wall-free and wall bodies of the step kernels differs and decides a rounding
to 16 bits), and the diagnostics must agree: F_w and the budgets to their
summation order, the front exactly."""
import os
import socket

import numpy as np
import pytest

from paper_2112_08479_gb300 import lbm

from helpers import stored_phi

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

STEPS = [1, 1, 2, 5, 31]


def _params(model, storage, periodic):
    return lbm.lock_exchange(256, 8, 16, H=16, x0=120, u_b=0.05, Re=1000.0, model=model,
                             storage=storage, geometry="periodic" if periodic else "walls")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, port, case, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE="2", MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    import torch
    import torch.distributed as dist
    from paper_2112_08479_gb300 import lbm, slab
    lbm.load()
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", rank=rank, world_size=2)
    try:
        s = slab.SlabLattice(_params(*case), rank, 2, device="cuda:0")
        out = []
        for n in STEPS:
            s.step(n)
            d = s.diag()
            st = s.lat.get_state().cpu()
            parts = [torch.empty_like(st) for _ in range(2)]
            dist.all_gather(parts, st)
            if rank == 0:
                Q = s.local.Q + s.local.NS
                full = torch.cat([p.view(Q, s.local.nz, s.local.ny, -1) for p in parts], dim=3)
                out.append((full.numpy(), d, s.lat.step_count))
        torch.cuda.synchronize()
        if rank == 0:
            q.put(out)
    finally:
        dist.destroy_process_group()


CASES = [("bgk", "fp32", False), ("bgk", "fp32", True), ("cumulant", "fp32", False),
         ("cumulant", "fp16s", True), ("bgk", "bf16s", False)]


@pytest.mark.parametrize("case", CASES)
def test_two_slabs_equal_whole_box(case):
    import torch.multiprocessing as mp
    model, storage, periodic = case
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, port, case, q)) for r in range(2)]
    for p in ps:
        p.start()
    got = q.get(timeout=600)
    for p in ps:
        p.join(timeout=120)
        assert p.exitcode == 0
    p = _params(*case)
    whole = lbm.Lattice(p, device="cuda")
    ulp = {"fp32": 0.0, "fp16s": 2.0**-10, "bf16s": 2.0**-7}[storage]
    scale = np.r_[[p.scale_f] * p.Q, [p.scale_phi] * p.NS][:, None] if ulp else 1.0
    for n, (state, d, step) in zip(STEPS, got):
        whole.step(n)
        assert step == whole.step_count
        want = whole.get_state().cpu().numpy()
        got_s = state.reshape(p.Q + p.NS, -1)
        if ulp == 0.0:
            bad = np.argwhere(got_s != want)
            assert bad.size == 0, (step, bad[:5].tolist())
        else:
            diff = np.abs(got_s.astype(np.float64) - want)
            mag = np.maximum(np.abs(got_s), np.abs(want)).astype(np.float64)
            mag[p.Q:] = np.maximum(stored_phi(got_s[p.Q:], p), stored_phi(want[p.Q:], p))
            tol = np.maximum(mag * scale * ulp, 2.0**-24) / scale
            tol[p.Q] = stored_phi(want[p.Q + 1:], p, 1).sum(axis=0) * ulp + 2.0**-20   # FP32 rest
            assert np.all(diff <= tol * 1.0001), step
            assert np.count_nonzero(diff) <= max(16, 1e-3 * diff.size), step
        dw = whole.diag()
        assert d["front_node"] == pytest.approx(dw["front_node"], abs=1e-9 if ulp == 0 else 1e-3)
        assert d["Fw"] == pytest.approx(dw["Fw"], rel=1e-5, abs=1e-12)
        assert d["scalar_mass"] == pytest.approx(dw["scalar_mass"], rel=1e-9)
        assert d["mass_delta"] == pytest.approx(dw["mass_delta"], abs=1e-6 * p.N)
        assert d["flags"] == 0
