"""x-slab decomposition on CPU (gloo, world sizes 2 and 3): the exchange
protocol of paper_2112_08479_gb300.slab against the whole box.

The lattice of each rank is a numpy stand-in that streams in the AA pattern
with no collision (every stored value moves, none changes) and packs and
unpacks its faces as include/lbm.h specifies; the library's own kernels are
checked the same way on the GPU (tests/test_gpu_slab.py).  A pure streaming
permutation of distinct values exposes any value delivered to the wrong slot,
node or rank: after even and odd steps, with walls and with periodic ends,
the gathered canonical slab states (the streamed populations of every node)
must equal the whole box's exactly, and the slab diagnostics (sums over
slabs, front from the gathered column maxima) the whole box's."""
import os
import socket

import numpy as np
import pytest

C27 = np.array([[0, 0, 0], [1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1],
                [1, 1, 0], [-1, -1, 0], [1, -1, 0], [-1, 1, 0], [1, 0, 1], [-1, 0, -1],
                [1, 0, -1], [-1, 0, 1], [0, 1, 1], [0, -1, -1], [0, 1, -1], [0, -1, 1],
                [1, 1, 1], [-1, -1, -1], [1, 1, -1], [-1, -1, 1], [1, -1, 1], [-1, 1, -1],
                [-1, 1, 1], [1, -1, -1]])


def opp(d):
    return 0 if d == 0 else (d + 1 if d % 2 else d - 1)


class StreamLattice:
    """AA streaming (no collision) of Q fluid and 7 scalar populations on an
    [k][z][y][x] array: walls at both x ends (unless periodic x, whole box
    only) and both z ends, y periodic; the face buffers of lbm_halo_pack /
    lbm_halo_unpack."""

    def __init__(self, params, device="cpu"):
        import torch
        self.torch, self.params = torch, params
        self.Q = params.Q
        self.nx, self.ny, self.nz = params.nx, params.ny, params.nz
        self.px = bool(params.flags & 2)
        x = np.arange(params.nx) + params.x_offset
        gnx = params.nx_global or params.nx
        y = np.arange(params.ny)[:, None]
        z = np.arange(params.nz)[:, None, None]
        # distinct values (exact in FP32), falling along x so that the front
        # (largest x whose column maximum reaches the threshold) lies inside
        node = (gnx - 1 - x) + gnx * (y + params.ny * z)
        k = np.arange(self.Q + 7)[:, None, None, None]
        self.a = (node[None] * 64 + k).astype(np.float32)
        self.odd = False
        self.steps = 0

    @property
    def next_step_odd(self):
        return self.odd

    def _inside(self, x, z):
        okx = np.ones_like(x, dtype=bool) if self.px else (x >= 0) & (x < self.nx)
        return okx & (z >= 0) & (z < self.nz)

    def step(self, n=1):
        for _ in range(n):
            a, out = self.a, self.a.copy()
            Z, Y, X = np.meshgrid(np.arange(self.nz), np.arange(self.ny), np.arange(self.nx),
                                  indexing="ij")
            for base, q in ((0, self.Q), (self.Q, 7)):
                for d in range(q):
                    c = C27[d]
                    if not self.odd:
                        out[base + opp(d)] = a[base + d]
                        continue
                    if d == 0:
                        continue
                    xs, ys, zs = X - c[0], (Y - c[1]) % self.ny, Z - c[2]
                    ins = self._inside(xs, zs)
                    v = np.where(ins, a[base + opp(d), np.clip(zs, 0, self.nz - 1), ys,
                                        xs % self.nx], a[base + d])
                    xt, yt, zt = X + c[0], (Y + c[1]) % self.ny, Z + c[2]
                    int_ = self._inside(xt, zt)
                    out[base + d, zt[int_], yt[int_], xt[int_] % self.nx] = v[int_]
                    out[base + opp(d), Z[~int_], Y[~int_], X[~int_]] = v[~int_]
            self.a = out
            self.odd = not self.odd
            self.steps += 1

    def _face_dirs(self, s):
        return ([d for d in range(self.Q) if C27[d][0] == s],
                [k for k in range(7) if C27[k][0] == s])

    def halo_pack(self, face, buf):
        s = 1 if face == 0 else -1
        x = 0 if face == 0 else self.nx - 1
        fd, sd = self._face_dirs(s)
        rows = [self.a[d, :, :, x] for d in fd] + [self.a[self.Q + k, :, :, x] for k in sd]
        buf.copy_(self.torch.from_numpy(np.stack(rows).astype(np.float32).ravel()
                                        .view(np.uint8)))

    def halo_unpack(self, face, buf):
        s = 1 if face == 0 else -1
        x = 0 if face == 0 else self.nx - 1
        nb = buf.numpy().view(np.float32).reshape(-1, self.nz, self.ny)
        nfd, nsd = self._face_dirs(-s)                   # the neighbour's buffer order
        fd, sd = self._face_dirs(s)
        for base, dirs, ndirs, off in ((0, fd, nfd, 0), (self.Q, sd, nsd, len(nfd))):
            for d in dirs:
                c = C27[d]
                j = off + ndirs.index(opp(d))
                for z in range(self.nz):
                    zs = z - c[2]
                    if zs < 0 or zs >= self.nz:
                        continue
                    for y in range(self.ny):
                        self.a[base + d, z, y, x] = nb[j, zs, (y - c[1]) % self.ny]

    def state(self):
        """Canonical view (the streamed populations of every node): after an
        even AA step population i of node m sits in slot opp(i) of the
        upwind node m - c_i, or in slot i of m itself where that node lies
        beyond a wall (here the slab faces too)."""
        if not self.odd:
            return self.a
        out = self.a.copy()
        Z, Y, X = np.meshgrid(np.arange(self.nz), np.arange(self.ny), np.arange(self.nx),
                              indexing="ij")
        for base, q in ((0, self.Q), (self.Q, 7)):
            for d in range(1, q):
                c = C27[d]
                xs, ys, zs = X - c[0], (Y - c[1]) % self.ny, Z - c[2]
                ins = self._inside(xs, zs)
                out[base + d] = np.where(ins, self.a[base + opp(d), np.clip(zs, 0, self.nz - 1),
                                                     ys, xs % self.nx], self.a[base + d])
        return out

    def diag(self, raise_unstable=False):
        a = self.state()
        chi = a[self.Q:].sum(0)
        return {"Fw": float(a[1, 0].sum() - a[2, 1].sum()),
                "mass_delta": float(a[: self.Q].sum()), "scalar_mass": float(chi.sum()),
                "flags": 0, "front": 0.0, "front_node": 0.0, "step": self.steps}

    def column_max(self):
        chi = self.state()[self.Q:].sum(0)
        return self.torch.from_numpy(chi.mean(1).max(0).astype(np.float32))

    def front_of_columns(self, m, nx, thr, x0, H, periodic):
        m = m.numpy().astype(np.float64)
        xlim = nx if not periodic else max(1, (nx + x0) // 2)
        hits = np.nonzero(m[:xlim] >= thr)[0]
        if hits.size == 0:
            xn = -1.0
        else:
            x = int(hits[-1])
            xn = float(x) if x == xlim - 1 else x + (m[x] - thr) / (m[x] - m[x + 1])
        return (xn + 0.5 - x0) / H, xn


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _params(periodic, model=1):
    from paper_2112_08479_gb300 import lbm
    # the front threshold sits inside the stored values' range so that the
    # front lands on some column
    return lbm.Params(nx=24, ny=3, nz=4, model=model, x0=5, H=4,
                      flags=lbm.LBM_FLAG_PERIODIC_X if periodic else 0,
                      front_threshold=1.12e5)


def _worker(rank, world, port, periodic, steps, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    import torch
    import torch.distributed as dist
    from paper_2112_08479_gb300 import slab
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        s = slab.SlabLattice(_params(periodic), rank, world, device="cpu", align=4,
                             factory=StreamLattice)
        out = []
        for n in steps:
            s.step(n)
            d = s.diag()
            a = torch.from_numpy(np.ascontiguousarray(s.lat.state()))
            # slabs differ in width: gather each padded to the widest
            w = max(hi - lo for lo, hi in s.ranges)
            pad = torch.zeros(a.shape[:3] + (w,), dtype=a.dtype)
            pad[..., : a.shape[3]] = a
            allp = [torch.empty_like(pad) for _ in range(world)]
            dist.all_gather(allp, pad)
            if rank == 0:
                full = torch.cat([allp[r][..., : hi - lo] for r, (lo, hi) in enumerate(s.ranges)],
                                 dim=3)
                out.append((full.numpy(), d))
        if rank == 0:
            q.put(out)
    finally:
        dist.destroy_process_group()


def _run(world, periodic, steps):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, world, port, periodic, steps, q))
          for r in range(world)]
    for p in ps:
        p.start()
    out = q.get(timeout=300)
    for p in ps:
        p.join(timeout=120)
        assert p.exitcode == 0
    return out


@pytest.mark.parametrize("world,periodic", [(2, False), (2, True), (3, True), (3, False)])
def test_slabs_equal_whole_box(world, periodic):
    import torch  # noqa: F401
    from paper_2112_08479_gb300 import slab
    steps = [1, 1, 1, 2, 3]           # even, odd, even, then pairs and a triple
    got = _run(world, periodic, steps)
    whole = slab.SlabLattice(_params(periodic), 0, 1, device="cpu", factory=StreamLattice)
    assert len(got) == len(steps)
    for n, (state, d) in zip(steps, got):
        whole.step(n)
        assert np.array_equal(state, whole.lat.state()), n
        dw = whole.diag()
        for k in ("Fw", "mass_delta", "scalar_mass"):
            assert d[k] == pytest.approx(dw[k], rel=1e-12, abs=1e-6), k
        assert d["front_node"] == dw["front_node"] and d["front"] == dw["front"]
    # the values did move across the slab faces
    assert not np.array_equal(got[-1][0], StreamLattice(_params(periodic)).state())


def test_split_covers_the_box():
    from paper_2112_08479_gb300 import slab
    assert slab.split(2048, 8) == [(256 * r, 256 * (r + 1)) for r in range(8)]
    r = slab.split(2048, 3)
    assert r[0][0] == 0 and r[-1][1] == 2048 and all(a[1] == b[0] for a, b in zip(r, r[1:]))
    assert all((hi - lo) % 128 == 0 for lo, hi in r)
    with pytest.raises(ValueError):
        slab.split(2000, 2)
    with pytest.raises(ValueError):
        slab.split(256, 4)
