"""x-slab decomposition of a lock-exchange box over the ranks of a process
group, one slab per GPU.

The box of nx columns is cut along x (the direction the current travels)
into `world` slabs of whole tiles of `align` columns.  Each rank runs its slab
as an ordinary context of the library (lbm_params.x_offset / nx_global), with
walls at its x ends to the step kernels; after every step touching faces
swap their face buffers (lbm_halo_pack, the exchange, lbm_halo_unpack), which
makes the slab faces fluid for the next step and for every read of the state
in between (diagnostics, lbm_get_state).  With periodic x the ring closes
over the last and first slab.  The result equals the whole-box run bit for
bit.

Exchange: NCCL point-to-point on device buffers, or any other backend (gloo)
through pinned host copies.  The diagnostics sum F_w and the FP64 budgets
over the slabs (all-reduce) and take the front (Sec. 3.1) from the column
maxima of all slabs gathered in x order (lbm_column_max,
lbm_front_of_columns).  All arithmetic of the method runs in the library's
kernels; this module moves buffers between ranks.
"""
from __future__ import annotations

import dataclasses

from . import lbm


def split(nx: int, world: int, align: int = 128):
    """Column ranges [lo, hi) of `world` slabs covering nx columns, each a
    whole number of `align`-column tiles, as equal as possible."""
    if nx % align:
        raise ValueError(f"nx = {nx} is not a multiple of the slab alignment {align}")
    units = nx // align
    if units < world:
        raise ValueError(f"{nx} columns give fewer than {world} slabs of {align}")
    base, extra = divmod(units, world)
    out, lo = [], 0
    for r in range(world):
        w = (base + (1 if r < extra else 0)) * align
        out.append((lo, lo + w))
        lo += w
    return out


def slab_params(p: lbm.Params, rank: int, world: int, align: int = 128) -> lbm.Params:
    """Parameters of rank's slab of the box p (p itself when world == 1)."""
    if world == 1:
        return p
    lo, hi = split(p.nx, world, align)[rank]
    return dataclasses.replace(p, nx=hi - lo, x_offset=lo, nx_global=p.nx,
                              flags=p.flags & ~lbm.LBM_FLAG_PERIODIC_X)


class SlabLattice:
    """One rank's slab of a box.  `factory(params, device)` builds the local
    lattice (default: lbm.Lattice); it must offer step, next_step_odd,
    halo_pack, halo_unpack, diag, column_max and front_of_columns."""

    def __init__(self, params: lbm.Params, rank: int = 0, world: int = 1, group=None,
                 device="cuda", align: int = 128, factory=None):
        import torch
        import torch.distributed as dist
        self.torch, self.dist = torch, dist
        self.params, self.rank, self.world, self.group = params, rank, world, group
        self.ranges = split(params.nx, world, align) if world > 1 else [(0, params.nx)]
        self.local = slab_params(params, rank, world, align)
        self.lat = (factory or (lambda q, dev: lbm.Lattice(q, device=dev)))(self.local, device)
        periodic = bool(params.flags & lbm.LBM_FLAG_PERIODIC_X)
        self.periodic = periodic
        self.left = self.right = None
        if world > 1:
            if rank > 0 or periodic:
                self.left = (rank - 1) % world
            if rank < world - 1 or periodic:
                self.right = (rank + 1) % world
        self.peer = {0: self.left, 1: self.right}
        self.device = torch.device(device)
        on_gpu = self.device.type == "cuda"
        self.nccl = world > 1 and on_gpu and dist.get_backend(group) == "nccl"
        nbytes = lbm.lbm_halo_bytes(self.local.c()) if world > 1 else 0
        mk = lambda dev: {f: torch.empty(nbytes, dtype=torch.uint8, device=dev)
                          for f in (0, 1) if self.peer[f] is not None}
        self.send, self.recv = mk(self.device), mk(self.device)
        # host staging for backends without device tensors (gloo)
        self.stage = on_gpu and world > 1 and not self.nccl
        if self.stage:
            pin = lambda: {f: torch.empty(nbytes, dtype=torch.uint8).pin_memory()
                           for f in (0, 1) if self.peer[f] is not None}
            self.hsend, self.hrecv = pin(), pin()

    # -- halo exchange ---------------------------------------------------------
    def _exchange(self):
        torch, dist = self.torch, self.dist
        faces = [f for f in (0, 1) if self.peer[f] is not None]
        for f in faces:
            self.lat.halo_pack(f, self.send[f])
        if self.stage:
            for f in faces:
                self.hsend[f].copy_(self.send[f])
            torch.cuda.current_stream(self.device).synchronize()
            send, recv = self.hsend, self.hrecv
        else:
            send, recv = self.send, self.recv
        # sends in the order (face 1, face 0), receives in the order (face 0,
        # face 1): a pair of ranks then matches in issue order even when both
        # faces of a rank touch the same peer (two slabs with periodic ends);
        # the tag is the face the buffer was packed from
        ops = []
        for f in (1, 0):
            if self.peer[f] is not None:
                ops.append(dist.P2POp(dist.isend, send[f], self.peer[f], self.group, tag=f))
        for f in (0, 1):
            if self.peer[f] is not None:
                ops.append(dist.P2POp(dist.irecv, recv[f], self.peer[f], self.group, tag=1 - f))
        for w in dist.batch_isend_irecv(ops):
            w.wait()
        if self.stage:
            for f in faces:
                self.recv[f].copy_(self.hrecv[f], non_blocking=True)
        for f in faces:
            self.lat.halo_unpack(f, self.recv[f])

    @property
    def stream(self):
        return self.lat.stream

    @property
    def N(self) -> int:
        """Nodes of this rank's slab."""
        return self.local.nx * self.local.ny * self.local.nz

    def set_scalar(self, chi0_local):
        """Re-initialises the slab from its part of a scalar field (the slab's
        N floats, host or device)."""
        self.lat.set_scalar(chi0_local)

    def step(self, n: int = 1):
        for _ in range(n):
            self.lat.step(1)
            if self.world > 1:
                self._exchange()

    # -- diagnostics -------------------------------------------------------------
    def diag(self) -> dict:
        torch, dist = self.torch, self.dist
        d = self.lat.diag(raise_unstable=False)
        m = self.lat.column_max()
        if self.world > 1:
            dev = self.device if self.nccl else torch.device("cpu")
            sums = torch.tensor([d["Fw"], d["mass_delta"], d["scalar_mass"]],
                                dtype=torch.float64, device=dev)
            dist.all_reduce(sums, group=self.group)
            flags = torch.tensor([d["flags"]], dtype=torch.int64, device=dev)
            allf = [torch.zeros_like(flags) for _ in range(self.world)]
            dist.all_gather(allf, flags, group=self.group)
            wmax = max(hi - lo for lo, hi in self.ranges)
            mp = torch.full((wmax,), float("-inf"), dtype=torch.float32, device=dev)
            mp[: m.numel()] = m.to(dev)
            parts = [torch.empty_like(mp) for _ in range(self.world)]
            dist.all_gather(parts, mp, group=self.group)
            m = torch.cat([parts[r][: hi - lo] for r, (lo, hi) in enumerate(self.ranges)])
            m = m.to(self.device)
            d["Fw"], d["mass_delta"], d["scalar_mass"] = (float(v) for v in sums.cpu())
            fl = 0
            for t in allf:
                fl |= int(t.item())
            d["flags"] = fl
        p = self.params
        d["front"], d["front_node"] = self.lat.front_of_columns(
            m, p.nx, p.front_threshold, p.x0, p.H, self.periodic)
        return d
