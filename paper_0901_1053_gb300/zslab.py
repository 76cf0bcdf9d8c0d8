"""One solve split along z into slabs that advance side by side.

The scheme couples neighbouring planes only (Sec. 4: the method is easily
parallelised): updating planes [k0, k1) reads the state at planes k0 - 1 ..
k1. Before every step each slab therefore receives the six components of the
last plane of the slab below (into its ghost plane below) and e_x, e_y of the
first plane of the slab above (into the plane above its last one): two
messages per interface and step, point to point, no collective. Bunch current
and wake stay with the planes that carry them; the grid's wake is the sum of
the slabs' wakes, formed once at the end.

The slab objects are tetm.Solver instances created with k_range (the C ABI's
tetm_create_slab, tetm_export_plane, tetm_import_plane); the drivers below
only move their messages:
  LocalChain   every slab in this process (one GPU), messages through host
               buffers;
  DistSlab     one slab per rank, messages by torch.distributed point-to-point
               sends (gloo on host buffers, NCCL on device buffers).
"""
from __future__ import annotations

from typing import List, Sequence, Tuple

import numpy as np

UP, DOWN = 0, 1  # TETM_PLANES_UP / TETM_PLANES_DOWN


def split_planes(nz: int, parts: int) -> List[Tuple[int, int]]:
    """Contiguous plane ranges of nearly equal length (each at least 2)."""
    if parts < 1 or 2 * parts > nz:
        raise ValueError("cannot split %d planes into %d slabs of at least 2" % (nz, parts))
    edges = [round(p * nz / parts) for p in range(parts + 1)]
    return [(edges[p], edges[p + 1]) for p in range(parts)]


class LocalChain:
    """Slabs of one grid in one process, bottom to top. Per step: every slab
    exports its two messages, the exports complete, every slab imports its
    neighbours' messages, every slab steps."""

    def __init__(self, slabs: Sequence):
        self.slabs = list(slabs)
        self.up = [np.empty(s.plane_bytes(UP), np.uint8) for s in self.slabs[:-1]]
        self.down = [np.empty(s.plane_bytes(DOWN), np.uint8) for s in self.slabs[1:]]

    def exchange(self):
        for i in range(len(self.slabs) - 1):
            self.slabs[i].export_plane(UP, self.up[i])
            self.slabs[i + 1].export_plane(DOWN, self.down[i])
        for s in self.slabs:
            s.sync()
        for i in range(len(self.slabs) - 1):
            self.slabs[i + 1].import_plane(UP, self.up[i])
            self.slabs[i].import_plane(DOWN, self.down[i])

    def step(self, n: int = 1):
        for _ in range(n):
            self.exchange()
            for s in self.slabs:
                s.step(1)

    def wake(self):
        """The grid's wake: the slabs' wakes summed bottom to top."""
        w, s0, ds = self.slabs[0].wake()
        total = np.array(w, dtype=np.float64)
        for s in self.slabs[1:]:
            total = total + s.wake()[0]
        return total, s0, ds


class DistSlab:
    """The slab of this rank of a torch.distributed group (ranks in plane
    order). Messages travel in buffers on `device` ("cpu" for gloo)."""

    def __init__(self, slab, rank: int, world: int, device="cpu", group=None):
        import torch
        self.slab, self.rank, self.world, self.group = slab, rank, world, group
        self.host = str(device) == "cpu"

        def buf(direction):
            return torch.empty(slab.plane_bytes(direction), dtype=torch.uint8, device=device)
        self.send_up = buf(UP) if rank < world - 1 else None
        self.recv_down = buf(DOWN) if rank < world - 1 else None
        self.send_down = buf(DOWN) if rank > 0 else None
        self.recv_up = buf(UP) if rank > 0 else None

    def exchange(self):
        import torch.distributed as dist
        if self.send_up is not None:
            self.slab.export_plane(UP, self.send_up)
        if self.send_down is not None:
            self.slab.export_plane(DOWN, self.send_down)
        self.slab.sync()
        reqs = []
        if self.send_up is not None:
            reqs.append(dist.isend(self.send_up, self.rank + 1, group=self.group))
            reqs.append(dist.irecv(self.recv_down, self.rank + 1, group=self.group))
        if self.send_down is not None:
            reqs.append(dist.isend(self.send_down, self.rank - 1, group=self.group))
            reqs.append(dist.irecv(self.recv_up, self.rank - 1, group=self.group))
        for r in reqs:
            r.wait()
        if not self.host:
            import torch
            torch.cuda.synchronize()  # the received bytes are in place before the solve's stream reads them
        if self.recv_up is not None:
            self.slab.import_plane(UP, self.recv_up)
        if self.recv_down is not None:
            self.slab.import_plane(DOWN, self.recv_down)

    def step(self, n: int = 1):
        for _ in range(n):
            self.exchange()
            self.slab.step(1)

    def wake(self):
        """The grid's wake on every rank: one sum over the ranks."""
        import torch
        import torch.distributed as dist
        w, s0, ds = self.slab.wake()
        t = torch.tensor(np.asarray(w, dtype=np.float64))
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=self.group)
        return t.numpy(), s0, ds
