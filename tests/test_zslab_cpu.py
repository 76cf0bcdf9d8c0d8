"""The z-slab split's host logic on CPU: the exchange drivers of
paper_0901_1053_gb300/zslab.py move the right plane messages in the right
direction at the right time. A toy stepper with the scheme's plane coupling
(plane k reads every component of plane k - 1 and e_x, e_y of plane k + 1,
a current on moving planes and one wake sample per window point and step)
stands in for the GPU solve: split into slabs it must give the whole grid's
fields bit for bit and its wake up to the order of the final sum, in one
process (LocalChain) and on two gloo ranks (DistSlab)."""
import os
import socket

import numpy as np
import pytest

from paper_0901_1053_gb300 import zslab

M = 5           # values per component and plane
C0, NW = 3, 12  # bunch extent and wake window of the toy


def toy_rule(below, here, above, k_global, n):
    """New values of one plane: every component of the plane below, e_x and
    e_y of the plane above (components 0, 1), a moving current on e_z."""
    new = here + 0.1 * np.outer(np.arange(1, 7), below.sum(axis=0)) / 6.0 \
        + 0.05 * (above[0] - 0.5 * above[1])[None, :]
    d = k_global - n + C0
    if -C0 <= d < C0:
        new[2] -= 0.3 * (1.0 + 0.1 * d)
    return new


class ToySlab:
    """Planes [k_lo, k_hi) of an nz-plane toy grid with ghost planes below
    and above; the message interface of tetm.Solver (plane_bytes,
    export_plane, import_plane, step, sync, wake)."""

    def __init__(self, nz, k_lo, k_hi, seed=3):
        self.nz, self.k_lo, self.k_hi = nz, k_lo, k_hi
        rng = np.random.default_rng(seed)
        full = rng.standard_normal((nz, 6, M))
        self.y = np.zeros((k_hi - k_lo + 2, 6, M))        # local planes -1 .. nz_local
        self.y[1:-1] = full[k_lo:k_hi]
        self.n = 0
        self.w = np.zeros(NW)

    def owned(self):
        return self.y[1:-1]

    def plane_bytes(self, direction):
        return (6 if direction == zslab.UP else 2) * M * 8

    def export_plane(self, direction, buf):
        src = self.y[-2] if direction == zslab.UP else self.y[1][:2]
        b = np.frombuffer(np.ascontiguousarray(src).tobytes(), np.uint8)
        if hasattr(buf, "numpy"):
            buf.numpy()[:] = b
        else:
            buf[:] = b

    def import_plane(self, direction, buf):
        raw = buf.numpy() if hasattr(buf, "numpy") else buf
        v = np.frombuffer(raw.tobytes(), np.float64)
        if direction == zslab.UP:
            self.y[0] = v.reshape(6, M)
        else:
            self.y[-1][:2] = v.reshape(2, M)

    def sync(self):
        pass

    def step(self, n=1):
        for _ in range(n):
            old = self.y.copy()
            for kl in range(1, self.y.shape[0] - 1):
                kg = self.k_lo + kl - 1
                self.y[kl] = toy_rule(old[kl - 1], old[kl], old[kl + 1], kg, self.n)
                m = self.n - kg - C0
                if 0 <= m < NW:
                    self.w[m] += self.y[kl][2][0]
            self.n += 1

    def wake(self):
        return self.w.copy(), 0.0, 1.0


def whole(nz, steps):
    t = ToySlab(nz, 0, nz)
    t.step(steps)
    return t


def test_split_planes():
    assert zslab.split_planes(10, 3) == [(0, 3), (3, 7), (7, 10)]
    assert zslab.split_planes(4, 2) == [(0, 2), (2, 4)]
    with pytest.raises(ValueError):
        zslab.split_planes(5, 3)


@pytest.mark.parametrize("parts", [2, 3, 5])
def test_local_chain_equals_the_whole_grid(parts):
    nz, steps = 23, 30
    ref = whole(nz, steps)
    slabs = [ToySlab(nz, a, b) for a, b in zslab.split_planes(nz, parts)]
    chain = zslab.LocalChain(slabs)
    chain.step(steps)
    got = np.concatenate([s.owned() for s in slabs])
    assert np.array_equal(got, ref.owned())
    assert np.allclose(chain.wake()[0], ref.wake()[0], rtol=1e-14, atol=0)
    assert np.any(ref.wake()[0] != 0)


def test_a_missing_exchange_changes_the_result():
    """The check is sharp: stepping without the exchange differs."""
    nz, steps = 23, 10
    ref = whole(nz, steps)
    slabs = [ToySlab(nz, a, b) for a, b in zslab.split_planes(nz, 2)]
    for s in slabs:
        s.step(steps)
    assert not np.array_equal(np.concatenate([s.owned() for s in slabs]), ref.owned())


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, nz, steps, q):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world)})
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    a, b = zslab.split_planes(nz, world)[rank]
    d = zslab.DistSlab(ToySlab(nz, a, b), rank, world, device="cpu")
    d.step(steps)
    w = d.wake()[0]
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, a, b, d.slab.owned().copy(), w))


@pytest.mark.parametrize("world", [2])
def test_gloo_ranks_equal_the_whole_grid(world):
    import torch.multiprocessing as mp
    nz, steps = 21, 25
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, nz, steps, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=180) for _ in procs), key=lambda r: r[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    ref = whole(nz, steps)
    for rank, a, b, owned, w in res:
        assert np.array_equal(owned, ref.owned()[a:b]), rank
        assert np.allclose(w, ref.wake()[0], rtol=1e-14, atol=0), rank
