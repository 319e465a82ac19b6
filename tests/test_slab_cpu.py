"""The z-slab decomposition's exchange (paper_1704_07559_gb300/slab.py) on CPU, with gloo ranks:
each rank steps its slab with the FP64 oracle (its own planes plus one ghost plane per z face,
the halo contract of lbm_halo_pack / lbm_halo_unpack written out in numpy here) and exchanges the
crossing populations with its neighbours through slab.Slabs; the planes gathered from the ranks
equal the whole lattice stepped by the oracle, bit for bit.  Two and three ranks, the channel's
walls at y and a uniform force; a single slab exchanges with itself."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle as O
from paper_1704_07559_gb300 import inputs as I
from paper_1704_07559_gb300 import slab

TAU0 = 0.51
RATES = [0, 1.19, 1.4, 0, 1.2, 0, 1.2, 0, 1.2, 1 / TAU0, 1.4, 1 / TAU0, 1.4, 1 / TAU0, 1 / TAU0, 1 / TAU0, 1.98,
         1.98, 1.98]
CHANNEL = [O.PERIODIC, O.PERIODIC, O.WALL, O.WALL, O.PERIODIC, O.PERIODIC]
DIMS = (10, 8, 9)
F = np.array([1e-5, 0.0, 2e-6])
STEPS = 4


def params():
    return O.make_params(19, RATES, closure=O.SMAG, smag_cs=0.17, formula=O.CHAI, bc=CHANNEL)


def global_start():
    nx, ny, nz = DIMS
    G = O.Grid(params(), nx, ny, nz)
    drho, u = I.channel_profile(nx, ny, nz, u_centre=0.1, noise=0.01, seed=2)
    return G, G.init(drho, u, force=F)


class OracleSlab:
    """Planes [z0, z1) of the lattice and a ghost plane on each side, stepped by the oracle; the
    crossing populations (c_z = +1 up, c_z = -1 down, increasing index) packed and unpacked as
    the library does."""

    def __init__(self, fglobal, z0, z1):
        q, nz, ny, nx = fglobal.shape
        self.nl = z1 - z0
        planes = np.arange(z0 - 1, z1 + 1) % nz
        self.f = np.ascontiguousarray(fglobal[:, planes])  # the ghost planes as the global init left them
        self.G = O.Grid(params(), nx, ny, self.nl + 2)  # z periodic: the own planes never wrap
        c = O.tables(19)[0]
        self.up = [i for i in range(q) if c[i][2] == 1]
        self.dn = [i for i in range(q) if c[i][2] == -1]
        self.storage_dtype = torch.float64
        self.device = torch.device("cpu")

    def halo_layout(self):
        return len(self.up), len(self.up) * self.f.shape[2] * self.f.shape[3]

    def halo_pack(self, lo, hi):
        hi.copy_(torch.from_numpy(self.f[self.up, self.nl].ravel()))
        lo.copy_(torch.from_numpy(self.f[self.dn, 1].ravel()))

    def halo_unpack(self, lo, hi):
        shape = (len(self.up),) + self.f.shape[2:]
        self.f[self.up, 0] = lo.numpy().reshape(shape)
        self.f[self.dn, self.nl + 1] = hi.numpy().reshape(shape)

    def step(self, n):
        for _ in range(n):
            self.f, _ = self.G.step(self.f, force=F)

    def own(self):
        return self.f[:, 1:self.nl + 1]


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        _, f0 = global_start()
        z0, z1 = slab.split_planes(DIMS[2], world, rank)
        s = OracleSlab(f0, z0, z1)
        slab.Slabs(s, dist).step(STEPS)
        out[rank] = (z0, z1, s.own().copy())
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_slabs_over_gloo_ranks_equal_the_whole_lattice(world):
    G, f0 = global_start()
    want = G.run(f0, STEPS, force=F)
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, free_port(), out), nprocs=world, join=True)
        res = dict(out)
    got = np.zeros_like(want)
    for r in range(world):
        z0, z1, own = res[r]
        got[:, z0:z1] = own
    assert np.array_equal(got, want)


def test_one_slab_is_its_own_neighbour():
    G, f0 = global_start()
    s = OracleSlab(f0, 0, DIMS[2])
    slab.Slabs(s).step(STEPS)
    assert np.array_equal(s.own(), G.run(f0, STEPS, force=F))


def test_split_planes():
    for nz, world in ((9, 2), (128, 8), (7, 7), (10, 3)):
        spans = [slab.split_planes(nz, world, r) for r in range(world)]
        assert spans[0][0] == 0 and spans[-1][1] == nz
        assert all(spans[r][1] == spans[r + 1][0] for r in range(world - 1))
        sizes = [b - a for a, b in spans]
        assert max(sizes) - min(sizes) <= 1
