"""The z-slab decomposition through the library (lattices with halo z faces, lbm_halo_pack /
lbm_halo_unpack) against the same lattice stepped whole, on one GPU.

Slabs compute each node with the same arithmetic as the whole lattice, so after every step the
slabs' own planes equal the whole lattice's planes bit for bit (populations, and after an
exchange the read-outs of both formulas); the slabs' sums add up to the lattice's.  Exchanges run
in one process (copies between the slabs' device buffers, two and three slabs, and one slab that
is its own neighbour) and between two processes sharing the GPU through gloo and host memory
(slab.Slabs, the path a multi-GPU run takes with NCCL).  No kernel waits on another process: each
process steps, then exchanges on the host.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1704_07559_gb300 import inputs as I
from paper_1704_07559_gb300 import lbm, slab

pytestmark = pytest.mark.gpu

TAU0 = 0.51
RATES19 = [0, 1.19, 1.4, 0, 1.2, 0, 1.2, 0, 1.2, 1 / TAU0, 1.4, 1 / TAU0, 1.4, 1 / TAU0, 1 / TAU0, 1 / TAU0, 1.98,
           1.98, 1.98]
RATES15 = [0, 1.19, 1.4, 0, 1.2, 0, 1.2, 0, 1.2] + [1 / TAU0] * 5 + [1.98]
CHANNEL = ["periodic", "periodic", "wall", "wall"]
DIMS = (64, 24, 20)
FORCE = [1e-5, 0.0, 2e-6]


def fields(dims):
    nx, ny, nz = dims
    drho, u = I.channel_profile(nx, ny, nz, u_centre=0.08, noise=0.01, seed=2)
    g = np.random.default_rng(3).normal(scale=1e-3, size=(9, nz, ny, nx))
    return drho, u, g


def with_ghosts(a, z0, z1):
    """The planes [z0 - 1, z1 + 1) of a field (periodic in z), for a slab's init."""
    nz = a.shape[-3]
    return np.ascontiguousarray(np.take(a, np.arange(z0 - 1, z1 + 1) % nz, axis=-3))


def make(q, dims, precision, formula, halo):
    bc = CHANNEL + (["halo", "halo"] if halo else ["periodic", "periodic"])
    return lbm.Lattice(q, *dims, rates=RATES19 if q == 19 else RATES15, precision=precision, closure="smag",
                       smag_cs=0.17, formula=formula, bc=bc, force=FORCE)


def exchange(slabs, bufs):
    """Pack every slab, then unpack into each slab what its neighbours packed (periodic)."""
    k = len(slabs)
    for s, (lo, hi) in zip(slabs, bufs):
        s.halo_pack(lo, hi)
    for i, s in enumerate(slabs):
        s.halo_unpack(bufs[(i - 1) % k][1], bufs[(i + 1) % k][0])


@pytest.mark.parametrize("q,precision,formula,nslab", [
    (19, "fp32", "yu", 2), (19, "fp32", "chai", 3), (19, "fp16s", "yu", 2), (19, "bf16s", "chai", 3),
    (19, "fp64", "yu", 2), (15, "fp32", "chai", 2), (19, "fp32", "yu", 1)])
def test_slabs_equal_the_whole_lattice(q, precision, formula, nslab):
    drho, u, g = fields(DIMS)
    whole = make(q, DIMS, precision, formula, halo=False)
    whole.init(drho, u, g)
    spans = [slab.split_planes(DIMS[2], nslab, r) for r in range(nslab)]
    slabs = []
    for z0, z1 in spans:
        s = make(q, DIMS[:2] + (z1 - z0,), precision, formula, halo=True)
        s.init(with_ghosts(drho, z0, z1), with_ghosts(u, z0, z1), with_ghosts(g, z0, z1))
        slabs.append(s)
    pops, elems = slabs[0].halo_layout()
    assert pops == 5 and elems == 5 * DIMS[0] * DIMS[1]
    bufs = [(torch.empty(elems, dtype=s.storage_dtype, device="cuda"),
             torch.empty(elems, dtype=s.storage_dtype, device="cuda")) for s in slabs]
    for step in range(6):
        whole.step(1)
        for s in slabs:
            s.step(1)
        exchange(slabs, bufs)
        fw = whole.get_state()
        for (z0, z1), s in zip(spans, slabs):
            assert torch.equal(s.get_state()[:, 1:-1], fw[:, z0:z1]), (step, z0)
    for fm in ("yu", "chai"):
        Sw = whole.strain_rate(fm)
        for (z0, z1), s in zip(spans, slabs):
            assert torch.equal(s.strain_rate(fm)[:, 1:-1], Sw[:, z0:z1]), fm
    total = sum(s.sums() for s in slabs)
    ref = whole.sums()
    scale = whole.N * float(fw.abs().max().double())
    assert np.abs(total - ref).max() <= (1e-13 if precision == "fp64" else 1e-6) * scale


def test_halo_rules():
    s = make(19, (16, 8, 4), "fp32", "yu", halo=True)
    drho, u, g = fields((16, 8, 6))
    s.init(drho, u)
    with pytest.raises(lbm.LBMError) as ei:
        s.step(2)  # the exchange sits between steps
    assert ei.value.code == -1
    s.step(1)
    with pytest.raises(lbm.LBMError) as ei:
        s.set_watchdog(3, 1e-6)
    assert ei.value.code == -1
    w = make(19, (16, 8, 4), "fp32", "yu", halo=False)
    with pytest.raises(lbm.LBMError) as ei:
        w.halo_layout()
    assert ei.value.code == -1
    t = torch.empty(16, device="cuda")
    with pytest.raises(lbm.LBMError) as ei:
        w.halo_pack(t, t)
    assert ei.value.code == -1


def free_port():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def _rank(rank, world, port, steps, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        torch.cuda.set_device(0)
        drho, u, g = fields(DIMS)
        z0, z1 = slab.split_planes(DIMS[2], world, rank)
        s = make(19, DIMS[:2] + (z1 - z0,), "fp32", "chai", halo=True)
        s.init(with_ghosts(drho, z0, z1), with_ghosts(u, z0, z1), with_ghosts(g, z0, z1))
        slab.Slabs(s, dist).step(steps)
        out[rank] = (z0, z1, s.get_state()[:, 1:-1].cpu().numpy())
    finally:
        dist.destroy_process_group()


def test_two_processes_exchange_through_gloo():
    steps = 5
    drho, u, g = fields(DIMS)
    whole = make(19, DIMS, "fp32", "chai", halo=False)
    whole.init(drho, u, g)
    whole.step(steps)
    want = whole.get_state().cpu().numpy()
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(2, free_port(), steps, out), nprocs=2, join=True)
        res = dict(out)
    for r in range(2):
        z0, z1, own = res[r]
        assert np.array_equal(own, want[:, z0:z1])
