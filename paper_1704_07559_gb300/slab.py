"""Domain decomposition of a lattice into z-slabs, one per rank (usually one per GPU).

The method is local in space: a step reads each node's nearest neighbours only (the pull of
eq. (mrteq)), the natural parallelism Sec. 1 of the paper points to.  Cut along z, a slab needs
from each neighbouring slab only the populations that cross the shared face: after every step
its top own plane sends the populations with c_z = +1 up and its bottom own plane those with
c_z = -1 down (5 of 19 in D3Q19), and the slab writes what it receives into its ghost planes,
which its next step pulls from.  The library holds the slab (a lattice created with 'halo' z faces)
and packs and unpacks those populations on the GPU (lbm_halo_pack / lbm_halo_unpack); this module
moves them between ranks with torch.distributed point-to-point messages: NCCL between the GPUs'
own memories, or gloo through host copies.  The lattice as a whole is periodic in z: slab k's
upper neighbour is slab k + 1 modulo the number of slabs, and a single slab exchanges with itself.

Each step is lat.step(1) then exchange(); after lat.init(...) the ghost planes already hold what
the first step pulls, so no exchange precedes it.
"""
import torch


def split_planes(nz, world, rank):
    """Planes [z0, z1) of the global lattice owned by `rank`: the nz planes in `world` contiguous
    slabs whose sizes differ by at most one."""
    base, extra = divmod(nz, world)
    z0 = rank * base + min(rank, extra)
    return z0, z0 + base + (1 if rank < extra else 0)


class Slabs:
    """The exchange of one rank's slab.

    lat: a lattice with halo z faces (lbm.Lattice, or anything with halo_layout(),
    halo_pack(lo, hi), halo_unpack(lo, hi), step(n), storage_dtype and device; a CUDA lattice's
    stream must be torch's current stream).  dist: an initialised torch.distributed (or None for
    a single slab).  With a gloo process group the halos of a CUDA lattice travel through host
    memory."""

    def __init__(self, lat, dist=None):
        self.lat = lat
        self.dist = dist
        self.world = dist.get_world_size() if dist is not None else 1
        self.rank = dist.get_rank() if dist is not None else 0
        _, elems = lat.halo_layout()
        mk = lambda: torch.empty(elems, dtype=lat.storage_dtype, device=lat.device)  # noqa: E731
        self.send_lo, self.send_hi, self.recv_lo, self.recv_hi = mk(), mk(), mk(), mk()
        self.host = dist is not None and dist.get_backend() == "gloo" and lat.device.type == "cuda"
        if self.host:
            mkh = lambda: torch.empty(elems, dtype=lat.storage_dtype).pin_memory()  # noqa: E731
            self.h = [mkh() for _ in range(4)]

    def exchange(self):
        """Send this slab's outgoing populations to its neighbours and unpack theirs."""
        self.lat.halo_pack(self.send_lo, self.send_hi)
        if self.world == 1:
            self.recv_lo.copy_(self.send_hi)  # periodic in z: the slab is its own neighbour
            self.recv_hi.copy_(self.send_lo)
        else:
            up, down = (self.rank + 1) % self.world, (self.rank - 1) % self.world
            if self.host:
                s_lo, s_hi, r_lo, r_hi = self.h
                s_lo.copy_(self.send_lo)
                s_hi.copy_(self.send_hi)
            else:
                s_lo, s_hi, r_lo, r_hi = self.send_lo, self.send_hi, self.recv_lo, self.recv_hi
            # NCCL orders its messages after the work queued on the current stream (the pack) and
            # req.wait() orders the current stream after them (the unpack); the host copies of the
            # gloo path are synchronous
            d = self.dist
            # the messages going up carry tag 0, those going down tag 1 (with two slabs both
            # neighbours are the same rank); every rank posts them in the same order
            ops = [d.P2POp(d.isend, s_hi, up, tag=0), d.P2POp(d.irecv, r_lo, down, tag=0),
                   d.P2POp(d.isend, s_lo, down, tag=1), d.P2POp(d.irecv, r_hi, up, tag=1)]
            for req in d.batch_isend_irecv(ops):
                req.wait()
            if self.host:
                self.recv_lo.copy_(r_lo)
                self.recv_hi.copy_(r_hi)
        self.lat.halo_unpack(self.recv_lo, self.recv_hi)

    def step(self, n=1):
        """n steps of the whole decomposed lattice (this rank's share), exchanging after each."""
        for _ in range(n):
            self.lat.step(1)
            self.exchange()
        return self
