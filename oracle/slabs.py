"""The oracle's time step over a large lattice, run as z-slabs in parallel processes.

Test infrastructure, like the rest of oracle/: only the tests call it.  It adds no arithmetic of
its own.  A step reads each node's nearest neighbours only (the pull of eq. (mrteq)), so after k
steps a node depends on the nodes within k planes of it.  A slab of z-planes [z0, z1), cut out
with k halo planes on each side and stepped k times on its own (z faces periodic), therefore
holds on its own planes exactly the values of the whole lattice stepped k times; the halo planes'
results are dropped.  This needs the lattice's z faces to be periodic (the halo planes are then
the wrapped neighbours).

Workers are spawned processes, never forked, so a caller that holds a CUDA context can use it.
"""
import multiprocessing as mp
import os

import numpy as np


def _job(args):
    """One worker: (read-outs of the slab's input state for each formula,) k steps."""
    import oracle as O

    kw, dims, fslab, force, k, halo, readouts = args
    nx, ny, nzs = dims
    out = {}
    for fm in readouts:
        p = O.make_params(**dict(kw, formula=O.YU if fm == "yu" else O.CHAI))
        r = O.Grid(p, nx, ny, nzs).readout(fslab, force=force)
        out[fm] = (r["S"][:, halo:nzs - halo], r["tau"][halo:nzs - halo])
    G = O.Grid(O.make_params(**kw), nx, ny, nzs)
    f = fslab
    for _ in range(k):
        f, _ = G.step(f, force=force)
    return f[:, halo:nzs - halo], out


def run(params_kw, f, steps=1, force=None, readouts=(), workers=None):
    """`steps` oracle steps of the post-collision state f (q, nz, ny, nx, float64) with the
    parameters make_params(**params_kw) (bc with periodic z faces), and the read-outs (S, tau)
    of f's pre-collision state by each formula named in `readouts` ("yu", "chai").  force: None
    or a uniform force (a per-node field is not supported here).  Returns (f_after,
    {formula: (S, tau)})."""
    import oracle as O

    bc = params_kw.get("bc")
    assert bc is None or (bc[4] == O.PERIODIC and bc[5] == O.PERIODIC), "z faces must be periodic"
    q, nz, ny, nx = f.shape
    workers = workers or os.cpu_count() or 1
    workers = max(1, min(workers, nz))
    halo = max(steps, 1)
    bounds = np.linspace(0, nz, workers + 1).astype(int)
    jobs = []
    for w in range(workers):
        z0, z1 = int(bounds[w]), int(bounds[w + 1])
        planes = np.arange(z0 - halo, z1 + halo) % nz
        jobs.append((params_kw, (nx, ny, len(planes)), np.ascontiguousarray(f[:, planes]), force, steps, halo,
                     tuple(readouts)))
    with mp.get_context("spawn").Pool(workers) as pool:
        res = pool.map(_job, jobs)
    f_after = np.concatenate([r[0] for r in res], axis=1)
    reads = {}
    for fm in readouts:
        reads[fm] = (np.concatenate([r[1][fm][0] for r in res], axis=1),
                     np.concatenate([r[1][fm][1] for r in res], axis=0))
    return f_after, reads
