"""The oracle's time step over a large lattice, run as slabs in parallel processes.

Test infrastructure, like the rest of oracle/: only the tests call it.  It adds no arithmetic of
its own.  A step reads each node's nearest neighbours only (the pull of eq. (mrteq)), so after k
steps a node depends on the nodes within k planes of it.  A slab of planes [a, b) along the cut
axis, cut out with k halo planes on each side and stepped k times on its own, therefore holds on
its own planes exactly the values of the whole lattice stepped k times; the halo planes' results
are dropped.  Along a periodic axis the halo planes are the wrapped neighbours.  Along an axis with
walls, a slab that reaches a face of the lattice keeps that face's boundary kind, and an interior
cut gets a wall: whatever a wall does there stays within the halo planes, which are dropped.

Workers are spawned processes, never forked, so a caller that holds a CUDA context can use it.
"""
import multiprocessing as mp
import os

import numpy as np


def _job(args):
    """One worker: (read-outs of the slab's input state for each formula,) k steps."""
    import oracle as O

    kw, dims, fslab, force, k, lo, hi, readouts, ax = args
    nx, ny, nz = dims
    own = [slice(None)] * 4
    own[ax] = slice(lo, fslab.shape[ax] - hi)
    own_f = tuple(own)
    own_s = tuple(own[1:])
    out = {}
    for fm in readouts:
        p = O.make_params(**dict(kw, formula=O.YU if fm == "yu" else O.CHAI))
        r = O.Grid(p, nx, ny, nz).readout(fslab, force=force)
        out[fm] = (r["S"][(slice(None),) + own_s], r["tau"][own_s])
    G = O.Grid(O.make_params(**kw), nx, ny, nz)
    f = fslab
    for _ in range(k):
        f, _ = G.step(f, force=force)
    return f[own_f], out


def run(params_kw, f, steps=1, force=None, readouts=(), workers=None, axis="z"):
    """`steps` oracle steps of the post-collision state f (q, nz, ny, nx, float64) with the
    parameters make_params(**params_kw), and the read-outs (S, tau) of f's pre-collision state by
    each formula named in `readouts` ("yu", "chai"); the lattice is cut along `axis` ("z" or "y").
    force: None or a uniform force (a per-node field is not supported here).  Returns (f_after,
    {formula: (S, tau)})."""
    import oracle as O

    q, nz, ny, nx = f.shape
    ax = {"z": 1, "y": 2}[axis]
    faces = (4, 5) if axis == "z" else (2, 3)
    n = f.shape[ax]
    bc = list(params_kw.get("bc") or [O.PERIODIC] * 6)
    periodic = bc[faces[0]] == O.PERIODIC
    workers = max(1, min(workers or os.cpu_count() or 1, n))
    halo = max(steps, 1)
    bounds = np.linspace(0, n, workers + 1).astype(int)
    jobs = []
    for w in range(workers):
        a, b = int(bounds[w]), int(bounds[w + 1])
        kw = dict(params_kw)
        if periodic:
            planes = np.arange(a - halo, b + halo) % n
            lo = hi = halo
        else:
            planes = np.arange(max(0, a - halo), min(n, b + halo))
            lo, hi = a - planes[0], planes[-1] + 1 - b
            sub = list(bc)
            if a > 0:
                sub[faces[0]] = O.WALL  # an interior cut: its effect stays in the dropped halo
            if b < n:
                sub[faces[1]] = O.WALL
            kw["bc"] = sub
        fs = np.ascontiguousarray(np.take(f, planes, axis=ax))
        dims = (nx, len(planes) if ax == 2 else ny, len(planes) if ax == 1 else nz)
        jobs.append((kw, dims, fs, force, steps, int(lo), int(hi), tuple(readouts), ax))
    with mp.get_context("spawn").Pool(workers) as pool:
        res = pool.map(_job, jobs)
    f_after = np.concatenate([r[0] for r in res], axis=ax)
    reads = {}
    for fm in readouts:
        reads[fm] = (np.concatenate([r[1][fm][0] for r in res], axis=ax),
                     np.concatenate([r[1][fm][1] for r in res], axis=ax - 1))
    return f_after, reads
