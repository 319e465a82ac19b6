"""The visiting order of the multi-step launch (csrc/step_stream.cuh), checked on the CPU.

The launch hands out tickets t = k * units + p (step k of the launch, position p); position p
is the unit (zigzag(p // tiles, nz), zigzag(p % tiles, tiles)) with zigzag(i, n) = i/2 for even i
and n - 1 - i/2 for odd i.  A unit runs step k once its nine neighbours (z +-1, band +-1, both
wrapped) have finished step k - 1.  The claims the kernel relies on:
  - the order is a permutation of the units (every unit runs every step exactly once);
  - every dependency of a ticket is an earlier ticket (so the earliest unfinished ticket can run:
    no deadlock, whatever the number of resident blocks);
  - a unit's dependencies sit at most 2 * tiles + 2 positions after its own position in the
    previous step (nz > 1), or 2 positions (nz = 1), which is the span the launcher leaves
    between a ticket and its dependencies beyond the resident blocks.
"""
import itertools

import pytest


def zigzag(i, n):
    return n - 1 - i // 2 if i & 1 else i // 2


def position_of(nz, tiles):
    pos = {}
    for p in range(nz * tiles):
        pos[(zigzag(p // tiles, nz), zigzag(p % tiles, tiles))] = p
    return pos


def deps(z, ty, nz, tiles):
    return {((z + dz) % nz, (ty + dy) % tiles) for dz, dy in itertools.product((-1, 0, 1), repeat=2)}


@pytest.mark.parametrize("nz,tiles", [(1, 1), (1, 2), (1, 7), (1, 4096), (2, 3), (3, 1), (5, 8), (6, 7),
                                      (32, 16), (128, 32), (129, 5)])
def test_zigzag_order_is_a_permutation_with_bounded_span(nz, tiles):
    pos = position_of(nz, tiles)
    units = nz * tiles
    assert sorted(pos.values()) == list(range(units))
    assert set(pos) == {(z, t) for z in range(nz) for t in range(tiles)}
    span = 2 * tiles + 2 if nz > 1 else 2
    for (z, ty), p in pos.items():
        for d in deps(z, ty, nz, tiles):
            q = pos[d]
            # step k at position p waits for step k - 1 at position q: ticket (k-1)*units + q
            assert (0 * units + q) < (1 * units + p)  # an earlier ticket
            assert q - p <= span, ((z, ty), d, p, q)


@pytest.mark.parametrize("nz,tiles,resident", [(128, 32, 1216), (128, 16, 1064), (64, 7, 200), (1, 4096, 1824)])
def test_no_block_waits_when_units_exceed_resident_plus_span(nz, tiles, resident):
    """Simulated launch with `resident` blocks taking tickets in order, every unit taking the same
    time: with units >= resident + span no ticket ever finds a dependency unfinished."""
    units = nz * tiles
    span = (2 * tiles if nz > 1 else 0) + 3
    if units < resident + span:
        pytest.skip("the launcher would not stream this shape")
    pos = position_of(nz, tiles)
    unit_at = {p: u for u, p in pos.items()}
    steps = 4
    finish = {}  # ticket -> finishing time
    free_at = [0] * resident  # time at which each block takes its next ticket
    for t in range(steps * units):
        b = min(range(resident), key=lambda i: free_at[i])
        start = free_at[b]
        k, p = divmod(t, units)
        if k > 0:
            z, ty = unit_at[p]
            for d in deps(z, ty, nz, tiles):
                dep_t = (k - 1) * units + pos[d]
                assert finish[dep_t] <= start, (t, dep_t)
        finish[t] = start + 1
        free_at[b] = start + 1
