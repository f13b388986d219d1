"""Independent solves split across ranks (one process per GPU).

Batched tubes and served requests are independent units: each is a whole
shock-tube solve with its own state, so several GPUs share them without any
exchange on the data path.  This module only decides who solves what and
collects the results; every step of every solve runs in the CUDA library on
the rank that owns it.

* ``assign`` gives every unit to exactly one rank, balancing the work
  (node updates) by the longest-first greedy rule: units in decreasing
  order of work, each to the rank with the least work so far (ties to the
  lower rank).  It is deterministic, so every rank computes the same
  assignment without communicating.
* ``solve_partitioned`` runs a rank's units through a caller-given solve
  function and, when a process group is given, gathers every rank's results
  so that all ranks end with the full set (a host-side collective after the
  solves, not part of any step).
"""
from __future__ import annotations

import heapq
from typing import Callable, Sequence


def assign(work: Sequence[float], world: int) -> list[list[int]]:
    """Indices of the units each of `world` ranks solves (each index exactly
    once, ascending within a rank)."""
    if world < 1:
        raise ValueError("world must be at least 1")
    order = sorted(range(len(work)), key=lambda i: (-float(work[i]), i))
    heap = [(0.0, r) for r in range(world)]
    heapq.heapify(heap)
    parts: list[list[int]] = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        parts[r].append(i)
        heapq.heappush(heap, (load + float(work[i]), r))
    return [sorted(p) for p in parts]


def solve_partitioned(units: Sequence, work: Sequence[float],
                      solve: Callable[[list], dict], rank: int, world: int,
                      group=None) -> dict:
    """Solves this rank's share of `units` with ``solve(list_of_units)``,
    which returns {unit index within that list: result}.  Returns {global
    index: result} for this rank's units, or for all units when a
    torch.distributed process group is given (gathered after the solves)."""
    mine = assign(work, world)[rank]
    got = solve([units[i] for i in mine]) if mine else {}
    local = {mine[k]: v for k, v in got.items()}
    if group is None or world == 1:
        return local
    import torch.distributed as dist
    parts: list = [None] * world
    dist.all_gather_object(parts, local, group=group)
    out: dict = {}
    for p in parts:
        for k, v in p.items():
            if k in out:
                raise RuntimeError(f"unit {k} solved twice")
            out[k] = v
    return out
