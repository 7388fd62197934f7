"""Partition of independent patches across ranks (one process per GPU).

Patches never exchange data, so a batch is split across ranks by cost with no collective
on the data path: largest patch first, each to the rank with the least assigned cells so
far (greedy longest-processing-time order; ties go to the lower rank).  Every rank computes
the same assignment from the same descriptor list.  Timing across ranks is reduced with a
max, the only collective used.
"""
from __future__ import annotations


def partition(cells, world: int):
    """Return, for each rank, the list of patch indices it owns."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(cells)), key=lambda i: (-cells[i], i))
    load = [0] * world
    owned = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda q: (load[q], q))
        owned[r].append(i)
        load[r] += cells[i]
    for lst in owned:
        lst.sort()
    return owned


def imbalance(cells, owned) -> float:
    """max over ranks of assigned cells / mean (1.0 = perfect balance)."""
    loads = [sum(cells[i] for i in lst) for lst in owned]
    mean = sum(loads) / len(loads)
    return max(loads) / mean if mean > 0 else 1.0
