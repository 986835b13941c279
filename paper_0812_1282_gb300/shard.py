"""Multi-GPU split of a batch of independent domains (one process per GPU).

The domains of a batch (many sessile drops or channels of uneven sizes)
never exchange data, so the multi-GPU form of a batched job gives each rank
a subset of the domains and lets it step them alone: no collective touches
the data path.  Only the per-domain results (a few numbers each: contact
angle, spurious-current norm, a non-finite count) meet at the end, summed
over ranks into one table that every rank holds.

The split balances node counts (the work of a step is proportional to the
nodes a rank owns): domains are taken largest first and each goes to the
rank with the fewest nodes so far, the greedy longest-processing-time rule.
"""
from __future__ import annotations

import math


def partition(nodes, world: int):
    """Split domains with the given node counts over `world` ranks.

    Returns one ascending list of domain indices per rank.  Every domain
    appears exactly once.  Ties (equal sizes, equal loads) go to the lower
    index / lower rank, so every rank computes the same split."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(nodes)), key=lambda d: (-int(nodes[d]), d))
    load = [0] * world
    owned = [[] for _ in range(world)]
    for d in order:
        r = min(range(world), key=lambda k: (load[k], k))
        owned[r].append(d)
        load[r] += int(nodes[d])
    return [sorted(o) for o in owned]


def rank_loads(nodes, parts):
    """Node count per rank under a split."""
    return [sum(int(nodes[d]) for d in p) for p in parts]


def gather_rows(n_dom: int, width: int, mine: dict, device="cpu"):
    """Per-domain rows (`width` floats each) from every rank, as one list of
    n_dom rows on every rank.  `mine` maps this rank's domain indices to
    their rows.  Each domain is owned by exactly one rank, so a sum over
    ranks of tables that are zero outside the owned rows assembles the
    table (NaN or inf of an owned row survives the sum)."""
    import torch
    import torch.distributed as dist

    t = torch.zeros((n_dom, width), dtype=torch.float64)
    for d, row in mine.items():
        if len(row) != width:
            raise ValueError("row of domain %d has %d values, not %d" % (d, len(row), width))
        t[d] = torch.tensor([float(v) for v in row], dtype=torch.float64)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        t = t.to(device)
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        t = t.cpu()
    return [[float(v) for v in t[d]] for d in range(n_dom)]


def finite_or_none(v: float):
    return v if math.isfinite(v) else None
