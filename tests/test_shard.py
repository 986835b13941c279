"""Multi-GPU split of the batched workload, on CPU: the node-balanced
partition of the domains over ranks, and the gather of per-domain results
(gloo, world size 2).  Each rank steps its share of small sessile drops with
the FP64 oracle (standing in for its GPU) and the gathered table must equal
the one a single process computes over all domains."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

import lbinputs
from paper_0812_1282_gb300 import shard

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _nodes(specs):
    return [s["nx"] * s["ny"] for s in specs]


@pytest.mark.parametrize("world", [1, 2, 3, 4, 8])
def test_partition_covers_every_domain_once_and_balances(world):
    nodes = _nodes(lbinputs.batch_specs())
    parts = shard.partition(nodes, world)
    assert len(parts) == world
    flat = sorted(d for p in parts for d in p)
    assert flat == list(range(len(nodes)))
    for p in parts:
        assert p == sorted(p)
    loads = shard.rank_loads(nodes, parts)
    # greedy largest-first: no rank exceeds the mean by more than the
    # largest domain
    assert max(loads) - sum(loads) / world <= max(nodes)
    if world > 1:
        assert max(loads) / min(loads) < 1.02   # 256 domains split evenly
    assert shard.partition(nodes, world) == parts  # deterministic


def test_partition_small_cases():
    assert shard.partition([5, 1, 1, 1, 1, 1], 2) == [[0], [1, 2, 3, 4, 5]]
    assert shard.partition([3, 3, 3], 3) == [[0], [1], [2]]
    assert shard.partition([], 2) == [[], []]
    assert shard.partition([7, 2], 4) == [[0], [1], [], []]
    with pytest.raises(ValueError):
        shard.partition([1], 0)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


SPECS = dict(n=6, seed=5, lo=24, hi=44)
STEPS = 60


def _run_domain(oracle, s):
    p = oracle.params(**lbinputs.BASE, collision="mrt", tau_alpha=s["tau_alpha"],
                      tau_beta=s["tau_beta"], h_bottom=oracle.wetting_h(s["theta"]),
                      step2_relax_momentum=True)
    lat = oracle.OracleLattice(p, s["nx"], s["ny"])
    lat.init_drop(s["R"], s["cx"], s["cy"])
    lat.step(STEPS)
    _, phi, ux, uy = lat.moments()
    return [oracle.contact_angle(phi)[0], float(np.hypot(ux, uy).max()),
            float((~np.isfinite(phi)).sum())]


def _rank_main(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    import oracle

    dist.init_process_group("gloo", rank=rank, world_size=ws)
    oracle.set_threads(1)
    specs = lbinputs.batch_specs(**SPECS)
    parts = shard.partition(_nodes(specs), ws)
    rows = {d: _run_domain(oracle, specs[d]) for d in parts[rank]}
    table = shard.gather_rows(len(specs), 3, rows)
    slowest = bench.max_over_ranks(ws, float(len(parts[rank])))
    out[rank] = (parts[rank], table, slowest)
    dist.destroy_process_group()


def test_split_run_gathers_the_single_process_table_gloo():
    import oracle

    oracle.build()
    specs = lbinputs.batch_specs(**SPECS)
    single = [_run_domain(oracle, s) for s in specs]
    ws, port = 2, _free_port()
    with mp.get_context("spawn").Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank_main, args=(ws, port, out), nprocs=ws, join=True)
        res = dict(out)
    owned = sorted(d for r in range(ws) for d in res[r][0])
    assert owned == list(range(len(specs)))
    assert all(res[r][0] for r in range(ws))  # both ranks got work
    for r in range(ws):
        table = res[r][1]
        assert table == single  # bit for bit: the same oracle runs, gathered
        assert res[r][2] == max(len(res[k][0]) for k in range(ws))


def test_gather_rows_keeps_nonfinite_and_checks_width():
    table = shard.gather_rows(3, 2, {0: [1.0, 2.0], 2: [float("nan"), 3.0]})
    assert table[0] == [1.0, 2.0] and table[1] == [0.0, 0.0]
    assert np.isnan(table[2][0]) and table[2][1] == 3.0
    with pytest.raises(ValueError):
        shard.gather_rows(2, 2, {0: [1.0]})
