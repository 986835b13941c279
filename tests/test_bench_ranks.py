"""Multi-rank logic of bench.py on CPU (gloo, world size 2): the timing
reduction takes the slowest rank, the whole-job value counts every rank's
replica, and under torchrun the reference arm prints exactly one line."""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, elapsed, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", rank=rank, world_size=ws)
    m = bench.max_over_ranks(ws, elapsed[rank])
    bench.barrier(ws)
    out[rank] = (m, bench.job_value(1000, 10, ws, m))
    dist.destroy_process_group()


def test_max_over_ranks_and_job_value_gloo():
    ws, port = 2, _free_port()
    elapsed = [0.5, 2.0]
    with mp.get_context("spawn").Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank_main, args=(ws, port, elapsed, out), nprocs=ws, join=True)
        res = dict(out)
    for rank in range(ws):
        m, v = res[rank]
        assert m == 2.0
        assert v == pytest.approx(1000 * 10 * 2 / 2.0 / 1e6)


def test_reference_arm_under_torchrun_prints_one_line():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl",
           "reference", "--gpus", "2", "--steps", "2", "--warmup", "3"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle"
    assert d["e2e"]["h2d_bytes_per_step"] == 0
