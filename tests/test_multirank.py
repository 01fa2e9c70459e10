"""Multi-rank host logic of the benchmark on CPU (gloo, world size 2): each
rank gets its own seeded edges over the same robot and scene, and the only
collective reduces times (max) and work (sum).  No GPU involved."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import vpgen
    w = bench.rank_workload(vpgen.DUAL14_SHELVES, 300, rank)
    times = [10.0 + rank, 20.0 - rank]
    sums = [float(w.counts.sum()), 300.0]
    mx, sm = bench.reduce_over_ranks(times, sums, torch.device("cpu"))
    out[rank] = (mx, sm, float(w.counts.sum()), w.q0[:2].copy(), w.robot.n_spheres, w.env.n_prims)
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_shard_and_reduce():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=240)
        assert p.exitcode == 0
    (mx0, sm0, c0, q0a, s0, p0), (mx1, sm1, c1, q0b, s1, p1) = out[0], out[1]
    assert mx0 == mx1 == [11.0, 20.0]
    assert sm0 == sm1 == [c0 + c1, 600.0]
    assert not np.array_equal(q0a, q0b)          # different edges per rank
    assert (s0, p0) == (s1, p1)                  # same robot and scene


def test_single_process_reduce_is_identity():
    import torch
    import bench
    assert bench.reduce_over_ranks([1.5, 2.0], [3.0], torch.device("cpu")) == ([1.5, 2.0], [3.0])


def test_reference_arm_under_two_ranks_prints_one_line():
    """`bench.py --impl reference` launched as two ranks: rank 0 times the
    oracle and prints the one JSON line, with the contract's keys; rank 1
    exits 0 without work or output."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    outs = []
    for rank in (1, 0):
        env = dict(os.environ, RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE="2",
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(_free_port()))
        r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--gpus", "2", "--steps", "2",
                            "--warmup", "1", "--edges", "4096"], cwd=root, env=env, capture_output=True, text=True,
                           timeout=600)
        assert r.returncode == 0, r.stderr[-2000:]
        outs.append(r.stdout.strip())
    assert outs[0] == ""
    line = json.loads(outs[1])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["steps"] == 2
    assert line["value"] > 0 and line["unit"] == "states/s" and line["higher_is_better"] is True
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": "states/s", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
