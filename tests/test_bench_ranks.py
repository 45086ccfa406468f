"""Host logic of bench.py's multi-process path on CPU (gloo, world size 2):
the whole-job time is the slowest rank's, and the reference arm runs on rank 0
only.  (The GPU replicas themselves need one GPU per rank.)"""
import os
import socket
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    v = bench.max_over_ranks(10.0 * (rank + 1), world, "cpu")
    dist.barrier()
    dist.destroy_process_group()
    out.put((rank, v))


def test_max_over_ranks_gloo_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert got == {0: 20.0, 1: 20.0}


def test_single_rank_and_reference_arm_rank(capsys):
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5

    class Args:
        workload = "poisson2d_64_B16"
        steps = 1
        warmup = 0
        gpus = 2
    bench.run_reference(Args(), rank=1)           # a non-zero rank does no work
    assert capsys.readouterr().out == ""


def test_reference_arm_json_line(capsys):
    """bench.py --impl reference on rank 0: one JSON line timing the oracle on
    the host, with the keys of the bench contract (the line's own value in
    cpu_baseline and e2e, no host<->device bytes)."""
    import json
    sys.path.insert(0, ROOT)
    import bench

    class Args:
        workload = "poisson2d_64_B16"
        steps = 1
        warmup = 0
        gpus = 1
    bench.run_reference(Args(), rank=0)
    lines = [ln for ln in capsys.readouterr().out.splitlines() if ln.strip()]
    assert len(lines) == 1
    out = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config"):
        assert key in out, key
    assert out["impl"] == "reference" and out["higher_is_better"] is False
    assert out["value"] > 0 and out["config"]["workload"] == "poisson2d_64_B16"
    cb = out["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == out["value"]
    assert out["e2e"] == {"value": out["value"], "unit": out["unit"], "h2d_bytes_per_step": 0,
                          "d2h_bytes_per_step": 0}
