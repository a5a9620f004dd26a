"""Replica parallelism host logic on CPU with two gloo ranks: distinct
per-rank seeds, the max-over-ranks timing and the whole-job rate, and the
reference arm's rank handling (rank 1 returns without work)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist

    from paper_2212_07848_gb300 import replicas as R
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, lr = R.rank_info()
    seconds = 1.0 + rank                       # rank 1 is the slower one
    smax = R.max_over_ranks(seconds, dist)
    rate = R.whole_job_rate(1000.0, w, smax)
    seed = R.replica_seed(100, r)
    dist.barrier()
    dist.destroy_process_group()
    out.put((r, w, lr, smax, rate, seed))


def test_two_gloo_ranks():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[0] for r in res] == [0, 1] and all(r[1] == 2 and r[2] == r[0] for r in res)
    assert all(r[3] == 2.0 for r in res)               # both see the slowest rank's time
    assert all(r[4] == pytest.approx(1000.0) for r in res)   # 2 x 1000 units / 2 s
    assert res[0][5] != res[1][5]                      # independent replicas


def test_single_process_defaults():
    from paper_2212_07848_gb300 import replicas as R
    assert R.max_over_ranks(3.5) == 3.5
    assert R.whole_job_rate(10.0, 4, 2.0) == 20.0
    with pytest.raises(ValueError):
        R.whole_job_rate(1.0, 1, 0.0)


def test_reference_arm_rank1_does_no_work(capsys):
    import argparse

    import bench
    args = argparse.Namespace(steps=1, warmup=0, gpus=2)
    bench.run_reference(args, rank=1, world=2)
    assert capsys.readouterr().out == ""


def test_reference_arm_prints_the_contract_line(capsys):
    """`bench.py --impl reference` at N = 1: one JSON line with the keys of the
    benchmark contract, the oracle as the timed program."""
    import argparse
    import json

    import bench
    args = argparse.Namespace(steps=1, warmup=0, gpus=1)
    bench.run_reference(args, rank=0, world=1)
    lines = [l for l in capsys.readouterr().out.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["n_gpus"] == 1 and d["value"] > 0
    assert d["metric"] == bench.METRIC and d["config"]["workload"] == bench.WORKLOAD
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
