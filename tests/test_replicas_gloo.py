"""The N > 1 host path of the benchmark on CPU: two gloo ranks, per-rank
seeds and inputs, max-over-ranks timing and sum-over-ranks work."""
import os
import socket

import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2604_16590_gb300 import replicas
from paper_2604_16590_gb300.inputs import qkv


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        seed = replicas.replica_seed(20262, rank)
        (x,) = qkv((2, 8, 4), seed, 0.5, "bf16", n=1)
        ms = 100.0 + 25.0 * rank  # rank 1 is slower
        t_max = replicas.max_over_ranks(ms)
        units = replicas.sum_over_ranks(4 * 1024)
        xs = [torch.zeros_like(x.float()) for _ in range(world)]
        dist.all_gather(xs, x.float())
        q.put((rank, seed, t_max, units, replicas.weak_scaling_value(4 * 1024, world, t_max * 1e-3),
               bool(torch.equal(xs[0], xs[1]))))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_like_the_benchmark():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    seeds = {r[1] for r in res}
    assert len(seeds) == 2 and replicas.replica_seed(20262, 0) == 20262
    for rank, seed, t_max, units, value, same in res:
        assert t_max == 125.0  # the slowest rank's time
        assert units == 2 * 4 * 1024  # work of both ranks
        assert abs(value - 2 * 4 * 1024 / 0.125) < 1e-6
        assert not same  # replicas draw different inputs


def test_single_process_reductions_are_identity():
    assert replicas.max_over_ranks(3.5) == 3.5
    assert replicas.sum_over_ranks(7.0) == 7.0


def test_bench_gpus_flag_launches_that_many_ranks():
    """`bench.py --gpus 2` started without torchrun launches two ranks itself
    (torch.distributed.run, rendezvous on 127.0.0.1); rank 0 alone prints the
    line and reports the real world size.  --dry-run does no GPU work."""
    import json
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = {k: v for k, v in os.environ.items() if k not in ("WORLD_SIZE", "RANK", "LOCAL_RANK")}
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--gpus", "2", "--dry-run"],
                       capture_output=True, text=True, timeout=300, env=env, cwd=root)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [json.loads(x) for x in r.stdout.splitlines() if x.startswith("{")]
    assert len(lines) == 1
    assert lines[0]["n_gpus"] == 2 and lines[0]["ranks_seen"] == 2
