"""CPU: the benchmark's multi-rank logic with two gloo ranks (the path
shards by frame: replicas only).  Each rank draws its own scenes, the
timing reduction takes the slowest rank, and the reference arm runs on
rank 0 alone."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(ws), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        t = bench.max_over_ranks(1.0 + rank * 0.5, ws, torch.device("cpu"))
        radar, grid, scenes = bench.make_scenes(rank)
        first = float(np.asarray(scenes[0].V, np.float64).sum())
        out.put((rank, t, first, len(scenes), bench.dist_env()))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    (r0, t0, f0, n0, e0), (r1, t1, f1, n1, e1) = res
    assert (r0, r1) == (0, 1)
    assert t0 == t1 == 1.5                 # both ranks see the slowest rank's time
    assert n0 == n1 and f0 != f1           # same frame count, different scenes per rank
    assert e0 == (2, 0, 0) and e1 == (2, 1, 1)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    import bench
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    args = type("A", (), {"steps": 1, "warmup": 0, "gpus": 2})()
    assert bench.run_reference(args) is None
    assert capsys.readouterr().out == ""
