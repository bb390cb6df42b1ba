"""The multi-process path on CPU: two gloo ranks (world_size 2, 127.0.0.1)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as d
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    d.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2501_14534_gb300 import dist
    res = {}
    res["shard"] = dist.shard_views(7, rank, world)
    res["max"] = dist.reduce_max(10.0 + rank)
    n = 5
    grads = {"means": torch.full((n, 3), float(rank + 1)), "opacity_logits": torch.arange(n, dtype=torch.float32) * (rank + 1)}
    stats = {"grad_norm_accum": torch.full((n,), 0.5 * (rank + 1)),
             "vis_count": torch.full((n,), rank + 1, dtype=torch.int32),
             "max_radius": torch.tensor([3, 9, 1, 7, 2], dtype=torch.int32) * (1 + rank * (torch.arange(n) % 2)),
             "hit_count": torch.arange(n, dtype=torch.int32) * (10 + rank)}
    dist.allreduce_grads(grads, stats)
    res["means"] = grads["means"].tolist()
    res["op"] = grads["opacity_logits"].tolist()
    res["acc"] = stats["grad_norm_accum"].tolist()
    res["cnt"] = stats["vis_count"].tolist()
    res["maxr"] = stats["max_radius"].tolist()
    res["hits"] = stats["hit_count"].tolist()
    g2 = {"x": torch.ones(3)}
    dist.allreduce_grads(g2, None, views_per_rank=(3 if rank == 0 else 1, 4))
    res["scaled"] = g2["x"].tolist()
    out[rank] = res
    d.barrier()
    d.destroy_process_group()


def test_two_gloo_ranks_reduce_grads_stats_and_times():
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    a, b = out[0], out[1]
    assert sorted(a["shard"] + b["shard"]) == list(range(7)) and len(a["shard"]) == 4
    assert a["max"] == b["max"] == 11.0
    for r in (a, b):
        assert all(v == 3.0 for row in r["means"] for v in row)          # 1 + 2
        assert r["op"] == [0.0, 3.0, 6.0, 9.0, 12.0]
        assert r["acc"] == [1.5] * 5
        assert r["cnt"] == [3] * 5
        assert r["maxr"] == [3, 18, 1, 14, 2]
        assert r["hits"] == [0, 21, 42, 63, 84]                           # k (10 + 11)
        assert r["scaled"] == [1.0] * 3                                   # 3/4 + 1/4
