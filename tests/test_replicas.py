"""Scene sharding and the host-side reductions of the replica path, on 2 gloo ranks (CPU)."""
import os
import socket

import pytest

from paper_1301_1714_gb300 import replicas


def test_shard_is_a_partition_balanced_by_footprint():
    fp = [5.0, 1.0, 1.0, 3.0, 2.0, 2.0, 8.0, 1.0]
    for world in (1, 2, 3, 4):
        sh = replicas.shard_by_footprint(fp, world)
        flat = sorted(k for s in sh for k in s)
        assert flat == list(range(len(fp)))
        loads = [sum(fp[k] for k in s) for s in sh]
        assert max(loads) - min(loads) <= max(fp)
    assert replicas.shard_by_footprint(fp, 2) == replicas.shard_by_footprint(list(fp), 2)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, fp, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = replicas.my_scenes(fp, rank, world)
        n_mine = sum(fp[k] for k in mine)
        tmax = replicas.reduce_max(10.0 + rank)
        total = replicas.reduce_sum(n_mine)
        gathered = [None] * world
        dist.all_gather_object(gathered, mine)
        q.put((rank, mine, tmax, total, gathered))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_shards_and_reductions():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    fp = [1024.0, 65536.0, 4096.0, 2048.0, 30000.0, 777.0, 12345.0]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, fp, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    for rank, mine, tmax, total, gathered in res:
        assert tmax == 11.0
        assert total == sum(fp)
        assert gathered[rank] == mine
        assert sorted(k for s in gathered for k in s) == list(range(len(fp)))
    assert res[0][4] == res[1][4]


def test_launcher_starts_ranks_with_their_bookkeeping(tmp_path):
    """bench.py --gpus N without torchrun launches N ranks through replicas.launch_ranks:
    every rank sees world N, its own rank, and the reductions the benchmark uses."""
    probe = os.path.join(os.path.dirname(os.path.abspath(__file__)), "rank_probe.py")
    rc = replicas.launch_ranks(2, [probe, str(tmp_path)], timeout=300)
    assert rc == 0
    import json
    got = sorted((json.load(open(tmp_path / f"rank{k}.json")) for k in range(2)), key=lambda d: d["rank"])
    assert [d["rank"] for d in got] == [0, 1]
    assert all(d["world"] == 2 and d["group_size"] == 2 for d in got)
    assert [d["local_rank"] for d in got] == [0, 1]
    assert all(d["n_total"] == 3000.0 and d["t_max"] == 1.5 for d in got)
