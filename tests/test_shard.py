"""Host logic of the multi-GPU batched path: matrices are sharded over ranks by
longest-processing-time on n^3 cost, with no collective on the data path.
Checked with two gloo ranks on CPU: both compute the same partition, the
shares are disjoint and cover the batch, and the loads are balanced to within
the largest single cost."""
import os
import socket

import numpy as np
import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, sizes, out):
    import torch.distributed as dist
    import paper_1912_04062_gb300 as sk
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    parts = sk.shard_lpt(sizes, world)
    gathered = [None] * world
    dist.all_gather_object(gathered, (rank, parts[rank], parts))
    dist.destroy_process_group()
    out.put(gathered)


def test_lpt_partition_two_gloo_ranks():
    import torch.multiprocessing as mp
    import inputs
    sizes = [int(x) for x in inputs.batch_sizes(300, seed=5)]
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, sizes, q)) for r in range(world)]
    for p in procs:
        p.start()
    results = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    gathered = results[0]
    # every rank derived the same full partition
    assert all(g[2] == gathered[0][2] for g in gathered)
    shares = [g[1] for g in sorted(gathered)]
    flat = sorted(i for sh in shares for i in sh)
    assert flat == list(range(len(sizes)))
    loads = [sum(sizes[i] ** 3 for i in sh) for sh in shares]
    assert max(loads) - min(loads) <= max(s ** 3 for s in sizes)


def test_lpt_partition_edge_cases():
    import paper_1912_04062_gb300 as sk
    assert sk.shard_lpt([], 3) == [[], [], []]
    assert sk.shard_lpt([10], 4) == [[0], [], [], []]
    parts = sk.shard_lpt([100, 100, 100, 100], 2)
    assert sorted(len(p) for p in parts) == [2, 2]
    with pytest.raises(ValueError):
        sk.shard_lpt([1], 0)
    # the largest matrix goes first to rank 0
    assert 1 in sk.shard_lpt(np.array([5, 50, 7]), 2)[0]


def test_tuning_table_lookup(tmp_path):
    # the batched solve's tuned launch configurations: exact size class, the
    # nearest recorded class on the same GPU, the default elsewhere, and a
    # round trip through the JSON file
    from paper_1912_04062_gb300 import tuning
    assert tuning.bucket([32, 1024, 500]) == "nmax<=1024,count<=16"
    assert tuning.bucket(list(range(2, 2002))) == "nmax<=inf,count<=8192"
    assert tuning.bucket([40] * 200) == "nmax<=64,count<=1024"
    path = str(tmp_path / "t.json")
    t = tuning.record("GPU A", [32] * 2000 + [1024], (3, 96), [(1, 0, 9.0), (3, 96, 4.5)], path=path)
    assert t["GPU A"]["nmax<=1024,count<=8192"]["ctas_per_sm"] == 3
    tuning.record("GPU A", [50] * 10, (4, 64), [(4, 64, 1.0)], path=path)
    table = tuning.load(path)
    assert tuning.lookup("GPU A", [32] * 2000 + [1024], table) == (3, 96)
    assert tuning.lookup("GPU A", [60] * 12, table) == (4, 64)
    # nearest class: order class 1024 first, then the count class
    assert tuning.lookup("GPU A", [900] * 100, table) == (3, 96)
    assert tuning.lookup("GPU B", [900] * 100, table) == tuning.DEFAULT
    assert tuning.lookup("GPU A", [], {}) == tuning.DEFAULT
