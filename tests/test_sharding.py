"""Multi-process path on CPU (gloo, world size 2): contiguous shards of the
candidates, one all-gather of (best, index, second) per rank, merged with the
lowest-index tie rule; the result equals the single-process argmax."""
import os
import socket

import numpy as np
import pytest

from paper_2110_15425_gb300.sharding import combine_top2, shard_range


def test_shard_range_covers_exactly():
    for n in [0, 1, 7, 27000, 1 << 20]:
        for world in [1, 2, 3, 8]:
            spans = [shard_range(n, r, world) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(spans, spans[1:]))
            sizes = [h - l for l, h in spans]
            assert max(sizes) - min(sizes) <= 1


def test_combine_top2_ties_and_gap():
    assert combine_top2([(3.0, 5, 1.0), (3.0, 2, 2.5)]) == (3.0, 2, 0.0)
    assert combine_top2([(1.0, 0, 0.5), (4.0, 9, 3.0), (2.0, 4, -1.0)]) == (4.0, 9, 1.0)
    assert combine_top2([(1.0, 0, float("-inf"))]) == (1.0, 0, 0.0)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    import oracle
    from paper_2110_15425_gb300 import workloads as W
    from paper_2110_15425_gb300.sharding import gather_top2, shard_range
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = W.predator_prey(n_trials=8, levels=5)
    lo, hi = shard_range(125, rank, world)
    ids = np.arange(lo, hi, dtype=np.uint32)
    m = oracle.pp_means(w["pos"], w["levels"], w["seed"], cand_ids=ids)
    b, bv, g = oracle.argmax(m)
    local = (bv, lo + b, bv - g if hi - lo > 1 else float("-inf"))
    q.put((rank, gather_top2(local)))
    dist.barrier()
    dist.destroy_process_group()


def test_gloo_two_ranks_grid_argmax():
    import multiprocessing as mp
    pytest.importorskip("torch.distributed")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    import oracle
    from paper_2110_15425_gb300 import workloads as W
    w = W.predator_prey(n_trials=8, levels=5)
    m = oracle.pp_means(w["pos"], w["levels"], w["seed"])
    b, bv, g = oracle.argmax(m)
    for _, (v, i, gap) in res:
        assert i == b and v == bv and abs(gap - g) < 1e-12
