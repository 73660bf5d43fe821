"""Multi-rank host logic of the benchmark on CPU (gloo, world size 2): each
rank codes its own shard of patches (weak scaling, no collective on the data
path), shards are disjoint and reproducible, and the reported time is the max
over ranks."""
import os
import socket

import numpy as np
import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    d, x, wl = bench.rank_inputs(rank, 3000)
    # fingerprint of this rank's shard
    fp = torch.tensor([float(x[:, 0, 0, 0].sum()), float(x[-1].sum())], dtype=torch.float64)
    fps = [torch.zeros(2, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(fps, fp)
    t = torch.tensor([10.0 * (rank + 1)])
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    # the shard of rank r equals the generator's chunks [r*n, (r+1)*n)
    from paper_1806_04374_gb300 import synth
    n = (3000 + synth.CHUNK - 1) // synth.CHUNK
    ref, _ = synth.make_patches(d, (rank + 1) * n * synth.CHUNK, wl.n_terms, wl.sigma,
                                wl.seed + 1, chunk_ids=[rank * n])
    q.put((rank, [f.tolist() for f in fps], float(t.item()), bool(np.array_equal(ref[:3000], x))))
    dist.destroy_process_group()


def test_two_rank_shards_and_max_time():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=180) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    fps = res[0][1]
    assert res[1][1] == fps                 # every rank saw the same gathered fingerprints
    assert fps[0] != fps[1]                 # disjoint shards
    assert all(r[2] == 20.0 for r in res)   # max over ranks
    assert all(r[3] for r in res)           # shard = the generator's chunks for that rank
