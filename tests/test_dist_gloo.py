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


def test_merge_top_order_ties_and_padding():
    """The merged list of largest-error patches is what one rank holding all
    patches would keep: descending error, ties to the smaller global index,
    short lists padded with index -1."""
    from paper_1806_04374_gb300.rksvd import merge_top
    errs = [np.array([3.0, 1.0, 0.5, -1.0], np.float32), np.array([3.0, 2.0, -1.0, -1.0], np.float32)]
    gidx = [np.array([5, 2, 7, -1]), np.array([10, 11, -1, -1])]
    vecs = [np.arange(4, dtype=np.float32)[:, None] * np.ones((4, 3), np.float32),
            10 + np.arange(4, dtype=np.float32)[:, None] * np.ones((4, 3), np.float32)]
    idx, vec = merge_top(errs, gidx, vecs, ntop=6)
    assert idx.tolist() == [5, 10, 11, 2, 7, -1]
    assert vec[:, 0].tolist() == [0.0, 10.0, 11.0, 1.0, 2.0, 0.0]


def _ksvd_worker(rank, world, port, q):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1806_04374_gb300.rksvd import _all_reduce_sum, gather_top
    # this rank's partial covariance and its list (host tensors)
    C = torch.full((2, 3, 3), float(rank + 1), dtype=torch.float64)
    _all_reduce_sum(C, None)
    err = torch.tensor([5.0 - rank, 1.0, -1.0], dtype=torch.float32)
    idx = torch.tensor([0, 1, -1], dtype=torch.int64)
    vec = torch.full((3, 2), float(rank), dtype=torch.float32)
    top_idx, top_vec = gather_top(err, idx, vec, offset=100 * rank, group=None)
    q.put((rank, float(C[1, 2, 0]), top_idx.tolist(), top_vec[:, 0].tolist()))
    dist.destroy_process_group()


def test_two_rank_ksvd_exchange():
    """The R-K-SVD exchange on two gloo ranks: covariances summed, the ranks'
    largest-error lists gathered with global indices and merged identically
    on every rank."""
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_ksvd_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in res:
        assert r[1] == 3.0                           # 1 + 2
        assert r[2] == [0, 100, 1]                   # 5.0 (rank 0), 4.0 (rank 1), then 1.0 tie -> 1
        assert r[3] == [0.0, 1.0, 0.0]
