"""End-to-end rotational K-SVD through the C ABI (paper_1806_04374_gb300.rksvd):
the learned atoms recover planted ones, and the coding-error trajectory
follows the same loop run with the oracle (oracle.romp + oracle.ksvd)."""
import numpy as np
import pytest

import oracle
from oracle import ksvd as oksvd
from paper_1806_04374_gb300 import synth

pytestmark = pytest.mark.gpu


def test_recovers_planted_atoms(cuda_ok):
    import torch
    import bench
    from paper_1806_04374_gb300 import rksvd
    R, K, M = 16, 2, 6
    d_true = synth.make_dictionary(M, 6, 8, 901)
    x, _ = synth.make_patches(d_true, 6000, 2, 0.02, 902)
    d0 = synth.make_dictionary(M, 6, 8, 903)
    d, codes, hist = rksvd.learn(torch.from_numpy(x).cuda(), torch.from_numpy(d0).cuda(), R, K,
                                 iters=15, precision="f16")
    mse = [h["mse"] for h in hist]
    assert mse[-1] < 0.5 * mse[0]
    rec = bench.recovery(d.cpu().numpy(), d_true, R)
    print("mse", mse, "recovery", rec)
    assert rec >= 0.65


def test_trajectory_matches_oracle_loop(cuda_ok):
    import torch
    from paper_1806_04374_gb300 import rksvd
    R, K, M = 16, 2, 6
    d_true = synth.make_dictionary(M, 6, 8, 911)
    x, _ = synth.make_patches(d_true, 1500, 2, 0.05, 912)
    d0 = synth.make_dictionary(M, 6, 8, 913)
    iters = 3
    _, _, hist = rksvd.learn(torch.from_numpy(x).cuda(), torch.from_numpy(d0).cuda(), R, K,
                             iters=iters, precision="fp32")
    n = 6 * 17
    d = d0.astype(np.float64)
    ref = []
    for it in range(iters):
        o = oracle.romp(x, d.astype(np.float32), R, K)
        ref.append(o["rn2"].mean() / n)
        d, _ = oksvd.ksvd_update(x, d.astype(np.float32), R, o["atom"], o["angle"], o["coef"])
    got = [h["mse"] for h in hist[:iters]]
    print("gpu", got, "oracle", ref)
    assert np.allclose(got, ref, rtol=1e-3)


def _learn_rank(rank, world, port, q):
    import os
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    torch.cuda.set_device(0)
    from paper_1806_04374_gb300 import rksvd
    R, K, M, P = 16, 2, 10, 4000
    d_true = synth.make_dictionary(6, 6, 8, 921)
    x, _ = synth.make_patches(d_true, P, 2, 0.05, 922)
    d0 = synth.make_dictionary(M, 6, 8, 923)
    lo, hi = rank * P // world, (rank + 1) * P // world
    d, _, hist = rksvd.learn(torch.from_numpy(x[lo:hi]).cuda(), torch.from_numpy(d0).cuda(), R, K,
                             iters=3, precision="f16", group=dist.group.WORLD, offset=lo)
    q.put((rank, d.cpu().numpy()))
    dist.destroy_process_group()


def test_two_rank_learning_matches_one_gpu(cuda_ok):
    """R-K-SVD with the patches split over two ranks (two processes on this
    GPU, gloo for the exchange; their kernels never wait on one another)
    learns the same dictionary as one process holding all the patches."""
    import socket
    import torch
    import torch.multiprocessing as mp
    from paper_1806_04374_gb300 import rksvd
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_learn_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=300) for _ in procs), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    R, K, M, P = 16, 2, 10, 4000
    d_true = synth.make_dictionary(6, 6, 8, 921)
    x, _ = synth.make_patches(d_true, P, 2, 0.05, 922)
    d0 = synth.make_dictionary(M, 6, 8, 923)
    d, _, _ = rksvd.learn(torch.from_numpy(x).cuda(), torch.from_numpy(d0).cuda(), R, K, iters=3,
                          precision="f16")
    d = d.cpu().numpy()
    assert np.abs(res[0][1] - res[1][1]).max() == 0.0   # every rank holds the same atoms
    assert np.abs(res[0][1] - d).max() < 1e-4, np.abs(res[0][1] - d).max()


def test_checkpoint_resume_is_bit_identical(cuda_ok, tmp_path):
    """Four R-K-SVD iterations in one run, and the same loop stopped after two
    (its checkpoint written) and resumed from the file: the same atoms bit
    for bit and the same history."""
    import torch
    from paper_1806_04374_gb300 import rksvd
    R, K, M = 16, 3, 8
    d_true = synth.make_dictionary(M, 6, 8, 931)
    x, _ = synth.make_patches(d_true, 5000, 3, 0.05, 932)
    xd = torch.from_numpy(x).cuda()
    d0 = torch.from_numpy(synth.make_dictionary(M, 6, 8, 933)).cuda()
    d_full, _, h_full = rksvd.learn(xd, d0, R, K, iters=4, precision="f16")
    ck = str(tmp_path / "rksvd.npz")
    rksvd.learn(xd, d0, R, K, iters=2, precision="f16", checkpoint=ck)
    d_saved, it, _ = rksvd.load_checkpoint(ck, R, K)
    assert it == 2
    d_res, _, h_res = rksvd.learn(xd, d0, R, K, iters=4, precision="f16", checkpoint=ck,
                                  resume=True)
    assert np.array_equal(d_res.cpu().numpy(), d_full.cpu().numpy())
    assert h_res == h_full
    assert rksvd.load_checkpoint(ck, R, K)[1] == 4
