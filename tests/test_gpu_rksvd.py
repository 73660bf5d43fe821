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
