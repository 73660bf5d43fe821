"""The library's scratch pool (include/rsc.h, "Scratch"): a call's device
scratch comes from a pool that keeps its memory between calls, so a second
call of the same size takes no new device memory, and rsc_dict_destroy gives
the unused memory back."""
import numpy as np
import pytest

from paper_1806_04374_gb300 import synth

pytestmark = pytest.mark.gpu


def test_scratch_is_kept_between_calls_and_trimmed_on_destroy(cuda_ok):
    import torch
    import paper_1806_04374_gb300 as rsc
    rsc.load_library()
    d, x, _, wl = synth.workload_inputs("omp_1m", P=400_000)
    P, K = x.shape[0], wl.K
    dic = rsc.Dictionary(torch.from_numpy(d).cuda(), wl.R)
    xd = torch.from_numpy(x).cuda()
    out = {"atom": torch.empty((P, K), dtype=torch.int32, device="cuda"),
           "angle_idx": torch.empty((P, K), dtype=torch.int32, device="cuda"),
           "angle": torch.empty((P, K), dtype=torch.float32, device="cuda"),
           "coef": torch.empty((P, K), dtype=torch.float64, device="cuda"),
           "resid_norm2": torch.empty((P,), dtype=torch.float32, device="cuda")}
    need = rsc.rsc_workspace_bytes(dic.handle, 0, P, 0, K, rsc.RSC_F16_RESCORE)
    assert need > 100 << 20  # residual rows, candidates, state: hundreds of MB
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    first = rsc.encode(dic, xd, K, "f16", out=out)
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    codes = {k: v.cpu().numpy().copy() for k, v in first.items()}
    # the pool kept the first call's scratch (the device's default pool
    # would have given it back at the synchronisation)
    assert free0 - free1 >= need // 2, (free0, free1, need)
    for _ in range(3):
        again = rsc.encode(dic, xd, K, "f16", out=out)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free1  # reused, nothing new
        for k, v in again.items():
            assert np.array_equal(v.cpu().numpy(), codes[k]), k
    assert rsc.rsc_dict_check(dic.handle) == 0
    dic.close()  # rsc_dict_destroy trims the pool
    torch.cuda.synchronize()
    free2 = torch.cuda.mem_get_info()[0]
    assert free2 - free1 >= need // 2, (free1, free2, need)
