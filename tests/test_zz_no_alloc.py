"""rsc_encode_noalloc: the FP16 coding path for callers that cannot allocate
device memory while they code (its scratch list lives in a fixed device
array inside the library).  Called through the C ABI and compared with
rsc_encode (RSC_F16_RESCORE) on the same inputs, twice in a row, since every
call reuses the same array.  Collected last on purpose."""
import numpy as np
import pytest

from paper_1806_04374_gb300 import synth

pytestmark = pytest.mark.gpu


def _outputs(torch, P, K):
    return {
        "atom": torch.empty((P, K), dtype=torch.int32, device="cuda"),
        "angle_idx": torch.empty((P, K), dtype=torch.int32, device="cuda"),
        "angle": torch.empty((P, K), dtype=torch.float32, device="cuda"),
        "coef": torch.empty((P, K), dtype=torch.float64, device="cuda"),
        "resid_norm2": torch.empty((P,), dtype=torch.float32, device="cuda"),
    }


def _call(rsc, dic, xd, P, K, out, stream):
    return rsc.rsc_encode_noalloc(dic.handle, xd.data_ptr(), P, K, out["atom"].data_ptr(),
                                  out["angle_idx"].data_ptr(), out["angle"].data_ptr(),
                                  out["coef"].data_ptr(), out["resid_norm2"].data_ptr(), stream)


def test_noalloc_matches_encode_twice(cuda_ok):
    import torch
    import paper_1806_04374_gb300 as rsc
    rsc.load_library()
    d, x, _, wl = synth.workload_inputs("omp_1m", P=300_000)
    P, K = x.shape[0], wl.K
    dic = rsc.Dictionary(torch.from_numpy(d).cuda(), wl.R)
    xd = torch.from_numpy(x).cuda()
    ref = rsc.encode(dic, xd, K, "f16")
    torch.cuda.synchronize()
    stream = int(torch.cuda.current_stream().cuda_stream)
    outs = [_outputs(torch, P, K) for _ in range(3)]
    # the first call on the device is the set-up: it looks up the array's
    # device address, and the CUDA runtime may load the array (4 MiB) then
    assert _call(rsc, dic, xd, P, K, outs[0], stream) == rsc.RSC_OK
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for out in outs[1:]:
        assert _call(rsc, dic, xd, P, K, out, stream) == rsc.RSC_OK
        torch.cuda.synchronize()
        assert rsc.rsc_dict_check(dic.handle) == 0
    free1 = torch.cuda.mem_get_info()[0]
    assert free1 == free0, (free0, free1)  # no device memory taken by the calls
    r = {k: v.cpu().numpy() for k, v in ref.items()}
    for out in outs:
        o = {k: v.cpu().numpy() for k, v in out.items()}
        assert np.array_equal(o["atom"], r["atom"])
        assert np.array_equal(o["angle_idx"], r["angle_idx"])
        scale = np.abs(r["coef"]).max()
        assert np.abs(o["coef"] - r["coef"]).max() <= 1e-12 * scale
        assert np.allclose(o["resid_norm2"], r["resid_norm2"], rtol=1e-6, atol=1e-6)
    # sizes beyond the fixed array are refused before any work
    big = 1 << 20
    assert rsc.rsc_encode_noalloc(dic.handle, xd.data_ptr(), big + 1, K, 0, 0, 0, 0, 0,
                                  stream) == rsc.RSC_ERR_UNSUPPORTED
    dic.close()
