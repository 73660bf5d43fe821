"""rsc_encode_noalloc: the FP16 coding path for callers that cannot allocate
device memory while they code (its scratch list lives in a fixed device
array inside the library).  Called through the C ABI and compared with
rsc_encode (RSC_F16_RESCORE) and with the FP64 oracle on the same inputs,
on calls in a row, since every call reuses the same array.  Collected last on
purpose."""
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


def _host(out):
    return {k: v.cpu().numpy() for k, v in out.items()}


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
    r = _host(ref)
    for out in outs:
        o = _host(out)
        assert np.array_equal(o["atom"], r["atom"])
        assert np.array_equal(o["angle_idx"], r["angle_idx"])
        scale = np.abs(r["coef"]).max()
        assert np.abs(o["coef"] - r["coef"]).max() <= 1e-12 * scale
        assert np.allclose(o["resid_norm2"], r["resid_norm2"], rtol=1e-6, atol=1e-6)
    # sizes beyond the fixed array are refused before any work
    big = 1 << 20
    assert rsc.rsc_encode_noalloc(dic.handle, xd.data_ptr(), big + 1, K, 0, 0, 0, 0, 0,
                                  stream) == rsc.RSC_ERR_UNSUPPORTED
    # misaligned optional outputs are refused like rsc_encode refuses them
    o = outs[0]
    assert rsc.rsc_encode_noalloc(dic.handle, xd.data_ptr(), P, K, o["atom"].data_ptr(),
                                  o["angle_idx"].data_ptr(), o["angle"].data_ptr() + 2,
                                  o["coef"].data_ptr(), o["resid_norm2"].data_ptr(),
                                  stream) == rsc.RSC_ERR_INVALID
    assert rsc.rsc_encode_noalloc(dic.handle, xd.data_ptr(), P, K, o["atom"].data_ptr(),
                                  o["angle_idx"].data_ptr(), o["angle"].data_ptr(),
                                  o["coef"].data_ptr(), o["resid_norm2"].data_ptr() + 1,
                                  stream) == rsc.RSC_ERR_INVALID
    dic.close()


@pytest.mark.parametrize("K", [3, 8])
def test_noalloc_other_step_counts_against_oracle(cuda_ok, K):
    """The K = 3 and K = 8 instances of the fused kernel, twice in a row,
    against the FP64 oracle on a sample (selection margin 1e-6, weights
    1e-3) and equal between the two calls."""
    import torch
    import paper_1806_04374_gb300 as rsc
    import parity
    rsc.load_library()
    d, x, _, wl = synth.workload_inputs("omp_1m", P=20_000)
    P = x.shape[0]
    dic = rsc.Dictionary(torch.from_numpy(d).cuda(), wl.R)
    xd = torch.from_numpy(x).cuda()
    stream = int(torch.cuda.current_stream().cuda_stream)
    outs = [_outputs(torch, P, K) for _ in range(2)]
    for out in outs:
        assert _call(rsc, dic, xd, P, K, out, stream) == rsc.RSC_OK
        torch.cuda.synchronize()
        assert rsc.rsc_dict_check(dic.handle) == 0
    o0, o1 = _host(outs[0]), _host(outs[1])
    for k in ("atom", "angle_idx", "coef", "resid_norm2"):
        assert np.array_equal(o0[k], o1[k]), k
    idx = np.random.default_rng(K).choice(P, 600, replace=False)
    parity.check(x[idx], d, wl.R, K, {k: v[idx] for k, v in o1.items()}, coef_tol=1e-3)
    dic.close()


def _symmetric_workload(P=4096):
    """M = 16 atoms (J = 6, kmax = 8), of which atoms 0 and 1 carry only the
    harmonics k = 0 and k = 8: their scores repeat every eighth of a turn, so
    at R = 32 each has 8 exactly tied angles.  Half of the patches are one of
    them, steered and weighted, plus noise 1e-5, so 8 units fall inside the
    FP16 path's certification window and the patch is handed to the FP32
    path; the other half are plain 3-atom patches."""
    d = synth.make_dictionary(16, 6, 8, 20180701).astype(np.float64)
    rng = np.random.default_rng(20180702)
    for m in (0, 1):
        s = np.zeros((9, 6, 2))
        s[0, :, 0] = rng.standard_normal(6)
        s[8] = rng.standard_normal((6, 2))
        d[m] = s / np.sqrt(synth.coef_norm2(s))
    d = d.astype(np.float32)
    x, _ = synth.make_patches(d, P, 3, 0.05, 20180703)
    n_sym = P // 2
    dc = d[..., 0].astype(np.float64) + 1j * d[..., 1]
    m = rng.integers(0, 2, n_sym)
    th = rng.uniform(0, 2 * np.pi, n_sym)
    w = rng.choice([-1.0, 1.0], n_sym) * rng.uniform(0.5, 2.0, n_sym)
    z = w[:, None, None] * dc[m] * np.exp(-1j * np.arange(9)[None, :, None] * th[:, None, None])
    noise = rng.standard_normal((n_sym, 9, 6, 2)) * 1e-5
    x[:n_sym, ..., 0] = (z.real + noise[..., 0]).astype(np.float32)
    x[:n_sym, ..., 1] = (z.imag + noise[..., 1]).astype(np.float32)
    x[:n_sym, 0, :, 1] = 0.0
    return d, x


def test_noalloc_handoffs_reuse_the_array(cuda_ok):
    """Two calls in a row that hand patches to the FP32 path through the
    fixed array: both hand some off, both give the same codes, and those
    codes pass the oracle rule (the handed-off patches included)."""
    import torch
    import paper_1806_04374_gb300 as rsc
    import parity
    rsc.load_library()
    d, x = _symmetric_workload()
    P, K, R = x.shape[0], 3, 32
    dic = rsc.Dictionary(torch.from_numpy(d).cuda(), R)
    xd = torch.from_numpy(x).cuda()
    stream = int(torch.cuda.current_stream().cuda_stream)
    rsc.rsc_dict_fallback_count(dic.handle)  # reset
    outs, counts = [_outputs(torch, P, K) for _ in range(2)], []
    for out in outs:
        assert _call(rsc, dic, xd, P, K, out, stream) == rsc.RSC_OK
        torch.cuda.synchronize()
        assert rsc.rsc_dict_check(dic.handle) == 0
        counts.append(rsc.rsc_dict_fallback_count(dic.handle))
    assert counts[0] > 0 and counts[0] == counts[1], counts
    o0, o1 = _host(outs[0]), _host(outs[1])
    for k in ("atom", "angle_idx", "coef", "resid_norm2"):
        assert np.array_equal(o0[k], o1[k]), k
    idx = np.concatenate([np.arange(0, 512), np.arange(P // 2, P // 2 + 256)])
    parity.check(x[idx], d, R, K, {k: v[idx] for k, v in o1.items()}, coef_tol=1e-3)
    dic.close()
