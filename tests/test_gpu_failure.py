"""Failure detection on the GPU without faulting it.

* A bounded device wait that runs out: the FP16 scoring kernel's pipeline
  waits are given a 1 ns limit (rsc_dict_set_limits), so they give up on a
  small case; the kernel records RSC_ERR_TIMEOUT, drains what it issued and
  returns.  rsc_dict_check reports the timeout, the stream stays usable, and
  the next call with the default limit is oracle-correct.
* An allocation failure injected on the host: a scratch budget below what the
  FP16 path needs makes rsc_encode return RSC_ERR_OOM before any device work;
  no device error is recorded and the next call succeeds."""
import numpy as np
import pytest

from paper_1806_04374_gb300 import synth

from parity import check

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def case(cuda_ok):
    import torch
    import paper_1806_04374_gb300 as rsc
    rsc.load_library()
    d, x, _, wl = synth.workload_inputs("omp_1m", P=8192)
    dic = rsc.Dictionary(torch.from_numpy(d).cuda(), wl.R)
    yield rsc, dic, d, x, wl
    dic.close()


def test_pipeline_wait_timeout_is_reported_and_recovers(case):
    import torch
    rsc, dic, d, x, wl = case
    xd = torch.from_numpy(x).cuda()
    stream = torch.cuda.Stream()
    sh = int(stream.cuda_stream)
    assert rsc.rsc_dict_check(dic.handle, sh) == 0
    assert rsc.rsc_dict_set_limits(dic.handle, 1, 0) == 0
    with torch.cuda.stream(stream):
        rsc.encode(dic, xd, wl.K, "f16", stream=stream)
    assert rsc.rsc_dict_check(dic.handle, sh) == rsc.RSC_ERR_TIMEOUT
    assert rsc.rsc_dict_check(dic.handle, sh) == 0  # the check clears it
    # the stream and the context are usable
    with torch.cuda.stream(stream):
        y = (xd * 2.0).sum()
    stream.synchronize()
    assert torch.isfinite(y).item()
    # default limit again: correct codes
    assert rsc.rsc_dict_set_limits(dic.handle, 0, 0) == 0
    with torch.cuda.stream(stream):
        out = rsc.encode(dic, xd, wl.K, "f16", stream=stream)
    stream.synchronize()
    assert rsc.rsc_dict_check(dic.handle, sh) == 0
    g = {k: v.cpu().numpy()[:512] for k, v in out.items()}
    check(x[:512], d, wl.R, wl.K, g, coef_tol=1e-3)


def test_scratch_budget_reports_oom(case):
    import torch
    rsc, dic, d, x, wl = case
    xd = torch.from_numpy(x).cuda()
    need = rsc.rsc_workspace_bytes(dic.handle, None, x.shape[0], 0, wl.K, rsc.RSC_F16_RESCORE)
    assert need > 0
    assert rsc.rsc_dict_set_limits(dic.handle, 0, need - 1) == 0
    with pytest.raises(rsc.RscError) as ei:
        rsc.encode(dic, xd, wl.K, "f16")
    assert ei.value.status == rsc.RSC_ERR_OOM
    torch.cuda.synchronize()
    assert rsc.rsc_dict_check(dic.handle) == 0
    # the FP32 path takes no scratch and is not limited
    out32 = rsc.encode(dic, xd[:256], wl.K, "fp32")
    # a budget of exactly the need is enough; then no limit
    assert rsc.rsc_dict_set_limits(dic.handle, 0, need) == 0
    out = rsc.encode(dic, xd, wl.K, "f16")
    assert rsc.rsc_dict_set_limits(dic.handle, 0, 0) == 0
    torch.cuda.synchronize()
    assert rsc.rsc_dict_check(dic.handle) == 0
    g = {k: v.cpu().numpy()[:256] for k, v in out.items()}
    g32 = {k: v.cpu().numpy() for k, v in out32.items()}
    check(x[:256], d, wl.R, wl.K, g, coef_tol=1e-3)
    check(x[:256], d, wl.R, wl.K, g32, coef_tol=1e-5)
