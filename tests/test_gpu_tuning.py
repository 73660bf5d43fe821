"""Tuning of the FP16 path on the GPU: every tuning gives the same codes bit
for bit; overrides and their source are reported; a ring depth the layout was
not built with is refused; the committed table's entries reach the
dictionaries of their sizes."""
import os

import numpy as np
import pytest

from paper_1806_04374_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rsc(cuda_ok):
    import paper_1806_04374_gb300 as rsc
    rsc.load_library()
    return rsc


@pytest.mark.parametrize("sizes", [(6, 8, 64, 64, 5), (10, 12, 32, 16, 4)])
def test_every_tuning_gives_the_same_codes(rsc, sizes):
    import torch
    J, kmax, M, R, K = sizes
    d = synth.make_dictionary(M, J, kmax, 20180910)
    x, _ = synth.make_patches(d, 150_000, 3, 0.1, 20180911)
    dic = rsc.Dictionary(torch.from_numpy(d).cuda(), R)
    xd = torch.from_numpy(x).cuda()
    base = {k: v.cpu().numpy() for k, v in rsc.encode(dic, xd, K, "f16").items()}
    from paper_1806_04374_gb300 import autotune
    opts = autotune.stage_options(dic)
    assert len(opts) == 2, opts
    dflt, other = opts
    for t in ({"groups": 1}, {"groups": 3, "group_min": 20000},
              {"refine_blocks_per_sm": 8, "score_stages": other},
              {"groups": 2, "refine_blocks_per_sm": 64, "score_stages": dflt}):
        rsc.rsc_dict_set_tuning(dic.handle, **t)
        got = rsc.rsc_dict_tuning(dic.handle, K)
        assert got["source"] == 2 and all(got[k] == v for k, v in t.items()), (t, got)
        out = {k: v.cpu().numpy() for k, v in rsc.encode(dic, xd, K, "f16").items()}
        torch.cuda.synchronize()
        assert rsc.rsc_dict_check(dic.handle) == 0
        for k in base:
            assert np.array_equal(out[k], base[k]), (t, k)
    with pytest.raises(rsc.RscError):
        rsc.rsc_dict_set_tuning(dic.handle, score_stages=next(v for v in range(2, 7)
                                                            if v not in opts))
    with pytest.raises(rsc.RscError):
        rsc.rsc_dict_set_tuning(dic.handle, groups=7)
    rsc.rsc_dict_set_tuning(dic.handle, clear=True)
    assert rsc.rsc_dict_tuning(dic.handle, K)["source"] in (0, 1)
    dic.close()


def test_committed_table_reaches_dictionaries(rsc):
    import torch
    from paper_1806_04374_gb300 import autotune
    if os.environ.get("RSC_TUNING_TABLE") or not os.path.exists(autotune.TABLE):
        pytest.skip("no committed table in use")
    lines = [ln.split("#")[0].split() for ln in open(autotune.TABLE)]
    entries = [list(map(int, f)) for f in lines if len(f) == 8]
    assert entries
    for n, M, R, K, g, gm, rb, st in entries:
        J = next(j for j in range(1, 64) if n % j == 0 and (n // j - 1) % 2 == 0
                 and (n // j - 1) // 2 in (8, 12))
        kmax = (n // J - 1) // 2
        d = synth.make_dictionary(M, J, kmax, 20180912)
        dic = rsc.Dictionary(torch.from_numpy(d).cuda(), R)
        t = rsc.rsc_dict_tuning(dic.handle, K)
        assert t["source"] == 1, (n, M, R, K, t)
        assert (t["groups"], t["refine_blocks_per_sm"], t["score_stages"]) == (g, rb, st)
        dic.close()
