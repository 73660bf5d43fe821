"""The tuning table (CPU, no GPU): librsc's parser finds the entry of an
(n, M, R, K), skips comments and malformed or out-of-range lines, and reads
back what the autotuner writes."""
import ctypes

import pytest

from paper_1806_04374_gb300 import autotune


@pytest.fixture(scope="module")
def rsc():
    from paper_1806_04374_gb300 import build
    build.build()
    import paper_1806_04374_gb300 as rsc
    rsc.load_library()
    return rsc


def test_parser(rsc, tmp_path):
    p = tmp_path / "t.txt"
    p.write_text("# comment\n102 64 64 5 3 0 16 4  # trailing comment\n"
                 "250 256 128 8 1 0 8 5\nnot a line\n102 64 64 3 9 0 8 4\n")
    t = rsc.rsc_tuning_table_lookup(str(p), 102, 64, 64, 5)
    assert t == {"groups": 3, "group_min": 0, "refine_blocks_per_sm": 16, "score_stages": 4,
                 "source": 1}
    assert rsc.rsc_tuning_table_lookup(str(p), 250, 256, 128, 8)["score_stages"] == 5
    # groups 9 is out of range: the line is ignored
    assert rsc.rsc_tuning_table_lookup(str(p), 102, 64, 64, 3)["source"] == 0
    assert rsc.rsc_tuning_table_lookup(str(p), 102, 64, 64, 4)["source"] == 0
    with pytest.raises(rsc.RscError):
        rsc.rsc_tuning_table_lookup(str(tmp_path / "missing.txt"), 1, 1, 1, 1)
    lib = rsc.load_library()
    assert lib.rsc_dict_set_tuning(ctypes.c_void_p(None), None) == rsc.RSC_ERR_INVALID
    assert lib.rsc_dict_tuning(ctypes.c_void_p(None), 5, None) == rsc.RSC_ERR_INVALID


def test_autotuner_table_reads_back(rsc, tmp_path):
    entries = [{"workload": "w", "n": 102, "M": 64, "R": 64, "K": 5, "patches": 10,
                "default_ms": 2.0, "best": {"groups": 3, "refine_blocks_per_sm": 8,
                                            "score_stages": 4, "ms": 1.5}}]
    path = str(tmp_path / "rsc_tuning.txt")
    autotune.write_table(path, entries, "test")
    t = rsc.rsc_tuning_table_lookup(path, 102, 64, 64, 5)
    assert (t["groups"], t["refine_blocks_per_sm"], t["score_stages"], t["source"]) == (3, 8, 4, 1)
