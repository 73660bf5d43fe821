"""Host logic of bench.py (CPU only): the kernel count the line reports, and
the oracle-parity counts that the benchmark line carries for its timed
outputs (zero for the oracle's own results; a planted wrong pick, a wrong
weight and a wrong residual norm are counted)."""
import numpy as np

import bench
import oracle
from paper_1806_04374_gb300 import synth


def _case():
    d, x, _, wl = synth.workload_inputs("omp_small", P=64)
    free = oracle.romp(x, d, wl.R, wl.K)
    gpu = {"atom": free["atom"].copy(), "angle_idx": free["angle"].copy(),
           "coef": free["coef"].copy(), "resid_norm2": free["rn2"].astype(np.float32)}
    return d, x, wl, free, gpu


def test_oracle_parity_of_the_oracle_itself_is_clean():
    d, x, wl, free, gpu = _case()
    r = bench.oracle_parity(x, d, wl, gpu, free, 1e-5)
    assert r["mismatches"] == 0 and r["pinned_steps"] > 0
    assert r["max_rel_coef_err"] < 1e-12


def test_oracle_parity_counts_planted_errors():
    d, x, wl, free, gpu = _case()
    p = int(np.argmax(free["margin"][:, 0]))  # a patch whose first step is pinned
    gpu["angle_idx"][p, 0] = (gpu["angle_idx"][p, 0] + 1) % wl.R
    q = (p + 1) % x.shape[0]
    gpu["coef"][q] *= 1.01
    r = bench.oracle_parity(x, d, wl, gpu, free, 1e-5)
    assert r["selection_mismatches"] >= 1
    assert r["coef_violations"] >= 1
    assert r["mismatches"] >= 2
    gpu2 = dict(_case()[4])
    gpu2["resid_norm2"] = gpu2["resid_norm2"] * 1.5 + 1.0
    r2 = bench.oracle_parity(x, d, wl, gpu2, free, 1e-5)
    assert r2["rn2_violations"] == x.shape[0]


def test_kernel_launch_count_from_event_slots():
    # one call of 3 stream groups at K = 5: per group 5 scoring slots, one
    # hand-off slot, and 6 refine-phase slots (the init kernel, then 5 slots
    # of two refine passes): 5 + 1 + 1 + 10 = 17 kernels a group
    assert bench.kernel_launch_count([15, 3, 18], 5, "f16") == 51
    # the FP32 path: one kernel a call, timed in the scoring phase
    assert bench.kernel_launch_count([4, 0, 0], 5, "fp32") == 4
