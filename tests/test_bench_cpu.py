"""Host logic of bench.py (CPU only): the oracle-parity counts that the
benchmark line carries for its timed outputs are zero for the oracle's own
results and count a planted wrong pick, a wrong weight and a wrong residual
norm."""
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
