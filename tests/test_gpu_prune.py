"""RSC_FP32_PRUNE: the FP32 path with the exact |G| bound pruning of the angle
transform (an atom whose bound |G_0| + 2 sum_k |G_k| >= max_r |score(m, r)|
cannot reach the window of the running best is not transformed).  The
pruning is exact, so every code must equal the plain FP32 path's bit for bit,
on every edge shape of the parity suite, on the 10^6-patch workload's patches
and on patches built to sit on ties; and the pruned codes pass the oracle
parity rule."""
import numpy as np
import pytest

import parity
from paper_1806_04374_gb300 import synth
from test_gpu_parity import CASES, run_gpu

pytestmark = pytest.mark.gpu

KEYS = ("atom", "angle_idx", "angle", "coef", "resid_norm2")


@pytest.fixture(scope="module")
def rsc(cuda_ok):
    import paper_1806_04374_gb300 as rsc
    rsc.load_library()
    return rsc


def _same(a, b):
    for k in KEYS:
        assert np.array_equal(a[k], b[k]), k


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_pruned_codes_equal_plain_fp32(rsc, case):
    name, M, J, kmax, R, K, P, n_terms, sigma = case
    d = synth.make_dictionary(M, J, kmax, 1000 + M + R)
    x, _ = synth.make_patches(d, max(P, 200), n_terms, sigma, 2000 + R)
    plain = run_gpu(rsc, x, d, R, K, "fp32")
    pruned = run_gpu(rsc, x, d, R, K, "fp32_prune")
    _same(plain, pruned)


def test_pruned_workload_sample_and_oracle(rsc):
    d, x, _, wl = synth.workload_inputs("omp_1m", P=100_000)
    plain = run_gpu(rsc, x, d, wl.R, wl.K, "fp32")
    pruned = run_gpu(rsc, x, d, wl.R, wl.K, "fp32_prune")
    _same(plain, pruned)
    idx = np.random.default_rng(20181206).choice(x.shape[0], 400, replace=False)
    s = parity.check(x[idx], d, wl.R, wl.K, {k: pruned[k][idx] for k in KEYS}, 1e-5)
    print("pruned sample", s)


def test_pruned_on_ties(rsc):
    """Atoms that carry only harmonics 0 and 8 score the same at angles r and
    r + R/8, and several atoms share one bound: the pruning must keep every
    tie the plain path keeps."""
    M, J, kmax, R, K = 24, 6, 8, 64, 4
    d = synth.make_dictionary(M, J, kmax, 20181207)
    d[:8, 1:8] = 0.0  # atoms 0..7: harmonics 0 and 8 only
    d[:8] /= np.sqrt(np.einsum("mkjc,mkjc->m", d[:8], d[:8]) * 2
                     - np.einsum("mjc,mjc->m", d[:8, 0], d[:8, 0]))[:, None, None, None]
    x, _ = synth.make_patches(d, 3000, 3, 0.02, 20181208)
    plain = run_gpu(rsc, x, d, R, K, "fp32")
    pruned = run_gpu(rsc, x, d, R, K, "fp32_prune")
    _same(plain, pruned)
