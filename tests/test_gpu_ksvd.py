"""GPU rotational K-SVD update (rsc_ksvd_update, through the C ABI) against
the FP64 oracle of oracle/ksvd.py, from identical codes."""
import numpy as np
import pytest

from oracle import ksvd
from paper_1806_04374_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rsc(cuda_ok):
    import paper_1806_04374_gb300 as rsc
    rsc.load_library()
    return rsc


def gpu_update(rsc, x, d, R, atom, angle, coef):
    import torch
    dic = rsc.Dictionary(torch.from_numpy(np.ascontiguousarray(d, np.float32)).cuda(), R)
    codes = {"atom": torch.from_numpy(np.ascontiguousarray(atom, np.int32)).cuda(),
             "angle_idx": torch.from_numpy(np.ascontiguousarray(angle, np.int32)).cuda(),
             "coef": torch.from_numpy(np.ascontiguousarray(coef, np.float64)).cuda()}
    new, used = rsc.ksvd_update(dic, torch.from_numpy(np.ascontiguousarray(x)).cuda(), codes)
    torch.cuda.synchronize()
    out = new.cpu().numpy(), used.cpu().numpy()
    dic.close()
    return out


def eig_ratio(x, d, R, atom, angle, coef, m):
    """lambda_1 / (lambda_1 - lambda_2) of the aligned-residual covariance of
    atom m: the conditioning of its leading eigenvector (Davis-Kahan)."""
    from test_oracle_ksvd import _direct_columns
    Y = _direct_columns(x, np.asarray(d, np.float64), R, atom, angle, coef, m)
    lam = np.linalg.eigvalsh(Y @ Y.T)
    return lam[-1] / max(lam[-1] - lam[-2], 1e-300)


def assert_atoms_close(d_gpu, d_ref, ratios=None):
    """The GPU covariance is FP64-grade (double-float columns, exact products,
    FP64 sums: ~1e-11 relative), the leading eigenvector comes from at most
    5000 FP64 power iterations started at the old atom, and the atoms are
    returned as float32.  So an atom may differ from the exact singular vector
    by the float32 rounding (~1e-7 per entry), ~1e-11 r with
    r = lambda_1 / (lambda_1 - lambda_2) (Davis-Kahan), and the iteration's
    own residual (1 - 1/r)^5000 <= exp(-5000 / r); the tolerance allows 2e-6,
    1e-9 r and that residual."""
    for m in range(d_ref.shape[0]):
        u, v = ksvd.pack(d_gpu[m]), ksvd.pack(d_ref[m])
        assert abs(np.linalg.norm(u) - 1.0) < 1e-6, m
        r = ratios.get(m) if ratios is not None else None
        tol = 2e-6 + (1e-9 * r + np.exp(-5000.0 / r) if r else 0.0)
        assert np.max(np.abs(u - v)) < tol, (m, np.max(np.abs(u - v)), tol)


def test_single_atom_closed_form(rsc):
    rng = np.random.default_rng(1)
    R = 16
    d_true = synth.make_dictionary(1, 6, 8, 11)
    d_old = synth.make_dictionary(1, 6, 8, 12)
    P = 200
    r = rng.integers(0, R, P)
    w = rng.standard_normal(P)
    x = np.stack([w[p] * ksvd.steer(d_true[0], 2 * np.pi * r[p] / R) for p in range(P)])
    x = x.astype(np.float32)
    new, used = gpu_update(rsc, x, d_old, R, np.zeros((P, 1), np.int32), r[:, None], w[:, None])
    assert used[0] == P
    u, v = ksvd.pack(new[0]), ksvd.pack(d_true[0])
    assert abs(abs(u @ v) / np.linalg.norm(v) - 1.0) < 1e-6


def test_update_matches_oracle_on_encoded_codes(rsc):
    """Codes from rsc_encode on the small workload (1000 patches, M = 16,
    R = 32, K = 3); both updates start from the same codes."""
    import torch
    d, x, _, wl = synth.workload_inputs("omp_small")
    dic = rsc.Dictionary(torch.from_numpy(d).cuda(), wl.R)
    codes = rsc.encode(dic, torch.from_numpy(x).cuda(), wl.K, "fp32")
    torch.cuda.synchronize()
    c = {k: v.cpu().numpy() for k, v in codes.items()}
    dic.close()
    ref, used_ref = ksvd.ksvd_update(x, d, wl.R, c["atom"], c["angle_idx"], c["coef"])
    new, used = gpu_update(rsc, x, d, wl.R, c["atom"], c["angle_idx"], c["coef"])
    assert np.array_equal(used, used_ref)
    ratios = {m: eig_ratio(x, d, wl.R, c["atom"], c["angle_idx"], c["coef"], m)
              for m in range(d.shape[0]) if used[m] > 0}
    assert_atoms_close(new, ref, ratios)
    # the same update again: bit-identical (sample lists in patch order, the
    # covariance's partial sums added in a fixed order)
    new2, used2 = gpu_update(rsc, x, d, wl.R, c["atom"], c["angle_idx"], c["coef"])
    assert np.array_equal(used2, used) and np.array_equal(new2, new)


def test_unused_atoms_reset_and_repeated_atoms(rsc):
    """Atoms 3 and 4 are used by no patch: reset to the two patches with the
    largest coding error; atom 0 appears twice in some codes."""
    rng = np.random.default_rng(7)
    M, R, K, P = 5, 8, 3, 300
    d = synth.make_dictionary(M, 6, 8, 70)
    x, _ = synth.make_patches(d[:3], P, 2, 0.2, 71)
    atom = rng.integers(0, 3, (P, K)).astype(np.int32)
    atom[::7, 1] = atom[::7, 0]
    angle = rng.integers(0, R, (P, K)).astype(np.int32)
    angle[::7, 1] = (angle[::7, 0] + 3) % R
    coef = rng.standard_normal((P, K))
    atom[::5, 2] = -1
    angle[::5, 2] = -1
    coef[::5, 2] = 0.0
    ref, used_ref = ksvd.ksvd_update(x, d, R, atom, angle, coef)
    new, used = gpu_update(rsc, x, d, R, atom, angle, coef)
    assert np.array_equal(used, used_ref) and used[3] == 0 and used[4] == 0
    ratios = {m: eig_ratio(x, d, R, atom, angle, coef, m) for m in range(3)}
    assert_atoms_close(new, ref, ratios)


def test_split_update_over_two_shards_equals_single_update(rsc):
    """rsc_ksvd_accumulate on two shards of the patches (as two ranks would),
    the covariances and counts summed, the largest-error lists merged, then
    rsc_ksvd_finish: the same atoms and counts as rsc_ksvd_update on all the
    patches, including the resets of unused atoms (M exceeds the atoms the
    planted data use, so some atoms go unused)."""
    import torch
    from paper_1806_04374_gb300.rksvd import merge_top
    M, J, kmax, R, K, P = 24, 6, 8, 16, 2, 3001
    d_true = synth.make_dictionary(4, J, kmax, 31)
    x, _ = synth.make_patches(d_true, P, 2, 0.05, 32)
    d0 = synth.make_dictionary(M, J, kmax, 33)
    dic = rsc.Dictionary(torch.from_numpy(d0).cuda(), R)
    xd = torch.from_numpy(x).cuda()
    codes = rsc.encode(dic, xd, K, "fp32")
    # atoms 20..23 taken out of the codes: they go unused and are reset
    drop = codes["atom"] >= 20
    codes["atom"][drop] = -1
    codes["angle_idx"][drop] = -1
    codes["coef"][drop] = 0.0
    ref_new, ref_used = rsc.ksvd_update(dic, xd, codes)
    split = 1700
    parts = []
    for lo, hi in ((0, split), (split, P)):
        sub = {k: v[lo:hi].contiguous() for k, v in codes.items()}
        parts.append((lo, rsc.ksvd_accumulate(dic, xd[lo:hi].contiguous(), sub)))
    C = parts[0][1]["C"] + parts[1][1]["C"]
    count = (parts[0][1]["count"] + parts[1][1]["count"]).to(torch.int32)
    errs, gidx, vecs = [], [], []
    for lo, acc in parts:
        idx = acc["top_idx"].cpu().numpy()
        errs.append(acc["top_err"].cpu().numpy())
        gidx.append(np.where(idx >= 0, idx + lo, -1))
        vecs.append(acc["top_vec"].cpu().numpy())
    top_idx, top_vec = merge_top(errs, gidx, vecs)
    new, used = rsc.ksvd_finish(dic, C, count, torch.from_numpy(top_idx).cuda(),
                                torch.from_numpy(top_vec).cuda())
    torch.cuda.synchronize()
    ref_used = ref_used.cpu().numpy()
    assert np.array_equal(used.cpu().numpy(), ref_used)
    assert (ref_used == 0).sum() >= 4          # resets exercised
    assert np.abs(new.cpu().numpy() - ref_new.cpu().numpy()).max() < 1e-6
    dic.close()
