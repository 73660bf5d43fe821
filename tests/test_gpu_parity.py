"""GPU parity: librsc (through the C ABI) against the FP64 oracle.

Selections must match the oracle wherever its top-two margin exceeds 1e-6
relative; weights must match the oracle's least-squares weights along the
GPU's path within 1e-5 relative (FP32 scoring path) -- see tests/parity.py.
"""
import numpy as np
import pytest

import oracle
from paper_1806_04374_gb300 import synth

from parity import check

pytestmark = pytest.mark.gpu

COEF_TOL = {"fp32": 1e-5, "f16": 1e-3}


@pytest.fixture(scope="module")
def rsc(cuda_ok):
    import paper_1806_04374_gb300 as rsc
    rsc.load_library()
    return rsc


def run_gpu(rsc, x, d, R, K, precision="fp32"):
    import torch
    dev = torch.device("cuda:0")
    dic = rsc.Dictionary(torch.from_numpy(np.ascontiguousarray(d)).to(dev), R)
    xt = torch.from_numpy(np.ascontiguousarray(x)).to(dev)
    out = rsc.encode(dic, xt, K, precision)
    torch.cuda.synchronize()
    assert rsc.rsc_dict_check(dic.handle) == 0
    res = {k: v.cpu().numpy() for k, v in out.items()}
    res["fallbacks"] = rsc.rsc_dict_fallback_count(dic.handle)
    dic.close()
    return res


@pytest.mark.parametrize("precision", ["fp32", "f16"])
def test_small_workload_full(rsc, precision):
    """1000 patches, M=16, R=32, K=3, sigma 0.05 (plus 3 ragged extra)."""
    d, x, _, wl = synth.workload_inputs("omp_small")
    x2, _ = synth.make_patches(d, 3, wl.n_terms, wl.sigma, 777)
    x = np.concatenate([x, x2])
    g = run_gpu(rsc, x, d, wl.R, wl.K, precision)
    s = check(x, d, wl.R, wl.K, g, COEF_TOL[precision])
    assert s["pinned_steps"] > 0.99 * x.shape[0] * wl.K - 50
    print(precision, s, "fallbacks", g["fallbacks"])


@pytest.mark.parametrize("precision", ["fp32", "f16"])
def test_1m_workload_sampled(rsc, precision):
    """The 1,000,000-patch workload (M=64, R=64, K=5) coded in one launch as
    the benchmark does; 768 sampled patches (incl. the first and last) are
    checked against the oracle one by one."""
    d, x, _, wl = synth.workload_inputs("omp_1m")
    g = run_gpu(rsc, x, d, wl.R, wl.K, precision)
    rng = np.random.default_rng(5)
    idx = np.unique(np.concatenate([[0, wl.P - 1], rng.choice(wl.P, 766, replace=False)]))
    sub = {k: (v[idx] if isinstance(v, np.ndarray) else v) for k, v in g.items()}
    s = check(x[idx], d, wl.R, wl.K, sub, COEF_TOL[precision])
    print(precision, s, "fallbacks", g["fallbacks"])
    # every patch coded: no atom index out of range, no NaN weights
    assert g["atom"].min() >= -1 and g["atom"].max() < wl.M
    assert np.isfinite(g["coef"]).all()


@pytest.mark.parametrize("shape", [
    # (name, M, J, kmax, R, K, P): plain rows of 112 slots (odd R), one
    # 256-row chunk per tile; rows of 256 slots, 8 chunks per tile, two
    # stream groups (P >= 2 x 65,536)
    ("plain112_R33", 7, 6, 8, 33, 3, 60000),
    ("long_rows_n250", 32, 10, 12, 64, 4, 140000),
], ids=lambda c: c[0])
def test_many_tiles_per_cta_sampled(rsc, shape):
    """Enough patches that every scoring CTA codes several 128-patch tiles
    in one launch, so its residual-row buffers are reused (the paired layout
    is covered by test_1m_workload_sampled): 400 sampled patches, including
    tile edges and both ends, checked against the oracle."""
    name, M, J, kmax, R, K, P = shape
    d = synth.make_dictionary(M, J, kmax, 3000 + M)
    x, _ = synth.make_patches(d, P, 3, 0.05, 4000 + R)
    g = run_gpu(rsc, x, d, R, K, "f16")
    rng = np.random.default_rng(11)
    edges = [0, 127, 128, 255, 256, P // 2 - 1, P // 2, P - 129, P - 128, P - 1]
    idx = np.unique(np.concatenate([edges, rng.choice(P, 390, replace=False)]))
    sub = {k: (v[idx] if isinstance(v, np.ndarray) else v) for k, v in g.items()}
    s = check(x[idx], d, R, K, sub, COEF_TOL["f16"])
    print(name, s, "fallbacks", g["fallbacks"])
    assert g["atom"].min() >= -1 and g["atom"].max() < M
    assert np.isfinite(g["coef"]).all()


CASES = [
    # (name, M, J, kmax, R, K, P, n_terms, sigma)
    ("R1_textbook_omp", 12, 6, 8, 1, 4, 97, 3, 0.05),
    ("R60_paper_angles", 10, 6, 8, 60, 3, 131, 3, 0.05),
    ("R33_ragged_lanes", 7, 6, 8, 33, 3, 67, 2, 0.1),
    ("R128_max", 9, 6, 8, 128, 3, 45, 3, 0.05),
    ("K16_reuse_atoms", 2, 6, 8, 16, 16, 41, 4, 0.2),
    ("K1", 20, 6, 8, 64, 1, 100, 3, 0.05),
    ("M256_global_dict", 256, 6, 8, 64, 4, 60, 3, 0.05),
    ("kmax12_J10", 32, 10, 12, 64, 4, 40, 3, 0.05),
    ("kmax16_J4", 16, 4, 16, 64, 3, 40, 3, 0.05),
    ("kmax0_rotation_invariant", 8, 6, 0, 16, 3, 30, 3, 0.05),
    # even R codes atom pairs (r, r + R/2) in one unit: the smallest pairs
    ("R2_one_pair_per_atom", 9, 6, 8, 2, 3, 60, 2, 0.05),
    ("R4_two_pairs", 11, 6, 8, 4, 3, 60, 3, 0.05),
    ("kmax1_minimal_odd_half", 12, 6, 1, 16, 3, 60, 2, 0.05),
    # the image workload's coder sizes: 21x21 patches, J=10, kmax=12 (n=250),
    # M=256, R=128, K=8 (tensor-core rows of 256 slots)
    ("c2_sizes_n250_M256_R128_K8", 256, 10, 12, 128, 8, 24, 4, 0.05),
]


def tc_supported(J, kmax, K):
    """Shapes the tensor-core path handles: packed length J(2 kmax + 1) <= 256
    and K <= 8."""
    return J * (2 * kmax + 1) <= 256 and K <= 8


@pytest.mark.parametrize("precision", ["fp32", "f16"])
@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_edge_shapes(rsc, case, precision):
    name, M, J, kmax, R, K, P, n_terms, sigma = case
    d = synth.make_dictionary(M, J, kmax, 1000 + M + R)
    x, _ = synth.make_patches(d, P, n_terms, sigma, 2000 + R)
    if precision == "f16" and not tc_supported(J, kmax, K):
        with pytest.raises(rsc.RscError) as ei:
            run_gpu(rsc, x, d, R, K, precision)
        assert ei.value.status == rsc.RSC_ERR_UNSUPPORTED
        return
    g = run_gpu(rsc, x, d, R, K, precision)
    s = check(x, d, R, K, g, COEF_TOL[precision])
    print(name, precision, s, "fallbacks", g["fallbacks"])


@pytest.mark.parametrize("precision", ["fp32", "f16"])
def test_degenerate_patches(rsc, precision):
    """Zero patch (no step), exactly one steered atom on the grid (one step,
    then stop), and an exactly sparse patch recovered with zero residual."""
    M, J, kmax, R = 6, 6, 8, 8
    d = synth.make_dictionary(M, J, kmax, 42)
    xs = [np.zeros((kmax + 1, J, 2), np.float32), d[3].copy()]
    q = oracle.steer(d[1].astype(np.float64), 2 * np.pi * 2 / R)  # a quarter turn: exact
    xs.append(q.astype(np.float32))
    x = np.stack(xs)
    g = run_gpu(rsc, x, d, R, 3, precision)
    assert np.all(g["atom"][0] == -1) and np.all(g["coef"][0] == 0)
    assert g["atom"][1, 0] == 3 and g["angle_idx"][1, 0] == 0 and np.all(g["atom"][1, 1:] == -1)
    assert g["atom"][2, 0] == 1 and g["angle_idx"][2, 0] == 2 and np.all(g["atom"][2, 1:] == -1)
    assert abs(g["coef"][1, 0] - 1.0) < 1e-9 and abs(g["coef"][2, 0] - 1.0) < 1e-9
    check(x, d, R, 3, g, COEF_TOL[precision])


@pytest.mark.parametrize("precision", ["fp32", "f16"])
def test_half_turn_ties_take_the_smaller_angle(rsc, precision):
    """Atoms with even harmonics only score the same at r and r + R/2 (half a
    turn multiplies harmonic k by (-1)^k, Eq. (Sr)): the tie must go to the
    smaller flat index, i.e. the angle below R/2, as the oracle's rule says."""
    M, J, kmax, R = 6, 6, 8, 16
    d = synth.make_dictionary(M, J, kmax, 4242).astype(np.float64)
    d[:, 1::2] = 0.0
    d /= np.sqrt(synth.coef_norm2(d))[:, None, None, None]
    d = d.astype(np.float32)
    xs = []
    for m, r0 in [(0, 3), (2, 11), (5, 0), (4, 7)]:  # 11 = 3 + R/2: ties with 3
        xs.append(oracle.steer(d[m].astype(np.float64), 2 * np.pi * r0 / R).astype(np.float32))
    x = np.stack(xs)
    g = run_gpu(rsc, x, d, R, 1, precision)
    o = oracle.romp(x, d, R, 1)
    assert np.array_equal(g["atom"][:, 0], [0, 2, 5, 4])
    assert np.array_equal(g["angle_idx"][:, 0], [3, 3, 0, 7])
    assert np.array_equal(g["angle_idx"][:, 0], o["angle"][:, 0])


@pytest.mark.parametrize("precision", ["fp32", "f16"])
@pytest.mark.parametrize("scale", [1e-12, 1e12])
def test_patch_scale(rsc, precision, scale):
    """Selections and weights scale with the patch: the FP16 path stores each
    residual row times a power of two chosen from its norm bound, so patches
    far outside fp16's range (1e-12, 1e12 times the unit-scale workload) are
    coded like the oracle codes them."""
    d, x, _, wl = synth.workload_inputs("omp_small", P=300)
    xs = (x.astype(np.float64) * scale).astype(np.float32)
    g = run_gpu(rsc, xs, d, wl.R, wl.K, precision)
    s = check(xs, d, wl.R, wl.K, g, COEF_TOL[precision])
    assert s["pinned_steps"] > 0.98 * xs.shape[0] * wl.K - 20
    print(precision, scale, s, "fallbacks", g["fallbacks"])


@pytest.mark.parametrize("precision", ["fp32", "f16"])
def test_rotation_covariance_gpu(rsc, precision):
    """Rotating every patch by s grid steps shifts every GPU-selected angle by
    s (Eq. 3) wherever the oracle's margins pin the selections."""
    d, x, _, wl = synth.workload_inputs("omp_small", P=200)
    s = 5
    xr = np.stack([oracle.steer(v.astype(np.float64), 2 * np.pi * s / wl.R) for v in x]).astype(
        np.float32)
    g0 = run_gpu(rsc, x, d, wl.R, wl.K, precision)
    g1 = run_gpu(rsc, xr, d, wl.R, wl.K, precision)
    o0 = oracle.romp(x, d, wl.R, wl.K)
    o1 = oracle.romp(xr, d, wl.R, wl.K)
    ok = np.all(o0["margin"] > 1e-4, axis=1) & np.all(o1["margin"] > 1e-4, axis=1)
    assert ok.sum() > 150
    assert np.array_equal(g1["atom"][ok], g0["atom"][ok])
    assert np.array_equal(g1["angle_idx"][ok], (g0["angle_idx"][ok] + s) % wl.R)


def test_empty_and_errors(rsc):
    import torch
    d = synth.make_dictionary(4, 6, 8, 1)
    dic = rsc.Dictionary(torch.from_numpy(d).cuda(), 8)
    x = torch.zeros((0, 9, 6, 2), device="cuda")
    out = rsc.encode(dic, x, 3)
    assert out["atom"].shape == (0, 3)
    x = torch.from_numpy(synth.make_patches(d, 4, 2, 0.1, 3)[0]).cuda()
    outs = rsc.encode(dic, x, 2)
    p = {k: v.data_ptr() for k, v in outs.items()}
    bad = [
        (dict(K=0), rsc.RSC_ERR_INVALID),
        (dict(K=17), rsc.RSC_ERR_INVALID),
        (dict(prec=7), rsc.RSC_ERR_INVALID),
        (dict(x_ptr=x.data_ptr() + 4), rsc.RSC_ERR_INVALID),  # misaligned
        (dict(atom_ptr=0), rsc.RSC_ERR_INVALID),
        (dict(P=-1), rsc.RSC_ERR_INVALID),
    ]
    for kw, want in bad:
        args = dict(handle=dic.handle, x_ptr=x.data_ptr(), P=4, K=2, prec=0, atom_ptr=p["atom"],
                    angle_idx_ptr=p["angle_idx"], angle_ptr=p["angle"], coef_ptr=p["coef"],
                    resid_norm2_ptr=p["resid_norm2"])
        args.update(kw)
        assert rsc.rsc_encode(**args) == want, kw
    torch.cuda.synchronize()
    # a dictionary whose atoms are not unit norm is rejected
    with pytest.raises(rsc.RscError):
        rsc.Dictionary(torch.from_numpy(2.0 * d).cuda(), 8)
    # sizes beyond this build
    with pytest.raises(rsc.RscError):
        rsc.Dictionary(torch.from_numpy(d).cuda(), 129)


@pytest.mark.parametrize("precision,P", [("fp32", 300_000), ("f16", 300_000),
                                         ("f16", (1 << 20) + 5_000)])
def test_host_entry_point_matches_device(rsc, precision, P):
    """rsc_encode_host (chunks of up to 2^20 patches on two streams, each
    stream group copying its own patches in and its outputs out) returns the
    same codes as rsc_encode on device buffers; the larger case takes two
    chunks."""
    import torch
    d, x, _, wl = synth.workload_inputs("omp_1m", P=P)
    dic = rsc.Dictionary(torch.from_numpy(d).cuda(), wl.R)
    xd = torch.from_numpy(x).cuda()
    a = rsc.encode(dic, xd, wl.K, precision)
    torch.cuda.synchronize()
    b = rsc.encode_host(dic, torch.from_numpy(x).pin_memory(), wl.K, precision)
    for k in ("atom", "angle_idx", "coef", "resid_norm2", "angle"):
        assert np.array_equal(a[k].cpu().numpy(), b[k].numpy()), k


def test_f16_and_fp32_paths_agree(rsc):
    """Both scoring paths certify their picks against exact re-scoring, so on
    the 1M workload they return the same selections wherever the oracle's
    margin pins them; compared here on every patch of the first 200k, with
    the weights equal to ~1e-12 relative (both solve the same FP64 system)."""
    d, x, _, wl = synth.workload_inputs("omp_1m", P=200_000)
    g32 = run_gpu(rsc, x, d, wl.R, wl.K, "fp32")
    g16 = run_gpu(rsc, x, d, wl.R, wl.K, "f16")
    same = np.all((g32["atom"] == g16["atom"]) & (g32["angle_idx"] == g16["angle_idx"]), axis=1)
    assert same.mean() > 0.9999, same.mean()
    rel = np.abs(g32["coef"][same] - g16["coef"][same]).max() / np.abs(g32["coef"]).max()
    assert rel < 1e-9, rel
    print("identical patches", same.sum(), "of", same.size, "max rel coef diff", rel,
          "f16 handed to fp32:", g16["fallbacks"])


def test_final_residual_norm_from_the_factor(rsc):
    """On the FP16 path a patch that takes all K steps reports
    ||x||^2 - z^T z (L z = b, the least-squares factor; ||x||^2 in
    double-float): within the float32 rounding of ||r|| and of its square
    (4 ulps) of the forced-path oracle's FP64 residual norm^2, far inside the
    1e-5 ||x||^2 of the general rule (the FP32 residual's own norm is off by
    up to ~3e-7 ||x||^2)."""
    d, x, _, wl = synth.workload_inputs("omp_1m", P=4096)
    g = run_gpu(rsc, x, d, wl.R, wl.K, "f16")
    forced = oracle.romp(x, d, wl.R, wl.K, forced_atom=g["atom"], forced_angle=g["angle_idx"])
    xd = x.astype(np.float64)
    xn2 = 2 * np.einsum("phjc,phjc->p", xd, xd) - np.einsum("pjc,pjc->p", xd[:, 0], xd[:, 0])
    full = g["atom"][:, -1] >= 0
    assert full.sum() > 0.99 * x.shape[0]
    gn = g["resid_norm2"].astype(np.float64)
    ref = forced["rn2"]
    err = np.abs(gn - ref)[full]
    bound = (2.0 ** -21 * ref + 1e-12 * xn2)[full]
    assert np.all(err <= bound), (err.max(), (err / xn2[full]).max())
