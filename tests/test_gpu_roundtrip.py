"""GPU reconstruction (rsc_reconstruct) and synthesis (rsc_synthesize),
through the C ABI, against the FP64 oracle (oracle/ksvd.py reconstruct,
oracle/basis.py synthesize)."""
import numpy as np
import pytest

from oracle import basis as obasis
from oracle import ksvd
from paper_1806_04374_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rsc(cuda_ok):
    import paper_1806_04374_gb300 as rsc
    rsc.load_library()
    return rsc


def test_reconstruct_matches_oracle_and_residual(rsc):
    """Codes of the small workload (1000 patches, M = 16, R = 32, K = 3) from
    rsc_encode, reconstructed on the GPU: equal to the oracle's
    sum_i a_i S_i d_i, and |x - x_rec|^2 equals the coder's resid_norm2."""
    import torch
    d, x, _, wl = synth.workload_inputs("omp_small")
    dic = rsc.Dictionary(torch.from_numpy(d).cuda(), wl.R)
    xd = torch.from_numpy(x).cuda()
    codes = rsc.encode(dic, xd, wl.K, "f16")
    rec = rsc.reconstruct(dic, codes)
    torch.cuda.synchronize()
    c = {k: v.cpu().numpy() for k, v in codes.items()}
    got = rec.cpu().numpy().astype(np.float64)
    ref = ksvd.reconstruct(d, wl.R, c["atom"], c["angle_idx"], c["coef"])
    scale = np.abs(ref).max()
    assert np.abs(got - ref).max() < 2e-6 * scale
    err = ((ksvd.pack(x.astype(np.float64) - got)) ** 2).sum(1)
    xn = (ksvd.pack(x.astype(np.float64)) ** 2).sum(1)
    assert np.allclose(err, c["resid_norm2"], rtol=1e-3, atol=1e-5 * xn.max())
    dic.close()


def test_reconstruct_skips_steps_not_taken(rsc):
    import torch
    M, J, kmax, R = 4, 6, 8, 12
    d = synth.make_dictionary(M, J, kmax, 21)
    dic = rsc.Dictionary(torch.from_numpy(d).cuda(), R)
    atom = np.array([[1, -1], [-1, -1], [3, 0]], np.int32)
    angle = np.array([[7, -1], [-1, -1], [11, 4]], np.int32)
    coef = np.array([[0.5, 0.0], [0.0, 0.0], [-1.25, 2.0]])
    codes = {"atom": torch.from_numpy(atom).cuda(), "angle_idx": torch.from_numpy(angle).cuda(),
             "coef": torch.from_numpy(coef).cuda()}
    got = rsc.reconstruct(dic, codes).cpu().numpy()
    ref = ksvd.reconstruct(d, R, atom, angle, coef)
    assert np.abs(got - ref).max() < 1e-6 * np.abs(ref).max()
    assert np.all(got[1] == 0.0)
    dic.close()


@pytest.mark.parametrize("shape", [(11, 6, 8), (21, 10, 12), (21, 10, 6)],
                         ids=["11x11", "21x21", "21x21_lowpass"])
def test_synthesize_matches_oracle(rsc, shape):
    """Random half spectra to pixels; the 21 x 21 lowpass basis (kmax halved)
    is the paper's smoother variant of the same construction."""
    import torch
    N, J, kmax = shape
    rng = np.random.default_rng(8)
    c = rng.standard_normal((300, kmax + 1, J, 2)).astype(np.float32)
    c[:, 0, :, 1] = 0.0
    b = rsc.Basis(N, J, kmax)
    got = rsc.synthesize(b, torch.from_numpy(c).cuda()).cpu().numpy()
    ref = obasis.synthesize(c, N, J, kmax)
    assert got.shape == ref.shape == (300, obasis.grid(N)[0].size)
    assert np.abs(got - ref).max() < 2e-5 * np.abs(ref).max()
    b.close()


def test_image_round_trip(rsc):
    """Windows of a 21 x 21 image: projected, coded, reconstructed and
    synthesised on the GPU; the pixels equal the oracle's synthesis of the
    GPU codes' reconstruction, and synthesising the projection alone gives
    the oracle's synthesis of its own projection."""
    import torch
    N, J, kmax, M, R, K = 21, 10, 12, 16, 16, 4
    rng = np.random.default_rng(9)
    img = rng.standard_normal((30, 27)).astype(np.float32)
    d = synth.make_dictionary(M, J, kmax, 22)
    b = rsc.Basis(N, J, kmax)
    dic = rsc.Dictionary(torch.from_numpy(d).cuda(), R)
    xt = rsc.project(b, torch.from_numpy(img).cuda())
    pix = rsc.synthesize(b, xt).cpu().numpy()
    ref = obasis.synthesize(obasis.project(img, N, J, kmax), N, J, kmax)
    # the projection's error (about 1e-6 of |x_hat|, split-fp16 products and
    # FP32 sums) passes through Phi Phi^+, whose condition number the
    # pseudo-inverse cutoff bounds by 1e3: the round trip holds to 1e-3
    assert np.abs(pix - ref).max() < 1e3 * 1e-6 * np.abs(ref).max()
    codes = rsc.encode(dic, xt, K, "f16")
    rec_pix = rsc.synthesize(b, rsc.reconstruct(dic, codes)).cpu().numpy()
    c = {k: v.cpu().numpy() for k, v in codes.items()}
    ref_rec = obasis.synthesize(ksvd.reconstruct(d, R, c["atom"], c["angle_idx"], c["coef"]),
                                N, J, kmax)
    assert np.abs(rec_pix - ref_rec).max() < 2e-5 * np.abs(ref_rec).max()
    dic.close()
    b.close()
