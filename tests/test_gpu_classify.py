"""GPU multi-dictionary labelling (rsc_classify_images, through the C ABI)
against the FP64 oracle (oracle.classify on the oracle's projection)."""
import numpy as np
import pytest

import oracle
from oracle import basis as obasis
from paper_1806_04374_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rsc(cuda_ok):
    import paper_1806_04374_gb300 as rsc
    rsc.load_library()
    return rsc


@pytest.mark.parametrize("precision", ["fp32", "f16"])
def test_classify_matches_oracle(rsc, precision):
    """Three dictionaries (different M and R), line-texture images of uneven
    sizes (one smaller than a window).  Labels must equal the oracle's
    wherever the two smallest coding errors differ by more than 1e-3
    relative (the coders' weights agree to 1e-5 / 1e-3); the histogram is
    the per-image count of the GPU's own labels."""
    import torch
    N, J, kmax, K = 11, 6, 8, 3
    specs = [(12, 16), (8, 32), (16, 12)]  # (M, R)
    ds = [synth.make_dictionary(M, J, kmax, 60 + c) for c, (M, R) in enumerate(specs)]
    Rs = [R for _, R in specs]
    shapes = [(24, 30), (9, 40), (31, 19), (16, 16)]
    imgs = [synth.make_line_image(h, w, 0.02, 70 + i) for i, (h, w) in enumerate(shapes)]
    b = rsc.Basis(N, J, kmax)
    dics = [rsc.Dictionary(torch.from_numpy(d).cuda(), R) for d, R in zip(ds, Rs)]
    labels, hist = rsc.classify_images(dics, b, [torch.from_numpy(im).cuda() for im in imgs],
                                       K, precision)
    torch.cuda.synchronize()
    labels, hist = labels.cpu().numpy(), hist.cpu().numpy()
    xs = [obasis.project(im, N, J, kmax).astype(np.float32) for im in imgs]
    ref_labels, rn2, ref_hist = oracle.classify(xs, ds, Rs, K)
    ref = np.concatenate(ref_labels)
    counts = [x.shape[0] for x in xs]
    assert labels.shape == ref.shape == (sum(counts),)
    srt = np.sort(rn2, 0)
    gap = (srt[1] - srt[0]) / np.maximum(srt[1], 1e-30)
    clear = gap > 1e-3
    assert clear.mean() > 0.9
    assert np.array_equal(labels[clear], ref[clear])
    lo = 0
    for i, n in enumerate(counts):
        assert np.array_equal(hist[i], np.bincount(labels[lo:lo + n], minlength=3))
        lo += n
    assert hist[1].sum() == 0 and hist.sum() == sum(counts)
    print(precision, "clear", clear.mean(), "agree", (labels == ref).mean())
    for dd in dics:
        dd.close()
    b.close()


def test_classify_no_windows(rsc):
    """Every image smaller than a window: no labels, an all-zero histogram."""
    import torch
    N, J, kmax = 11, 6, 8
    b = rsc.Basis(N, J, kmax)
    dics = [rsc.Dictionary(torch.from_numpy(synth.make_dictionary(6, J, kmax, 80 + c)).cuda(), 8)
            for c in range(2)]
    imgs = [torch.ones((5, 40), device="cuda"), torch.ones((10, 10), device="cuda")]
    labels, hist = rsc.classify_images(dics, b, imgs, 3, "f16")
    torch.cuda.synchronize()
    assert labels.numel() == 0
    assert hist.shape == (2, 2) and int(hist.abs().sum()) == 0
    for dd in dics:
        dd.close()
    b.close()
