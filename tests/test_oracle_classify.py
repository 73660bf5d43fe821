"""Pins for the oracle's multi-dictionary labelling (the coding stage of the
paper's texture classifier, Sec. III-B; CPU only)."""
import numpy as np

import oracle
from paper_1806_04374_gb300 import synth


def test_identical_dictionaries_label_the_first():
    """Equal coding errors: the smaller dictionary index wins."""
    d = synth.make_dictionary(8, 6, 8, 31)
    x, _ = synth.make_patches(d, 40, 2, 0.1, 32)
    labels, rn2, hist = oracle.classify([x[:25], x[25:]], [d, d, d], [16, 16, 16], 3)
    assert np.all(rn2[0] == rn2[1]) and np.all(rn2[1] == rn2[2])
    assert all(np.all(li == 0) for li in labels)
    assert hist.tolist() == [[25, 0, 0], [15, 0, 0]]


def test_patches_take_the_label_of_their_generating_dictionary():
    """Patches planted from dictionary c (two steered atoms plus little noise)
    are coded best by c: the label is the argmin of the coding error, not
    the argmax, and the histogram counts each image's patches."""
    ds = [synth.make_dictionary(8, 6, 8, 40 + c) for c in range(3)]
    xs = []
    for c in range(3):
        x, _ = synth.make_patches(ds[c], 30, 2, 0.01, 50 + c)
        xs.append(x)
    labels, rn2, hist = oracle.classify(xs, ds, [32, 32, 32], 3)
    for c in range(3):
        assert np.all(labels[c] == c)
    assert np.array_equal(hist, 30 * np.eye(3, dtype=np.int64))
    # the winning error is the smallest of the three for every patch
    lab = np.concatenate(labels)
    assert np.all(rn2[lab, np.arange(lab.size)] == rn2.min(0))
