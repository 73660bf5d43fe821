"""The R-K-SVD checkpoint file on CPU: the dictionary, iteration count and
history come back as written; a file written for another R or K is refused;
a write replaces the previous file only once complete."""
import numpy as np
import pytest

from paper_1806_04374_gb300 import rksvd, synth


def test_checkpoint_round_trip(tmp_path):
    d = synth.make_dictionary(5, 6, 8, 7)
    hist = [{"iter": 0, "mse": 0.25, "unused": 1}, {"iter": 1, "mse": 0.125, "unused": 0}]
    path = str(tmp_path / "ck.npz")
    rksvd.save_checkpoint(path, d, 2, hist, R=32, K=3)
    d2, it, h2 = rksvd.load_checkpoint(path, R=32, K=3)
    assert np.array_equal(d2, d) and d2.dtype == np.float32
    assert it == 2 and h2 == hist
    with pytest.raises(ValueError):
        rksvd.load_checkpoint(path, R=16, K=3)
    rksvd.save_checkpoint(path, d * 0.5, 3, hist + [{"iter": 2, "mse": 0.1, "unused": 0}], 32, 3)
    d3, it3, h3 = rksvd.load_checkpoint(path, 32, 3)
    assert it3 == 3 and len(h3) == 3 and np.array_equal(d3, d * 0.5)
    assert not (tmp_path / "ck.npz.tmp.npz").exists()
