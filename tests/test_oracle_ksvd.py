"""Pins for the FP64 rotational K-SVD update oracle (CPU only).

* Closed forms: patches built from steered copies of true atoms with their
  exact codes give back exactly those atoms (Fig. "code": aligning each
  residual with S_{-r0} undoes the rotation, so every column is w * d_m).
* The aligned-residual columns of the literal pseudocode (materialised
  augmented dictionary, code vectors with one entry zeroed) equal the direct
  formula S_{-r0}(x - sum_{i != i0} a_i S_{r_i} d_{m_i}).
* The first singular vector equals the leading eigenvector of Y Y^T
  (numpy eigh), the unused-atom reset and the repeated-atom reading.
"""
import numpy as np

from oracle import ksvd
from paper_1806_04374_gb300 import synth

J, KMAX = 6, 8
H = KMAX + 1


def test_pack_unpack_roundtrip_and_norm():
    rng = np.random.default_rng(0)
    c = rng.standard_normal((4, H, J, 2))
    c[:, 0, :, 1] = 0
    assert np.allclose(ksvd.unpack(ksvd.pack(c), H, J), c)
    n2 = (c[:, 0, :, 0] ** 2).sum(-1) + 2 * (c[:, 1:] ** 2).sum((-1, -2, -3))
    assert np.allclose((ksvd.pack(c) ** 2).sum(-1), n2)


def test_single_atom_recovered_exactly():
    rng = np.random.default_rng(1)
    R = 16
    d_true = synth.make_dictionary(1, J, KMAX, 11).astype(np.float64)
    d_old = synth.make_dictionary(1, J, KMAX, 12).astype(np.float64)
    P = 40
    r = rng.integers(0, R, P)
    w = rng.standard_normal(P)
    x = np.stack([w[p] * ksvd.steer(d_true[0], 2 * np.pi * r[p] / R) for p in range(P)])
    atom = np.zeros((P, 1), int)
    d_new, n_used = ksvd.ksvd_update(x, d_old, R, atom, r[:, None], w[:, None])
    assert n_used[0] == P
    v_new, v_true = ksvd.pack(d_new[0]), ksvd.pack(d_true[0])
    v_true /= np.linalg.norm(v_true)
    assert abs(abs(v_new @ v_true) - 1.0) < 1e-12
    assert v_new[np.abs(v_new).argmax()] > 0  # sign reading


def test_two_atoms_exact_codes_recovered():
    rng = np.random.default_rng(2)
    R = 12
    d = synth.make_dictionary(2, J, KMAX, 21).astype(np.float64)
    P = 30
    r = rng.integers(0, R, (P, 2))
    w = rng.standard_normal((P, 2))
    x = np.stack([w[p, 0] * ksvd.steer(d[0], 2 * np.pi * r[p, 0] / R) +
                  w[p, 1] * ksvd.steer(d[1], 2 * np.pi * r[p, 1] / R) for p in range(P)])
    atom = np.tile(np.array([0, 1]), (P, 1))
    d_new, n_used = ksvd.ksvd_update(x, d, R, atom, r, w)
    for m in range(2):
        v = ksvd.pack(d[m])
        assert abs(abs(ksvd.pack(d_new[m]) @ v) / np.linalg.norm(v) - 1.0) < 1e-12


def _direct_columns(x, d, R, atom, angle, coef, m, rule="largest"):
    """S_{-r0}(x - sum of a_i S_{r_i} d_{m_i} over the steps whose (atom,
    angle) is not (m, r0)) for the patches using m.  r0 is the occurrence of m
    with the largest |weight|, ties to the earliest (rule "largest", the
    reading of Sec. II-C's arbitrary choice), or, to show that the pins tell
    the readings apart, the first ("first") or last ("last") occurrence."""
    cols = []
    for p in range(x.shape[0]):
        occ = [i for i in range(atom.shape[1]) if atom[p, i] == m]
        if not occ:
            continue
        if rule == "first":
            i0 = occ[0]
        elif rule == "last":
            i0 = occ[-1]
        else:
            i0 = max(occ, key=lambda i: (abs(coef[p, i]), -i))
        r0 = angle[p, i0]
        res = x[p].astype(np.float64).copy()
        for i in range(atom.shape[1]):
            if atom[p, i] >= 0 and not (atom[p, i] == m and angle[p, i] == r0):
                res -= coef[p, i] * ksvd.steer(d[atom[p, i]], 2 * np.pi * angle[p, i] / R)
        cols.append(ksvd.pack(ksvd.steer(res, -2 * np.pi * angle[p, i0] / R)))
    return np.stack(cols, 1)


def test_literal_columns_equal_direct_formula_and_svd_equals_eigh():
    import oracle
    d, x, _, wl = synth.workload_inputs("omp_small", P=120)
    o = oracle.romp(x, d, wl.R, wl.K)
    d_new, n_used = ksvd.ksvd_update(x, d, wl.R, o["atom"], o["angle"], o["coef"])
    for m in range(d.shape[0]):
        if n_used[m] == 0:
            continue
        Y = _direct_columns(x, d.astype(np.float64), wl.R, o["atom"], o["angle"], o["coef"], m)
        assert Y.shape[1] == n_used[m]
        wv, V = np.linalg.eigh(Y @ Y.T)
        u = V[:, -1]
        if u[np.abs(u).argmax()] < 0:
            u = -u
        assert np.allclose(ksvd.pack(d_new[m]), u, atol=1e-9), m


def test_repeated_atom_uses_largest_weight_and_unused_reset():
    R = 8
    d = synth.make_dictionary(3, J, KMAX, 31).astype(np.float64)
    rng = np.random.default_rng(3)
    P = 6
    x = rng.standard_normal((P, H, J, 2))
    x[:, 0, :, 1] = 0
    # patch 0 uses atom 0 twice (weights 0.2 at r=1, -0.9 at r=5); atom 2 unused
    atom = np.array([[0, 0], [1, -1], [1, 0], [0, 1], [1, -1], [0, -1]])
    angle = np.array([[1, 5], [2, -1], [3, 4], [6, 7], [0, -1], [2, -1]])
    coef = np.array([[0.2, -0.9], [1.0, 0], [0.5, 0.4], [0.3, 0.7], [0.8, 0], [1.1, 0]])
    d_new, n_used = ksvd.ksvd_update(x, d, R, atom, angle, coef)
    assert list(n_used) == [4, 4, 0]
    Y = _direct_columns(x, d, R, atom, angle, coef, 0)
    # the column of patch 0 is aligned with the -0.9 occurrence (r0 = 5)
    res = x[0] - 0.2 * ksvd.steer(d[0], 2 * np.pi * 1 / R)
    assert np.allclose(Y[:, 0], ksvd.pack(ksvd.steer(res, -2 * np.pi * 5 / R)))
    # atom 2 reset to the unit-normalised patch with the largest coding error
    Aug = ksvd.augmented(d, R)
    X = ksvd.pack(x)
    errs = []
    for p in range(P):
        b = np.zeros(3 * R)
        for i in range(2):
            if atom[p, i] >= 0:
                b[atom[p, i] * R + angle[p, i]] += coef[p, i]
        errs.append(np.sum((X[p] - Aug @ b) ** 2))
    p_star = int(np.argmax(errs))
    assert np.allclose(ksvd.pack(d_new[2]), X[p_star] / np.linalg.norm(X[p_star]))
    # the oracle's atom 0 is the leading singular direction of exactly these
    # columns (sign reading applied), and not that of the columns a "first
    # occurrence" reading would give
    assert np.allclose(ksvd.pack(d_new[0]), _leading(Y), atol=1e-12)
    Y_first = _direct_columns(x, d, R, atom, angle, coef, 0, rule="first")
    assert not np.allclose(Y_first[:, 0], Y[:, 0], atol=1e-3)
    assert np.abs(_leading(Y_first) - ksvd.pack(d_new[0])).max() > 1e-3


def _leading(Y):
    """Leading eigenvector of Y Y^T with its largest-magnitude entry positive."""
    _, V = np.linalg.eigh(Y @ Y.T)
    u = V[:, -1]
    return -u if u[np.abs(u).argmax()] < 0 else u


def _twin_case(first_is_larger):
    """Two patches that use atom 0 twice at different angles, with inexact
    codes (the residual is not aligned with the atom), so the angle r0 that
    aligns a patch's column decides the updated atom."""
    R = 16
    d = synth.make_dictionary(2, J, KMAX, 41).astype(np.float64)
    rng = np.random.default_rng(4)
    P = 5
    x = rng.standard_normal((P, H, J, 2))
    x[:, 0, :, 1] = 0
    big, small = -1.3, 0.4
    w = [big, small] if first_is_larger else [small, big]
    atom = np.array([[0, 0], [0, 0], [0, 1], [1, -1], [0, -1]])
    angle = np.array([[3, 11], [14, 6], [9, 2], [5, -1], [0, -1]])
    coef = np.array([w, w[::-1], [0.7, 0.2], [0.9, 0.0], [-0.6, 0.0]])
    return x, d, R, atom, angle, coef


def test_repeated_atom_twin_cases_pin_the_largest_weight_reading():
    # twin A: in patch 0 the larger |weight| comes second, in patch 1 first;
    # twin B swaps which occurrence is larger.  In both, the oracle's atom 0
    # must be the leading direction of the columns aligned with the larger
    # |weight|, which differs from the one a first-occurrence rule gives.
    for first_is_larger in (False, True):
        x, d, R, atom, angle, coef = _twin_case(first_is_larger)
        d_new, n_used = ksvd.ksvd_update(x, d, R, atom, angle, coef)
        assert n_used[0] == 4 and n_used[1] == 2
        Y = _direct_columns(x, d, R, atom, angle, coef, 0)
        assert np.allclose(ksvd.pack(d_new[0]), _leading(Y), atol=1e-12)
        Y_first = _direct_columns(x, d, R, atom, angle, coef, 0, rule="first")
        assert np.abs(_leading(Y_first) - ksvd.pack(d_new[0])).max() > 1e-3
    # equal |weights|: the earliest occurrence aligns the column
    x, d, R, atom, angle, coef = _twin_case(False)
    coef[0] = [0.8, -0.8]
    d_new, _ = ksvd.ksvd_update(x, d, R, atom, angle, coef)
    Y = _direct_columns(x, d, R, atom, angle, coef, 0)
    assert np.allclose(ksvd.pack(d_new[0]), _leading(Y), atol=1e-12)
    Y_last = _direct_columns(x, d, R, atom, angle, coef, 0, rule="last")
    assert np.abs(_leading(Y_last) - ksvd.pack(d_new[0])).max() > 1e-3
