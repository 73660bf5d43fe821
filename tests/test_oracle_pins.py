"""Pins for the FP64 oracle: checks against what the paper and mathematics fix,
independent of the oracle's own code (CPU only).

* Eq. (Sr): S_0 = I, S_a S_b = S_{a+b}, S_{2 pi} = I, norm preserved.
* Eq. (rotation): steering equals rotating the continuous function
  f(rho, phi) = sum_{j,k} c_jk b_j(rho) e^{i k phi} (evaluated point-wise here).
* Eq. (rearrange): the coefficient inner product equals the L2 inner product
  of the synthesised functions for an orthonormal radial family (quadrature).
* Eq. (3): rotating a patch by r0 grid steps shifts every selected angle by
  r0 (mod R) and leaves atoms and weights unchanged.
* OMP (Sec. II-C): residual orthogonal to the selected steered atoms,
  Pythagoras, K = 1 brute force over (m, theta, a), R = 1 and general R equal
  to a textbook OMP (scikit-learn) on the materialised augmented dictionary,
  tiny brute force of the step-wise definition, closed form for an
  orthonormal dictionary, degenerate inputs.
"""
import numpy as np
import pytest

import oracle
from paper_1806_04374_gb300 import synth

J, KMAX = 6, 8
H = KMAX + 1


def rand_half(rng, J=J, kmax=KMAX):
    c = rng.standard_normal((kmax + 1, J, 2))
    c[0, :, 1] = 0.0
    return c


def pack(c):
    """Real vector whose Euclidean dot product is the full-spectrum inner
    product: k = 0 real parts, then sqrt(2) (Re, Im) of k >= 1."""
    c = np.asarray(c, np.float64)
    return np.concatenate([c[0, :, 0].ravel(), np.sqrt(2.0) * c[1:].ravel()])


def full_spectrum(c):
    """Complex array F[k + kmax, j] for k = -kmax..kmax from a half spectrum."""
    c = np.asarray(c, np.float64)
    kmax = c.shape[0] - 1
    z = c[..., 0] + 1j * c[..., 1]
    z[0] = z[0].real
    F = np.zeros((2 * kmax + 1, c.shape[1]), complex)
    F[kmax:] = z
    F[:kmax] = np.conj(z[1:][::-1])
    return F


# ---------------------------------------------------------------- Eq. (Sr)

def test_steer_identity_compose_period_norm():
    rng = np.random.default_rng(1)
    c = rand_half(rng)
    assert np.allclose(oracle.steer(c, 0.0), c, atol=1e-15)
    a, b = 0.7, -2.3
    ab = oracle.steer(oracle.steer(c, a), b)
    assert np.allclose(ab, oracle.steer(c, a + b), atol=1e-13)
    assert np.allclose(oracle.steer(c, 2 * np.pi), c, atol=1e-12)
    R = 32
    s1 = oracle.steer(c, 2 * np.pi * 5 / R)
    assert np.allclose(oracle.steer(s1, 2 * np.pi * (R - 5) / R), c, atol=1e-12)
    n0 = oracle.inner(c, c)
    for th in rng.uniform(0, 2 * np.pi, 5):
        assert abs(oracle.inner(oracle.steer(c, th), oracle.steer(c, th)) - n0) < 1e-12 * n0


# ---------------------------------------------------------------- Eq. (rotation)

def synth_fn(c, rho, phi):
    """f(rho, phi) = sum_{k=-kmax..kmax} sum_j c_jk b_j(rho) e^{i k phi} with
    Gaussian rings b_j centred at j*5/6, width 1 (the real patch function)."""
    F = full_spectrum(c)
    kmax = c.shape[0] - 1
    ks = np.arange(-kmax, kmax + 1)
    centres = (np.arange(c.shape[1]) + 1) * 5.0 / 6.0
    b = np.exp(-0.5 * (rho[:, None] - centres[None, :]) ** 2)  # [npts, J]
    e = np.exp(1j * ks[None, :] * phi[:, None])  # [npts, 2kmax+1]
    val = np.einsum("pk,kj,pj->p", e, F, b)
    return val


def test_steering_is_rotation_of_the_function():
    rng = np.random.default_rng(2)
    c = rand_half(rng)
    rho = rng.uniform(0, 5.5, 200)
    phi = rng.uniform(-np.pi, np.pi, 200)
    f = synth_fn(c, rho, phi)
    assert np.max(np.abs(f.imag)) < 1e-10  # Hermitian spectrum => real patch
    for theta in (0.3, 2 * np.pi * 7 / 32, -1.1):
        rotated = synth_fn(c, rho, phi - theta)  # (R_theta f)(rho, phi) = f(rho, phi - theta)
        steered = synth_fn(oracle.steer(c, theta), rho, phi)
        assert np.allclose(rotated.real, steered.real, atol=1e-10)


# ---------------------------------------------------------------- Eq. (rearrange)

def test_inner_product_is_L2_inner_product_of_functions():
    """With radial functions q_j orthonormal on [0, 5.5] w.r.t. rho d rho,
    psi_jk = q_j(rho) e^{ik phi} / sqrt(2 pi) is orthonormal on the disk, so
    the L2 product of two real synthesised patches equals the coefficient
    inner product (full spectrum, i.e. weights 1 for k = 0, 2 for k >= 1)."""
    rng = np.random.default_rng(3)
    kmax, Jr = 4, 3
    xg, wg = np.polynomial.legendre.leggauss(60)
    rho = 0.5 * 5.5 * (xg + 1)
    wr = 0.5 * 5.5 * wg * rho
    Q = np.stack([rho ** i for i in range(Jr)], 1)
    # orthonormalise w.r.t. the weighted product (Gram-Schmidt via Cholesky)
    G = Q.T @ (wr[:, None] * Q)
    Lc = np.linalg.cholesky(G)
    Qo = Q @ np.linalg.inv(Lc).T
    nphi = 64
    phi = 2 * np.pi * np.arange(nphi) / nphi

    def func(c):
        F = full_spectrum(c)
        ks = np.arange(-kmax, kmax + 1)
        e = np.exp(1j * ks[None, :] * phi[:, None]) / np.sqrt(2 * np.pi)
        return np.einsum("ak,kj,rj->ra", e, F, Qo).real  # [rho, phi]

    for _ in range(3):
        u = rand_half(rng, Jr, kmax)
        v = rand_half(rng, Jr, kmax)
        fu, fv = func(u), func(v)
        l2 = np.sum(wr[:, None] * fu * fv) * (2 * np.pi / nphi)
        assert abs(l2 - oracle.inner(u, v)) < 1e-9 * (1 + abs(l2))


def test_pack_matches_inner():
    rng = np.random.default_rng(4)
    u, v = rand_half(rng), rand_half(rng)
    assert abs(pack(u) @ pack(v) - oracle.inner(u, v)) < 1e-12


# ---------------------------------------------------------------- helpers

def augmented_packed(d, R):
    """Columns pack(S_{2 pi r / R} d_m), column index m*R + r."""
    M = d.shape[0]
    cols = [pack(oracle.steer(d[m].astype(np.float64), 2 * np.pi * r / R))
            for m in range(M) for r in range(R)]
    return np.stack(cols, 1)


def small_case(seed, M=8, R=16, P=40, n_terms=3, sigma=0.05):
    d = synth.make_dictionary(M, J, KMAX, seed)
    x, truth = synth.make_patches(d, P, n_terms, sigma, seed + 1)
    return d, x, truth


# ---------------------------------------------------------------- Eq. (3)

def test_rotation_covariance_on_grid():
    d, x, _ = small_case(10, M=8, R=32, P=60)
    R, K = 32, 3
    o = oracle.romp(x, d, R, K)
    for s in (1, 7, 31):
        xr = np.stack([oracle.steer(xi.astype(np.float64), 2 * np.pi * s / R) for xi in x])
        xr32 = xr.astype(np.float32)
        # the float32 rounding of the rotated patch perturbs scores by ~1e-7;
        # compare only patches whose every step has a clear margin
        o2 = oracle.romp(xr32, d, R, K)
        ok = np.all(o["margin"] > 1e-4, axis=1)
        assert ok.sum() > 40
        assert np.array_equal(o2["atom"][ok], o["atom"][ok])
        assert np.array_equal(o2["angle"][ok], (o["angle"][ok] + s) % R)
        assert np.allclose(o2["coef"][ok], o["coef"][ok], rtol=1e-5, atol=1e-6)


# ---------------------------------------------------------------- OMP properties

def test_residual_orthogonal_and_pythagoras():
    d, x, _ = small_case(11, M=8, R=16, P=30)
    R, K = 16, 4
    o = oracle.romp(x, d, R, K)
    for p in range(x.shape[0]):
        xp = x[p].astype(np.float64)
        approx = np.zeros_like(xp)
        atoms = []
        for i in range(K):
            if o["atom"][p, i] < 0:
                continue
            A = oracle.steer(d[o["atom"][p, i]].astype(np.float64), 2 * np.pi * o["angle"][p, i] / R)
            atoms.append(A)
            approx += o["coef"][p, i] * A
        res = xp - approx
        nx = np.sqrt(oracle.inner(xp, xp))
        for A in atoms:
            assert abs(oracle.inner(A, res)) < 1e-10 * nx
        assert abs(oracle.inner(xp, xp) - oracle.inner(approx, approx) - o["rn2"][p]) < 1e-10 * nx ** 2
        assert abs(oracle.inner(res, res) - o["rn2"][p]) < 1e-10 * nx ** 2


def test_k1_brute_force_over_atom_angle_weight():
    d, x, _ = small_case(12, M=6, R=12, P=25)
    R = 12
    o = oracle.romp(x, d, R, 1)
    Aug = augmented_packed(d, R)
    for p in range(x.shape[0]):
        xv = pack(x[p])
        best = None
        for c in range(Aug.shape[1]):
            A = Aug[:, [c]]
            a, *_ = np.linalg.lstsq(A, xv, rcond=None)
            err = np.sum((xv - A[:, 0] * a[0]) ** 2)
            if best is None or err < best[0] - 1e-12:
                best = (err, c, a[0])
        err, c, a = best
        assert o["atom"][p, 0] == c // R and o["angle"][p, 0] == c % R
        assert abs(o["coef"][p, 0] - a) < 1e-10
        assert abs(o["rn2"][p] - err) < 1e-10


@pytest.mark.parametrize("R", [1, 8])
def test_matches_textbook_omp(R):
    lm = pytest.importorskip("sklearn.linear_model")
    d, x, _ = small_case(13, M=10, R=max(R, 1), P=30)
    K = 4
    o = oracle.romp(x, d, R, K)
    Aug = augmented_packed(d, R)
    for p in range(x.shape[0]):
        if np.min(o["margin"][p]) < 1e-6:
            continue
        coef = lm.orthogonal_mp(Aug, pack(x[p]), n_nonzero_coefs=K)
        nz = np.flatnonzero(coef)
        got = o["atom"][p] * R + o["angle"][p]
        assert set(nz.tolist()) == set(got.tolist())
        assert np.allclose(coef[got], o["coef"][p], rtol=1e-8, atol=1e-10)


def test_tiny_brute_force_stepwise_definition():
    """M <= 3, R <= 8, K = 2: every candidate support enumerated; step 1 must
    maximise |<A, x>|, step 2 must maximise |<A, x - P_1 x>| with the LS
    projection P_1, and the final weights must be the LS solution."""
    rng = np.random.default_rng(14)
    for trial in range(6):
        M, R = 1 + trial % 3, (4, 8)[trial % 2]
        d = synth.make_dictionary(M, J, KMAX, 100 + trial)
        x, _ = synth.make_patches(d, 5, 2, 0.1, 200 + trial)
        o = oracle.romp(x, d, R, 2)
        Aug = augmented_packed(d, R)
        for p in range(x.shape[0]):
            xv = pack(x[p])
            s = np.abs(Aug.T @ xv)
            c1 = int(np.argmax(s))
            if np.sort(s)[-1] - np.sort(s)[-2] < 1e-9:
                continue
            assert c1 == o["atom"][p, 0] * R + o["angle"][p, 0]
            A1 = Aug[:, [c1]]
            a1, *_ = np.linalg.lstsq(A1, xv, rcond=None)
            r1 = xv - A1 @ a1
            s2 = np.abs(Aug.T @ r1)
            c2 = int(np.argmax(s2))
            top = np.sort(s2)
            if top[-1] - top[-2] < 1e-9:
                continue
            assert c2 == o["atom"][p, 1] * R + o["angle"][p, 1]
            A12 = Aug[:, [c1, c2]]
            a12, *_ = np.linalg.lstsq(A12, xv, rcond=None)
            assert np.allclose(a12, o["coef"][p], atol=1e-10)
            assert abs(np.sum((xv - A12 @ a12) ** 2) - o["rn2"][p]) < 1e-10
    _ = rng


def test_orthonormal_dictionary_closed_form():
    """Atoms on disjoint rings, each carrying harmonics 1 and 2 (no rotational
    symmetry): any steered copies of different atoms are orthogonal, so a
    noise-free x = sum w_m S_{theta_m} d_m on grid angles is recovered exactly,
    in order of decreasing |w_m|, with zero residual."""
    rng = np.random.default_rng(15)
    M, R = 5, 24
    d = np.zeros((M, H, J, 2))
    for m in range(M):
        d[m, 1, m] = rng.standard_normal(2)
        d[m, 2, m] = rng.standard_normal(2)
        d[m] /= np.sqrt(oracle.inner(d[m], d[m]))
    d32 = d.astype(np.float32)
    w = np.array([2.0, -1.5, 1.0, 0.6, -0.3])
    r_true = np.array([3, 17, 0, 23, 11])
    x = sum(w[m] * oracle.steer(d32[m].astype(np.float64), 2 * np.pi * r_true[m] / R)
            for m in range(M))
    x32 = x.astype(np.float32)[None]
    o = oracle.romp(x32, d32, R, M)
    order = np.argsort(-np.abs(w))
    assert np.array_equal(o["atom"][0], order)
    assert np.array_equal(o["angle"][0], r_true[order])
    # x was rounded to float32: weights within float32 rounding
    assert np.allclose(o["coef"][0], w[order], rtol=1e-6, atol=1e-6)
    assert o["rn2"][0] < 1e-12


def test_degenerate_inputs_stop():
    d = synth.make_dictionary(4, J, KMAX, 5)
    R = 8
    # zero patch: nothing to explain
    o = oracle.romp(np.zeros((1, H, J, 2), np.float32), d, R, 3)
    assert np.all(o["atom"] == -1) and np.all(o["coef"] == 0) and o["rn2"][0] == 0
    # exactly one steered atom (a quarter turn permutes re/im exactly in
    # float32), K = 3: one step, then the residual is ~0 and coding stops
    for r in (0, 2):
        x = oracle.steer(d[2].astype(np.float64), 2 * np.pi * r / R)[None].astype(np.float32)
        o = oracle.romp(x, d, R, 3)
        assert o["atom"][0, 0] == 2 and o["angle"][0, 0] == r
        assert abs(o["coef"][0, 0] - 1.0) < 1e-12
        assert np.all(o["atom"][0, 1:] == -1) and np.all(o["angle"][0, 1:] == -1)


def test_forced_mode_reproduces_free_mode():
    d, x, _ = small_case(16, M=8, R=16, P=20)
    o = oracle.romp(x, d, 16, 4)
    f = oracle.romp(x, d, 16, 4, forced_atom=o["atom"], forced_angle=o["angle"])
    assert np.array_equal(f["atom"], o["atom"]) and np.array_equal(f["angle"], o["angle"])
    assert np.allclose(f["coef"], o["coef"], atol=1e-12)
    taken = o["atom"] >= 0
    assert np.allclose(f["pick_score"][taken], f["best_score"][taken], rtol=1e-12)


def test_generator_recovers_truth_on_small_workload():
    """Sanity of the inputs: on the small workload the first pick of most
    patches is one of the planted atoms at the nearest grid angle."""
    d, x, truth, wl = synth.workload_inputs("omp_small", P=200)
    o = oracle.romp(x, d, wl.R, wl.K)
    hit = 0
    for p in range(200):
        i = np.argmax(np.abs(truth["w"][p]))
        r_near = int(np.round(truth["theta"][p, i] * wl.R / (2 * np.pi))) % wl.R
        hit += (o["atom"][p, 0] == truth["atom"][p, i]) and (o["angle"][p, 0] == r_near)
    assert hit > 120


def test_scores_equal_packed_augmented_products():
    """oracle.scores(x) = [pack(S_r d_m) . pack(x)] for every (m, r)."""
    d, x, _ = small_case(17, M=5, R=12, P=3)
    Aug = augmented_packed(d, 12)
    for p in range(3):
        s = oracle.scores(x[p], d, 12)
        assert np.allclose(s.ravel(), Aug.T @ pack(x[p]), atol=1e-12)
