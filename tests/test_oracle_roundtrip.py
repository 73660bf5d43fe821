"""Pins for the oracle's way back from codes to patches (CPU only):
reconstruction in steerable coordinates (Sec. II-C's sparse code with the
steering of Eq. (Sr)) and synthesis to pixels (step 4 of the proposed
algorithm, Sec. II-E: D = Phi D_hat)."""
import numpy as np

import oracle
from oracle import basis, ksvd
from paper_1806_04374_gb300 import synth


def test_reconstruction_error_is_the_omp_residual():
    """|x - sum_i a_i S_i d_i|^2 equals the residual norm the C OMP oracle
    computes from its own residual vector (an independent route)."""
    d, x, _, wl = synth.workload_inputs("omp_small")
    x = x[:200]
    out = oracle.romp(x, d, wl.R, wl.K)
    rec = ksvd.reconstruct(d, wl.R, out["atom"], out["angle"], out["coef"])
    err = ksvd.pack(x.astype(np.float64) - rec)
    rn2 = (err ** 2).sum(1)
    assert np.allclose(rn2, out["rn2"], rtol=1e-9, atol=1e-12 * (ksvd.pack(x) ** 2).sum(1).max())


def test_reconstruction_of_planted_codes_is_exact():
    """Codes that plant atoms at grid angles reconstruct the planted sum."""
    rng = np.random.default_rng(4)
    M, J, kmax, R = 5, 6, 8, 16
    d = synth.make_dictionary(M, J, kmax, 9)
    atom = np.array([[0, 3, -1], [4, 4, 2]])
    angle = np.array([[5, 0, -1], [1, 9, 15]])
    coef = rng.standard_normal((2, 3))
    coef[0, 2] = 0.0
    rec = ksvd.reconstruct(d, R, atom, angle, coef)
    # steering by a grid angle is a phase exp(-i k 2 pi r / R) per harmonic
    k = np.arange(kmax + 1)[:, None]
    for p in range(2):
        z = np.zeros((kmax + 1, J), complex)
        for i in range(3):
            if atom[p, i] >= 0:
                dz = d[atom[p, i], ..., 0] + 1j * d[atom[p, i], ..., 1]
                z += coef[p, i] * dz * np.exp(-1j * k * 2 * np.pi * angle[p, i] / R)
        assert np.allclose(rec[p, ..., 0], z.real, atol=1e-12)
        assert np.allclose(rec[p, 1:, :, 1], z.imag[1:], atol=1e-12)
        assert np.all(rec[p, 0, :, 1] == 0.0)


def _patch_image(pix, N):
    rows, cols, _, _ = basis.grid(N)
    img = np.zeros((N, N))
    img[rows, cols] = pix
    return img


def test_synthesis_then_projection_returns_the_kept_coordinates():
    """project(synthesize(c)) = P c with P = Pr Xr the orthogonal projector
    pinned in test_oracle_basis (identity on its range)."""
    rng = np.random.default_rng(5)
    for N, J, kmax in ((11, 6, 8), (21, 10, 12)):
        Pr, _ = basis.analysis(N, J, kmax)
        Phi, _ = basis.synthesis(N, J, kmax)
        Xr = basis.real_synthesis(Phi, kmax, J)
        v = (Pr @ Xr) @ rng.standard_normal(Xr.shape[1])   # in the kept span
        c = basis.unpack_half(v, J, kmax)
        pix = basis.synthesize(c[None], N, J, kmax)[0]
        back = basis.project(_patch_image(pix, N), N, J, kmax)[0]
        assert np.allclose(back, c, atol=1e-9 * np.abs(c).max())


def test_synthesis_of_a_quarter_turn_is_the_rotated_patch():
    """Steering by pi/2 (Eq. (rotation), harmonic k times exp(-i k pi/2))
    synthesises the patch turned by +90 degrees on the pixel grid (np.rot90
    maps the circular mask onto itself)."""
    rng = np.random.default_rng(6)
    for N, J, kmax in ((11, 6, 8), (21, 10, 12)):
        c = rng.standard_normal((1, kmax + 1, J, 2))
        c[:, 0, :, 1] = 0.0
        img = _patch_image(basis.synthesize(c, N, J, kmax)[0], N)
        img90 = _patch_image(basis.synthesize(ksvd.steer(c, np.pi / 2), N, J, kmax)[0], N)
        assert np.allclose(img90, np.rot90(img), atol=1e-10 * np.abs(img).max())


def test_lowpass_basis_round_trip():
    """The lowpass variant (kmax halved, Sec. III's comparison of rotation
    methods) is the same construction with fewer harmonics: its synthesis is
    the full basis's synthesis restricted to harmonics 0..kmax/2."""
    rng = np.random.default_rng(7)
    N, J, kmax = 21, 10, 12
    c = rng.standard_normal((3, kmax // 2 + 1, J, 2))
    c[:, 0, :, 1] = 0.0
    full = np.zeros((3, kmax + 1, J, 2))
    full[:, : kmax // 2 + 1] = c
    low = basis.synthesize(c, N, J, kmax // 2)
    assert np.allclose(low, basis.synthesize(full, N, J, kmax), atol=1e-12)
