"""Pins for the oracle's steerable basis and projection (CPU only)."""
import json
import os

import numpy as np

from oracle import basis
from oracle import ksvd

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_counts.json")


def test_circular_patch_pixel_count_matches_paper():
    g = json.load(open(GOLDEN))["circular_patch_pixels"]
    rows, cols, rho, phi = basis.grid(g["diameter"])
    assert rows.size == g["pixels"]


def test_loewdin_orthonormal_within_each_harmonic_and_hermitian():
    N, J, kmax = 11, 6, 8
    Phi, _ = basis.synthesis(N, J, kmax)
    for k in range(-kmax, kmax + 1):
        B = Phi[:, k + kmax, :]
        assert np.allclose(B.conj().T @ B, np.eye(J), atol=1e-10)
        assert np.allclose(Phi[:, -k + kmax, :], B.conj(), atol=1e-14)


def test_real_synthesis_equals_complex_sum():
    N, J, kmax = 11, 6, 8
    Phi, _ = basis.synthesis(N, J, kmax)
    rng = np.random.default_rng(0)
    c = rng.standard_normal((kmax + 1, J, 2))
    c[0, :, 1] = 0
    z = c[..., 0] + 1j * c[..., 1]
    full = np.concatenate([np.conj(z[1:][::-1]), z], 0)  # k = -kmax..kmax
    x = np.einsum("pkj,kj->p", Phi, full)
    assert np.max(np.abs(x.imag)) < 1e-12
    Xr = basis.real_synthesis(Phi, kmax, J)
    assert np.allclose(Xr @ ksvd.pack(c), x.real, atol=1e-12)


def test_quarter_turn_of_the_patch_is_steering_by_half_pi():
    """rot90 maps the grid and mask onto themselves, so projecting a patch
    rotated by +90 degrees equals steering its coefficients by pi/2 (Eq.
    (rotation): harmonic k times exp(-i k pi/2))."""
    rng = np.random.default_rng(1)
    for N, J, kmax in ((11, 6, 8), (21, 10, 12)):
        img = rng.standard_normal((N, N))
        c = basis.project(img, N, J, kmax)[0]
        c90 = basis.project(np.rot90(img), N, J, kmax)[0]
        assert np.allclose(c90, ksvd.steer(c, np.pi / 2), atol=1e-10)


def test_pseudo_inverse_properties():
    """Truncated pseudo-inverse: singular values <= 1e-3 sigma_max are
    dropped.  Pr Xr is then the orthogonal projector onto the kept right
    singular vectors (symmetric, idempotent, exact on its range), the
    operator norm is at most 1e3 / sigma_max (a cutoff of 1e-10 gives
    2.5e7 / sigma_max at 21 x 21), and Xr Pr Xr differs from Xr by at most
    the largest dropped singular value."""
    rng = np.random.default_rng(3)
    for N, J, kmax, dropped in ((21, 10, 12, 12), (11, 6, 8, 8)):
        Phi, _ = basis.synthesis(N, J, kmax)
        Xr = basis.real_synthesis(Phi, kmax, J)
        Pr, _ = basis.analysis(N, J, kmax)
        s = np.linalg.svd(Xr, compute_uv=False)
        n = Xr.shape[1]
        assert (s <= basis.RCOND * s[0]).sum() + (n - s.size) == dropped
        P = Pr @ Xr
        assert np.allclose(P, P.T, atol=1e-9)
        assert np.allclose(P @ P, P, atol=1e-9)
        assert abs(np.trace(P) - (n - dropped)) < 1e-8
        c = P @ rng.standard_normal(n)
        assert np.allclose(Pr @ (Xr @ c), c, atol=1e-9)
        assert np.linalg.norm(Pr, 2) <= 1.0 / (basis.RCOND * s[0]) * (1 + 1e-9)
        assert np.linalg.norm(Xr - Xr @ Pr @ Xr, 2) <= basis.RCOND * s[0]


def test_project_windows_order():
    rng = np.random.default_rng(2)
    img = rng.standard_normal((14, 13))
    c = basis.project(img, 11, 6, 8)
    assert c.shape == ((14 - 10) * (13 - 10), 9, 6, 2)
    c_12 = basis.project(img[1:12, 2:13], 11, 6, 8)[0]
    assert np.allclose(c[1 * 3 + 2], c_12)
