"""FP64 oracle of the discrete steerable basis and the patch projection --
TEST INFRASTRUCTURE ONLY (tests, smoke check and CPU baseline only).

Steps of Sec. II-D / II-E in the paper's order, with the Gaussian-ring radial
profiles of the synthetic workloads in place of the paper's annulus
indicators (Eq. (basis-cont)):
  1. sample b_j(rho) e^{i k phi} on the pixel grid of an N x N patch,
     keeping the pixels with rho <= N/2 (a circular patch);
  2. normalise: within each harmonic k the J sampled profiles are made
     orthonormal (Loewdin: B_k (B_k^H B_k)^{-1/2}), which keeps every column
     a radial profile times e^{i k phi}, hence steerable (Eq. (rotation));
  3. the analysis operator is the pseudo-inverse of the synthesis matrix
     (the paper's (Phi^* Phi)^{-1} Phi^* of step 2 of the proposed
     algorithm, generalised because Phi^* Phi is singular when there are
     more basis vectors than pixels);
  4. x_hat = Phi^+ x for every stride-1 window of an image; the way back,
     pixels = Phi x_hat, is synthesize (the proposed algorithm's step 4,
     D = Phi D_hat).
Readings: pixel (row, col) sits at x = col - c, y = c - row (c = (N-1)/2),
phi = atan2(y, x); e^{i k phi} is taken as 0 at the centre pixel for k != 0;
ring centres r_j = j * (N - 1) / (2 J), width 1 pixel; pseudo-inverse cutoff
1e-3 relative to the largest singular value (the paper's operator presumes
Phi^* Phi invertible; at 21 x 21 with J = 10, kmax = 12 the synthesis matrix
has singular values down to 4e-8 of the largest, and inverting those would
put pixel noise, amplified up to 2.5e7 times, into coefficient directions
that synthesise almost nothing; 1e-3 leaves the 11 x 11, J = 6, kmax = 8
operator unchanged).
Coefficients are returned as half spectra [k = 0..kmax][j][re, im].
"""
from __future__ import annotations

import numpy as np


def grid(N: int):
    """Pixel offsets (dy, dx) in the circular mask, row-major, with their
    polar coordinates."""
    c = (N - 1) / 2.0
    rows, cols = np.mgrid[0:N, 0:N]
    x = cols - c
    y = c - rows
    rho = np.hypot(x, y)
    keep = rho <= N / 2.0
    return rows[keep], cols[keep], rho[keep], np.arctan2(y[keep], x[keep])


def synthesis(N: int, J: int, kmax: int, sigma: float = 1.0, spacing: float | None = None):
    """Complex synthesis columns phi_{j,k}[pixel] for k = -kmax..kmax, Loewdin
    orthonormalised within each k.  Returns (Phi [npix, 2kmax+1, J], mask)."""
    if spacing is None:
        spacing = (N - 1) / (2.0 * J)
    rows, cols, rho, phi = grid(N)
    centres = spacing * (np.arange(J) + 1)
    prof = np.exp(-0.5 * ((rho[:, None] - centres[None, :]) / sigma) ** 2)  # [npix, J]
    Phi = np.zeros((rho.size, 2 * kmax + 1, J), complex)
    centre = rho == 0
    for k in range(-kmax, kmax + 1):
        e = np.exp(1j * k * phi)
        if k != 0:
            e = np.where(centre, 0.0, e)
        Bk = prof * e[:, None]
        G = Bk.conj().T @ Bk
        w, V = np.linalg.eigh(G)
        Bk = Bk @ (V @ np.diag(w ** -0.5) @ V.conj().T)
        Phi[:, k + kmax, :] = Bk
    return Phi, (rows, cols)


def real_synthesis(Phi, kmax: int, J: int):
    """Real matrix mapping packed coefficients (c_j0, sqrt2 Re c_jk, sqrt2 Im
    c_jk) to pixels of a real patch x = sum_{j,k} c_jk phi_jk."""
    cols = [Phi[:, kmax, j].real for j in range(J)]
    for k in range(1, kmax + 1):
        for j in range(J):
            ph = Phi[:, kmax + k, j]
            cols.append(np.sqrt(2.0) * ph.real)
            cols.append(-np.sqrt(2.0) * ph.imag)
    return np.stack(cols, 1)


RCOND = 1e-3


def analysis(N: int, J: int, kmax: int, **kw):
    """Packed pseudo-inverse [n, npix] (singular values at most RCOND times
    the largest treated as zero) and the mask."""
    Phi, mask = synthesis(N, J, kmax, **kw)
    Pr = np.linalg.pinv(real_synthesis(Phi, kmax, J), rcond=RCOND)
    return Pr, mask


def unpack_half(v, J: int, kmax: int):
    """Packed coefficients [..., n] -> half spectra [..., kmax+1, J, 2]."""
    out = np.zeros(v.shape[:-1] + (kmax + 1, J, 2))
    out[..., 0, :, 0] = v[..., :J]
    rest = v[..., J:].reshape(v.shape[:-1] + (kmax, J, 2)) / np.sqrt(2.0)
    out[..., 1:, :, :] = rest
    return out


def synthesize(c, N: int, J: int, kmax: int, **kw):
    """Pixels Phi x_hat of half spectra c [P, kmax+1, J, 2] over the circular
    patch (step 4 of the proposed algorithm, Sec. II-E: D = Phi D_hat):
    [P, npix], pixels in the row-major order of grid()."""
    Phi, _ = synthesis(N, J, kmax, **kw)
    X = real_synthesis(Phi, kmax, J)
    c = np.asarray(c, np.float64)
    v = np.concatenate([c[:, 0, :, 0], np.sqrt(2.0) * c[:, 1:].reshape(c.shape[0], -1)], 1)
    return v @ X.T


def project(image, N: int, J: int, kmax: int, **kw):
    """Half-spectrum coefficients of every stride-1 N x N window of a 2-D
    image, windows in row-major order of their top-left corner."""
    image = np.asarray(image, np.float64)
    Pr, (rows, cols) = analysis(N, J, kmax, **kw)
    h, w = image.shape
    out = []
    for r0 in range(h - N + 1):
        for c0 in range(w - N + 1):
            out.append(Pr @ image[r0 + rows, c0 + cols])
    return unpack_half(np.array(out).reshape(-1, Pr.shape[0]), J, kmax)
