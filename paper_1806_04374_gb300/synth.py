"""Seeded synthetic inputs for rotational sparse coding (numpy, host).

This module is the only thing the oracle side and the CUDA side share: it
draws the dictionaries and patches both are given.  It contains none of the
coder's arithmetic (no scores, selection, least squares or residuals).  To
synthesise a rotated atom it applies the rotation model of Eq. (rotation)
directly, c[j,k] -> exp(-i k theta) c[j,k], in numpy complex arithmetic of its
own, at continuous angles drawn uniformly on [0, 2 pi).

Coefficient layout everywhere: ``[..., kmax+1, J, 2]`` float32 half spectra
(harmonics k = 0..kmax of a real patch, J radial rings, re/im).  A real patch
has c[j,-k] = conj(c[j,k]), so the negative harmonics are implicit and the
k = 0 entries are real (their Im slot is 0).  The coefficient-space norm is
sum_j c_j0^2 + 2 sum_{k>=1} |c_jk|^2, i.e. the norm of the full spectrum.

Workloads (shapes from the paper's 11x11 circular patches, Sec. III-A: J = 6
Gaussian rings and harmonics |k| <= 8 give n = J (2 kmax + 1) = 102 real
degrees of freedom):
  * ``omp_small``  : P = 1000, M = 16, R = 32, K = 3, 3 atoms/patch, sigma 0.05
  * ``omp_1m``     : P = 1,000,000, M = 64, R = 64, K = 5, 3 atoms/patch,
                     sigma 0.1
Noise is i.i.d. N(0, sigma^2) per real degree of freedom of the full
spectrum (so N(0, sigma^2/2) on Re and Im of each k >= 1 entry).
"""
from __future__ import annotations

import dataclasses

import numpy as np

CHUNK = 65536  # patches per independently seeded chunk


@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    P: int
    M: int
    J: int
    kmax: int
    R: int
    K: int
    n_terms: int
    sigma: float
    seed: int


WORKLOADS = {
    "omp_small": Workload("omp_small", 1000, 16, 6, 8, 32, 3, 3, 0.05, 20180611),
    "omp_1m": Workload("omp_1m", 1_000_000, 64, 6, 8, 64, 5, 3, 0.1, 20180612),
}


def coef_norm2(c: np.ndarray) -> np.ndarray:
    """Squared coefficient-space norm of half spectra [..., H, J, 2] (fp64)."""
    c = np.asarray(c, np.float64)
    k0 = (c[..., 0, :, 0] ** 2).sum(-1)
    rest = (c[..., 1:, :, :] ** 2).sum((-1, -2, -3))
    return k0 + 2.0 * rest


def make_dictionary(M: int, J: int, kmax: int, seed: int) -> np.ndarray:
    """M unit-norm atoms with Hermitian N(0,1) spectra: the k = 0 entries are
    real N(0,1), the k >= 1 entries have independent N(0,1) real and
    imaginary parts.  Normalised in fp64, returned as float32."""
    rng = np.random.Generator(np.random.PCG64(seed))
    d = rng.standard_normal((M, kmax + 1, J, 2))
    d[:, 0, :, 1] = 0.0
    d /= np.sqrt(coef_norm2(d))[:, None, None, None]
    return d.astype(np.float32)


def _rotate(c: np.ndarray, theta: np.ndarray) -> np.ndarray:
    """Rotation model of Eq. (rotation) for the generator: complex half
    spectra c [..., H, J] times exp(-i k theta[...])."""
    H = c.shape[-2]
    k = np.arange(H)
    phase = np.exp(-1j * k[None, :] * theta[..., None])
    return c * phase[..., None]


def make_patches(d: np.ndarray, P: int, n_terms: int, sigma: float, seed: int,
                 chunk_ids=None):
    """Patches x = sum_{i<n_terms} w_i S_{theta_i} d_{m_i} + noise.

    m_i uniform over the M atoms, theta_i ~ U[0, 2 pi), w_i ~ N(0, 1).
    Chunk c (patches [c*CHUNK, (c+1)*CHUNK)) is drawn from its own seed, so
    any chunk can be regenerated alone.  Returns (x float32 [P, H, J, 2],
    truth dict with 'atom', 'theta', 'w').
    """
    d = np.asarray(d, np.float64)
    M, H, J, _ = d.shape
    dc = d[..., 0] + 1j * d[..., 1]
    nchunks = (P + CHUNK - 1) // CHUNK
    ids = range(nchunks) if chunk_ids is None else chunk_ids
    xs, atoms, thetas, ws = [], [], [], []
    for c in ids:
        lo = c * CHUNK
        n = min(CHUNK, P - lo)
        rng = np.random.Generator(np.random.PCG64([seed, c]))
        # full-chunk draws sliced to n, so a short last chunk is a prefix of
        # the full one and patch i is the same whatever P is
        m = rng.integers(0, M, size=(CHUNK, n_terms))[:n]
        th = rng.uniform(0.0, 2.0 * np.pi, size=(CHUNK, n_terms))[:n]
        w = rng.standard_normal((CHUNK, n_terms))[:n]
        x = np.zeros((n, H, J), np.complex128)
        for i in range(n_terms):
            x += w[:, i, None, None] * _rotate(dc[m[:, i]], th[:, i])
        noise = rng.standard_normal((CHUNK, H, J, 2))[:n] * sigma
        noise[:, 1:] *= np.sqrt(0.5)
        noise[:, 0, :, 1] = 0.0
        out = np.empty((n, H, J, 2), np.float32)
        out[..., 0] = x.real + noise[..., 0]
        out[..., 1] = x.imag + noise[..., 1]
        out[:, 0, :, 1] = 0.0
        xs.append(out)
        atoms.append(m.astype(np.int32))
        thetas.append(th)
        ws.append(w)
    return (np.concatenate(xs), {"atom": np.concatenate(atoms), "theta": np.concatenate(thetas),
                                 "w": np.concatenate(ws)})


def workload_inputs(name: str, P: int | None = None):
    """Dictionary and patches of a named workload (optionally the first P
    patches only).  Returns (d, x, truth, workload)."""
    wl = WORKLOADS[name]
    d = make_dictionary(wl.M, wl.J, wl.kmax, wl.seed)
    P = wl.P if P is None else P
    x, truth = make_patches(d, P, wl.n_terms, wl.sigma, wl.seed + 1)
    return d, x, truth, wl


def make_line_image(h: int, w: int, density: float, seed: int, noise: float = 0.1,
                    width: float = 1.0, length: float = 9.0) -> np.ndarray:
    """A pixel image for the image workloads: background N(0, noise^2) plus
    randomly placed and oriented line segments (Poisson count density * h * w,
    centres uniform, angles U[0, pi), weights N(0, 1)) with a Gaussian cross
    profile of the given width and a soft end taper, i.e. rotated copies of
    one line template, the structure of the paper's toy example (Fig. 1)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    img = rng.normal(0.0, noise, (h, w))
    n = rng.poisson(density * h * w)
    ys, xs = np.mgrid[0:h, 0:w].astype(np.float64)
    cy = rng.uniform(0, h, n)
    cx = rng.uniform(0, w, n)
    th = rng.uniform(0, np.pi, n)
    wt = rng.standard_normal(n)
    half = length / 2.0
    reach = int(np.ceil(half + 3 * width)) + 1
    for i in range(n):
        y0, y1 = max(0, int(cy[i]) - reach), min(h, int(cy[i]) + reach + 1)
        x0, x1 = max(0, int(cx[i]) - reach), min(w, int(cx[i]) + reach + 1)
        dy, dx = ys[y0:y1, x0:x1] - cy[i], xs[y0:y1, x0:x1] - cx[i]
        along = dx * np.cos(th[i]) + dy * np.sin(th[i])
        across = -dx * np.sin(th[i]) + dy * np.cos(th[i])
        taper = np.clip(half + 1.0 - np.abs(along), 0.0, 1.0)
        img[y0:y1, x0:x1] += wt[i] * taper * np.exp(-0.5 * (across / width) ** 2)
    return img.astype(np.float32)
