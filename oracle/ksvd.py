"""FP64 oracle of the rotational K-SVD atom update -- TEST INFRASTRUCTURE ONLY.

Only the tests, the smoke check and the CPU-baseline leg of the benchmark may
import this module; the product library never does.

It follows the inner loop of the R-K-SVD pseudocode (Fig. "code", Sec. II-C)
literally, in coefficient space where R_r is the steering matrix S_r of
Eq. (Sr):
  * the augmented dictionary [S_0 D ... S_{R-1} D] is built once, before the
    atom loop, and used for every atom (so all atoms are updated from the
    same dictionary and the same codes);
  * for atom m, every patch whose code uses m at some angle r0 contributes the
    column S_{-r0} (x_p - D_aug b), where b is the patch's code with the entry
    of (m, r0) set to zero;
  * D_m becomes the first left singular vector of the matrix of those columns.
Readings where the paper is silent (Sec. II-C, "implementation details"):
  * an atom used more than once by a patch: r0 is the occurrence with the
    largest |weight| (ties: the earliest selected);
  * an unused atom is reset to the unit-normalised patch with the largest
    coding error ||x_p - D_aug a_p||; several unused atoms take successive
    patches in descending error (ties: smaller patch index);
  * the singular vector's sign makes its largest-magnitude entry positive.
Vectors are handled as packed reals (k = 0 real parts, sqrt(2) Re and Im of
k >= 1), whose Euclidean product is the coefficient inner product, so the SVD
is taken in the right geometry.
"""
from __future__ import annotations

import numpy as np


def pack(c):
    """Half spectrum [..., H, J, 2] -> packed real [..., J + 2 kmax J]."""
    c = np.asarray(c, np.float64)
    k0 = c[..., 0, :, 0]
    rest = np.sqrt(2.0) * c[..., 1:, :, :]
    return np.concatenate([k0.reshape(c.shape[:-3] + (-1,)),
                           rest.reshape(c.shape[:-3] + (-1,))], axis=-1)


def unpack(v, H, J):
    """Inverse of pack."""
    v = np.asarray(v, np.float64)
    out = np.zeros(v.shape[:-1] + (H, J, 2))
    out[..., 0, :, 0] = v[..., :J]
    out[..., 1:, :, :] = v[..., J:].reshape(v.shape[:-1] + (H - 1, J, 2)) / np.sqrt(2.0)
    return out


def steer(c, theta):
    """S_theta of Eq. (Sr) on half spectra: harmonic k times exp(-i k theta)."""
    c = np.asarray(c, np.float64)
    H = c.shape[-3]
    z = c[..., 0] + 1j * c[..., 1]
    z = z * np.exp(-1j * np.arange(H) * theta)[:, None]
    out = np.stack([z.real, z.imag], -1)
    out[..., 0, :, 1] = 0.0
    return out


def reconstruct(d, R, atom, angle, coef):
    """The coded patches in steerable coordinates, sum_i a_i S_{theta_i} d_{m_i}
    (Sec. II-C's sparse code, steering of Eq. (Sr), theta = 2 pi r / R); steps
    with atom -1 contribute nothing.  Returns half spectra [P, H, J, 2]."""
    d = np.asarray(d, np.float64)
    atom, angle, coef = np.asarray(atom), np.asarray(angle), np.asarray(coef, np.float64)
    P, K = atom.shape
    out = np.zeros((P,) + d.shape[1:])
    for p in range(P):
        for i in range(K):
            if atom[p, i] >= 0:
                out[p] += coef[p, i] * steer(d[atom[p, i]], 2 * np.pi * angle[p, i] / R)
    return out


def augmented(d, R):
    """Packed columns S_{2 pi r / R} d_m, column index m*R + r."""
    M = d.shape[0]
    cols = [pack(steer(d[m], 2 * np.pi * r / R)) for m in range(M) for r in range(R)]
    return np.stack(cols, 1)


def ksvd_update(x, d, R, atom, angle, coef):
    """One R-K-SVD dictionary update from given codes.

    x: [P, H, J, 2], d: [M, H, J, 2] (float32 or float64); atom, angle: int
    [P, K] (-1 = no step); coef: float [P, K].  Returns (d_new [M, H, J, 2]
    float64, n_used [M] int)."""
    x = np.asarray(x, np.float64)
    d = np.asarray(d, np.float64)
    P, H, J, _ = x.shape
    M = d.shape[0]
    K = atom.shape[1]
    Aug = augmented(d, R)
    X = pack(x)                                   # [P, n]
    B = np.zeros((P, M * R))                      # codes as M*R vectors
    for p in range(P):
        for i in range(K):
            if atom[p, i] >= 0:
                B[p, atom[p, i] * R + angle[p, i]] += coef[p, i]
    err = np.sum((X - B @ Aug.T) ** 2, axis=1)    # coding error of each patch
    d_new = d.copy()
    n_used = np.zeros(M, np.int64)
    unused = []
    for m in range(M):
        cols = []
        for p in range(P):
            occ = [i for i in range(K) if atom[p, i] == m]
            if not occ:
                continue
            i0 = occ[0]
            for i in occ[1:]:
                if abs(coef[p, i]) > abs(coef[p, i0]):
                    i0 = i
            r0 = angle[p, i0]
            b = B[p].copy()
            b[m * R + r0] = 0.0
            res = unpack(X[p] - Aug @ b, H, J)
            cols.append(pack(steer(res, -2 * np.pi * r0 / R)))
        n_used[m] = len(cols)
        if not cols:
            unused.append(m)
            continue
        Y = np.stack(cols, 1)                     # [n, N_m]
        U, _, _ = np.linalg.svd(Y, full_matrices=False)
        u = U[:, 0]
        if u[np.argmax(np.abs(u))] < 0:
            u = -u
        d_new[m] = unpack(u, H, J)
    order = sorted(range(P), key=lambda p: (-err[p], p))
    for q, m in enumerate(unused):
        p = order[q]
        v = X[p] / np.linalg.norm(X[p])
        d_new[m] = unpack(v, H, J)
    return d_new, n_used
