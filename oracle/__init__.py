"""FP64 CPU oracle for rotational OMP -- TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never loads it and
shares no code with it.

The arithmetic lives in ``rsc_oracle.c`` (plain C, FP64): the augmented
dictionary [S_0 D ... S_{R-1} D] of Fig. "code" is materialised with the
steering matrix of Eq. (Sr), and OMP (Sec. II-C) is run on it with a Cholesky
least-squares solve rebuilt from scratch at every step.  This module only
compiles that file and marshals numpy arrays to it.

Layout of every coefficient array: ``[..., kmax+1, J, 2]`` float32 half
spectra (harmonics k = 0..kmax, rings j, re/im); Im of k = 0 is ignored.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sysconfig

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rsc_oracle.c")
_LIB = os.path.join(_HERE, "librsc_oracle.so")

# Readings of the paper shared by nothing: the oracle's own copies.
STOP_REL = 1e-10
PIVOT_REL = 1e-12

_lib = None


def build(force: bool = False) -> str:
    """Compile rsc_oracle.c into librsc_oracle.so with gcc + OpenMP."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-fPIC", "-shared", "-fopenmp",
           _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        i32p = ctypes.POINTER(ctypes.c_int32)
        f32p = ctypes.POINTER(ctypes.c_float)
        f64p = ctypes.POINTER(ctypes.c_double)
        lib.rsc_oracle_romp.restype = ctypes.c_int
        lib.rsc_oracle_romp.argtypes = [f32p, ctypes.c_int64, f32p, ctypes.c_int, ctypes.c_int,
                                        ctypes.c_int, ctypes.c_int, ctypes.c_int, i32p, i32p,
                                        i32p, i32p, f64p, f64p, f64p, f64p, f64p, ctypes.c_int]
        lib.rsc_oracle_scores.restype = ctypes.c_int
        lib.rsc_oracle_scores.argtypes = [f32p, f32p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                          ctypes.c_int, f64p]
        lib.rsc_oracle_steer.restype = None
        lib.rsc_oracle_steer.argtypes = [f64p, ctypes.c_int, ctypes.c_int, ctypes.c_double, f64p]
        lib.rsc_oracle_inner.restype = ctypes.c_double
        lib.rsc_oracle_inner.argtypes = [f64p, f64p, ctypes.c_int, ctypes.c_int]
        lib.rsc_oracle_max_threads.restype = ctypes.c_int
        lib.rsc_oracle_max_threads.argtypes = []
        _lib = lib
    return _lib


def _ptr(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct)) if a is not None else None


def _dims(d):
    d = np.asarray(d)
    M, H, J, two = d.shape
    assert two == 2
    return M, J, H - 1


def max_threads() -> int:
    return _load().rsc_oracle_max_threads()


def romp(x, d, R: int, K: int, nthreads: int = 0, forced_atom=None, forced_angle=None):
    """Rotational OMP (free mode) or, with ``forced_atom``/``forced_angle``,
    the same loop along given picks (forced-path mode).

    Returns a dict with ``atom``, ``angle`` (int32, P x K, -1 where no step),
    ``coef`` (float64, P x K), ``rn2`` (float64, P, squared residual norm),
    ``margin`` (float64, P x K: (s1-s2)/s1 of the exact scores at each step,
    -1 where no step), ``pick_score`` and ``best_score`` (float64, P x K:
    |score| of the pick and the largest |score| at each step).
    """
    lib = _load()
    x = np.ascontiguousarray(x, dtype=np.float32)
    d = np.ascontiguousarray(d, dtype=np.float32)
    M, J, kmax = _dims(d)
    P = x.shape[0]
    assert x.shape[1:] == d.shape[1:], (x.shape, d.shape)
    atom = np.empty((P, K), np.int32)
    angle = np.empty((P, K), np.int32)
    coef = np.empty((P, K), np.float64)
    rn2 = np.empty((P,), np.float64)
    margin = np.empty((P, K), np.float64)
    pick = np.empty((P, K), np.float64)
    best = np.empty((P, K), np.float64)
    fa = fr = None
    if forced_atom is not None:
        fa = np.ascontiguousarray(forced_atom, dtype=np.int32).reshape(P, K)
        fr = np.ascontiguousarray(forced_angle, dtype=np.int32).reshape(P, K)
    i32 = ctypes.c_int32
    rc = lib.rsc_oracle_romp(_ptr(x, ctypes.c_float), P, _ptr(d, ctypes.c_float), M, J, kmax, R, K,
                             _ptr(fa, i32), _ptr(fr, i32), _ptr(atom, i32), _ptr(angle, i32),
                             _ptr(coef, ctypes.c_double), _ptr(rn2, ctypes.c_double),
                             _ptr(margin, ctypes.c_double), _ptr(pick, ctypes.c_double),
                             _ptr(best, ctypes.c_double), int(nthreads))
    if rc != 0:
        raise ValueError("rsc_oracle_romp rejected its arguments")
    return {"atom": atom, "angle": angle, "coef": coef, "rn2": rn2, "margin": margin,
            "pick_score": pick, "best_score": best}


def classify(xs, ds, Rs, K: int, nthreads: int = 0):
    """The coding stage of the paper's texture classifier (Sec. III-B): every
    patch coded with each dictionary (``romp``), labelled with the index of
    the dictionary of least squared coding error (ties: the smaller index).
    ``xs`` is a list of per-image patch arrays [P_i, kmax+1, J, 2]; returns
    (labels per image, rn2 [C, P_total], histogram [n_images, C])."""
    x = np.concatenate(xs) if xs else np.zeros((0,))
    C = len(ds)
    rn2 = np.stack([romp(x, ds[c], Rs[c], K, nthreads)["rn2"] for c in range(C)])
    label = np.argmin(rn2, 0)  # first minimum: the smaller index on ties
    hist, labels, lo = np.zeros((len(xs), C), np.int64), [], 0
    for i, xi in enumerate(xs):
        li = label[lo:lo + xi.shape[0]]
        labels.append(li)
        hist[i] = np.bincount(li, minlength=C)
        lo += xi.shape[0]
    return labels, rn2, hist


def scores(x1, d, R: int):
    """Exact scores <S_r d_m, x> of one patch, shape (M, R)."""
    lib = _load()
    x1 = np.ascontiguousarray(x1, dtype=np.float32)
    d = np.ascontiguousarray(d, dtype=np.float32)
    M, J, kmax = _dims(d)
    out = np.empty((M * R,), np.float64)
    rc = lib.rsc_oracle_scores(_ptr(x1, ctypes.c_float), _ptr(d, ctypes.c_float), M, J, kmax, R,
                               _ptr(out, ctypes.c_double))
    if rc != 0:
        raise MemoryError
    return out.reshape(M, R)


def steer(c, theta: float):
    """S_theta applied to one FP64 half spectrum of shape (kmax+1, J, 2)."""
    lib = _load()
    c = np.ascontiguousarray(c, dtype=np.float64)
    H, J, _ = c.shape
    out = np.empty_like(c)
    lib.rsc_oracle_steer(_ptr(c, ctypes.c_double), J, H - 1, float(theta),
                         _ptr(out, ctypes.c_double))
    return out


def inner(u, v) -> float:
    """Coefficient-space inner product of two FP64 half spectra."""
    lib = _load()
    u = np.ascontiguousarray(u, dtype=np.float64)
    v = np.ascontiguousarray(v, dtype=np.float64)
    H, J, _ = u.shape
    return lib.rsc_oracle_inner(_ptr(u, ctypes.c_double), _ptr(v, ctypes.c_double), J, H - 1)
