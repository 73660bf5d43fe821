"""GPU rotational sparse coding (rotational OMP, McCann et al., "Fast
Rotational Sparse Coding") for NVIDIA GB300.

The compute lives in librsc.so (CUDA, sm_103a) behind the C ABI of
include/rsc.h.  This module is a thin ctypes binding with the same names: it
marshals pointers, sizes and CUDA streams, and never computes anything
itself.  PyTorch is used only to own device memory and streams.  There is no
CPU fallback: if the library is missing the import of the binding fails.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "librsc.so")

RSC_OK = 0
RSC_ERR_INVALID = -1
RSC_ERR_OOM = -2
RSC_ERR_CUDA = -3
RSC_ERR_TIMEOUT = -4
RSC_ERR_UNSUPPORTED = -5

RSC_FP32 = 0
RSC_F16_RESCORE = 2
RSC_FP32_PRUNE = 3
PRECISIONS = {"fp32": RSC_FP32, "f16": RSC_F16_RESCORE, "fp32_prune": RSC_FP32_PRUNE}

# every symbol include/rsc.h declares
EXPORTS = (
    "rsc_dict_create", "rsc_dict_destroy", "rsc_dict_dims", "rsc_encode", "rsc_encode_host",
    "rsc_dict_check", "rsc_dict_fallback_count", "rsc_dict_set_timing", "rsc_dict_timing",
    "rsc_status_string", "rsc_last_cuda_error", "rsc_version", "rsc_encode_noalloc",
    "rsc_ksvd_update", "rsc_basis_create", "rsc_basis_destroy", "rsc_basis_info", "rsc_project",
    "rsc_encode_images", "rsc_ksvd_accumulate", "rsc_ksvd_finish", "rsc_reconstruct",
    "rsc_synthesize", "rsc_classify_images", "rsc_workspace_bytes", "rsc_dict_set_limits",
    "rsc_dict_set_tuning", "rsc_dict_tuning", "rsc_tuning_table_lookup",
)


class rsc_dims(ctypes.Structure):
    _fields_ = [("M", ctypes.c_int32), ("J", ctypes.c_int32), ("kmax", ctypes.c_int32),
                ("R", ctypes.c_int32)]


class rsc_tuning(ctypes.Structure):
    _fields_ = [("groups", ctypes.c_int32), ("group_min", ctypes.c_int32),
                ("refine_blocks_per_sm", ctypes.c_int32), ("score_stages", ctypes.c_int32),
                ("source", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class RscError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        msg = f"{what}: {rsc_status_string(status)} ({status})"
        if status == RSC_ERR_CUDA:
            msg += f" [{rsc_last_cuda_error()}]"
        super().__init__(msg)


_lib = None


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Loads librsc.so (built by ``build.build()``); raises if it is absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"librsc.so not built ({path}); run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    lib.rsc_dict_create.argtypes = [vp, rsc_dims, vp, ctypes.POINTER(vp)]
    lib.rsc_dict_destroy.argtypes = [vp]
    lib.rsc_dict_dims.argtypes = [vp, ctypes.POINTER(rsc_dims)]
    lib.rsc_encode.argtypes = [vp, vp, i64, i32, i32, vp, vp, vp, vp, vp, vp]
    lib.rsc_encode_host.argtypes = [vp, vp, i64, i32, i32, vp, vp, vp, vp, vp]
    lib.rsc_encode_noalloc.argtypes = [vp, vp, i64, i32, vp, vp, vp, vp, vp, vp]
    lib.rsc_ksvd_update.argtypes = [vp, vp, i64, i32, vp, vp, vp, vp, vp, vp]
    lib.rsc_ksvd_accumulate.argtypes = [vp, vp, i64, i32, vp, vp, vp, vp, vp, vp, vp, vp, i32, vp]
    lib.rsc_ksvd_finish.argtypes = [vp, vp, vp, vp, vp, i32, vp, vp, vp]
    lib.rsc_basis_create.argtypes = [i32, i32, i32, ctypes.c_double, ctypes.c_double,
                                     ctypes.POINTER(vp)]
    lib.rsc_basis_destroy.argtypes = [vp]
    lib.rsc_basis_info.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(i32)]
    lib.rsc_project.argtypes = [vp, vp, i32, i32, vp, vp]
    lib.rsc_reconstruct.argtypes = [vp, i64, i32, vp, vp, vp, vp, vp]
    lib.rsc_synthesize.argtypes = [vp, vp, i64, vp, vp]
    lib.rsc_classify_images.argtypes = [ctypes.POINTER(vp), i32, vp, ctypes.POINTER(vp),
                                        ctypes.POINTER(i32), ctypes.POINTER(i32), i32, i32, i32,
                                        vp, vp, vp]
    lib.rsc_encode_images.argtypes = [vp, vp, ctypes.POINTER(vp), ctypes.POINTER(i32),
                                      ctypes.POINTER(i32), i32, i32, i32, vp, vp, vp, vp, vp, vp]
    lib.rsc_workspace_bytes.argtypes = [vp, vp, i64, i32, i32, i32, ctypes.POINTER(ctypes.c_uint64)]
    lib.rsc_workspace_bytes.restype = ctypes.c_int
    lib.rsc_dict_check.argtypes = [vp, vp]
    lib.rsc_dict_fallback_count.argtypes = [vp, ctypes.POINTER(i64)]
    lib.rsc_dict_set_timing.argtypes = [vp, ctypes.c_int]
    lib.rsc_dict_set_limits.argtypes = [vp, ctypes.c_uint64, ctypes.c_uint64]
    lib.rsc_dict_set_limits.restype = ctypes.c_int
    lib.rsc_dict_set_tuning.argtypes = [vp, ctypes.POINTER(rsc_tuning)]
    lib.rsc_dict_set_tuning.restype = ctypes.c_int
    lib.rsc_dict_tuning.argtypes = [vp, i32, ctypes.POINTER(rsc_tuning)]
    lib.rsc_dict_tuning.restype = ctypes.c_int
    lib.rsc_tuning_table_lookup.argtypes = [ctypes.c_char_p, i32, i32, i32, i32,
                                            ctypes.POINTER(rsc_tuning)]
    lib.rsc_tuning_table_lookup.restype = ctypes.c_int
    lib.rsc_dict_timing.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(i64)]
    lib.rsc_status_string.argtypes = [ctypes.c_int]
    lib.rsc_status_string.restype = ctypes.c_char_p
    lib.rsc_last_cuda_error.argtypes = []
    lib.rsc_last_cuda_error.restype = ctypes.c_char_p
    lib.rsc_version.argtypes = []
    for name in ("rsc_dict_create", "rsc_dict_destroy", "rsc_dict_dims", "rsc_encode",
                 "rsc_encode_host", "rsc_dict_check", "rsc_dict_fallback_count",
                 "rsc_dict_set_timing", "rsc_dict_timing", "rsc_version", "rsc_encode_noalloc",
                 "rsc_ksvd_update", "rsc_basis_create", "rsc_basis_destroy", "rsc_basis_info",
                 "rsc_project", "rsc_encode_images"):
        getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


# ----------------------------------------------------------- raw C-ABI calls

def rsc_status_string(status: int) -> str:
    return load_library().rsc_status_string(int(status)).decode()


def rsc_last_cuda_error() -> str:
    return load_library().rsc_last_cuda_error().decode()


def rsc_version() -> int:
    return load_library().rsc_version()


def rsc_dict_create(coef_ptr: int, M: int, J: int, kmax: int, R: int, stream: int = 0) -> int:
    """Returns the handle (int) or raises RscError."""
    h = ctypes.c_void_p()
    st = load_library().rsc_dict_create(ctypes.c_void_p(coef_ptr), rsc_dims(M, J, kmax, R),
                                        ctypes.c_void_p(stream), ctypes.byref(h))
    if st != RSC_OK:
        raise RscError(st, "rsc_dict_create")
    return h.value


def rsc_dict_destroy(handle: int) -> int:
    return load_library().rsc_dict_destroy(ctypes.c_void_p(handle))


def rsc_encode(handle: int, x_ptr: int, P: int, K: int, prec: int, atom_ptr: int, angle_idx_ptr: int,
               angle_ptr: int, coef_ptr: int, resid_norm2_ptr: int, stream: int = 0) -> int:
    """Raw call; returns the status code."""
    vp = ctypes.c_void_p
    return load_library().rsc_encode(vp(handle), vp(x_ptr), int(P), int(K), int(prec), vp(atom_ptr),
                                     vp(angle_idx_ptr), vp(angle_ptr or None), vp(coef_ptr),
                                     vp(resid_norm2_ptr or None), vp(stream))


def rsc_encode_host(handle: int, x_ptr: int, P: int, K: int, prec: int, atom_ptr: int,
                    angle_idx_ptr: int, angle_ptr: int, coef_ptr: int, resid_norm2_ptr: int) -> int:
    vp = ctypes.c_void_p
    return load_library().rsc_encode_host(vp(handle), vp(x_ptr), int(P), int(K), int(prec),
                                          vp(atom_ptr), vp(angle_idx_ptr), vp(angle_ptr or None),
                                          vp(coef_ptr), vp(resid_norm2_ptr or None))


def rsc_encode_noalloc(handle: int, x_ptr: int, P: int, K: int, atom_ptr: int, angle_idx_ptr: int,
                       angle_ptr: int, coef_ptr: int, resid_norm2_ptr: int, stream: int = 0) -> int:
    """Raw call of the allocation-free FP16 entry point; returns the status."""
    vp = ctypes.c_void_p
    return load_library().rsc_encode_noalloc(vp(handle), vp(x_ptr), int(P), int(K), vp(atom_ptr),
                                             vp(angle_idx_ptr), vp(angle_ptr or None),
                                             vp(coef_ptr), vp(resid_norm2_ptr or None), vp(stream))


def rsc_ksvd_update(handle: int, x_ptr: int, P: int, K: int, atom_ptr: int, angle_idx_ptr: int,
                    coef_ptr: int, new_coef_ptr: int, n_used_ptr: int, stream: int = 0) -> int:
    """Raw call of the rotational K-SVD dictionary update; returns the status."""
    vp = ctypes.c_void_p
    return load_library().rsc_ksvd_update(vp(handle), vp(x_ptr), int(P), int(K), vp(atom_ptr),
                                          vp(angle_idx_ptr), vp(coef_ptr), vp(new_coef_ptr),
                                          vp(n_used_ptr or None), vp(stream))


def rsc_workspace_bytes(handle: int, basis_handle, P: int, n_images: int, K: int, prec: int) -> int:
    """Device scratch (bytes) one rsc_encode (basis_handle None) or
    rsc_encode_images call on P patches takes; raises RscError."""
    v = ctypes.c_uint64()
    st = load_library().rsc_workspace_bytes(ctypes.c_void_p(handle),
                                            ctypes.c_void_p(basis_handle or None), int(P),
                                            int(n_images), int(K), int(prec), ctypes.byref(v))
    if st != RSC_OK:
        raise RscError(st, "rsc_workspace_bytes")
    return v.value


def rsc_dict_check(handle: int, stream: int = 0) -> int:
    return load_library().rsc_dict_check(ctypes.c_void_p(handle), ctypes.c_void_p(stream))


def rsc_dict_fallback_count(handle: int) -> int:
    v = ctypes.c_int64()
    st = load_library().rsc_dict_fallback_count(ctypes.c_void_p(handle), ctypes.byref(v))
    if st != RSC_OK:
        raise RscError(st, "rsc_dict_fallback_count")
    return v.value


def rsc_dict_set_timing(handle: int, enable) -> int:
    """enable: False/0 off, True/1 on, 2 on with the FP16 path's halves run
    one after the other (each kernel timed alone)."""
    return load_library().rsc_dict_set_timing(ctypes.c_void_p(handle), int(enable))


def rsc_dict_set_limits(handle: int, pipeline_wait_ns: int = 0, scratch_limit: int = 0) -> int:
    """Diagnostic limits for testing the error paths (0 = default): the FP16
    scoring kernel's pipeline wait limit and the FP16 path's scratch budget."""
    return load_library().rsc_dict_set_limits(ctypes.c_void_p(handle), int(pipeline_wait_ns),
                                              int(scratch_limit))


def rsc_dict_set_tuning(handle: int, groups: int = 0, group_min: int = 0,
                        refine_blocks_per_sm: int = 0, score_stages: int = 0, clear: bool = False):
    """Tuning overrides of a dictionary (0 = not set); clear=True removes them."""
    t = None if clear else rsc_tuning(groups, group_min, refine_blocks_per_sm, score_stages, 0)
    st = load_library().rsc_dict_set_tuning(ctypes.c_void_p(handle),
                                            None if t is None else ctypes.byref(t))
    if st != RSC_OK:
        raise RscError(st, "rsc_dict_set_tuning")


def rsc_dict_tuning(handle: int, K: int) -> dict:
    """The tuning an encode with K steps uses (fields and their source)."""
    t = rsc_tuning()
    st = load_library().rsc_dict_tuning(ctypes.c_void_p(handle), int(K), ctypes.byref(t))
    if st != RSC_OK:
        raise RscError(st, "rsc_dict_tuning")
    return t.as_dict()


def rsc_tuning_table_lookup(path: str, n: int, M: int, R: int, K: int) -> dict:
    t = rsc_tuning()
    st = load_library().rsc_tuning_table_lookup(path.encode(), n, M, R, K, ctypes.byref(t))
    if st != RSC_OK:
        raise RscError(st, "rsc_tuning_table_lookup")
    return t.as_dict()


def rsc_dict_timing(handle: int):
    """Returns ([ms per phase], [launches per phase]) for phases 0 (scoring),
    1 (FP32 hand-off) and 2 (refine)."""
    ms = (ctypes.c_double * 3)()
    n = (ctypes.c_int64 * 3)()
    st = load_library().rsc_dict_timing(ctypes.c_void_p(handle), ms, n)
    if st != RSC_OK:
        raise RscError(st, "rsc_dict_timing")
    return list(ms), list(n)


# ----------------------------------------------------------- torch helpers

def _stream_handle(stream) -> int:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


class Dictionary:
    """Owns an rsc_dict handle built from a CUDA float32 tensor [M, kmax+1, J, 2]."""

    def __init__(self, d, R: int, stream=None):
        import torch
        if not (isinstance(d, torch.Tensor) and d.is_cuda and d.dtype == torch.float32):
            raise TypeError("dictionary must be a CUDA float32 tensor [M, kmax+1, J, 2]")
        d = d.contiguous()
        M, H, J, two = d.shape
        if two != 2:
            raise ValueError("last dimension must be (re, im)")
        self.M, self.J, self.kmax, self.R, self.H = M, J, H - 1, int(R), H
        self.handle = rsc_dict_create(d.data_ptr(), M, J, H - 1, int(R), _stream_handle(stream))

    def close(self):
        if getattr(self, "handle", None):
            rsc_dict_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def encode(dic: Dictionary, x, K: int, precision: str = "fp32", stream=None, out=None):
    """rsc_encode on CUDA tensors.  x: float32 [P, kmax+1, J, 2] on the
    dictionary's device.  Returns a dict of output tensors (atom, angle_idx,
    angle, coef, resid_norm2); ``out`` may hold preallocated ones."""
    import torch
    if not (x.is_cuda and x.dtype == torch.float32 and x.is_contiguous()):
        raise TypeError("x must be a contiguous CUDA float32 tensor")
    P = x.shape[0]
    dev = x.device
    if out is None:
        out = {
            "atom": torch.empty((P, K), dtype=torch.int32, device=dev),
            "angle_idx": torch.empty((P, K), dtype=torch.int32, device=dev),
            "angle": torch.empty((P, K), dtype=torch.float32, device=dev),
            "coef": torch.empty((P, K), dtype=torch.float64, device=dev),
            "resid_norm2": torch.empty((P,), dtype=torch.float32, device=dev),
        }
    st = rsc_encode(dic.handle, x.data_ptr(), P, K, PRECISIONS[precision], out["atom"].data_ptr(),
                    out["angle_idx"].data_ptr(), out["angle"].data_ptr(), out["coef"].data_ptr(),
                    out["resid_norm2"].data_ptr(), _stream_handle(stream))
    if st != RSC_OK:
        raise RscError(st, "rsc_encode")
    return out


def encode_host(dic: Dictionary, x, K: int, precision: str = "fp32", out=None):
    """rsc_encode_host on host (ideally pinned) CPU tensors; blocks."""
    import torch
    if x.is_cuda or x.dtype != torch.float32 or not x.is_contiguous():
        raise TypeError("x must be a contiguous CPU float32 tensor")
    P = x.shape[0]
    if out is None:
        out = {
            "atom": torch.empty((P, K), dtype=torch.int32),
            "angle_idx": torch.empty((P, K), dtype=torch.int32),
            "angle": torch.empty((P, K), dtype=torch.float32),
            "coef": torch.empty((P, K), dtype=torch.float64),
            "resid_norm2": torch.empty((P,), dtype=torch.float32),
        }
    st = rsc_encode_host(dic.handle, x.data_ptr(), P, K, PRECISIONS[precision],
                         out["atom"].data_ptr(), out["angle_idx"].data_ptr(),
                         out["angle"].data_ptr(), out["coef"].data_ptr(),
                         out["resid_norm2"].data_ptr())
    if st != RSC_OK:
        raise RscError(st, "rsc_encode_host")
    return out


def ksvd_update(dic: Dictionary, x, codes: dict, stream=None):
    """rsc_ksvd_update on CUDA tensors: x [P, kmax+1, J, 2] float32 and the
    codes returned by encode().  Returns (new atoms [M, kmax+1, J, 2] float32,
    n_used [M] int32)."""
    import torch
    P, K = codes["atom"].shape
    new = torch.empty((dic.M, dic.H, dic.J, 2), dtype=torch.float32, device=x.device)
    used = torch.empty((dic.M,), dtype=torch.int32, device=x.device)
    st = rsc_ksvd_update(dic.handle, x.data_ptr(), P, K, codes["atom"].data_ptr(),
                         codes["angle_idx"].data_ptr(), codes["coef"].data_ptr(), new.data_ptr(),
                         used.data_ptr(), _stream_handle(stream))
    if st != RSC_OK:
        raise RscError(st, "rsc_ksvd_update")
    return new, used


KSVD_TOP = 64  # patches of largest coding error kept per rank for the atom resets


def ksvd_accumulate(dic: Dictionary, x, codes: dict, ntop: int = KSVD_TOP, stream=None):
    """rsc_ksvd_accumulate on CUDA tensors: this rank's share of an R-K-SVD
    update.  Returns dict(C [M, n, n] float64, count [M] int32, top_err
    [ntop] float32, top_idx [ntop] int64, top_vec [ntop, kmax+1, J, 2])."""
    import torch
    P, K = codes["atom"].shape
    n = dic.J * (2 * dic.kmax + 1)
    dev = x.device
    out = {"C": torch.empty((dic.M, n, n), dtype=torch.float64, device=dev),
           "count": torch.empty((dic.M,), dtype=torch.int32, device=dev),
           "top_err": torch.empty((ntop,), dtype=torch.float32, device=dev),
           "top_idx": torch.empty((ntop,), dtype=torch.int64, device=dev),
           "top_vec": torch.empty((ntop, dic.H, dic.J, 2), dtype=torch.float32, device=dev)}
    st = load_library().rsc_ksvd_accumulate(
        ctypes.c_void_p(dic.handle), ctypes.c_void_p(x.data_ptr()), P, K,
        ctypes.c_void_p(codes["atom"].data_ptr()), ctypes.c_void_p(codes["angle_idx"].data_ptr()),
        ctypes.c_void_p(codes["coef"].data_ptr()), ctypes.c_void_p(out["C"].data_ptr()),
        ctypes.c_void_p(out["count"].data_ptr()), ctypes.c_void_p(out["top_err"].data_ptr()),
        ctypes.c_void_p(out["top_idx"].data_ptr()), ctypes.c_void_p(out["top_vec"].data_ptr()),
        ntop, ctypes.c_void_p(_stream_handle(stream)))
    if st != RSC_OK:
        raise RscError(st, "rsc_ksvd_accumulate")
    return out


def ksvd_finish(dic: Dictionary, C, count, top_idx, top_vec, stream=None):
    """rsc_ksvd_finish on CUDA tensors (sums over the ranks and the merged
    top list).  Returns (new atoms, n_used)."""
    import torch
    new = torch.empty((dic.M, dic.H, dic.J, 2), dtype=torch.float32, device=C.device)
    used = torch.empty((dic.M,), dtype=torch.int32, device=C.device)
    st = load_library().rsc_ksvd_finish(
        ctypes.c_void_p(dic.handle), ctypes.c_void_p(C.data_ptr()),
        ctypes.c_void_p(count.data_ptr()), ctypes.c_void_p(top_idx.data_ptr()),
        ctypes.c_void_p(top_vec.data_ptr()), int(top_idx.shape[0]),
        ctypes.c_void_p(new.data_ptr()), ctypes.c_void_p(used.data_ptr()),
        ctypes.c_void_p(_stream_handle(stream)))
    if st != RSC_OK:
        raise RscError(st, "rsc_ksvd_finish")
    return new, used


class Basis:
    """Owns an rsc_basis handle (steerable basis + analysis operator)."""

    def __init__(self, N: int, J: int, kmax: int, ring_width: float = 0.0,
                 ring_spacing: float = 0.0):
        lib = load_library()
        h = ctypes.c_void_p()
        st = lib.rsc_basis_create(N, J, kmax, ring_width, ring_spacing, ctypes.byref(h))
        if st != RSC_OK:
            raise RscError(st, "rsc_basis_create")
        self.handle = h.value
        self.N, self.J, self.kmax, self.H = N, J, kmax, kmax + 1
        npix, n = ctypes.c_int32(), ctypes.c_int32()
        lib.rsc_basis_info(ctypes.c_void_p(self.handle), ctypes.byref(npix), ctypes.byref(n))
        self.npix, self.n = npix.value, n.value

    def close(self):
        if getattr(self, "handle", None):
            load_library().rsc_basis_destroy(ctypes.c_void_p(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def project(basis: Basis, image, stream=None):
    """rsc_project: coefficients of every stride-1 window of a CUDA float32
    image [h, w] -> [(h-N+1)(w-N+1), kmax+1, J, 2]."""
    import torch
    image = image.contiguous()
    h, w = image.shape
    P = max(h - basis.N + 1, 0) * max(w - basis.N + 1, 0)
    out = torch.empty((P, basis.H, basis.J, 2), dtype=torch.float32, device=image.device)
    st = load_library().rsc_project(ctypes.c_void_p(basis.handle), ctypes.c_void_p(image.data_ptr()),
                                    h, w, ctypes.c_void_p(out.data_ptr() if P else None),
                                    ctypes.c_void_p(_stream_handle(stream)))
    if st != RSC_OK:
        raise RscError(st, "rsc_project")
    return out


def reconstruct(dic: Dictionary, codes: dict, stream=None):
    """rsc_reconstruct: sum_i a_i S_{r_i} d_{m_i} of each patch's code (CUDA
    tensors atom, angle_idx [P, K] int32, coef [P, K] float64) -> half
    spectra [P, kmax+1, J, 2] float32."""
    import torch
    atom = codes["atom"].contiguous()
    ang = codes["angle_idx"].contiguous()
    coef = codes["coef"].contiguous()
    P, K = atom.shape
    out = torch.empty((P, dic.kmax + 1, dic.J, 2), dtype=torch.float32, device=atom.device)
    st = load_library().rsc_reconstruct(ctypes.c_void_p(dic.handle), P, K,
                                        ctypes.c_void_p(atom.data_ptr()),
                                        ctypes.c_void_p(ang.data_ptr()),
                                        ctypes.c_void_p(coef.data_ptr()),
                                        ctypes.c_void_p(out.data_ptr()),
                                        ctypes.c_void_p(_stream_handle(stream)))
    if st != RSC_OK:
        raise RscError(st, "rsc_reconstruct")
    return out


def synthesize(basis: Basis, coef, stream=None):
    """rsc_synthesize: pixels Phi x_hat of the circular patch for CUDA half
    spectra [P, kmax+1, J, 2] float32 -> [P, npix] float32 (the masked
    pixels in row-major order)."""
    import torch
    coef = coef.contiguous()
    P = coef.shape[0]
    out = torch.empty((P, basis.npix), dtype=torch.float32, device=coef.device)
    st = load_library().rsc_synthesize(ctypes.c_void_p(basis.handle), ctypes.c_void_p(coef.data_ptr()),
                                       P, ctypes.c_void_p(out.data_ptr()),
                                       ctypes.c_void_p(_stream_handle(stream)))
    if st != RSC_OK:
        raise RscError(st, "rsc_synthesize")
    return out


def classify_images(dicts, basis: Basis, images, K: int, precision: str = "f16", stream=None):
    """rsc_classify_images: windows of CUDA float32 images coded with each
    Dictionary in `dicts`; returns (labels [P] int32, hist [n_images, C]
    int32), the label being the index of the dictionary with the least
    squared coding error."""
    import torch
    images = [im.contiguous() for im in images]
    N = basis.N
    P = sum(max(im.shape[0] - N + 1, 0) * max(im.shape[1] - N + 1, 0) for im in images)
    dev = images[0].device if images else torch.device("cuda")
    C, n = len(dicts), len(images)
    labels = torch.empty((max(P, 1),), dtype=torch.int32, device=dev)
    hist = torch.empty((max(n, 1), C), dtype=torch.int32, device=dev)
    hs_ = (ctypes.c_void_p * C)(*[dd.handle for dd in dicts])
    ptrs = (ctypes.c_void_p * max(n, 1))(*[im.data_ptr() for im in images])
    hs = (ctypes.c_int32 * max(n, 1))(*[im.shape[0] for im in images])
    ws = (ctypes.c_int32 * max(n, 1))(*[im.shape[1] for im in images])
    st = load_library().rsc_classify_images(
        hs_, C, ctypes.c_void_p(basis.handle), ptrs, hs, ws, n, K, PRECISIONS[precision],
        ctypes.c_void_p(labels.data_ptr()), ctypes.c_void_p(hist.data_ptr()),
        ctypes.c_void_p(_stream_handle(stream)))
    if st != RSC_OK:
        raise RscError(st, "rsc_classify_images")
    return labels[:P], hist[:n]


def encode_images(dic: Dictionary, basis: Basis, images, K: int, precision: str = "fp32",
                  stream=None):
    """rsc_encode_images on a list of CUDA float32 images [h_i, w_i]."""
    import torch
    images = [im.contiguous() for im in images]
    N = basis.N
    P = sum(max(im.shape[0] - N + 1, 0) * max(im.shape[1] - N + 1, 0) for im in images)
    dev = images[0].device if images else torch.device("cuda")
    out = {
        "atom": torch.empty((P, K), dtype=torch.int32, device=dev),
        "angle_idx": torch.empty((P, K), dtype=torch.int32, device=dev),
        "angle": torch.empty((P, K), dtype=torch.float32, device=dev),
        "coef": torch.empty((P, K), dtype=torch.float64, device=dev),
        "resid_norm2": torch.empty((P,), dtype=torch.float32, device=dev),
    }
    n = len(images)
    ptrs = (ctypes.c_void_p * max(n, 1))(*[im.data_ptr() for im in images])
    hs = (ctypes.c_int32 * max(n, 1))(*[im.shape[0] for im in images])
    ws = (ctypes.c_int32 * max(n, 1))(*[im.shape[1] for im in images])
    st = load_library().rsc_encode_images(
        ctypes.c_void_p(dic.handle), ctypes.c_void_p(basis.handle), ptrs, hs, ws, n, K,
        PRECISIONS[precision], *[ctypes.c_void_p(out[k].data_ptr() if P else None)
                                 for k in ("atom", "angle_idx", "angle", "coef", "resid_norm2")],
        ctypes.c_void_p(_stream_handle(stream)))
    if st != RSC_OK:
        raise RscError(st, "rsc_encode_images")
    return out
