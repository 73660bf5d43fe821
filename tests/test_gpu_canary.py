"""Guard regions around every output: each entry point is called through the
C ABI with its outputs placed between two guard regions of a known byte
pattern, on ragged sizes (a partial last tile, partial warps), and must
leave the guards untouched and write every entry of its outputs.  A write
past either end of an output -- a tile or lane index that a bounds check
misses -- shows up as a changed guard byte."""
import ctypes

import numpy as np
import pytest

from paper_1806_04374_gb300 import synth

pytestmark = pytest.mark.gpu

GUARD = 64        # elements on each side (keeps every output 16-byte aligned)
PATTERN = 0xA5    # guard and fill byte


class Guarded:
    """A device tensor of `shape` inside a buffer with GUARD elements of
    guard before and after it, all bytes set to PATTERN."""

    def __init__(self, torch, shape, dtype):
        n = int(np.prod(shape))
        self.buf = torch.empty(n + 2 * GUARD, dtype=dtype, device="cuda")
        self.buf.view(torch.uint8).fill_(PATTERN)
        self.t = self.buf[GUARD:GUARD + n].view(*shape)
        self.esize = self.buf.element_size()

    @property
    def ptr(self):
        return ctypes.c_void_p(self.t.data_ptr())

    def guards_intact(self) -> bool:
        import torch
        b = self.buf.view(torch.uint8)
        nb = GUARD * self.esize
        return bool((b[:nb] == PATTERN).all().item()) and bool((b[-nb:] == PATTERN).all().item())

    def all_written(self) -> bool:
        """No element of the output still holds the fill pattern."""
        import torch
        v = self.t.reshape(-1).view(torch.uint8).reshape(-1, self.esize)
        return not bool((v == PATTERN).all(dim=1).any().item())


@pytest.fixture(scope="module")
def env(cuda_ok):
    import torch
    import paper_1806_04374_gb300 as rsc
    lib = rsc.load_library()
    M, J, kmax, R, K = 24, 6, 8, 32, 3
    d = synth.make_dictionary(M, J, kmax, 20181211)
    dic = rsc.Dictionary(torch.from_numpy(d).cuda(), R)
    basis = rsc.Basis(11, J, kmax)
    yield rsc, lib, torch, dic, basis, d, (M, J, kmax, R, K)
    dic.close()
    basis.close()


def _codes(torch, P, K):
    return {"atom": Guarded(torch, (P, K), torch.int32),
            "angle_idx": Guarded(torch, (P, K), torch.int32),
            "angle": Guarded(torch, (P, K), torch.float32),
            "coef": Guarded(torch, (P, K), torch.float64),
            "resid_norm2": Guarded(torch, (P,), torch.float32)}


def _check(outs, names=None):
    for k, g in outs.items():
        assert g.guards_intact(), f"{k}: guard region changed"
        if names is None or k in names:
            assert g.all_written(), f"{k}: entries left unwritten"


@pytest.mark.parametrize("prec", ["fp32", "fp32_prune", "f16"])
@pytest.mark.parametrize("P", [1, 37, 1037])
def test_encode_guards(env, prec, P):
    rsc, lib, torch, dic, basis, d, (M, J, kmax, R, K) = env
    x, _ = synth.make_patches(d, P, 2, 0.05, 20181212 + P)
    xd = torch.from_numpy(x).cuda()
    out = _codes(torch, P, K)
    st = torch.cuda.current_stream()
    rc = lib.rsc_encode(ctypes.c_void_p(dic.handle), ctypes.c_void_p(xd.data_ptr()), P, K,
                        rsc.PRECISIONS[prec], *[out[k].ptr for k in out],
                        ctypes.c_void_p(st.cuda_stream))
    assert rc == rsc.RSC_OK
    torch.cuda.synchronize()
    assert rsc.rsc_dict_check(dic.handle) == 0
    _check(out)
    a = out["atom"].t.cpu().numpy()
    assert ((a >= -1) & (a < M)).all()


@pytest.mark.parametrize("P", [37, 1037])
def test_noalloc_and_host_guards(env, P):
    rsc, lib, torch, dic, basis, d, (M, J, kmax, R, K) = env
    x, _ = synth.make_patches(d, P, 2, 0.05, 20181213 + P)
    xd = torch.from_numpy(x).cuda()
    out = _codes(torch, P, K)
    st = torch.cuda.current_stream()
    rc = lib.rsc_encode_noalloc(ctypes.c_void_p(dic.handle), ctypes.c_void_p(xd.data_ptr()), P,
                                K, *[out[k].ptr for k in out], ctypes.c_void_p(st.cuda_stream))
    assert rc == rsc.RSC_OK
    torch.cuda.synchronize()
    _check(out)
    # host buffers with guards
    hosts = {k: np.full(g.t.numel() + 2 * GUARD, 0, dtype=np.dtype(str(g.t.dtype).split(".")[1]))
             for k, g in out.items()}
    for h in hosts.values():
        h.view(np.uint8)[:] = PATTERN
    ptr = lambda h: ctypes.c_void_p(h[GUARD:].ctypes.data)  # noqa: E731
    rc = lib.rsc_encode_host(ctypes.c_void_p(dic.handle), ctypes.c_void_p(x.ctypes.data), P, K,
                             rsc.RSC_F16_RESCORE, *[ptr(hosts[k]) for k in out])
    assert rc == rsc.RSC_OK
    # the host entry point gives rsc_encode's codes (the fused coder behind
    # rsc_encode_noalloc agrees with them to ~1e-12 in the weights only)
    ref = rsc.encode(dic, xd, K, "f16")
    torch.cuda.synchronize()
    for k, h in hosts.items():
        g = h.view(np.uint8)
        nb = GUARD * h.itemsize
        assert (g[:nb] == PATTERN).all() and (g[-nb:] == PATTERN).all(), k
        assert np.array_equal(h[GUARD:-GUARD].reshape(out[k].t.shape), ref[k].cpu().numpy()), k


def _images(torch, sizes, seed):
    return [torch.from_numpy(synth.make_line_image(h, w, 0.01, seed + i)).cuda()
            for i, (h, w) in enumerate(sizes)]


SIZES = [(11, 11), (8, 30), (23, 41), (40, 17)]  # one window, none, ragged rows


def test_image_calls_guards(env):
    rsc, lib, torch, dic, basis, d, (M, J, kmax, R, K) = env
    imgs = _images(torch, SIZES, 20181214)
    N, n = basis.N, len(imgs)
    P = sum(max(h - N + 1, 0) * max(w - N + 1, 0) for h, w in SIZES)
    ptrs = (ctypes.c_void_p * n)(*[im.data_ptr() for im in imgs])
    hs = (ctypes.c_int32 * n)(*[h for h, _ in SIZES])
    ws = (ctypes.c_int32 * n)(*[w for _, w in SIZES])
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    # projection of one ragged image
    h, w = SIZES[2]
    coef = Guarded(torch, ((h - N + 1) * (w - N + 1), kmax + 1, J, 2), torch.float32)
    assert lib.rsc_project(ctypes.c_void_p(basis.handle), ctypes.c_void_p(imgs[2].data_ptr()),
                           h, w, coef.ptr, st) == rsc.RSC_OK
    torch.cuda.synchronize()
    assert coef.guards_intact() and coef.all_written()
    # project + code all images
    for prec in ("fp32", "f16"):
        out = _codes(torch, P, K)
        assert lib.rsc_encode_images(ctypes.c_void_p(dic.handle), ctypes.c_void_p(basis.handle),
                                     ptrs, hs, ws, n, K, rsc.PRECISIONS[prec],
                                     *[out[k].ptr for k in out], st) == rsc.RSC_OK
        torch.cuda.synchronize()
        _check(out)
    # classification with two dictionaries
    d2 = rsc.Dictionary(torch.from_numpy(synth.make_dictionary(M, J, kmax, 20181215)).cuda(), R)
    dicts = (ctypes.c_void_p * 2)(dic.handle, d2.handle)
    labels = Guarded(torch, (P,), torch.int32)
    hist = Guarded(torch, (n, 2), torch.int32)
    assert lib.rsc_classify_images(dicts, 2, ctypes.c_void_p(basis.handle), ptrs, hs, ws, n, K,
                                   rsc.RSC_F16_RESCORE, labels.ptr, hist.ptr, st) == rsc.RSC_OK
    torch.cuda.synchronize()
    assert labels.guards_intact() and labels.all_written()
    assert hist.guards_intact() and hist.all_written()
    assert hist.t.sum().item() == P
    d2.close()


def test_reconstruct_synthesize_ksvd_guards(env):
    rsc, lib, torch, dic, basis, d, (M, J, kmax, R, K) = env
    P = 1037
    x, _ = synth.make_patches(d, P, 2, 0.05, 20181216)
    xd = torch.from_numpy(x).cuda()
    codes = rsc.encode(dic, xd, K, "f16")
    torch.cuda.synchronize()
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rec = Guarded(torch, (P, kmax + 1, J, 2), torch.float32)
    assert lib.rsc_reconstruct(ctypes.c_void_p(dic.handle), P, K,
                               ctypes.c_void_p(codes["atom"].data_ptr()),
                               ctypes.c_void_p(codes["angle_idx"].data_ptr()),
                               ctypes.c_void_p(codes["coef"].data_ptr()), rec.ptr,
                               st) == rsc.RSC_OK
    torch.cuda.synchronize()
    assert rec.guards_intact() and rec.all_written()
    pix = Guarded(torch, (P, basis.npix), torch.float32)
    assert lib.rsc_synthesize(ctypes.c_void_p(basis.handle),
                              ctypes.c_void_p(rec.t.data_ptr()), P, pix.ptr, st) == rsc.RSC_OK
    torch.cuda.synchronize()
    assert pix.guards_intact() and pix.all_written()
    new = Guarded(torch, (M, kmax + 1, J, 2), torch.float32)
    used = Guarded(torch, (M,), torch.int32)
    assert lib.rsc_ksvd_update(ctypes.c_void_p(dic.handle), ctypes.c_void_p(xd.data_ptr()), P,
                               K, ctypes.c_void_p(codes["atom"].data_ptr()),
                               ctypes.c_void_p(codes["angle_idx"].data_ptr()),
                               ctypes.c_void_p(codes["coef"].data_ptr()), new.ptr, used.ptr,
                               st) == rsc.RSC_OK
    torch.cuda.synchronize()
    assert new.guards_intact() and used.guards_intact() and used.all_written()
