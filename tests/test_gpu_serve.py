"""The continuous-batching server (paper_1806_04374_gb300/serve.py) on the GPU:
each request's codes are the same alone, in a mix of overlapping and batched
requests, and from a direct rsc_encode_images call; admission by device
memory refuses a request larger than the budget and holds one that does not
fit beside a running request until that request's memory is released."""
import numpy as np
import pytest

from paper_1806_04374_gb300 import synth

pytestmark = pytest.mark.gpu

N, J, KMAX, M, R, K = 11, 6, 8, 32, 32, 5


@pytest.fixture(scope="module")
def setup(cuda_ok):
    import torch
    import paper_1806_04374_gb300 as rsc
    rsc.load_library()
    basis = rsc.Basis(N, J, KMAX)
    dic = rsc.Dictionary(torch.from_numpy(synth.make_dictionary(M, J, KMAX, 20180801)).cuda(), R)
    rng = np.random.default_rng(20180802)
    sides = [(int(a), int(b)) for a, b in rng.integers(14, 140, size=(9, 2))] + [(11, 11), (8, 30)]
    images = [synth.make_line_image(h, w, 0.01, 20180803 + i) for i, (h, w) in enumerate(sides)]
    yield rsc, dic, basis, images
    dic.close()
    basis.close()


def _equal(a, b):
    return all(np.array_equal(a[k], b[k]) for k in ("atom", "angle_idx", "angle", "coef",
                                                    "resid_norm2"))


@pytest.mark.parametrize("precision", ["f16", "fp32"])
def test_codes_same_alone_and_in_the_mix(setup, precision):
    import torch
    from paper_1806_04374_gb300 import serve
    rsc, dic, basis, images = setup
    # alone: one slot, no batching, each request submitted after the previous
    alone = []
    with serve.Server(dic, basis, K, precision, slots=1, batch_windows=1) as srv:
        for im in images:
            r = srv.submit(im)
            alone.append(r.result(timeout=60))
            assert r.batch_size == 1
    # in the mix: three slots, batching, everything submitted at once
    with serve.Server(dic, basis, K, precision, slots=3, batch_windows=20000) as srv:
        reqs = [srv.submit(im) for im in images]
        mixed = [r.result(timeout=60) for r in reqs]
        assert max(r.batch_size for r in reqs) > 1  # some were batched
    for i, (a, b) in enumerate(zip(alone, mixed)):
        assert a["atom"].shape[0] == reqs[i].windows
        assert _equal(a, b), i
    # and a direct call on one image gives the same codes
    d = rsc.encode_images(dic, basis, [torch.from_numpy(images[3]).cuda()], K, precision)
    torch.cuda.synchronize()
    assert _equal({k: v.cpu().numpy() for k, v in d.items()}, alone[3])
    assert rsc.rsc_dict_check(dic.handle) == 0


def test_admission_by_device_memory(setup):
    from paper_1806_04374_gb300 import serve
    rsc, dic, basis, images = setup
    big = synth.make_line_image(200, 180, 0.01, 20180810)
    mid = synth.make_line_image(150, 160, 0.01, 20180811)
    probe = serve.Server(dic, basis, K, "f16", mem_budget=1 << 40, slots=1)
    a_need = probe.need_bytes([serve.Request(0, big, N)])
    b_need = probe.need_bytes([serve.Request(1, mid, N)])
    probe.close()
    budget = a_need + b_need // 2  # each fits alone, not both at once
    with serve.Server(dic, basis, K, "f16", mem_budget=budget, slots=2,
                      batch_windows=1 << 20) as srv:
        with pytest.raises(serve.AdmissionError):
            srv.submit(synth.make_line_image(400, 400, 0.01, 20180812))
        ra = srv.submit(big)
        rb = srv.submit(mid)
        ca, cb = ra.result(timeout=60), rb.result(timeout=60)
        # b was admitted only after a finished and released its memory, even
        # though a second slot was free
        assert rb.t_admit >= ra.t_done
        assert srv.peak_reserved <= budget
    assert ca["atom"].shape[0] == ra.windows and cb["atom"].shape[0] == rb.windows
    # the codes are those of the images coded alone
    with serve.Server(dic, basis, K, "f16", slots=1) as srv:
        assert _equal(srv.submit(mid).result(timeout=60), cb)


class _Gate:
    """Wraps encode_images: calls wait until the test opens the gate, and a
    call whose batch holds an image of shape `poison` raises (a failure made
    on the host, before any device work)."""

    def __init__(self, rsc, poison=None):
        import threading
        self.real, self.poison = rsc.encode_images, poison
        self.open = threading.Event()
        self.calls = []

    def __call__(self, dic, basis, imgs, K, precision, **kw):
        self.open.wait(60)
        shapes = [tuple(im.shape) for im in imgs]
        self.calls.append(shapes)
        if self.poison in shapes:
            raise RuntimeError("injected failure")
        return self.real(dic, basis, imgs, K, precision, **kw)


def test_cancel_before_admission(setup, monkeypatch):
    from paper_1806_04374_gb300 import serve
    rsc, dic, basis, images = setup
    gate = _Gate(rsc)
    monkeypatch.setattr(rsc, "encode_images", gate)
    with serve.Server(dic, basis, K, "f16", slots=1, batch_windows=1) as srv:
        ra = srv.submit(images[0])
        for _ in range(600):  # the one worker has taken ra and waits at the gate
            if ra.t_admit is not None:
                break
            import time
            time.sleep(0.01)
        assert ra.t_admit is not None
        rb, rc = srv.submit(images[1]), srv.submit(images[2])
        assert rb.cancel() and not rb.cancel()
        assert not ra.cancel()  # already taken
        gate.open.set()
        ca, cc = ra.result(timeout=60), rc.result(timeout=60)
        with pytest.raises(serve.Cancelled):
            rb.result(timeout=60)
    assert len(gate.calls) == 2  # rb was never coded
    # the others' codes are those of a direct call
    monkeypatch.undo()
    for im, c in ((images[0], ca), (images[2], cc)):
        import torch
        d = rsc.encode_images(dic, basis, [torch.from_numpy(im).cuda()], K, "f16")
        assert _equal({k: v.cpu().numpy() for k, v in d.items()}, c)


def test_a_failing_request_fails_alone(setup, monkeypatch):
    from paper_1806_04374_gb300 import serve
    rsc, dic, basis, images = setup
    bad = synth.make_line_image(37, 41, 0.01, 20180813)
    with serve.Server(dic, basis, K, "f16", slots=1, batch_windows=1 << 20) as srv:
        clean = [srv.submit(im).result(timeout=60) for im in images[:4]]
    gate = _Gate(rsc, poison=bad.shape)
    monkeypatch.setattr(rsc, "encode_images", gate)
    with serve.Server(dic, basis, K, "f16", slots=1, batch_windows=1 << 20) as srv:
        first = srv.submit(images[0])  # taken at once, held at the gate
        for _ in range(600):
            if first.t_admit is not None:
                break
            import time
            time.sleep(0.01)
        rest = [srv.submit(im) for im in (images[1], bad, images[2], images[3])]
        gate.open.set()
        assert _equal(first.result(timeout=60), clean[0])
        with pytest.raises(RuntimeError, match="injected"):
            rest[1].result(timeout=60)
        for r, c in zip((rest[0], rest[2], rest[3]), clean[1:]):
            assert _equal(r.result(timeout=60), c)
        # the queued four went in one call, which failed; then one call each
        assert max(len(c) for c in gate.calls) == 4
        assert sum(1 for c in gate.calls if len(c) == 1) >= 4
        # and the server goes on serving
        assert _equal(srv.submit(images[1]).result(timeout=60), clean[1])
