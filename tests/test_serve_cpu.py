"""Host logic of the continuous-batching server (CPU only): admission by a
device-memory budget, batching in arrival order, the batch-size limit,
withdrawal before admission and failure isolation.  The coding call, the
memory model and the CUDA streams are replaced by host stand-ins; the
scheduling code under test is the server's own."""
import threading
import time

import numpy as np
import pytest

from paper_1806_04374_gb300 import serve

N = 11


class _Dims:
    """Stands in for the dictionary and the basis (sizes only)."""
    J, kmax, N, handle = 6, 8, N, None


class HostServer(serve.Server):
    """serve.Server with the device parts replaced: a request of W windows
    needs 100 W + 1000 bytes, and a call returns, for each request, its id
    in every window's atom entry.  ``gate`` (an Event) holds every call until
    it is set; a request whose image has the shape ``poison`` makes the call
    that contains it raise."""

    def __init__(self, gate=None, poison=None, **kw):
        self.gate, self.poison, self.batches = gate, poison, []
        super().__init__(_Dims(), _Dims(), 5, "f16", **kw)

    def _make_streams(self, slots):
        self.device = None
        return [None] * slots

    def _bind(self):
        pass

    def need_bytes(self, requests):
        return sum(100 * r.windows + 1000 for r in requests)

    def _code(self, batch, stream):
        self.batches.append([r.id for r in batch])
        if self.gate is not None:
            assert self.gate.wait(30)
        if self.poison is not None and any(r.image.shape == self.poison for r in batch):
            raise RuntimeError("poisoned request")
        return [{"atom": np.full((r.windows, self.K), r.id, np.int32)} for r in batch]


def _img(side):
    return np.zeros((side, side), np.float32)


def _wait_for(cond, timeout=10.0):
    t0 = time.perf_counter()
    while not cond():
        assert time.perf_counter() - t0 < timeout
        time.sleep(0.001)


def test_refuses_a_request_larger_than_the_budget():
    with HostServer(mem_budget=10_000, slots=1) as srv:
        with pytest.raises(serve.AdmissionError):
            srv.submit(_img(N + 9))  # 100 windows: 11,000 bytes
        r = srv.submit(_img(N + 8))  # 81 windows: 9,100 bytes
        assert r.result(10)["atom"].shape == (81, 5)


def test_admission_waits_for_memory_to_be_released():
    gate = threading.Event()
    # two slots, but the budget holds one of the two requests at a time
    with HostServer(gate=gate, mem_budget=15_000, slots=2) as srv:
        a = srv.submit(_img(N + 9), rid=1)   # 11,000 bytes
        _wait_for(lambda: a.t_admit is not None)
        b = srv.submit(_img(N + 9), rid=2)
        time.sleep(0.05)
        assert b.t_admit is None and srv.reserved == a.need
        gate.set()
        assert np.all(a.result(10)["atom"] == 1) and np.all(b.result(10)["atom"] == 2)
        assert b.t_admit >= a.t_done
        assert srv.peak_reserved <= srv.mem_budget


def test_queued_requests_are_batched_in_arrival_order():
    gate = threading.Event()
    with HostServer(gate=gate, slots=1, batch_windows=1 << 20) as srv:
        first = srv.submit(_img(N + 1), rid=0)
        _wait_for(lambda: len(srv.batches) == 1)
        rest = [srv.submit(_img(N + 1 + i), rid=i + 1) for i in range(3)]
        gate.set()
        for r in [first] + rest:
            codes = r.result(10)["atom"]
            assert codes.shape == (r.windows, 5) and np.all(codes == r.id)
        assert srv.batches == [[0], [1, 2, 3]]
        assert [r.batch_size for r in rest] == [3, 3, 3]


def test_batch_window_limit_splits_the_queue():
    gate = threading.Event()
    # requests of 4 windows each, at most 8 windows a call
    with HostServer(gate=gate, slots=1, batch_windows=8) as srv:
        first = srv.submit(_img(N + 1), rid=0)
        _wait_for(lambda: len(srv.batches) == 1)
        rest = [srv.submit(_img(N + 1), rid=i + 1) for i in range(5)]
        gate.set()
        for r in [first] + rest:
            r.result(10)
        assert srv.batches == [[0], [1, 2], [3, 4], [5]]


def test_memory_limits_a_batch():
    gate = threading.Event()
    # 4-window requests need 1,400 bytes each; the budget holds two at a time
    with HostServer(gate=gate, slots=1, mem_budget=3_000, batch_windows=1 << 20) as srv:
        first = srv.submit(_img(N + 1), rid=0)
        _wait_for(lambda: len(srv.batches) == 1)
        rest = [srv.submit(_img(N + 1), rid=i + 1) for i in range(3)]
        gate.set()
        for r in [first] + rest:
            r.result(10)
        assert srv.batches == [[0], [1, 2], [3]]


def test_cancel_withdraws_only_a_request_not_yet_admitted():
    gate = threading.Event()
    with HostServer(gate=gate, slots=1) as srv:
        running = srv.submit(_img(N + 2), rid=0)
        _wait_for(lambda: len(srv.batches) == 1)
        queued = srv.submit(_img(N + 2), rid=1)
        assert queued.cancel()
        assert not running.cancel()
        gate.set()
        assert running.result(10)["atom"].shape == (9, 5)
        with pytest.raises(serve.Cancelled):
            queued.result(10)
        assert srv.batches == [[0]]


def test_a_failing_request_fails_alone():
    gate = threading.Event()
    with HostServer(gate=gate, poison=(N + 3, N + 3), slots=1) as srv:
        first = srv.submit(_img(N + 1), rid=0)
        _wait_for(lambda: len(srv.batches) == 1)
        ok1 = srv.submit(_img(N + 1), rid=1)
        bad = srv.submit(_img(N + 3), rid=2)
        ok2 = srv.submit(_img(N + 2), rid=3)
        gate.set()
        first.result(10)
        assert np.all(ok1.result(10)["atom"] == 1) and np.all(ok2.result(10)["atom"] == 3)
        with pytest.raises(RuntimeError, match="poisoned"):
            bad.result(10)
        # the batch failed as a whole, then each of its requests ran alone
        assert srv.batches == [[0], [1, 2, 3], [1], [2], [3]]
        _wait_for(lambda: srv.reserved == 0)  # released after the results are handed out


def test_latency_summary_fields():
    with HostServer(slots=2) as srv:
        reqs = [srv.submit(_img(N + i)) for i in range(6)]
        for r in reqs:
            r.result(10)
    s = serve.latency_summary(reqs)
    assert s["requests"] == 6 and s["windows"] == sum(r.windows for r in reqs)
    assert 0 <= s["admit_wait_p50_ms"] <= s["p50_ms"] <= s["p99_ms"]
    assert s["windows_per_s"] > 0 and 1 <= s["mean_batch"] <= 6
