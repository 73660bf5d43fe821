"""Continuous-batching coding server over librsc.

Requests are whole images (host float32 arrays [h, w]) whose stride-1 N x N
windows are to be coded: projection onto the steerable basis, then rotational
OMP (the two coding steps of the paper's proposed algorithm, Sec. II-E), both
in one ``rsc_encode_images`` call.  This module only schedules: every step of
the coding runs in the library's kernels.

* Admission by device memory.  A request needs its image, its outputs and the
  library's own scratch for its windows (``rsc_workspace_bytes``).  Requests
  are admitted in arrival order while the sum of what the admitted ones need
  stays within ``mem_budget``; one that would overflow it waits until running
  requests finish and release theirs.  A request that alone needs more than
  the budget is refused by ``submit`` (``AdmissionError``).
* Slots.  ``slots`` host worker threads each own a CUDA stream.  The
  dictionary and the basis stay resident and are shared; a request's state on
  the device (its projected windows, the coder's residual rows and
  least-squares state) lives in its call's scratch until the call returns.
  Requests admitted while others run are coded on other streams, so their
  kernels overlap on the device.
* Batching.  A worker that takes the request at the head of the queue also
  takes the requests queued behind it, in order, while their windows stay
  within ``batch_windows`` and their memory fits, and codes them in one call.
  A window's code does not depend on the other windows of its call, so a
  request's codes are the same alone and in any batch.
* Times.  Each request records when it was submitted, admitted, started and
  finished (host clock, seconds); ``latency_summary`` gives p50 / p99.
* Failures.  A request that has not been admitted yet can be withdrawn
  (``Request.cancel``; its ``result`` raises ``Cancelled``).  When a batched
  call fails, each of its requests is coded again alone, so that only the
  requests that fail by themselves report the error (``result`` raises it);
  the worker goes on with the queue.
"""
from __future__ import annotations

import collections
import threading
import time

import numpy as np

import paper_1806_04374_gb300 as _rsc

_OUT_BYTES = {"atom": 4, "angle_idx": 4, "angle": 4, "coef": 8}  # per window and step


class AdmissionError(ValueError):
    """The request alone needs more device memory than the server's budget."""


class Cancelled(RuntimeError):
    """The request was withdrawn before it was admitted."""


class Request:
    """One submitted image.  ``result()`` waits for and returns its codes:
    numpy arrays atom, angle_idx [W, K] int32, angle [W, K] float32, coef
    [W, K] float64 and resid_norm2 [W] float32, W = its windows in row-major
    order."""

    def __init__(self, rid, image: np.ndarray, N: int, server=None):
        self.id = rid
        self._server = server
        self.image = image
        self.h, self.w = image.shape
        self.windows = max(self.h - N + 1, 0) * max(self.w - N + 1, 0)
        self.need = 0
        self.t_submit = time.perf_counter()
        self.t_admit = self.t_start = self.t_done = None
        self.batch_size = 0
        self.codes = None
        self.error = None
        self._done = threading.Event()

    def done(self) -> bool:
        return self._done.is_set()

    def wait(self, timeout=None) -> bool:
        return self._done.wait(timeout)

    def cancel(self) -> bool:
        """Withdraws the request if it is still waiting for admission; returns
        whether it was withdrawn (False once a worker has taken it)."""
        return self._server is not None and self._server._cancel(self)

    def result(self, timeout=None) -> dict:
        if not self._done.wait(timeout):
            raise TimeoutError(f"request {self.id} not finished")
        if self.error is not None:
            raise self.error
        return self.codes

    @property
    def latency(self) -> float:
        return self.t_done - self.t_submit


class Server:
    """Codes image requests with a resident dictionary and basis; see the
    module docstring.  ``close()`` (or leaving a ``with`` block) finishes the
    queued requests and stops the workers."""

    def __init__(self, dic: "_rsc.Dictionary", basis: "_rsc.Basis", K: int,
                 precision: str = "f16", mem_budget: int = 8 << 30, slots: int = 3,
                 batch_windows: int = 1 << 20):
        if basis.J != dic.J or basis.kmax != dic.kmax:
            raise ValueError("basis and dictionary differ in J or kmax")
        if slots < 1 or mem_budget <= 0 or batch_windows < 1:
            raise ValueError("slots, mem_budget and batch_windows must be positive")
        self.dic, self.basis, self.K = dic, basis, int(K)
        self.precision = precision
        self.prec = _rsc.PRECISIONS[precision]
        self.mem_budget = int(mem_budget)
        self.batch_windows = int(batch_windows)
        self.reserved = 0
        self.peak_reserved = 0
        self.calls = 0
        self._queue = collections.deque()
        self._cv = threading.Condition()
        self._closed = False
        self._next_id = 0
        self._streams = self._make_streams(slots)
        self._workers = [threading.Thread(target=self._work, args=(s,), daemon=True)
                         for s in self._streams]
        for t in self._workers:
            t.start()

    # ------------------------------------------------------------- device
    def _make_streams(self, slots: int) -> list:
        """The current CUDA device and one stream per slot."""
        import torch
        self.device = torch.device("cuda", torch.cuda.current_device())
        return [torch.cuda.Stream(device=self.device) for _ in range(slots)]

    def _bind(self):
        """Makes the server's device current in a worker thread."""
        import torch
        torch.cuda.set_device(self.device)

    # ------------------------------------------------------------- memory
    def need_bytes(self, requests) -> int:
        """Device bytes one call over `requests` takes: images, outputs and
        the library's scratch, each rounded up to the allocator's 512 bytes."""
        up = lambda v: (int(v) + 511) // 512 * 512  # noqa: E731
        W = sum(r.windows for r in requests)
        img = sum(up(r.h * r.w * 4) for r in requests)
        out = sum(up(W * self.K * b) for b in _OUT_BYTES.values()) + up(W * 4)
        ws = _rsc.rsc_workspace_bytes(self.dic.handle, self.basis.handle, W, len(requests),
                                      self.K, self.prec)
        return img + out + up(ws)

    # ------------------------------------------------------------- API
    def submit(self, image, rid=None) -> Request:
        """Queues one image (host, float32 [h, w]); returns its Request."""
        image = np.ascontiguousarray(image, dtype=np.float32)
        if image.ndim != 2:
            raise ValueError("an image is a 2-D array")
        with self._cv:
            if self._closed:
                raise RuntimeError("server closed")
            if rid is None:
                rid = self._next_id
            self._next_id += 1
        r = Request(rid, image, self.basis.N, self)
        r.need = self.need_bytes([r])
        if r.need > self.mem_budget:
            raise AdmissionError(f"request {rid} needs {r.need} bytes of device memory, "
                                 f"more than the budget of {self.mem_budget}")
        with self._cv:
            self._queue.append(r)
            self._cv.notify_all()
        return r

    def _cancel(self, r: Request) -> bool:
        with self._cv:
            try:
                self._queue.remove(r)
            except ValueError:
                return False
            r.error = Cancelled(f"request {r.id} withdrawn before admission")
            r.t_done = time.perf_counter()
            r._done.set()
            self._cv.notify_all()
        return True

    def close(self, wait: bool = True):
        with self._cv:
            self._closed = True
            self._cv.notify_all()
        if wait:
            for t in self._workers:
                t.join()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ------------------------------------------------------------- workers
    def _take(self):
        """Under the lock: waits until the head of the queue fits the free
        budget, then takes it and the requests behind it that fit the batch
        and the budget.  Returns (batch, bytes) or None when closed and empty."""
        while True:
            if self._queue and self.reserved + self._queue[0].need <= self.mem_budget:
                break
            if self._closed and not self._queue:
                return None
            self._cv.wait()
        batch = [self._queue.popleft()]
        need, W = batch[0].need, batch[0].windows
        while self._queue:
            r = self._queue[0]
            if W + r.windows > self.batch_windows:
                break
            trial = self.need_bytes(batch + [r])
            if self.reserved + trial > self.mem_budget:
                break
            batch.append(self._queue.popleft())
            need, W = trial, W + r.windows
        self.reserved += need
        self.peak_reserved = max(self.peak_reserved, self.reserved)
        self.calls += 1
        now = time.perf_counter()
        for r in batch:
            r.t_admit = now
            r.batch_size = len(batch)
        return batch, need

    def _work(self, stream):
        self._bind()
        while True:
            with self._cv:
                got = self._take()
            if got is None:
                return
            batch, need = got
            now = time.perf_counter()
            for r in batch:
                r.t_start = now
            try:
                results = self._code(batch, stream)
            except Exception as e:  # noqa: BLE001 -- retried alone, then handed to the callers
                if len(batch) == 1:
                    results = [e]
                else:
                    results = []
                    for r in batch:
                        try:
                            results.append(self._code([r], stream)[0])
                        except Exception as e1:  # noqa: BLE001
                            results.append(e1)
            now = time.perf_counter()
            for r, res in zip(batch, results):
                if isinstance(res, Exception):
                    r.error = res
                else:
                    r.codes = res
                r.t_done = now
                r._done.set()
            with self._cv:
                self.reserved -= need
                self._cv.notify_all()

    def _code(self, batch, stream) -> list:
        """One rsc_encode_images call over `batch` on `stream`; returns each
        request's codes (host numpy arrays, its windows in row-major order)."""
        import torch
        with torch.cuda.stream(stream):
            imgs = [torch.from_numpy(r.image).pin_memory().to(self.device, non_blocking=True)
                    for r in batch]
            out = _rsc.encode_images(self.dic, self.basis, imgs, self.K, self.precision,
                                     stream=stream)
            codes = {k: v.cpu().numpy() for k, v in out.items()}
            del out, imgs
        res, lo = [], 0
        for r in batch:
            res.append({k: v[lo:lo + r.windows] for k, v in codes.items()})
            lo += r.windows
        return res


def latency_summary(requests) -> dict:
    """p50 / p99 of request latency (done - submit) and of the wait for
    admission (admit - submit), in milliseconds, and the windows coded per
    second of wall time from the first submission to the last completion."""
    lat = np.array([r.latency for r in requests]) * 1e3
    wait = np.array([r.t_admit - r.t_submit for r in requests]) * 1e3
    t0 = min(r.t_submit for r in requests)
    t1 = max(r.t_done for r in requests)
    W = sum(r.windows for r in requests)
    return {"requests": len(requests), "windows": int(W), "wall_s": t1 - t0,
            "windows_per_s": W / (t1 - t0),
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "admit_wait_p50_ms": float(np.percentile(wait, 50)),
            "admit_wait_p99_ms": float(np.percentile(wait, 99)),
            "mean_batch": float(np.mean([r.batch_size for r in requests]))}
