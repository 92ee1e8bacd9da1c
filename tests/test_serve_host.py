"""Host logic of the serving loop that needs no GPU: the footprint estimates
used for admission, and the slot loop's handling of cancelled requests,
failures and shutdown (a fake slot whose search is a stub)."""
import concurrent.futures as cf
import queue
import threading
import time

import numpy as np
import pytest

from paper_1511_07343_gb300 import serve
from paper_1511_07343_gb300.serve import (DEFAULT_CLASSES, Result, Server, _Request, _Slot,
                                          batch_footprint, plan_footprint)


def test_footprint_covers_the_plane_and_grows_with_zmax():
    n = 1 << 23
    sizes = {z: plan_footprint(n, z, m, L) for z, (m, L) in DEFAULT_CLASSES.items()}
    assert sizes[50] < sizes[100] < sizes[200]
    # at least the float32 plane and its 4-bin maxima: 5 bytes per cell
    assert sizes[200] >= 201 * (n // 2) * 5
    assert plan_footprint(n // 2, 200, 512, 8192) < sizes[200]


def test_batch_footprint_is_one_largest_workspace_per_lane():
    """A multi-class batch holds one set of workspaces for its largest class
    per lane, not one per class."""
    n = 1 << 23
    one = batch_footprint(n, {200: (512, 8192)}, lanes=False)
    three = batch_footprint(n, DEFAULT_CLASSES, lanes=False)
    assert three < one + sum(plan_footprint(n, z, m, L) for z, (m, L) in DEFAULT_CLASSES.items()
                             if z != 200)
    assert three - one < 0.01 * one          # only templates and tables added
    two_lanes = batch_footprint(n, DEFAULT_CLASSES, lanes=True)
    assert 1.9 * three < two_lanes < 2.1 * three


class _FakeServer:
    """The parts of Server the slot loop uses, without a GPU."""

    def __init__(self, max_batch):
        self.max_batch = max_batch
        self._queue = queue.Queue()
        self._lock = threading.Lock()
        self.stats = {"admitted": 0, "batches": 0, "cancelled": 0, "largest_batch": 0}

    _take = Server._take

    def submit(self, x, zmax=50):
        fut = cf.Future()
        self._queue.put(_Request(np.asarray(x, np.float32), zmax, fut, time.perf_counter()))
        return fut


def _fake_slot(server, serve_fn):
    slot = _Slot.__new__(_Slot)
    threading.Thread.__init__(slot, daemon=True, name="fake-slot")
    slot.s = server
    slot._serve = serve_fn
    return slot


class _NoTorch:
    class cuda:
        @staticmethod
        def set_device(d):
            pass


def _echo(reqs):
    now = time.perf_counter()
    return [Result(np.zeros(0), int(r.series[0]), r.zmax, r.series.shape[0], r.arrival, now,
                   len(reqs)) for r in reqs]


def test_cancelled_request_is_skipped_and_the_rest_complete():
    srv = _FakeServer(max_batch=3)
    srv._torch = _NoTorch
    srv.device = None
    gate = threading.Event()
    served = []

    def slow_echo(reqs):
        gate.wait(5)
        served.extend(int(r.series[0]) for r in reqs)
        return _echo(reqs)

    futs = [srv.submit([i]) for i in range(7)]
    assert futs[1].cancel() and futs[4].cancel()     # cancelled while queued
    slot = _fake_slot(srv, slow_echo)
    slot.start()
    gate.set()
    for i, f in enumerate(futs):
        if i in (1, 4):
            assert f.cancelled()
        else:
            assert f.result(timeout=5).count == i
    srv._queue.put(None)
    slot.join(5)
    assert not slot.is_alive()
    assert sorted(served) == [0, 2, 3, 5, 6]
    assert srv.stats["cancelled"] == 2 and srv.stats["admitted"] == 5
    assert srv.stats["largest_batch"] <= 3


def test_a_failing_batch_fails_its_futures_and_the_slot_keeps_serving():
    srv = _FakeServer(max_batch=2)
    srv._torch = _NoTorch
    srv.device = None
    calls = []

    def flaky(reqs):
        calls.append(len(reqs))
        if len(calls) == 1:
            raise RuntimeError("stub failure")
        return _echo(reqs)

    first = [srv.submit([i]) for i in range(2)]   # taken together, fail together
    slot = _fake_slot(srv, flaky)
    slot.start()
    for f in first:
        with pytest.raises(RuntimeError, match="stub failure"):
            f.result(timeout=5)
    later = [srv.submit([10 + i]) for i in range(3)]
    assert [f.result(timeout=5).count for f in later] == [10, 11, 12]
    srv._queue.put(None)
    slot.join(5)
    assert not slot.is_alive()


def test_settle_never_raises_on_a_finished_future():
    f = cf.Future()
    assert f.set_running_or_notify_cancel()
    serve._settle(f, 1)
    serve._settle(f, 2)                      # already done: ignored
    serve._settle(f, error=RuntimeError())   # likewise
    assert f.result() == 1


def test_shutdown_sentinel_inside_a_batch_finishes_that_batch():
    srv = _FakeServer(max_batch=4)
    srv._torch = _NoTorch
    srv.device = None
    futs = [srv.submit([i]) for i in range(2)]
    srv._queue.put(None)
    slot = _fake_slot(srv, _echo)
    slot.start()
    slot.join(5)
    assert not slot.is_alive()
    assert [f.result(timeout=1).count for f in futs] == [0, 1]
