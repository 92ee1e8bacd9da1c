"""Continuous-batching serving loop for streams of DM trials.

De-dispersion produces many trials (~6000 per 530 s SKA observation,
Section 1) of possibly different lengths and acceleration ranges. A
`Server` keeps device-resident search state in worker slots, each slot with
its own CUDA stream and host thread:

* every slot holds one batch object of the C library with a zmax class per
  acceleration range served (templates and tables per class; one set of
  per-trial workspaces sized for the largest class, plus a second trial
  lane), built when the server starts;
* admission is by HBM footprint: the server starts only as many slots as the
  device-memory budget holds (a slot's footprint is fixed, so a request that
  a slot takes always fits);
* requests (host series + zmax) enter a FIFO queue as they arrive; an idle
  slot takes the oldest request and, without waiting, up to ``max_batch - 1``
  more that are already queued, and runs them as ONE fdas_search_batch call
  (mixed lengths and zmax classes; consecutive trials overlap on the slot's
  two lanes); slots run concurrently, so work from different requests
  overlaps on the GPU while new ones keep arriving;
* a request cancelled while queued is skipped; results are sorted candidate
  lists, the same as a single search of that trial gives.

Every arithmetic step runs in the CUDA library; this module only schedules.
"""
from __future__ import annotations

import concurrent.futures as cf
import dataclasses
import queue
import threading
import time

import numpy as np

from . import fdas

# Template width and segment length per zmax (the 128 / 256 / 512-tap
# pattern of the SKA-shaped configurations).
DEFAULT_CLASSES = {50: (128, 2048), 100: (256, 4096), 200: (512, 8192)}

_HS_LIST_BYTES = 8 << 20   # the harmonic-sum screen's list of 2^20 flagged pairs


def _trial_workspace_bytes(n_max: int, Z: int, seg_floats2: int, max_cands: int) -> int:
    """Per-trial workspaces of one lane: staging series, four-step scratch,
    spectra, segment spectra, plane and 4-bin maxima, candidate list,
    flagged-pair list."""
    nb = n_max // 2
    return (4 * n_max + 8 * 4 * nb + 8 * seg_floats2 + 5 * Z * nb + 16 * max_cands
            + _HS_LIST_BYTES)


def plan_footprint(n_max: int, zmax: int, m: int, L: int, dz: int = 2,
                   max_cands: int = 1 << 20) -> int:
    """Device bytes one plan of this class holds (an upper estimate of
    fdas_plan_get_info's device_bytes): its per-trial workspaces plus the
    templates (float64 taps and float32 spectra) and tables."""
    Z = 2 * (zmax // dz) + 1
    nb = n_max // 2
    S = (nb + (L - m) - 1) // (L - m)
    core = _trial_workspace_bytes(n_max, Z, S * L, max_cands) + 24 * Z * L
    # twiddle tables, tile orders and counters (a few MB at most), plus 2% headroom
    return int(core * 1.02) + (8 << 20)


def batch_footprint(n_max: int, classes: dict, dz: int = 2, max_cands: int = 1 << 20,
                    lanes: bool = True) -> int:
    """Device bytes of one multi-class batch (an upper estimate of
    fdas_batch_get_info's device_bytes): one set of per-trial workspaces sized
    for the largest class (two with the second trial lane) plus every class's
    templates and tables."""
    nb = n_max // 2
    Zmax = max(2 * (z // dz) + 1 for z in classes)
    seg = max(((nb + (L - m) - 1) // (L - m)) * L for (m, L) in classes.values())
    ws = _trial_workspace_bytes(n_max, Zmax, seg, max_cands)
    tables = sum(24 * (2 * (z // dz) + 1) * L + (2 << 20) for z, (m, L) in classes.items())
    core = ws * (2 if lanes else 1) + tables
    return int(core * 1.02) + (8 << 20)


@dataclasses.dataclass
class Result:
    candidates: np.ndarray      # fdas.CAND_DTYPE, sorted by (h, r_top, z_idx)
    count: int                  # exact number found (may exceed len(candidates))
    zmax: int
    n: int
    arrival: float              # time.perf_counter() at submit
    done: float                 # time.perf_counter() when the result was ready
    batch: int = 1              # trials in the fdas_search_batch call that served it

    @property
    def latency_ms(self) -> float:
        return (self.done - self.arrival) * 1e3


@dataclasses.dataclass
class _Request:
    series: np.ndarray
    zmax: int
    future: cf.Future
    arrival: float


class Server:
    def __init__(self, n_max: int, n_slots: int = 2, hbm_budget: int | None = None,
                 classes=None, dz: int = 2, nharm: int = 16, sigma: float = 6.0,
                 max_cands: int = 1 << 20, device: int = 0, max_batch: int = 2):
        import torch
        self._torch = torch
        self.n_max = int(n_max)
        self.classes = dict(classes or DEFAULT_CLASSES)
        self.dz, self.nharm, self.sigma, self.max_cands = dz, nharm, sigma, max_cands
        self.max_batch = max(1, int(max_batch))
        self.device = torch.device("cuda", device)
        if hbm_budget is None:
            free, _ = torch.cuda.mem_get_info(self.device)
            hbm_budget = int(0.8 * free)
        self.hbm_budget = int(hbm_budget)
        self.slot_bytes = batch_footprint(self.n_max, self.classes, dz, max_cands,
                                          lanes=self.max_batch > 1)
        n_fit = min(int(n_slots), self.hbm_budget // self.slot_bytes)
        self._lock = threading.Lock()
        self._queue: "queue.Queue[_Request | None]" = queue.Queue()
        self.stats = {"slots": n_fit, "admitted": 0, "batches": 0, "cancelled": 0,
                      "largest_batch": 0, "hbm_reserved": n_fit * self.slot_bytes}
        self._slots = []
        self._closed = False
        try:
            for i in range(n_fit):
                self._slots.append(_Slot(self, i))
        except Exception:
            for s in self._slots:
                s.release()
            raise
        for s in self._slots:
            s.start()

    # -- public API ---------------------------------------------------------
    def submit(self, series: np.ndarray, zmax: int) -> cf.Future:
        """Queue one DM trial (host float32 series); the future resolves to a
        Result. Cancelling the future before a slot takes the request drops
        the request."""
        if self._closed:
            raise RuntimeError("server is closed")
        if zmax not in self.classes:
            raise ValueError(f"unsupported zmax {zmax}; classes: {sorted(self.classes)}")
        x = np.ascontiguousarray(series, dtype=np.float32)
        if x.shape[0] > self.n_max:
            raise ValueError("series longer than the server's n_max")
        if not self._slots:
            raise ValueError("not one slot fits in the memory budget "
                             f"({self.slot_bytes} bytes per slot, budget {self.hbm_budget})")
        fut: cf.Future = cf.Future()
        self._queue.put(_Request(x, int(zmax), fut, time.perf_counter()))
        return fut

    def close(self):
        if self._closed:
            return
        self._closed = True
        for _ in self._slots:
            self._queue.put(None)
        for s in self._slots:
            s.join()
        for s in self._slots:
            s.release()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- scheduling -----------------------------------------------------------
    def _take(self):
        """The oldest request (blocking) plus up to max_batch - 1 more already
        queued; None when the server is closing. Requests cancelled while
        queued are dropped here: set_running_or_notify_cancel() marks the
        others running, after which they can no longer be cancelled."""
        got, stop = [], False
        req = self._queue.get()
        if req is None:
            return None
        pending = [req]
        while len(pending) < self.max_batch:
            try:
                nxt = self._queue.get_nowait()
            except queue.Empty:
                break
            if nxt is None:       # closing: finish this batch, then stop
                stop = True
                break
            pending.append(nxt)
        for r in pending:
            if r.future.set_running_or_notify_cancel():
                got.append(r)
            else:
                with self._lock:
                    self.stats["cancelled"] += 1
        return got, stop


def _settle(fut: cf.Future, result=None, error: BaseException | None = None):
    """Completes a running future; a future that is already done is left as
    it is (never raises into the slot thread)."""
    try:
        if error is not None:
            fut.set_exception(error)
        else:
            fut.set_result(result)
    except cf.InvalidStateError:
        pass


class _Slot(threading.Thread):
    def __init__(self, server: Server, idx: int):
        super().__init__(daemon=True, name=f"fdas-slot-{idx}")
        self.s = server
        torch = server._torch
        self.stream = torch.cuda.Stream(server.device)
        B = server.max_batch
        self.d_series = [torch.empty(server.n_max, dtype=torch.float32, device=server.device)
                         for _ in range(B)]
        self.h_series = [torch.empty(server.n_max, dtype=torch.float32).pin_memory()
                         for _ in range(B)]
        self.d_out = torch.empty(B * server.max_cands * 16, dtype=torch.uint8,
                                 device=server.device)
        self.d_cnt = torch.zeros(B, dtype=torch.int64, device=server.device)
        zs = sorted(server.classes, reverse=True)   # the largest class first
        m, L = server.classes[zs[0]]
        self.batch = fdas.fdas_batch_create(server.n_max, zs[0], server.dz, m, L, server.nharm,
                                            server.sigma, server.max_cands,
                                            self.stream.cuda_stream)
        try:
            for z in zs[1:]:
                fdas.fdas_batch_add_class(self.batch, z, *server.classes[z])
            # the mix changes from call to call, so launch directly rather
            # than capture a graph per call
            fdas.fdas_batch_set_graphs(self.batch, 0)
        except Exception:
            fdas.fdas_batch_destroy(self.batch)
            self.batch = None
            raise

    def run(self):
        torch = self.s._torch
        torch.cuda.set_device(self.s.device)
        while True:
            taken = self.s._take()
            if taken is None:
                return
            reqs, stop = taken
            if reqs:
                try:
                    results = self._serve(reqs)
                    with self.s._lock:
                        self.s.stats["admitted"] += len(reqs)
                        self.s.stats["batches"] += 1
                        self.s.stats["largest_batch"] = max(self.s.stats["largest_batch"],
                                                            len(reqs))
                    for r, res in zip(reqs, results):
                        _settle(r.future, res)
                except Exception as e:  # the error goes to every caller's future
                    for r in reqs:
                        _settle(r.future, error=e)
            if stop:
                return

    def _serve(self, reqs) -> list:
        torch = self.s._torch
        ns = [r.series.shape[0] for r in reqs]
        M = self.s.max_cands
        with torch.cuda.stream(self.stream):
            for i, r in enumerate(reqs):
                self.h_series[i][: ns[i]].numpy()[:] = r.series
                self.d_series[i][: ns[i]].copy_(self.h_series[i][: ns[i]], non_blocking=True)
            fdas.fdas_search_batch(self.batch, self.d_series[: len(reqs)], ns, self.d_out,
                                   self.d_cnt, [r.zmax for r in reqs])
            cnts = self.d_cnt[: len(reqs)].to("cpu", non_blocking=False).numpy()
            lists = []
            for i in range(len(reqs)):   # only the entries each trial filled
                keep = min(int(cnts[i]), M)
                lists.append(self.d_out[i * M * 16: (i * M + keep) * 16].to("cpu").numpy())
        done = time.perf_counter()
        out = []
        for i, r in enumerate(reqs):
            c = lists[i].view(fdas.CAND_DTYPE).copy()
            c.sort(order=["h", "r_top", "z_idx"])
            out.append(Result(c, int(cnts[i]), r.zmax, ns[i], r.arrival, done, len(reqs)))
        return out

    def release(self):
        if self.batch is not None:
            fdas.fdas_batch_destroy(self.batch)
            self.batch = None
