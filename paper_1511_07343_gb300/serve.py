"""Continuous-batching serving loop for streams of DM trials.

De-dispersion produces many trials (~6000 per 530 s SKA observation,
Section 1) of possibly different lengths and acceleration ranges. A
`Server` keeps device-resident plans (templates, twiddle tables, workspaces)
in worker slots, each slot with its own CUDA stream and host thread:

* requests (host series + zmax) enter a FIFO queue as they arrive;
* an idle slot takes the next request at once; a slot builds the plan of a
  zmax class the first time it needs it, and only if the device-memory
  budget still has room for that plan's footprint (otherwise the request
  waits for a slot that already holds such a plan);
* each slot copies its series to the device, enqueues the whole search on
  its stream (the same C ABI entry point as a single search) and returns the
  candidates; slots run concurrently, so work from different requests
  overlaps on the GPU.

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


def plan_footprint(n_max: int, zmax: int, m: int, L: int, dz: int = 2,
                   max_cands: int = 1 << 20) -> int:
    """Device bytes a plan of this class holds, for admission: plane and its
    4-bin maxima, spectra and workspaces, segment spectra, templates, the
    candidate list and the harmonic-sum screen's list of 2^20 flagged pairs
    (an upper estimate of fdas_plan_get_info's device_bytes)."""
    Z = 2 * (zmax // dz) + 1
    nb = n_max // 2
    S = (nb + (L - m) - 1) // (L - m)
    core = (4 * Z * nb + Z * nb + 8 * 4 * nb + 8 * S * L + 24 * Z * L
            + 16 * max_cands + 4 * n_max + 8 * (1 << 20))
    # twiddle tables and counters (a few MB at most), plus 2% headroom
    return int(core * 1.02) + (8 << 20)


class Budget:
    """Thread-safe reservation of a fixed number of device bytes."""

    def __init__(self, total: int):
        self.total = int(total)
        self.reserved = 0
        self._lock = threading.Lock()

    def try_reserve(self, nbytes: int) -> bool:
        with self._lock:
            if self.reserved + nbytes > self.total:
                return False
            self.reserved += nbytes
            return True

    def release(self, nbytes: int):
        with self._lock:
            if nbytes > self.reserved:
                raise ValueError("release of bytes never reserved")
            self.reserved -= nbytes


@dataclasses.dataclass
class Result:
    candidates: np.ndarray      # fdas.CAND_DTYPE, sorted by (h, r_top, z_idx)
    count: int                  # exact number found (may exceed len(candidates))
    zmax: int
    n: int
    arrival: float              # time.perf_counter() at submit
    done: float                 # time.perf_counter() when the result was ready

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
                 max_cands: int = 1 << 20, device: int = 0):
        import torch
        self._torch = torch
        self.n_max = int(n_max)
        self.classes = dict(classes or DEFAULT_CLASSES)
        self.dz, self.nharm, self.sigma, self.max_cands = dz, nharm, sigma, max_cands
        self.device = torch.device("cuda", device)
        if hbm_budget is None:
            free, _ = torch.cuda.mem_get_info(self.device)
            hbm_budget = int(0.8 * free)
        self.hbm_budget = int(hbm_budget)
        self._budget = Budget(self.hbm_budget)
        self._lock = threading.Lock()
        self._queue: "queue.Queue[_Request | None]" = queue.Queue()
        self._slots = [_Slot(self, i) for i in range(n_slots)]
        self._closed = False
        self.stats = {"admitted": 0, "plans_built": 0, "waits_for_memory": 0}
        for s in self._slots:
            s.start()

    # -- public API ---------------------------------------------------------
    def submit(self, series: np.ndarray, zmax: int) -> cf.Future:
        """Queue one DM trial (host float32 series); the future resolves to a
        Result."""
        if self._closed:
            raise RuntimeError("server is closed")
        if zmax not in self.classes:
            raise ValueError(f"unsupported zmax {zmax}; classes: {sorted(self.classes)}")
        x = np.ascontiguousarray(series, dtype=np.float32)
        if x.shape[0] > self.n_max:
            raise ValueError("series longer than the server's n_max")
        if self._footprint(int(zmax)) > self.hbm_budget:
            raise ValueError("one plan of this class does not fit in the memory budget")
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

    # -- admission ------------------------------------------------------------
    def _footprint(self, zmax: int) -> int:
        m, L = self.classes[zmax]
        return plan_footprint(self.n_max, zmax, m, L, self.dz, self.max_cands)

    def _try_reserve(self, nbytes: int) -> bool:
        return self._budget.try_reserve(nbytes)

    def _release(self, nbytes: int):
        self._budget.release(nbytes)


class _Slot(threading.Thread):
    def __init__(self, server: Server, idx: int):
        super().__init__(daemon=True, name=f"fdas-slot-{idx}")
        self.s = server
        torch = server._torch
        self.stream = torch.cuda.Stream(server.device)
        self.batches: dict[int, int] = {}     # zmax -> fdas_batch handle
        self.bytes: dict[int, int] = {}
        self.d_series = torch.empty(server.n_max, dtype=torch.float32, device=server.device)
        self.h_series = torch.empty(server.n_max, dtype=torch.float32).pin_memory()
        self.d_out = torch.empty(server.max_cands * 16, dtype=torch.uint8, device=server.device)
        self.d_cnt = torch.zeros(1, dtype=torch.int64, device=server.device)

    def _batch_for(self, zmax: int):
        if zmax in self.batches:
            return self.batches[zmax]
        s = self.s
        need = s._footprint(zmax)
        if not s._try_reserve(need):
            # this slot is idle, so its plans of other classes can go
            self.release()
            if not s._try_reserve(need):
                return None
        m, L = s.classes[zmax]
        try:
            b = fdas.fdas_batch_create(s.n_max, zmax, s.dz, m, L, s.nharm, s.sigma, s.max_cands,
                                       self.stream.cuda_stream)
        except Exception:
            s._release(need)
            raise
        self.batches[zmax] = b
        self.bytes[zmax] = need
        with s._lock:
            s.stats["plans_built"] += 1
        return b

    def run(self):
        torch = self.s._torch
        torch.cuda.set_device(self.s.device)
        while True:
            req = self.s._queue.get()
            if req is None:
                return
            try:
                b = self._batch_for(req.zmax)
                if b is None:
                    # no memory for a new plan: hand the request back and let a
                    # slot that holds this class (or a later free-up) take it
                    with self.s._lock:
                        self.s.stats["waits_for_memory"] += 1
                    self.s._queue.put(req)
                    time.sleep(0.001)
                    continue
                with self.s._lock:
                    self.s.stats["admitted"] += 1
                req.future.set_result(self._serve(b, req))
            except Exception as e:  # the error goes to the caller's future
                req.future.set_exception(e)

    def _serve(self, batch, req: _Request) -> Result:
        torch = self.s._torch
        n = req.series.shape[0]
        with torch.cuda.stream(self.stream):
            self.h_series[:n].numpy()[:] = req.series
            self.d_series[:n].copy_(self.h_series[:n], non_blocking=True)
            fdas.fdas_search_batch(batch, [self.d_series], [n], self.d_out, self.d_cnt)
            cnt = int(self.d_cnt.to("cpu", non_blocking=False).item())
            keep = min(cnt, self.s.max_cands)
            raw = self.d_out[: keep * 16].to("cpu").numpy().view(fdas.CAND_DTYPE).copy()
        raw.sort(order=["h", "r_top", "z_idx"])
        return Result(raw, cnt, req.zmax, n, req.arrival, time.perf_counter())

    def release(self):
        for z, b in self.batches.items():
            fdas.fdas_batch_destroy(b)
            self.s._release(self.bytes[z])
        self.batches.clear()
