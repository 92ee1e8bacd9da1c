#!/usr/bin/env python
"""Throughput of the FDAS path on the SKA-shaped single-trial workload:
N = 2^23 float32 samples (Gaussian noise + 20 accelerated sinusoids with up
to 8 harmonics), zmax = 200, dz = 2 (201 templates of 512 taps), segments of
8192 bins, float32 power plane, harmonic sums 1..16, 6-sigma threshold.

One step = one DM trial through the whole path (real FFT, whitening, segment
FFTs, fused correlation, harmonic sum, threshold, compaction) with the series
already resident in HBM; `e2e` repeats the measurement through the C ABI with
host buffers (host->device copy of the series and device->host copy of the
candidate list inside the timed region).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Multi-GPU: one process per GPU (torchrun); DM trials are independent, so
every rank processes its own trials with no data-path collective (weak
scaling); the timed region is bracketed by barriers and the max over ranks
is used.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "cfg2_n2e23_z200"
METRIC = "DM trials/s at N=2^23 zmax=200"
PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}
FP32_LANES_PER_SM = 128
# DRAM bytes (read + write) per launch at the benchmark size, from an ncu
# counter capture of the kernel, each valid only for the kernel source it was
# taken with (sha256 prefix of the file); None once that source changes.
# (A 2^21-sample capture, one launch per kernel, scaled to the 2^23-sample
# launch by the (segment, template) pairs or top bins it processes.)
MEASURED_TRAFFIC = {
    "k_correlate_fused": (4.055e+09, "paper_1511_07343_gb300/csrc/fdas_correlate.cu", "5095bcf9f5860ca7"),
    "k_harmsum_staged": (8.457e+08, "paper_1511_07343_gb300/csrc/fdas_harmsum.cu", "03294e1f8c59e47a"),
}


def measured_traffic(kernel):
    import hashlib
    if kernel not in MEASURED_TRAFFIC:
        return None
    nbytes, path, digest = MEASURED_TRAFFIC[kernel]
    with open(os.path.join(ROOT, path), "rb") as f:
        if hashlib.sha256(f.read()).hexdigest()[:16] != digest:
            return None  # the kernel changed since the counters were taken
    return nbytes


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    except Exception:
        return dict(PEAKS_FALLBACK, sm_max_mhz=2070.0), "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap,"
              "timestamp")
    PERIOD_MS = 20

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.file = None

    def __enter__(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", str(self.PERIOD_MS)],
                stdout=self.file, stderr=subprocess.DEVNULL)
            # wait (at most 5 s) for the first sample, so that sampling covers
            # the timed region that follows
            t_end = time.time() + 5.0
            while time.time() < t_end and os.path.getsize(self.file.name) == 0:
                time.sleep(0.02)
        except Exception:
            self.proc = None
        self.window = [None, None]
        return self

    def mark_start(self):
        self.window[0] = time.time()

    def mark_end(self):
        self.window[1] = time.time()

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if self.proc is None or self.file is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.file.flush()
        import datetime
        rows = []
        with open(self.file.name) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 10:
                    rows.append(parts)
        os.unlink(self.file.name)
        # samples inside the timed region (wall clock; one sample period of
        # slack on each side); all samples if none fell inside
        t0, t1 = self.window
        inside = []
        for r in rows:
            try:
                ts = datetime.datetime.strptime(r[9], "%Y/%m/%d %H:%M:%S.%f").timestamp()
            except ValueError:
                continue
            if t0 is not None and t1 is not None and \
                    t0 - self.PERIOD_MS / 1e3 <= ts <= t1 + self.PERIOD_MS / 1e3:
                inside.append(r)
        timed = bool(inside)
        rows = inside or rows
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = []
        for i, n in enumerate(names):
            if any(r[5 + i].lower().startswith("active") for r in rows):
                reasons.append(n)
        power = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows), "samples_in_timed_region": timed,
                "power_w_max": max(power) if power else None}


def reduce_max(value, world, device=None):
    """Max over ranks of a per-rank float (the slowest rank's time); identity
    for one rank."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def percentiles(xs):
    xs = np.asarray(xs, dtype=np.float64)
    if xs.size == 0:
        return {"p50": None, "p99": None}
    return {"p50": float(np.percentile(xs, 50)), "p99": float(np.percentile(xs, 99))}


# ---------------------------------------------------------------------------
# Same-GPU comparator: the paper's unfused step structure (Section 4) in FP32
# with cuFFT (through torch.fft) for steps 2, 4 and 6, a materialised complex
# plane for steps 5-6, and this library's whitening and harmonic-sum stages.
# ---------------------------------------------------------------------------
def plain_fp32_path(fdas, plan, info, p, dev, stream):
    import torch
    Z, L, m, V, S, nb = info.Z, info.L, info.m, info.V, info.S, info.nb
    bank = torch.empty(Z * L * 2, dtype=torch.float32, device=dev)
    fdas.fdas_template_bank(plan, bank)  # natural order, 1/L folded in
    # times L: torch's inverse FFT carries its own 1/L
    bank = torch.view_as_complex(bank.view(Z, L, 2)) * float(L)
    idx = (torch.arange(S, device=dev)[:, None] * V - m // 2
           + torch.arange(L, device=dev)[None, :])
    valid = (idx >= 0) & (idx < nb)
    idx = idx.clamp(0, nb - 1)
    zero = torch.zeros((), dtype=torch.complex64, device=dev)
    white = torch.empty(nb * 2, dtype=torch.float32, device=dev)
    plane = torch.empty(Z, nb, dtype=torch.float32, device=dev)
    cands = torch.empty(info.max_cands * 16, dtype=torch.uint8, device=dev)
    count = torch.zeros(1, dtype=torch.int64, device=dev)

    def step(x):
        with torch.cuda.stream(stream):
            X = torch.fft.rfft(x)[:nb].contiguous()                      # step 2
            fdas.fdas_stage_whiten(plan, torch.view_as_real(X), white)
            W = torch.view_as_complex(white.view(nb, 2))
            seg = torch.where(valid, W[idx], zero)                        # step 3
            F = torch.fft.fft(seg, dim=1)                                 # step 4
            Y = bank[:, None, :] * F[None, :, :]                          # step 5 (Z, S, L)
            y = torch.fft.ifft(Y, dim=2)                                  # step 6
            pw = torch.abs(y[:, :, m // 2: m // 2 + V])                   # step 7: power,
            pw.square_()                                                  # edge removal
            plane.copy_(pw.view(Z, S * V)[:, :nb])
            fdas.fdas_stage_harmsum(plan, plane, cands, count)
        return count
    step.cands = cands
    return step


def candidate_agreement(a, b, thresholds):
    """Key sets (r, z, h) of two candidate lists of the same series: common
    keys, keys only in one of them, and how many of the latter lie outside
    the 1e-4 T_h band around the threshold (judged by the power the list that
    has the key reports)."""
    def table(c):
        return {(int(x["r_top"]), int(x["z_idx"]), int(x["h"])): float(x["power"]) for x in c}
    ta, tb = table(a), table(b)
    lvl = {1 << i: float(thresholds[i]) for i in range(5)}

    def outside(keys, t):
        return sum(1 for k in keys if abs(t[k] - lvl[k[2]]) > 1e-4 * lvl[k[2]])
    only_a, only_b = set(ta) - set(tb), set(tb) - set(ta)
    return {"common": len(set(ta) & set(tb)), "only_fused": len(only_a),
            "only_plain": len(only_b), "only_fused_outside_band": outside(only_a, ta),
            "only_plain_outside_band": outside(only_b, tb)}


# ---------------------------------------------------------------------------
# Serving: a stream of DM trials with zmax drawn from {50, 100, 200}, one in
# ten at an uneven length from [2^21, 2^22] (snapped to 2^a 3^b 5^c), the rest
# 2^23 samples; continuous batching over device-resident plans.
# ---------------------------------------------------------------------------
def serve_measure(dev, n_sat=48, n_poisson=600, rate=11.32, seed=5, slots=2, max_batch=2):
    import torch
    from paper_1511_07343_gb300.serve import Server
    from synthetic import make_series, random_chirps, snap_235
    rng = np.random.default_rng(seed)
    pool = []
    for i in range(8):
        n = 1 << 23
        if i == 7:
            n = snap_235(np.exp(rng.uniform(np.log(2 ** 21), np.log(2 ** 22))))
        chirps = random_chirps(rng, int(rng.integers(0, 4)), n, 200.0)
        pool.append(make_series(n, 5000 + i, chirps, device=dev))
    zs = [50, 100, 200]
    with Server(n_max=1 << 23, n_slots=slots, nharm=16, max_cands=1 << 20,
                device=dev.index or 0, max_batch=max_batch) as srv:
        # every class and length once through every slot (first-use geometry)
        warm = [srv.submit(pool[i], z) for z in zs for i in (0, 7) for _ in range(slots)]
        for f in warm:
            f.result()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        futs = [srv.submit(pool[i % 8], zs[int(rng.integers(0, 3))]) for i in range(n_sat)]
        sat = [f.result() for f in futs]
        t_sat = time.perf_counter() - t0
        arrivals = np.cumsum(rng.exponential(1.0 / rate, size=n_poisson))
        t0 = time.perf_counter()
        futs = []
        for i, ta in enumerate(arrivals):
            dt = t0 + ta - time.perf_counter()
            if dt > 0:
                time.sleep(dt)
            futs.append(srv.submit(pool[i % 8], zs[int(rng.integers(0, 3))]))
        poi = [f.result() for f in futs]
        t_poi = time.perf_counter() - t0
        stats = dict(srv.stats)
        slot_gb = srv.slot_bytes / 1e9
    lat = percentiles([r.latency_ms for r in poi])
    by_class = {z: percentiles([r.latency_ms for r in poi if r.zmax == z]) for z in zs}
    return {"slots": stats["slots"], "max_batch": max_batch, "zmax_classes": zs,
            "slot_footprint_gb": slot_gb,
            "saturating": {"trials": n_sat, "trials_per_s": n_sat / t_sat,
                           "latency_ms": percentiles([r.latency_ms for r in sat]),
                           "mean_batch": float(np.mean([r.batch for r in sat]))},
            "poisson": {"rate_per_s": rate, "trials": n_poisson,
                        "sustained_trials_per_s": n_poisson / t_poi, "latency_ms": lat,
                        "latency_ms_by_zmax": by_class,
                        "trials_in_batches_of_2": sum(r.batch == 2 for r in poi)},
            "real_time_budget_trials_per_s": 6000 / 530.0, "stats": stats,
            "what": "host series in, sorted candidates out; arrival to result, wall clock; "
                    "each slot runs up to max_batch queued trials (mixed zmax and length) "
                    "as one fdas_search_batch call"}


# ---------------------------------------------------------------------------
# Batched uneven trials: 256 DM trials, N log-uniform in [2^20, 2^23] snapped
# to 2^a 3^b 5^c, 0-3 accelerated signals each, zmax = 200; one autotuned
# batch (segment length timed on a probe), each batch one CUDA graph launch.
# ---------------------------------------------------------------------------
def batch_measure(fdas, dev, n_trials=256, reps=2, seed=3):
    import torch
    from synthetic import make_series, random_chirps, snap_235
    rng = np.random.default_rng(seed)
    lens = [snap_235(math.exp(rng.uniform(math.log(2 ** 20), math.log(2 ** 23))))
            for _ in range(n_trials)]
    # 8 distinct series of 2^23 samples; trial t takes a prefix of one of them
    base = [torch.from_numpy(make_series(1 << 23, 9000 + i,
                                         random_chirps(rng, int(rng.integers(0, 4)),
                                                       1 << 20, 200.0),
                                         device=dev)).to(dev) for i in range(8)]
    xs = [base[t % 8][:lens[t]] for t in range(n_trials)]
    stream = torch.cuda.Stream(dev)
    maxc = 1 << 16
    t0 = time.perf_counter()
    batch = fdas.fdas_batch_create_tuned(1 << 23, 200, 2, 512, 16, 6.0, maxc, None,
                                         stream.cuda_stream)
    tune_s = time.perf_counter() - t0
    try:
        info = fdas.fdas_batch_get_info(batch)
        d_out = torch.empty(n_trials * maxc * 16, dtype=torch.uint8, device=dev)
        d_cnt = torch.zeros(n_trials, dtype=torch.int64, device=dev)
        torch.cuda.synchronize(dev)
        with torch.cuda.stream(stream):
            fdas.fdas_search_batch(batch, xs, lens, d_out, d_cnt)   # views + capture
        torch.cuda.synchronize(dev)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record(stream)
        with torch.cuda.stream(stream):
            for _ in range(reps):
                fdas.fdas_search_batch(batch, xs, lens, d_out, d_cnt)
        ev[1].record(stream)
        torch.cuda.synchronize(dev)
        g_ms = ev[0].elapsed_time(ev[1]) / reps
        cands = int(d_cnt.sum().item())
        fdas.fdas_batch_set_graphs(batch, 0)
        ev[0].record(stream)
        with torch.cuda.stream(stream):
            fdas.fdas_search_batch(batch, xs, lens, d_out, d_cnt)
        ev[1].record(stream)
        torch.cuda.synchronize(dev)
        d_ms = ev[0].elapsed_time(ev[1])
        info = fdas.fdas_batch_get_info(batch)
    finally:
        fdas.fdas_batch_destroy(batch)
    return {"trials": n_trials, "N_min": min(lens), "N_max": max(lens),
            "distinct_N": len(set(lens)), "zmax": 200, "template_width": 512,
            "segment": info.segment,
            "harmsum_block": info.hs_block,
            "tuner": {"segments": list(info.tuned_segment[:info.n_tuned]),
                      "harmsum_blocks": list(info.tuned_hs_block[:info.n_tuned]),
                      "trial_ms_at_N_max": [round(v, 4) for v in info.tuned_ms[:info.n_tuned]],
                      "seconds": tune_s},
            "graph": {"value": n_trials * 1e3 / g_ms, "unit": "trials/s", "ms_per_batch": g_ms,
                      "batches": reps, "builds": info.graph_builds,
                      "launches": info.graph_launches},
            "direct": {"value": n_trials * 1e3 / d_ms, "unit": "trials/s", "ms_per_batch": d_ms},
            "candidates_per_batch": cands,
            "what": "series resident in HBM; one fdas_search_batch = one graph launch of all "
                    "trials' kernels"}


# ---------------------------------------------------------------------------
# Precision variants: the correlation of Eq. 1 as a tensor-core GEMM with
# hi/lo-split bf16 or fp16 operands (float32 accumulation), same workload.
# Agreement is measured against the float32 FFT path on the same series (the
# error against the FP64 oracle comes from the GPU parity tests).
# ---------------------------------------------------------------------------
def precision_variants(fdas, p, dev, stream, d_series, ref_plane, ref_keys, steps, peaks,
                       peak_kind):
    import torch
    out = {}
    max_cands = 1 << 22
    for name, mode in (("bf16_hilo", fdas.FDAS_CORR_GEMM_BF16), ("fp16_hilo", fdas.FDAS_CORR_GEMM_FP16)):
        plan = fdas.fdas_plan_create(p["N"], p["zmax"], p["dz"], p["m"], p["L"], p["nharm"],
                                     p["sigma"], max_cands, stream.cuda_stream)
        try:
            fdas.fdas_plan_set_correlation(plan, mode)
            info = fdas.fdas_plan_get_info(plan)
            d_out = torch.empty(max_cands * 16, dtype=torch.uint8, device=dev)
            d_cnt = torch.zeros(1, dtype=torch.int64, device=dev)
            with torch.cuda.stream(stream):
                for i in range(3):
                    fdas.fdas_search_device(plan, d_series[i % len(d_series)], 1, d_out, d_cnt)
            torch.cuda.synchronize(dev)
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            ev[0].record(stream)
            for i in range(steps):
                fdas.fdas_search_device(plan, d_series[i % len(d_series)], 1, d_out, d_cnt)
            ev[1].record(stream)
            torch.cuda.synchronize(dev)
            ms = ev[0].elapsed_time(ev[1]) / steps
            prof = np.stack([fdas.fdas_profile_trial(plan, d_series[0]) for _ in range(3)])
            corr_ms = float(np.median(prof[:, 3]))
            # agreement with the float32 path on series 0
            h_out = np.zeros(max_cands, dtype=fdas.CAND_DTYPE)
            h_cnt = np.zeros(1, dtype=np.int64)
            fdas.fdas_search(plan, d_series[0], 1, h_out, h_cnt)
            keys = {(int(c["r_top"]), int(c["z_idx"]), int(c["h"]))
                    for c in h_out[:min(int(h_cnt[0]), max_cands)]}
            plane = torch.empty(info.Z * info.nb, dtype=torch.float32, device=dev)
            fdas.fdas_plane_debug(plan, plane)
            torch.cuda.synchronize(dev)
            rel = float(((plane - ref_plane).abs() / ref_plane.clamp(min=1.0)).max().item())
            del plane
        finally:
            fdas.fdas_plan_destroy(plan)
        Z, nb, m = info.Z, info.nb, info.m
        rows = -(-2 * Z // 128) * 128
        flops = 2.0 * 2 * Z * nb * 6 * m           # useful: 2Z rows x 6m x nb
        issued = 2.0 * rows * nb * 6 * m           # rows padded to the 128-row tile
        # the kernel is timed alone between events: the burst figure
        peak = peaks.get("bf16_tflops", PEAKS_FALLBACK["bf16_tflops"])
        ach = flops / (corr_ms / 1e3) / 1e12
        out[name] = {
            "value": 1e3 / ms, "unit": "trials/s", "ms_per_step": ms, "steps": steps,
            "stage_ms": {s: float(np.median(prof[:, i])) for i, s in
                         enumerate(["spectrum", "whiten", "segments", "correlate", "harmsum"])},
            "roofline": {"kernel": "k_gemm_correlate", "bound": "tensor", "achieved": ach,
                         "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                         "issued_frac": issued / (corr_ms / 1e3) / 1e12 / peak,
                         "peak_source": f"{peak_kind} bf16_tflops (fp16 dense rate = bf16)",
                         "algorithmic": f"2 x 2Z x nb x 6m = {flops:.3e} flop per launch "
                                        f"(3 hi/lo products, complex as 2 real rows)"},
            "vs_fp32_path": {"plane_max_rel": rel, "what": "max |dP|/max(P,1) over the whole "
                             "plane against the float32 FFT path, same series",
                             "candidates": len(keys), "fp32_candidates": len(ref_keys),
                             "common": len(keys & ref_keys)},
        }
    return out


# ---------------------------------------------------------------------------
# CPU baseline: the FP64 oracle as it stands, its plane rows spread over the
# host cores by a process pool (spawn: no worker inherits a CUDA context).
# ---------------------------------------------------------------------------
_W = {}


def _pool_init(xw_bytes, nb, m):
    _W["Xw"] = np.frombuffer(xw_bytes, dtype=np.complex128, count=nb)
    _W["m"] = m


def _pool_row(z):
    """One plane row of the oracle (template + zero-padded FFT correlation);
    returns the seconds it took in the worker."""
    from oracle import fdas_oracle as O
    t0 = time.perf_counter()
    tau = O.template_fresnel(float(z), _W["m"])
    O.correlate_row(_W["Xw"], tau)
    return time.perf_counter() - t0


def _pool_hs(args):
    """The oracle's harmonic sums and threshold over a (Z, width) sub-plane
    of unit exponentials (the whitened-noise plane's distribution)."""
    from oracle import fdas_oracle as O
    seed, Z, width, nharm, sigma = args
    P = np.random.default_rng(seed).exponential(size=(Z, width))
    H = O.harmonic_sums(P, nharm)
    T = O.thresholds(nharm, sigma)
    for h, v in H.items():
        np.nonzero(v >= T[h])
    return width


def _oracle_pool(Xw, m, cores):
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    return ctx.Pool(cores, initializer=_pool_init, initargs=(Xw.tobytes(), Xw.shape[0], m))


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_trial_estimate(x, p, rows=32, hs_width=1 << 16, small=None):
    """Trials/s of the oracle on this host's cores, from a bounded sample of
    one trial of the workload: the spectrum and whitening of the full series
    (one core), `rows` of the Z plane rows (one per task, on a pool of all
    cores, wall clock), and the harmonic sums and threshold over `hs_width` of
    the nb top bins (all Z rows); each part scaled to the whole trial. With
    `small` = (series, params) the whole oracle search of that (small)
    workload is also timed end to end."""
    from oracle import fdas_oracle as O
    cores = host_cores()
    t0 = time.perf_counter()
    Xw = O.whiten(O.spectrum(x))
    t_pre = time.perf_counter() - t0
    zs = O.z_values(p["zmax"], p["dz"])
    Z = len(zs)
    pick = zs[:: max(1, Z // rows)][:rows]
    with _oracle_pool(Xw, p["m"], cores) as pool:
        pool.map(_pool_row, pick[:cores])          # workers up and warm
        t0 = time.perf_counter()
        pool.map(_pool_row, pick, chunksize=1)
        t_rows = (time.perf_counter() - t0) * Z / len(pick)
        t0 = time.perf_counter()
        done = sum(pool.map(_pool_hs, [(i, Z, hs_width, p["nharm"], p["sigma"])
                                       for i in range(cores)], chunksize=1))
        t_hs = (time.perf_counter() - t0) * (x.shape[0] // 2) / done
    total = t_pre + t_rows + t_hs
    out = {"value": 1.0 / total, "unit": "trials/s", "cores": cores, "kind": "oracle",
           "sample": (f"FP64 oracle on {cores} host cores: full spectrum+whitening (1 core, "
                      f"{t_pre:.2f} s), {len(pick)} of {Z} plane rows on a {cores}-process pool "
                      f"({t_rows * len(pick) / Z:.2f} s wall), harmonic sums over {cores} x {hs_width} of "
                      f"{x.shape[0] // 2} bins x {Z} rows on the pool; rows and bins scaled to "
                      f"one trial"),
           "seconds_per_trial": total}
    if small is not None:
        xs, ps = small
        t0 = time.perf_counter()
        O.search(xs, ps["zmax"], ps["dz"], ps["m"], ps["nharm"], ps["sigma"])
        out["small_workload"] = {"workload": "cfg1_n2e17_z50", "trials": 1,
                                 "trials_per_s": 1.0 / (time.perf_counter() - t0),
                                 "cores": 1, "what": "whole oracle search of the 2^17-sample, "
                                                     "zmax = 50 trial, end to end"}
    return out


def run_reference(args):
    """The oracle as the reference arm, on a pool of all host cores: each
    step is 1/Z of a trial (one plane row, 1/Z of the harmonic sums and of
    the spectrum+whitening); steps run concurrently, one per core."""
    from oracle import fdas_oracle as O
    from synthetic import workload
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    x, p = workload(WORKLOAD)
    zs = O.z_values(p["zmax"], p["dz"])
    Z = len(zs)
    t0 = time.perf_counter()
    Xw = O.whiten(O.spectrum(x))
    t_pre = (time.perf_counter() - t0) / Z
    rng = np.random.default_rng(0)
    width = max(1, (x.shape[0] // 2) // Z)
    Psub = rng.exponential(size=(Z, width))
    T = O.thresholds(p["nharm"], p["sigma"])
    t0 = time.perf_counter()
    H = O.harmonic_sums(Psub, p["nharm"])
    for h, v in H.items():
        np.nonzero(v >= T[h])
    t_hs = time.perf_counter() - t0           # 1/Z of the harmonic sums (one core)
    cores = host_cores()
    with _oracle_pool(Xw, p["m"], cores) as pool:
        pool.map(_pool_row, [zs[i % Z] for i in range(args.warmup)], chunksize=1)
        t0 = time.perf_counter()
        pool.map(_pool_row, [zs[i % Z] for i in range(args.steps)], chunksize=1)
        wall = time.perf_counter() - t0
    dt = wall / args.steps + (t_pre + t_hs) / cores
    value = 1.0 / (Z * dt)
    sample = (f"each step = 1/{Z} of a trial (one plane row on one of {cores} pool processes, "
              f"plus 1/{Z} of the spectrum+whitening and of the harmonic sums over all bins, "
              f"timed on one core and shared over the {cores} cores)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "trials/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "N": p["N"], "zmax": p["zmax"], "dz": p["dz"],
                       "templates": Z, "template_width": p["m"], "segment": p["L"],
                       "nharm": p["nharm"], "sigma": p["sigma"]},
            "cpu_baseline": {"value": value, "unit": "trials/s", "cores": cores,
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "trials/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------------------
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=None)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--series", type=int, default=4, help="distinct resident series cycled")
    ap.add_argument("--log2n", type=int, default=None,
                    help="smaller series length for profiling captures (not a bench value)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-plain", action="store_true", help="skip the plain FP32 comparator")
    ap.add_argument("--plain-steps", type=int, default=10)
    ap.add_argument("--no-serve", action="store_true", help="skip the serving measurement")
    ap.add_argument("--no-batch", action="store_true",
                    help="skip the batched uneven-trial measurement")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the tensor-core precision variants")
    ap.add_argument("--corr", choices=["fft", "bf16", "fp16"], default="fft",
                    help="correlation mode of the timed path (profiling; default fft)")
    ap.add_argument("--segment", type=int, default=None,
                    help="overlap-save segment length (default: the workload's 8192)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)

    import __graft_entry__
    __graft_entry__.build()
    from paper_1511_07343_gb300 import fdas
    from synthetic import workload

    if args.log2n is not None:
        from synthetic import WORKLOADS, make_series, random_chirps
        p = dict(WORKLOADS[WORKLOAD])
        p["N"] = 1 << args.log2n
        rng = np.random.default_rng(11)
        series = [make_series(p["N"], 20 + i, random_chirps(rng, 20, p["N"], p["zmax"]),
                              device=dev) for i in range(args.series)]
    else:
        x0, p = workload(WORKLOAD, seed=2 + 1000 * rank, device=dev)
        series = [x0] + [workload(WORKLOAD, seed=3 + i + 1000 * rank, device=dev)[0]
                         for i in range(args.series - 1)]
    d_series = [torch.from_numpy(s).to(dev) for s in series]

    if args.segment is not None:
        p["L"] = args.segment
    stream = torch.cuda.Stream(dev)
    max_cands = 1 << 22
    plan = fdas.fdas_plan_create(p["N"], p["zmax"], p["dz"], p["m"], p["L"], p["nharm"],
                                 p["sigma"], max_cands, stream.cuda_stream)
    if args.corr != "fft":
        fdas.fdas_plan_set_correlation(plan, {"bf16": 1, "fp16": 2}[args.corr])
    info = fdas.fdas_plan_get_info(plan)
    # a step is one DM trial; the timed loop hands the library the resident
    # series several at a time (one fdas_search_device call of T trials,
    # which the library runs on two trial lanes that overlap on the GPU)
    T = len(d_series)
    d_all = torch.cat(d_series)
    d_out = torch.empty(T * max_cands * 16, dtype=torch.uint8, device=dev)
    d_cnt = torch.zeros(T, dtype=torch.int64, device=dev)

    def trials(n):
        fdas.fdas_search_device(plan, d_all, n, d_out, d_cnt)

    def step(i):  # one trial alone
        fdas.fdas_search_device(plan, d_series[i % T], 1, d_out, d_cnt)

    with torch.cuda.stream(stream):
        for i in range(-(-args.warmup // T)):
            trials(T)
    torch.cuda.synchronize(dev)

    calls = [min(T, args.steps - i) for i in range(0, args.steps, T)]
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    with ClockSampler(local) as clk:
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)
        clk.mark_start()
        evs[0].record(stream)
        for n in calls:
            trials(n)
        evs[1].record(stream)
        torch.cuda.synchronize(dev)
        clk.mark_end()
        if world > 1:
            dist.barrier()
    ms = reduce_max(evs[0].elapsed_time(evs[-1]), world, dev)
    clocks = clk.summary()
    ms_per_step = ms / args.steps
    value = args.steps * world / (ms / 1e3)
    n_cands = int(d_cnt[0].item())
    # per-trial device latency: single-trial calls back to back
    nlat = min(args.steps, 50)
    lev = [torch.cuda.Event(enable_timing=True) for _ in range(nlat + 1)]
    lev[0].record(stream)
    for i in range(nlat):
        step(i)
        lev[i + 1].record(stream)
    torch.cuda.synchronize(dev)
    step_ms = [lev[i].elapsed_time(lev[i + 1]) for i in range(nlat)]

    # per-stage times (CUDA events inside the library, same stream)
    stages = ["spectrum", "whiten", "segments", "correlate", "harmsum"]
    prof = np.stack([fdas.fdas_profile_trial(plan, d_series[i % len(d_series)])
                     for i in range(3)])
    stage_ms = {s: float(np.median(prof[:, i])) for i, s in enumerate(stages)}

    # end to end through the C ABI with host buffers: K page-locked host
    # series in one fdas_search_host call (the library overlaps each trial's
    # copies with the previous trial's kernels), candidates sorted on the host
    e2e_steps = 0 if args.no_e2e else (args.e2e_steps or 32)
    h_series = torch.from_numpy(series[0]).pin_memory()
    h_out = np.zeros(max(e2e_steps, 1) * max_cands, dtype=fdas.CAND_DTYPE)
    h_cnt = np.zeros(max(e2e_steps, 1), dtype=np.int64)
    e2e_s, d2h = None, 0
    if e2e_steps:
        h_multi = torch.from_numpy(np.concatenate([series[i % len(series)]
                                                   for i in range(e2e_steps)])).pin_memory()
        fdas.fdas_search_host(plan, h_multi.data_ptr(), e2e_steps, h_out, h_cnt)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        fdas.fdas_search_host(plan, h_multi.data_ptr(), e2e_steps, h_out, h_cnt)
        e2e_s = (time.perf_counter() - t0) / e2e_steps
        d2h = sum(8 + 16 * int(min(c, max_cands)) for c in h_cnt)
        del h_multi
    e2e_lat = []
    for i in range(min(e2e_steps, 10)):
        t1 = time.perf_counter()
        fdas.fdas_search_host(plan, h_series.data_ptr(), 1, h_out, h_cnt)
        e2e_lat.append((time.perf_counter() - t1) * 1e3)

    # the plain FP32 comparator on the same GPU, same series
    plain = None
    if not args.no_plain:
        pstep = plain_fp32_path(fdas, plan, info, p, dev, stream)
        for i in range(2):
            pstep(d_series[i % len(d_series)])
        torch.cuda.synchronize(dev)
        pe = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        pe[0].record(stream)
        for i in range(args.plain_steps):
            pcnt = pstep(d_series[i % len(d_series)])
        pe[1].record(stream)
        torch.cuda.synchronize(dev)
        pms = reduce_max(pe[0].elapsed_time(pe[1]), world, dev) / args.plain_steps
        # candidate recovery of both paths on the same series
        agree = []
        for i in range(min(2, len(d_series))):
            pcnt = pstep(d_series[i])
            torch.cuda.synchronize(dev)
            k = min(int(pcnt.item()), max_cands)
            plain_c = pstep.cands[: k * 16].cpu().numpy().view(fdas.CAND_DTYPE)
            fdas.fdas_search(plan, d_series[i], 1, h_out, h_cnt)
            fused_c = h_out[: min(int(h_cnt[0]), max_cands)]
            agree.append(candidate_agreement(fused_c, plain_c, info.thresholds))
        plain = {"value": world * 1e3 / pms, "unit": "trials/s", "ms_per_step": pms,
                 "steps": args.plain_steps, "speedup": value / (world * 1e3 / pms),
                 "candidates_last_step": int(pcnt.item()),
                 "recovery": agree,
                 "what": "unfused FP32 path: cuFFT (torch.fft) real FFT, segment and inverse FFTs, "
                         "elementwise multiply into a materialised complex plane, power, edge trim; "
                         "this library's whitening and harmonic sum"}
    # candidate distillation of the last timed step's list
    d_pk = torch.empty(max_cands * 24, dtype=torch.uint8, device=dev)
    d_npk = torch.zeros(1, dtype=torch.int64, device=dev)
    with torch.cuda.stream(stream):
        fdas.fdas_distill(plan, d_out, d_cnt, d_pk, d_npk)   # first call builds the table
        dev_ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        dev_ev[0].record(stream)
        for _ in range(5):
            fdas.fdas_distill(plan, d_out, d_cnt, d_pk, d_npk)
        dev_ev[1].record(stream)
    torch.cuda.synchronize(dev)
    distill = {"ms": dev_ev[0].elapsed_time(dev_ev[1]) / 5, "candidates": n_cands,
               "peaks": int(d_npk.item()),
               "what": "local maxima per level + cross-level matching, sigma per peak"}
    del d_pk
    # the block-median whitening variant on the same plan and series
    fdas.fdas_plan_set_whitening(plan, fdas.FDAS_WHITEN_BLOCK)
    prof_b = np.stack([fdas.fdas_profile_trial(plan, d_series[i % len(d_series)])
                       for i in range(3)])
    fdas.fdas_plan_set_whitening(plan, fdas.FDAS_WHITEN_RUNNING)
    whitening_variants = {
        "running_median_ms": stage_ms["whiten"],
        "block_median_ms": float(np.median(prof_b[:, 1])),
        "block_trial_ms": float(np.median(prof_b.sum(axis=1))),
        "what": "whitening stage time (CUDA events); block = medians of 64-bin blocks, "
                "linearly interpolated"}
    # half-bin planes (Z x 2 nb, the paper's Fig. 1 resolution) on the same plan
    half_bin = None
    if rank == 0 and not args.no_variants:
        fdas.fdas_plan_set_interbin(plan, 1)
        prof_h = np.stack([fdas.fdas_profile_trial(plan, d_series[i % len(d_series)])
                           for i in range(3)])
        fdas.fdas_plan_set_interbin(plan, 0)
        half_bin = {
            "trial_ms": float(np.median(prof_h.sum(axis=1))),
            "value": 1e3 / float(np.median(prof_h.sum(axis=1))), "unit": "trials/s",
            "stage_ms": {s: float(np.median(prof_h[:, i])) for i, s in enumerate(stages)},
            "what": "2Z template rows (offsets 0 and 1/2), plane of Z x 2nb half bins; "
                    "harmsum stage includes the 4-bin maxima kernel"}
    variants_ref = None
    if rank == 0 and not args.no_variants and args.corr == "fft":
        ref_plane = torch.empty(info.Z * info.nb, dtype=torch.float32, device=dev)
        fdas.fdas_search(plan, d_series[0], 1, h_out, h_cnt)
        fdas.fdas_plane_debug(plan, ref_plane)
        torch.cuda.synchronize(dev)
        ref_keys = {(int(c["r_top"]), int(c["z_idx"]), int(c["h"]))
                    for c in h_out[:min(int(h_cnt[0]), max_cands)]}
        variants_ref = (ref_plane, ref_keys)
    fdas.fdas_plan_destroy(plan)

    peaks, peak_kind = load_peaks()
    # dominant kernel and its roofline
    dom = max(stage_ms, key=stage_ms.get)
    N, Z, L, m, V, S, nb = p["N"], info.Z, info.L, info.m, info.V, info.S, info.nb
    if dom == "correlate" and args.corr != "fft":
        flops = 2.0 * 2 * Z * nb * 6 * m
        peak = peaks.get("bf16_tflops", PEAKS_FALLBACK["bf16_tflops"])
        achieved = flops / (stage_ms[dom] / 1e3) / 1e12
        roof = {"kernel": "k_gemm_correlate", "bound": "tensor", "achieved": achieved,
                "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak, "traffic": None,
                "peak_source": f"{peak_kind} bf16_tflops",
                "algorithmic": f"2 x 2Z x nb x 6m = {flops:.3e} flop per launch"}
    elif dom == "correlate":
        flops = S * Z * (5.0 * L * math.log2(L) + 6.0 * L + 3.0 * V)
        sm_max = peaks.get("sm_max_mhz", 2070.0)
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        peak = sms * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
        achieved = flops / (stage_ms[dom] / 1e3) / 1e12
        # HBM view of the same launch: the plane and 4-bin maxima it writes,
        # the segment spectra and template bank it reads (once each)
        hbm_bytes = Z * nb * 4.0 + Z * (nb // 4) * 4.0 + S * L * 8.0 + Z * L * 8.0
        hbm_ach = hbm_bytes / (stage_ms[dom] / 1e3) / 1e9
        roof = {"kernel": "k_correlate_fused", "bound": "alu", "achieved": achieved, "peak": peak,
                "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": measured_traffic("k_correlate_fused"),
                "peak_source": f"FP32 FMA: {sms} SMs x {FP32_LANES_PER_SM} lanes x 2 x "
                               f"{sm_max:.0f} MHz (derived; {peak_kind} sm_max_mhz)",
                "algorithmic": f"S*Z*(5 L log2 L + 6 L + 3 V) = {flops:.3e} flop per launch",
                "hbm": {"achieved": hbm_ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                        "frac": hbm_ach / peaks["hbm_gbs"], "bytes": hbm_bytes,
                        "peak_source": f"{peak_kind} hbm_gbs",
                        "algorithmic": "plane + 4-bin maxima written, segment spectra + "
                                       "template bank read once"}}
    else:
        nbytes = Z * (nb // 4) * 4.0  # one read of the 4-bin maxima
        peak = peaks["hbm_gbs"]
        achieved = nbytes / (stage_ms[dom] / 1e3) / 1e9
        roof = {"kernel": "k_harmsum_staged" if dom == "harmsum" else dom, "bound": "hbm",
                "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": measured_traffic("k_harmsum_staged") if dom == "harmsum" else None,
                "peak_source": f"{peak_kind} hbm_gbs",
                "algorithmic": f"one read of the Z x nb/4 float32 4-bin maxima = {nbytes:.3e} B "
                               "per launch"}

    line = {"metric": METRIC, "value": value, "unit": "trials/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "N": N, "zmax": p["zmax"], "dz": p["dz"],
                       "templates": Z, "template_width": m, "segment": L, "nharm": p["nharm"],
                       "sigma": p["sigma"], "parallelism": f"replicas{world}",
                       "l2": f"{len(d_series)} resident series cycled; each step writes a "
                             f"{Z * nb * 4 / 1e9:.2f} GB plane (> L2)",
                       "trials_per_call": len(d_series)},
            "stage_ms": stage_ms, "candidates_last_step": n_cands,
            "whitening_variants": whitening_variants,
            "distill": distill,
            "half_bin_plane": half_bin,
            "latency_ms": dict(percentiles(step_ms),
                               what="per-trial device time, single-trial calls back to back"),
            "vs_plain_fp32": plain,
            "roofline": roof,
            "clocks": clocks,
            "e2e": {"value": 1.0 / e2e_s if e2e_steps else None, "unit": "trials/s",
                    "h2d_bytes_per_step": 4 * N,
                    "d2h_bytes_per_step": int(d2h / max(e2e_steps, 1)),
                    "trials_per_call": e2e_steps,
                    "latency_ms": dict(percentiles(e2e_lat),
                                       what="one-trial fdas_search_host calls, wall clock")},
            "gpu_launches": int(info_kernels_per_trial() * args.steps),
            "peaks": {"source": peak_kind, "hbm_gbs": peaks.get("hbm_gbs")}}
    if variants_ref is not None:
        line["precision_variants"] = precision_variants(
            fdas, p, dev, stream, d_series, variants_ref[0], variants_ref[1], 10, peaks, peak_kind)
        del variants_ref
    if rank == 0 and not args.no_batch and args.log2n is None:
        line["batch_uneven"] = batch_measure(fdas, dev)
    if args.corr != "fft":
        line["config"]["correlation"] = args.corr + "_hilo_tensor_core"
    if rank == 0 and not args.no_serve and args.log2n is None:
        line["serving"] = serve_measure(dev)
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = oracle_trial_estimate(series[0], p,
                                                     small=workload("cfg1_n2e17_z50"))
    if world > 1:
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line))
    return 0


def info_kernels_per_trial():
    # real FFT (columns, rows, unpack), whitening, segment FFTs, correlation,
    # harmonic-sum screen and exact sums of the flagged pairs
    return 8


if __name__ == "__main__":
    sys.exit(main())
