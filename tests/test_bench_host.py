"""Host-side logic of bench.py: the max-over-ranks timing reduction used
when one process runs per GPU (checked here with two gloo ranks on CPU) and
the latency percentiles."""
import os
import socket

import numpy as np
import pytest

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # each rank reports its own step time; the job time is the slowest rank's
    got = bench.reduce_max(10.0 + 5.0 * rank, world)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, got))


def test_reduce_max_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert out == {0: 15.0, 1: 15.0}


def test_reduce_max_single_rank_is_identity():
    assert bench.reduce_max(3.5, 1) == 3.5


def test_percentiles():
    xs = np.arange(1, 101, dtype=float)
    p = bench.percentiles(xs)
    assert p["p50"] == pytest.approx(50.5)
    assert p["p99"] == pytest.approx(99.01)
    assert bench.percentiles([])["p50"] is None


def test_measured_traffic_follows_the_kernel_source(tmp_path, monkeypatch):
    """A stored DRAM-traffic figure is reported only while the kernel source
    it was captured with is unchanged (sha256 prefix); unknown kernels have
    none."""
    import hashlib
    src = tmp_path / "k.cu"
    src.write_bytes(b"__global__ void k() {}\n")
    digest = hashlib.sha256(src.read_bytes()).hexdigest()[:16]
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "MEASURED_TRAFFIC", {"k": (1.5e9, "k.cu", digest)})
    assert bench.measured_traffic("k") == 1.5e9
    assert bench.measured_traffic("other") is None
    src.write_bytes(b"__global__ void k() { /* changed */ }\n")
    assert bench.measured_traffic("k") is None


def test_committed_traffic_figures_match_their_sources():
    """Every stored figure names a committed kernel file; a mismatch makes the
    bench report null traffic, so the figure and the source move together."""
    for kernel, (nbytes, path, digest) in bench.MEASURED_TRAFFIC.items():
        assert os.path.exists(os.path.join(bench.ROOT, path)), path
        assert len(digest) == 16 and nbytes > 0
        assert bench.measured_traffic(kernel) == nbytes, kernel


def _sampler_with(tmp_path, lines, window):
    s = bench.ClockSampler(0)
    f = open(tmp_path / "clocks.csv", "w+")
    f.write("".join(l + "\n" for l in lines))
    s.file, s.proc, s.window = f, object(), list(window)
    return s


def _row(ts, sm, mx=2070, power=600.0, active="0x0", hw="Not Active", thermal="Not Active",
         swt="Not Active", cap="Not Active"):
    return f"0, {sm}, {mx}, {power}, {active}, {hw}, {thermal}, {swt}, {cap}, {ts}"


def test_clock_summary_keeps_samples_of_the_timed_region(tmp_path):
    """Median SM clock, maximum and throttle reasons come from the samples
    inside the timed window (one sample period of slack); samples outside
    (here a slow clock with hw_slowdown before the window) do not count."""
    import datetime
    base = datetime.datetime(2026, 1, 2, 3, 4, 5)
    stamp = lambda s: (base + datetime.timedelta(seconds=s)).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
    lines = [_row(stamp(0.0), 900, hw="Active")] + \
        [_row(stamp(1.0 + 0.02 * i), 2070 if i % 4 else 2040) for i in range(20)] + \
        [_row(stamp(3.0), 1200, cap="Active")]
    t0 = (base + datetime.timedelta(seconds=1.0)).timestamp()
    t1 = (base + datetime.timedelta(seconds=1.4)).timestamp()
    out = _sampler_with(tmp_path, lines, (t0, t1)).summary()
    assert out["samples_in_timed_region"] is True
    assert out["samples"] == 20
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == []
    assert out["power_w_max"] == 600.0


def test_clock_summary_reports_throttle_reasons(tmp_path):
    """Active throttle reasons inside the window are named; with no sample in
    the window all samples are used and the summary says so."""
    lines = [_row("2026/01/02 03:04:05.000", 1500, hw="Active", cap="Active"),
             _row("2026/01/02 03:04:05.020", 1600, thermal="Active")]
    out = _sampler_with(tmp_path, lines, (0.0, 1.0)).summary()
    assert out["samples_in_timed_region"] is False
    assert out["samples"] == 2 and out["sm_mhz"] == 1550.0
    assert out["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_power_cap"]


def test_clock_summary_without_nvidia_smi():
    s = bench.ClockSampler(0)
    assert s.summary()["reasons"] == ["nvidia-smi unavailable"]


def test_candidate_agreement_counts_keys_and_the_threshold_band():
    """Common keys, keys in one list only, and which of those lie outside the
    1e-4 T_h band (judged by the power the list holding the key reports)."""
    dt = np.dtype([("r_top", "<i4"), ("z_idx", "<i4"), ("h", "<i4"), ("power", "<f4")])
    thr = [10.0, 20.0, 30.0, 40.0, 50.0]
    a = np.array([(5, 1, 1, 12.0), (6, 1, 2, 25.0), (7, 2, 4, 30.0005), (8, 0, 16, 51.0)], dtype=dt)
    b = np.array([(5, 1, 1, 12.0), (6, 1, 2, 25.0), (9, 3, 8, 40.001), (10, 3, 8, 47.0)], dtype=dt)
    out = bench.candidate_agreement(a, b, thr)
    assert out == {"common": 2, "only_fused": 2, "only_plain": 2,
                   "only_fused_outside_band": 1, "only_plain_outside_band": 1}


def _run_bench(args, env_extra=None, timeout=900):
    import subprocess
    import sys
    env = dict(os.environ, **(env_extra or {}))
    return subprocess.run([sys.executable, os.path.join(bench.ROOT, "bench.py")] + args,
                          capture_output=True, text=True, timeout=timeout, env=env,
                          cwd=bench.ROOT)


def test_reference_arm_prints_one_line_of_the_contract():
    """`bench.py --impl reference` times the oracle on the host cores (no GPU)
    and prints one JSON line with the metric, the reference marker, the
    cpu_baseline description and an e2e entry without host-device bytes."""
    import json
    r = _run_bench(["--impl", "reference", "--steps", "2", "--warmup", "3"])
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC
    assert d["unit"] == "trials/s" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["steps"] == 2 and d["warmup"] == 3 and d["dtype"] == "f64"
    assert d["config"]["workload"] == bench.WORKLOAD and d["config"]["N"] == 1 << 23
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1
    assert d["e2e"] == {"value": d["value"], "unit": "trials/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_exit_quietly():
    r = _run_bench(["--impl", "reference", "--steps", "2", "--warmup", "3"],
                   env_extra={"RANK": "1", "WORLD_SIZE": "2"}, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == ""
