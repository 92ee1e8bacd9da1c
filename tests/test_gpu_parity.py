"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances (each follows from the float32 arithmetic of its stage):
  * template taps: float64 on both sides, |d tau| <= 1e-12;
  * template spectra (float32 store of a float64 DFT): <= 2e-7 * max |T|;
  * spectrum (float32 FFT of length N): max |dX| <= 2e-5 * rms(X);
  * whitened spectrum: max |dXw| <= 5e-5 (Xw has unit rms);
  * plane: |P_gpu - P_orc| <= 1e-4 * max(P_orc, 1);
  * candidates: identical (r, j, h) keys except keys whose oracle H_h lies
    within 1e-4 * T_h of T_h.
"""
import math

import numpy as np
import pytest
import torch

from oracle import fdas_oracle as O
from synthetic import Chirp, make_series, workload

pytestmark = pytest.mark.gpu

DEV = torch.device("cuda:0") if torch.cuda.is_available() else None


def make_plan(fd, N, zmax, dz, m, L, nharm, max_cands=1 << 20, sigma=6.0):
    stream = torch.cuda.current_stream(DEV).cuda_stream
    return fd.fdas_plan_create(N, zmax, dz, m, L, nharm, sigma, max_cands, stream)


def dev_c64(a):
    t = torch.from_numpy(np.ascontiguousarray(a.astype(np.complex64))).to(DEV)
    return t


def to_np_c(t):
    return t.cpu().numpy().astype(np.complex128)


def gpu_plane(fd, plan, info):
    plane = torch.empty(info.Z * info.nb, dtype=torch.float32, device=DEV)
    fd.fdas_plane_debug(plan, plane)
    torch.cuda.synchronize()
    return plane.cpu().numpy().reshape(info.Z, info.nb).astype(np.float64)


def search_one(fd, plan, info, x):
    d_x = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).to(DEV)
    out = np.zeros(info.max_cands, dtype=fd.CAND_DTYPE)
    counts = np.zeros(1, dtype=np.int64)
    fd.fdas_search(plan, d_x, 1, out, counts)
    return out[: min(counts[0], info.max_cands)], int(counts[0])


def keys(c):
    return {(int(a["r_top"]), int(a["z_idx"]), int(a["h"])) for a in c}


def assert_candidates_match(got_keys, cands, H, T):
    want = {(c[0], c[1], c[2]) for c in cands}
    bad = []
    for key in got_keys ^ want:
        r, j, h = key
        if abs(H[h][j, r] - T[h]) > 1e-4 * T[h]:
            bad.append((key, H[h][j, r], T[h], key in got_keys))
    assert not bad, bad[:10]


# --------------------------------------------------------------- templates --
@pytest.mark.parametrize("zmax,m,L", [(200, 512, 8192), (50, 128, 2048), (100, 256, 4096)])
def test_template_taps_and_spectra(gpu_lib, zmax, m, L):
    fd = gpu_lib
    plan = make_plan(fd, 1 << 12, zmax, 2, m, L, 1)
    try:
        info = fd.fdas_plan_get_info(plan)
        taps = torch.empty(info.Z * m * 2, dtype=torch.float64, device=DEV)
        bank = torch.empty(info.Z * L * 2, dtype=torch.float32, device=DEV)
        fd.fdas_template_taps(plan, taps)
        fd.fdas_template_bank(plan, bank)
        torch.cuda.synchronize()
    finally:
        fd.fdas_plan_destroy(plan)
    t_gpu = taps.cpu().numpy().view(np.complex128).reshape(info.Z, m)
    t_orc = O.template_bank(zmax, 2, m)
    assert np.max(np.abs(t_gpu - t_orc)) <= 1e-12
    b_gpu = bank.cpu().numpy().view(np.complex64).reshape(info.Z, L).astype(np.complex128)
    g = np.zeros((info.Z, L), dtype=np.complex128)
    d = np.arange(-m // 2, m // 2)
    g[:, np.mod(d, L)] = t_orc
    b_orc = np.fft.ifft(g, axis=1)          # (1/L) sum_j g[j] exp(+2 pi i j k / L)
    assert np.max(np.abs(b_gpu - b_orc)) <= 2e-7 * np.max(np.abs(b_orc))


# ---------------------------------------------------------------- spectrum --
@pytest.mark.parametrize("logn", [12, 13, 14, 17, 20, 23])
def test_spectrum_and_whitening(gpu_lib, logn):
    fd = gpu_lib
    N = 1 << logn
    x = make_series(N, 100 + logn, [Chirp(0.3 * N / 2, 10.0, 9.0, 1.1, 2)])
    plan = make_plan(fd, N, 20, 2, 64, 2048, 1)
    try:
        d_x = torch.from_numpy(x).to(DEV)
        spec = torch.empty(N, dtype=torch.float32, device=DEV)
        white = torch.empty(N, dtype=torch.float32, device=DEV)
        fd.fdas_stage_spectrum(plan, d_x, spec)
        fd.fdas_stage_whiten(plan, spec, white)
        torch.cuda.synchronize()
    finally:
        fd.fdas_plan_destroy(plan)
    X_gpu = spec.cpu().numpy().view(np.complex64).astype(np.complex128)
    X_orc = O.spectrum(x)
    rms = math.sqrt(np.mean(np.abs(X_orc) ** 2))
    assert np.max(np.abs(X_gpu - X_orc)) <= 2e-5 * rms
    W_gpu = white.cpu().numpy().view(np.complex64).astype(np.complex128)
    W_orc = O.whiten(X_orc)
    assert W_gpu[0] == 0
    assert np.max(np.abs(W_gpu - W_orc)) <= 5e-5


@pytest.mark.parametrize("N,two", [(1 << 15, False), (12288, False), (1 << 15, True)])
def test_whitening_exact_medians_with_ties(gpu_lib, N, two):
    """Small-integer spectra make every power exact in float32 and full of
    ties, so the medians are exact order statistics: the whitened spectrum
    must match the oracle to float32 rounding of the scale (N = 12288 gives a
    tile count that is not a multiple of a CTA's tiles). With `two` every
    power is 1 or 2, so most windows hold two long runs of equal keys and
    the median sits at or between them: a sort that lost or duplicated an
    entry among equal keys would move it."""
    fd = gpu_lib
    nb = N // 2
    rng = np.random.default_rng(N)
    if two:
        X = np.where(rng.random(nb) < 0.5, 1.0 + 0j, 1.0 + 1j).astype(np.complex64)
    else:
        X = (rng.integers(1, 4, nb) + 1j * rng.integers(0, 3, nb)).astype(np.complex64)
    plan = make_plan(fd, N, 20, 2, 64, 2048, 1)
    try:
        spec = torch.from_numpy(X.view(np.float32).copy()).to(DEV)
        white = torch.empty(N, dtype=torch.float32, device=DEV)
        fd.fdas_stage_whiten(plan, spec, white)
        torch.cuda.synchronize()
    finally:
        fd.fdas_plan_destroy(plan)
    W_gpu = white.cpu().numpy().view(np.complex64).astype(np.complex128)
    W_orc = O.whiten(X.astype(np.complex128))
    assert W_gpu[0] == 0
    assert np.max(np.abs(W_gpu - W_orc) / np.abs(W_orc[1:]).max()) <= 1e-6


# ------------------------------------------------------------------- plane --
@pytest.mark.parametrize("N,zmax,m,L", [
    (1 << 17, 50, 128, 2048),      # the 2^17-sample workload's shapes
    (1 << 14, 200, 512, 8192),     # zmax=200 templates, 2 segments, ragged tail
    (1 << 15, 100, 256, 4096),
    (1 << 12, 16, 64, 2048),       # a single segment longer than the spectrum
])
def test_plane_matches_oracle(gpu_lib, N, zmax, m, L):
    fd = gpu_lib
    rng = np.random.default_rng(N + zmax)
    nb = N // 2
    Xw = (rng.standard_normal(nb) + 1j * rng.standard_normal(nb)) / math.sqrt(2)
    Xw[100] += 12.0
    Xw = Xw.astype(np.complex64).astype(np.complex128)
    plan = make_plan(fd, N, zmax, 2, m, L, 1)
    try:
        info = fd.fdas_plan_get_info(plan)
        plane = torch.empty(info.Z * nb, dtype=torch.float32, device=DEV)
        fd.fdas_stage_plane(plan, dev_c64(Xw), plane)
        torch.cuda.synchronize()
    finally:
        fd.fdas_plan_destroy(plan)
    P_gpu = plane.cpu().numpy().reshape(info.Z, nb).astype(np.float64)
    P_orc = O.power_plane(Xw, O.template_bank(zmax, 2, m))
    rel = np.abs(P_gpu - P_orc) / np.maximum(P_orc, 1.0)
    assert rel.max() <= 1e-4, rel.max()


# ----------------------------------------------------------- harmonic sums --
@pytest.mark.parametrize("N", [1 << 13, 5 << 13])
@pytest.mark.parametrize("block", [32, 256])
def test_harmonic_sum_on_integer_plane_is_exact(gpu_lib, block, N):
    """Small integer powers make every float32 sum exact, so the GPU list
    must equal the oracle's list exactly (no threshold band needed), with
    either harmonic-sum block size; at N = 5 * 2^13 (20480 bins) the last
    256-thread tile runs past the spectrum, so its sub-harmonic slices end
    outside the rows."""
    fd = gpu_lib
    zmax, dz = 40, 2
    Z, nb = 41, N // 2
    rng = np.random.default_rng(9)
    P = rng.integers(0, 7, size=(Z, nb)).astype(np.float64)
    P[rng.integers(0, Z, 50), rng.integers(0, nb, 50)] = 25.0
    plan = make_plan(fd, N, zmax, dz, 64, 2048, 16, max_cands=1 << 22)
    try:
        fd.fdas_plan_set_harmsum_block(plan, block)
        with pytest.raises(fd.FdasError):
            fd.fdas_plan_set_harmsum_block(plan, 128)
        info = fd.fdas_plan_get_info(plan)
        d_p = torch.from_numpy(P.astype(np.float32).ravel()).to(DEV)
        d_out = torch.empty(info.max_cands * 4, dtype=torch.int32, device=DEV)
        d_cnt = torch.zeros(1, dtype=torch.int64, device=DEV)
        fd.fdas_stage_harmsum(plan, d_p, d_out, d_cnt)
        torch.cuda.synchronize()
        T_gpu = list(info.thresholds)
    finally:
        fd.fdas_plan_destroy(plan)
    n = int(d_cnt.item())
    arr = d_out.cpu().numpy().view(fd.CAND_DTYPE)[:n]
    cands, H = O.candidates(P, 16, 6.0)
    T = O.thresholds(16, 6.0)
    for i, h in enumerate((1, 2, 4, 8, 16)):
        assert abs(T_gpu[i] - T[h]) <= 1e-5 * T[h]
    assert n == len(cands)
    assert keys(arr) == {(c[0], c[1], c[2]) for c in cands}
    got = {(int(a["r_top"]), int(a["z_idx"]), int(a["h"])): float(a["power"]) for a in arr}
    for c in cands:
        assert got[(c[0], c[1], c[2])] == c[3]


@pytest.mark.parametrize("block", [32, 256])
def test_harmonic_sum_with_more_flags_than_the_list_holds(gpu_lib, block):
    """A plane of powers 3..5 flags every bin pair at h = 16 (1.34 million
    pairs, more than the screen's list of 2^20 entries), so the list kernel
    sums the first 2^20 and the screen the rest inline; integer powers keep
    every float32 sum exact, so the lists must be equal."""
    fd = gpu_lib
    N, zmax, dz = 1 << 17, 40, 2
    Z, nb = 41, N // 2
    rng = np.random.default_rng(10)
    P = rng.integers(3, 6, size=(Z, nb)).astype(np.float64)
    plan = make_plan(fd, N, zmax, dz, 64, 2048, 16, max_cands=1 << 23)
    try:
        fd.fdas_plan_set_harmsum_block(plan, block)
        info = fd.fdas_plan_get_info(plan)
        d_p = torch.from_numpy(P.astype(np.float32).ravel()).to(DEV)
        d_out = torch.empty(info.max_cands * 4, dtype=torch.int32, device=DEV)
        d_cnt = torch.zeros(1, dtype=torch.int64, device=DEV)
        fd.fdas_stage_harmsum(plan, d_p, d_out, d_cnt)
        torch.cuda.synchronize()
    finally:
        fd.fdas_plan_destroy(plan)
    n = int(d_cnt.item())
    arr = d_out.cpu().numpy().view(fd.CAND_DTYPE)[:n]
    cands, _ = O.candidates(P, 16, 6.0)
    assert n == len(cands) > (1 << 21)
    got = np.sort(arr[["h", "r_top", "z_idx"]].astype([("h", "<i4"), ("r_top", "<i4"),
                                                       ("z_idx", "<i4")]), order=["h", "r_top", "z_idx"])
    want = np.array([(c[2], c[0], c[1]) for c in cands],
                    dtype=[("h", "<i4"), ("r_top", "<i4"), ("z_idx", "<i4")])
    want.sort(order=["h", "r_top", "z_idx"])
    assert np.array_equal(got, want)


# --------------------------------------------------------------- full path --
def test_search_cfg1_matches_oracle(gpu_lib):
    fd = gpu_lib
    x, p = workload("cfg1_n2e17_z50")
    plan = make_plan(fd, p["N"], p["zmax"], p["dz"], p["m"], p["L"], p["nharm"])
    try:
        info = fd.fdas_plan_get_info(plan)
        got, n = search_one(fd, plan, info, x)
        P_gpu = gpu_plane(fd, plan, info)
    finally:
        fd.fdas_plan_destroy(plan)
    _, _, P, cands, H = O.search(x, p["zmax"], p["dz"], p["m"], p["nharm"], p["sigma"])
    assert (np.abs(P_gpu - P) / np.maximum(P, 1.0)).max() <= 1e-4
    assert_candidates_match(keys(got), cands, H, O.thresholds(p["nharm"]))
    assert any(abs(c["r_top"] - 10000) <= 1 for c in got)
    # host output is sorted by (h, r, j)
    order = [(int(c["h"]), int(c["r_top"]), int(c["z_idx"])) for c in got]
    assert order == sorted(order)


@pytest.mark.parametrize("L,m", [(2048, 128), (4096, 256), (8192, 512)])
def test_search_harmonics_matches_oracle(gpu_lib, L, m):
    fd = gpu_lib
    N, zmax, dz = 1 << 16, 60, 2
    chirps = [Chirp(1234.6, 14.0, 7.0, 0.2, 6), Chirp(9000.2, -30.0, 6.0, 2.0, 4),
              Chirp(20000.0, 3.0, 5.0, 1.0, 8)]
    x = make_series(N, 77, chirps)
    plan = make_plan(fd, N, zmax, dz, m, L, 16)
    try:
        info = fd.fdas_plan_get_info(plan)
        got, n = search_one(fd, plan, info, x)
        P_gpu = gpu_plane(fd, plan, info)
    finally:
        fd.fdas_plan_destroy(plan)
    _, _, P, cands, H = O.search(x, zmax, dz, m, 16, 6.0)
    assert (np.abs(P_gpu - P) / np.maximum(P, 1.0)).max() <= 1e-4
    assert_candidates_match(keys(got), cands, H, O.thresholds(16))
    assert {16, 8}.issubset({c[2] for c in cands})


def test_batch_host_device_paths_agree(gpu_lib):
    """Each trial gives the same candidates alone, in a batch, from host
    memory and through the device-output entry point."""
    fd = gpu_lib
    N = 1 << 15
    xs = np.stack([make_series(N, 300 + t, [Chirp(2000.0 + 500 * t, 6.0 * t, 8.0, 0.1, 4)])
                   for t in range(3)])
    plan = make_plan(fd, N, 30, 2, 128, 2048, 8, max_cands=4096)
    try:
        info = fd.fdas_plan_get_info(plan)
        single = [keys(search_one(fd, plan, info, xs[t])[0]) for t in range(3)]
        d_x = torch.from_numpy(xs.ravel()).to(DEV)
        out = np.zeros(3 * info.max_cands, dtype=fd.CAND_DTYPE)
        counts = np.zeros(3, dtype=np.int64)
        fd.fdas_search(plan, d_x, 3, out, counts)
        out_h = np.zeros_like(out)
        counts_h = np.zeros_like(counts)
        fd.fdas_search_host(plan, np.ascontiguousarray(xs.ravel()), 3, out_h, counts_h)
        d_out = torch.empty(3 * info.max_cands * 4, dtype=torch.int32, device=DEV)
        d_cnt = torch.zeros(3, dtype=torch.int64, device=DEV)
        fd.fdas_search_device(plan, d_x, 3, d_out, d_cnt)
        torch.cuda.synchronize()
        dev = d_out.cpu().numpy().view(fd.CAND_DTYPE)
        dcnt = d_cnt.cpu().numpy()
    finally:
        fd.fdas_plan_destroy(plan)
    M = info.max_cands
    for t in range(3):
        assert single[t]
        assert keys(out[t * M: t * M + counts[t]]) == single[t]
        assert keys(out_h[t * M: t * M + counts_h[t]]) == single[t]
        assert keys(dev[t * M: t * M + dcnt[t]]) == single[t]


@pytest.mark.parametrize("n_trials", [2, 3])
def test_trial_lanes_match_single_trials(gpu_lib, n_trials):
    """Multi-trial calls run odd trials on the plan's second lane: every
    trial's candidates equal a single-trial call's, and the debug plane is
    the last trial's whichever lane ran it."""
    fd = gpu_lib
    N = 1 << 15
    xs = np.stack([make_series(N, 500 + t, [Chirp(3000.0 + 700 * t, -4.0 * t, 9.0, 0.3, 4)])
                   for t in range(n_trials)])
    stream = torch.cuda.Stream(DEV)  # lanes need a stream other than the legacy default one
    plan = fd.fdas_plan_create(N, 30, 2, 128, 2048, 8, 6.0, 4096, stream.cuda_stream)
    try:
        info = fd.fdas_plan_get_info(plan)
        single, planes = [], []
        for t in range(n_trials):
            got, _ = search_one(fd, plan, info, xs[t])
            single.append(keys(got))
            planes.append(gpu_plane(fd, plan, info))
        bytes_before = fd.fdas_plan_get_info(plan).device_bytes
        d_x = torch.from_numpy(xs.ravel()).to(DEV)
        d_out = torch.empty(n_trials * info.max_cands * 4, dtype=torch.int32, device=DEV)
        d_cnt = torch.zeros(n_trials, dtype=torch.int64, device=DEV)
        torch.cuda.synchronize()
        fd.fdas_search_device(plan, d_x, n_trials, d_out, d_cnt)
        last_plane = gpu_plane(fd, plan, info)
        torch.cuda.synchronize()
        bytes_after = fd.fdas_plan_get_info(plan).device_bytes
        dev = d_out.cpu().numpy().view(fd.CAND_DTYPE)
        dcnt = d_cnt.cpu().numpy()
    finally:
        fd.fdas_plan_destroy(plan)
    M = info.max_cands
    for t in range(n_trials):
        assert single[t]
        assert keys(dev[t * M: t * M + dcnt[t]]) == single[t]
    assert np.array_equal(last_plane, planes[-1])
    assert bytes_after > bytes_before  # the lane's workspaces are counted


def test_candidate_overflow_reports_exact_count(gpu_lib):
    fd = gpu_lib
    N = 1 << 14
    x = make_series(N, 4, [Chirp(3000.0, 4.0, 20.0, 0.0, 4)])
    plan = make_plan(fd, N, 20, 2, 64, 2048, 4, max_cands=1 << 16)
    try:
        info = fd.fdas_plan_get_info(plan)
        _, n_full = search_one(fd, plan, info, x)
    finally:
        fd.fdas_plan_destroy(plan)
    assert n_full > 3
    plan = make_plan(fd, N, 20, 2, 64, 2048, 4, max_cands=2)
    try:
        info = fd.fdas_plan_get_info(plan)
        d_x = torch.from_numpy(x).to(DEV)
        out = np.zeros(2, dtype=fd.CAND_DTYPE)
        counts = np.zeros(1, dtype=np.int64)
        status = fd.fdas_search(plan, d_x, 1, out, counts)
    finally:
        fd.fdas_plan_destroy(plan)
    assert status == fd.FDAS_ERR_OVERFLOW
    assert counts[0] == n_full


# ---------------------------------------------------------- full-size case --
def _full_size_windows(chirps, nb, rng, n_random=4, half=1024):
    """Top-bin windows [r_a, r_a + 2 half): around h r0 for the injected
    signals with harmonics (h = 1..16 while h r0 stays inside the spectrum),
    then random ones."""
    starts = []
    for c in chirps:
        if c.nharm < 2:
            continue
        for h in (1, 2, 4, 8, 16):
            if h * c.r0 + half < nb - 1:
                starts.append(max(1, int(round(h * c.r0)) - half))
    starts = sorted(set(starts))
    starts = starts[:: max(1, len(starts) // 20)]  # about 20, spread over the spectrum
    starts += [int(v) for v in rng.integers(1, nb - 2 * half, n_random)]
    return [(a, a + 2 * half) for a in starts]


@pytest.mark.slow
def test_full_size_2e23_zmax200_windowed_candidates(gpu_lib):
    """The 2^23-sample, zmax=200, 16-harmonic workload in the launch
    configuration the benchmark times (several device-resident series in one
    call on a non-default stream, so consecutive trials run on the plan's two
    lanes, L = 8192). For every trial and every window of 2048 top bins (round
    the injected signals' harmonics, plus random ones), the GPU's candidate
    keys (r, z, h) at every level h = 1..16 equal the oracle's, whose sums
    come from plane rows formed only at the columns each ratio k/h reads
    (direct FFT correlation of the needed sub-band), apart from keys whose
    oracle H_h lies within 1e-4 T_h of T_h; common keys agree in power to
    1e-4 (H + h). The last trial's plane is also checked cell by cell at
    random and around every injected signal."""
    fd = gpu_lib
    x0, p = workload("cfg2_n2e23_z200", device=DEV)
    x1, p1 = workload("cfg2_n2e23_z200", seed=3, device=DEV)
    series = [(x0, p), (x1, p1)]
    stream = torch.cuda.Stream(DEV)
    plan = fd.fdas_plan_create(p["N"], p["zmax"], p["dz"], p["m"], p["L"], p["nharm"], 6.0,
                               1 << 22, stream.cuda_stream)
    try:
        info = fd.fdas_plan_get_info(plan)
        M = info.max_cands
        d_x = torch.from_numpy(np.concatenate([x0, x1])).to(DEV)
        d_out = torch.empty(2 * M * 4, dtype=torch.int32, device=DEV)
        d_cnt = torch.zeros(2, dtype=torch.int64, device=DEV)
        torch.cuda.synchronize()
        fd.fdas_search_device(plan, d_x, 2, d_out, d_cnt)
        plane = torch.empty(info.Z * info.nb, dtype=torch.float32, device=DEV)
        fd.fdas_plane_debug(plan, plane)   # the last trial's plane
        torch.cuda.synchronize()
        cnt = d_cnt.cpu().numpy()
        allc = d_out.cpu().numpy().view(fd.CAND_DTYPE)
    finally:
        fd.fdas_plan_destroy(plan)
    nb, Z = info.nb, info.Z
    T = O.thresholds(16)
    taus = O.template_bank(p["zmax"], p["dz"], p["m"])
    rng = np.random.default_rng(0)
    n_windows = n_harm_windows = 0
    levels_seen = set()
    for t, (x, pt) in enumerate(series):
        assert cnt[t] <= M
        got = allc[t * M: t * M + cnt[t]]
        Xw = O.whiten(O.spectrum(x))
        for r_a, r_b in _full_size_windows(pt["chirps"], nb, rng):
            Hw = O.harmonic_sums_window(Xw, taus, 16, r_a, r_b)
            sel = got[(got["r_top"] >= r_a) & (got["r_top"] < r_b)]
            have = {(int(c["r_top"]), int(c["z_idx"]), int(c["h"])): float(c["power"]) for c in sel}
            want = set()
            for h, Hh in Hw.items():
                jj, rr = np.nonzero(Hh >= T[h])
                want |= {(int(r) + r_a, int(j), h) for j, r in zip(jj, rr) if r + r_a >= 1}
            for (r, j, h) in set(have) ^ want:
                v = Hw[h][j, r - r_a]
                assert abs(v - T[h]) <= 1e-4 * T[h], (t, r_a, (r, j, h), v, T[h], (r, j, h) in have)
            for key in set(have) & want:
                r, j, h = key
                v = Hw[h][j, r - r_a]
                assert abs(have[key] - v) <= 1e-4 * (v + h), (t, key, have[key], v)
            n_windows += 1
            n_harm_windows += bool(want)
            levels_seen |= {h for (_, _, h) in want}
    assert n_windows >= 8 and n_harm_windows >= 4
    assert levels_seen == {1, 2, 4, 8, 16}
    # the last trial's plane, cell by cell
    x, pt = series[-1]
    Xw = O.whiten(O.spectrum(x))
    zs = O.z_values(pt["zmax"], pt["dz"])
    js = list(rng.integers(0, Z, 300))
    rs = list(rng.integers(0, nb, 300))
    for c in pt["chirps"]:
        if c.r0 < nb - 4:
            j0 = int(np.argmin(np.abs(zs - c.z0)))
            for dj in (-1, 0, 1):
                for dr in (-1, 0, 1):
                    js.append(min(max(j0 + dj, 0), Z - 1))
                    rs.append(int(round(c.r0)) + dr)
    js = np.array(js)
    rs = np.array(rs)
    ref = O.plane_cells(Xw, taus, js, rs)
    gp = plane.view(Z, nb)[torch.from_numpy(js).to(DEV), torch.from_numpy(rs).to(DEV)]
    gp = gp.cpu().numpy().astype(np.float64)
    assert (np.abs(gp - ref) / np.maximum(ref, 1.0)).max() <= 1e-4


def test_host_pipeline_equals_single_trials(gpu_lib):
    """Several series in one call on a non-default stream (copies and
    read-back overlapped with the neighbouring trials' kernels): every
    trial's sorted list and count equal those of one-trial calls, for
    page-locked and pageable host series (fdas_search_host) and for device
    series (fdas_search)."""
    fd = gpu_lib
    N = 1 << 15
    xs = np.stack([make_series(N, 900 + t, [Chirp(1500.0 + 700 * t, 4.0 * t - 8, 8.0, 0.2, 4)])
                   for t in range(5)])
    stream = torch.cuda.Stream(DEV)
    plan = fd.fdas_plan_create(N, 30, 2, 128, 2048, 8, 6.0, 2048, stream.cuda_stream)
    try:
        info = fd.fdas_plan_get_info(plan)
        single = []
        for t in range(5):
            o = np.zeros(info.max_cands, dtype=fd.CAND_DTYPE)
            c = np.zeros(1, dtype=np.int64)
            fd.fdas_search_host(plan, np.ascontiguousarray(xs[t]), 1, o, c)
            single.append((int(c[0]), o[:c[0]].tobytes()))
        pinned = torch.from_numpy(xs.ravel().copy()).pin_memory()
        d_all = torch.from_numpy(xs.ravel().copy()).to(DEV)
        torch.cuda.synchronize()
        for src in (pinned.numpy(), np.ascontiguousarray(xs.ravel()), d_all):
            out = np.zeros(5 * info.max_cands, dtype=fd.CAND_DTYPE)
            cnt = np.zeros(5, dtype=np.int64)
            if isinstance(src, torch.Tensor):   # device series: fdas_search
                fd.fdas_search(plan, src, 5, out, cnt)
            else:
                fd.fdas_search_host(plan, src, 5, out, cnt)
            for t in range(5):
                got = out[t * info.max_cands: t * info.max_cands + cnt[t]]
                assert (int(cnt[t]), got.tobytes()) == single[t], t
    finally:
        fd.fdas_plan_destroy(plan)
    assert all(c > 0 for c, _ in single)


@pytest.mark.parametrize("n_trials", [2, 3, 4, 6])
def test_pipelined_overflow_keeps_exact_counts(gpu_lib, n_trials):
    """Several host series through the lane pipeline (the read-back of trial
    t - 2 overlaps trials t - 1 and t) with a candidate list too small for
    them: the call returns FDAS_ERR_OVERFLOW after every trial, each count is
    the exact one a roomy plan reports, and each stored entry is one of that
    trial's candidates."""
    fd = gpu_lib
    N = 1 << 14
    xs = np.stack([make_series(N, 40 + t, [Chirp(2000.0 + 300 * t, 4.0, 20.0, 0.0, 4)])
                   for t in range(n_trials)])
    stream = torch.cuda.Stream(DEV)
    full = []
    plan = fd.fdas_plan_create(N, 20, 2, 64, 2048, 4, 6.0, 1 << 16, stream.cuda_stream)
    try:
        for t in range(n_trials):
            o = np.zeros(1 << 16, dtype=fd.CAND_DTYPE)
            c = np.zeros(1, dtype=np.int64)
            fd.fdas_search_host(plan, np.ascontiguousarray(xs[t]), 1, o, c)
            full.append((int(c[0]), keys(o[: c[0]])))
    finally:
        fd.fdas_plan_destroy(plan)
    M = 3
    plan = fd.fdas_plan_create(N, 20, 2, 64, 2048, 4, 6.0, M, stream.cuda_stream)
    try:
        out = np.zeros(n_trials * M, dtype=fd.CAND_DTYPE)
        cnt = np.zeros(n_trials, dtype=np.int64)
        status = fd.fdas_search_host(plan, np.ascontiguousarray(xs.ravel()), n_trials, out, cnt)
    finally:
        fd.fdas_plan_destroy(plan)
    assert status == fd.FDAS_ERR_OVERFLOW
    for t in range(n_trials):
        n_full, k_full = full[t]
        assert n_full > M and int(cnt[t]) == n_full
        assert keys(out[t * M: (t + 1) * M]) <= k_full
