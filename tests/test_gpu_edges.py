"""Edge cases of the CUDA path against the oracle: the largest supported
length (2^24 samples), a single template (zmax = 0, where Eq. 1 reduces to
the whitened power itself), the narrowest template (m = 8), an empty call,
and an all-zero series (every whitening median is 0)."""
import math

import numpy as np
import pytest
import torch

from oracle import fdas_oracle as O
from synthetic import Chirp, make_series

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0") if torch.cuda.is_available() else None


def plan_on(fd, N, zmax, m, L, nharm, maxc=1 << 16):
    stream = torch.cuda.current_stream(DEV).cuda_stream
    return fd.fdas_plan_create(N, zmax, 2, m, L, nharm, 6.0, maxc, stream)


def test_largest_length_2e24(gpu_lib):
    """N = 2^24: spectrum and whitening element by element, and sampled
    plane cells (zmax = 40) against direct sums of Eq. 1."""
    fd = gpu_lib
    N = 1 << 24
    chirps = [Chirp(3.0e6 + 0.3, 12.0, 10.0, 0.4, 2), Chirp(123456.0, -20.0, 9.0, 1.0, 1)]
    x = make_series(N, 24, chirps, device=DEV)
    plan = plan_on(fd, N, 40, 128, 2048, 4)
    try:
        info = fd.fdas_plan_get_info(plan)
        d_x = torch.from_numpy(x).to(DEV)
        d_X = torch.empty(info.nb, dtype=torch.complex64, device=DEV)
        d_W = torch.empty_like(d_X)
        fd.fdas_stage_spectrum(plan, d_x, d_X)
        fd.fdas_stage_whiten(plan, d_X, d_W)
        out = np.zeros(info.max_cands, dtype=fd.CAND_DTYPE)
        cnt = np.zeros(1, dtype=np.int64)
        fd.fdas_search(plan, d_x, 1, out, cnt)
        plane = torch.empty(info.Z * info.nb, dtype=torch.float32, device=DEV)
        fd.fdas_plane_debug(plan, plane)
        torch.cuda.synchronize()
    finally:
        fd.fdas_plan_destroy(plan)
    X = O.spectrum(x)
    Xg = d_X.cpu().numpy().astype(np.complex128)
    rms = math.sqrt(np.mean(np.abs(X) ** 2))
    assert np.abs(Xg - X).max() <= 2e-5 * rms
    Xw = O.whiten(X)
    assert np.abs(d_W.cpu().numpy().astype(np.complex128) - Xw).max() <= 5e-5
    taus = O.template_bank(40, 2, 128)
    rng = np.random.default_rng(24)
    js = np.concatenate([rng.integers(0, info.Z, 200), [26, 26, 10]])
    rs = np.concatenate([rng.integers(0, info.nb, 200), [3000000, 3000001, 123456]])
    ref = O.plane_cells(Xw, taus, js, rs)
    gp = plane.view(info.Z, info.nb)[torch.from_numpy(js).to(DEV), torch.from_numpy(rs).to(DEV)]
    rel = np.abs(gp.cpu().numpy() - ref) / np.maximum(ref, 1.0)
    assert rel.max() <= 1e-4
    got = out[:min(cnt[0], info.max_cands)]
    assert any(abs(int(c["r_top"]) - 3000000) <= 1 and c["h"] == 1 for c in got)


def test_single_template_is_the_whitened_power(gpu_lib):
    """zmax = 0: one template, tau_0 = delta, so P[0][r] = |Xw_r|^2 and the
    search is a plain threshold of the whitened power spectrum."""
    fd = gpu_lib
    N = 1 << 16
    x = make_series(N, 5, [Chirp(5000.0, 0.0, 9.0, 0.0, 4)])
    plan = plan_on(fd, N, 0, 64, 2048, 4)
    try:
        info = fd.fdas_plan_get_info(plan)
        assert info.Z == 1
        d_x = torch.from_numpy(x).to(DEV)
        out = np.zeros(info.max_cands, dtype=fd.CAND_DTYPE)
        cnt = np.zeros(1, dtype=np.int64)
        fd.fdas_search(plan, d_x, 1, out, cnt)
        plane = torch.empty(info.nb, dtype=torch.float32, device=DEV)
        fd.fdas_plane_debug(plan, plane)
        torch.cuda.synchronize()
    finally:
        fd.fdas_plan_destroy(plan)
    Xw = O.whiten(O.spectrum(x))
    P = np.abs(Xw) ** 2
    assert (np.abs(plane.cpu().numpy() - P) / np.maximum(P, 1.0)).max() <= 1e-4
    _, _, Po, cands, H = O.search(x, 0, 2, 64, 4)
    T = O.thresholds(4)
    want = {(c[0], c[1], c[2]) for c in cands}
    have = {(int(a["r_top"]), int(a["z_idx"]), int(a["h"])) for a in out[:cnt[0]]}
    for (r, j, h) in want ^ have:
        assert abs(H[h][j, r] - T[h]) <= 1e-4 * T[h], (r, j, h)
    assert (5000, 0, 1) in have and (20000, 0, 4) in have


def test_narrowest_template(gpu_lib):
    """m = 8 taps (the smallest width): plane element by element."""
    fd = gpu_lib
    N = 1 << 14
    rng = np.random.default_rng(8)
    nb = N // 2
    Xw = ((rng.standard_normal(nb) + 1j * rng.standard_normal(nb)) / math.sqrt(2)).astype(np.complex64)
    plan = plan_on(fd, N, 6, 8, 2048, 1)
    try:
        info = fd.fdas_plan_get_info(plan)
        plane = torch.empty(info.Z * nb, dtype=torch.float32, device=DEV)
        fd.fdas_stage_plane(plan, torch.from_numpy(Xw).to(DEV), plane)
        torch.cuda.synchronize()
    finally:
        fd.fdas_plan_destroy(plan)
    P = O.power_plane(Xw.astype(np.complex128), O.template_bank(6, 2, 8))
    rel = np.abs(plane.cpu().numpy().reshape(P.shape) - P) / np.maximum(P, 1.0)
    assert rel.max() <= 1e-4


def test_empty_call_and_zero_series(gpu_lib):
    """n_trials = 0 does nothing; an all-zero series has every whitening
    median 0, which gives a zero whitened spectrum (no NaN), a zero plane and
    no candidates."""
    fd = gpu_lib
    N = 1 << 14
    plan = plan_on(fd, N, 20, 64, 2048, 16)
    try:
        info = fd.fdas_plan_get_info(plan)
        out = np.zeros(info.max_cands, dtype=fd.CAND_DTYPE)
        cnt = np.zeros(1, dtype=np.int64)
        d_x = torch.zeros(N, dtype=torch.float32, device=DEV)
        fd.fdas_search(plan, d_x, 0, out, cnt)
        fd.fdas_search_host(plan, np.zeros(N, dtype=np.float32), 0, out, cnt)
        fd.fdas_search(plan, d_x, 1, out, cnt)
        plane = torch.empty(info.Z * info.nb, dtype=torch.float32, device=DEV)
        fd.fdas_plane_debug(plan, plane)
        torch.cuda.synchronize()
    finally:
        fd.fdas_plan_destroy(plan)
    assert cnt[0] == 0
    p = plane.cpu().numpy()
    assert np.all(np.isfinite(p)) and np.all(p == 0.0)


def test_misaligned_pointers_are_argument_errors(gpu_lib):
    """Views that start at an odd float are rejected with FDAS_ERR_INVALID
    before any launch, and the plan keeps working afterwards."""
    fd = gpu_lib
    N = 1 << 14
    plan = plan_on(fd, N, 20, 64, 2048, 4)
    try:
        info = fd.fdas_plan_get_info(plan)
        x = torch.from_numpy(np.random.default_rng(1).standard_normal(N + 4).astype(np.float32)).to(DEV)
        d_out = torch.empty(info.max_cands * 4, dtype=torch.int32, device=DEV)
        d_cnt = torch.zeros(2, dtype=torch.int64, device=DEV)
        spec = torch.empty(N + 8, dtype=torch.float32, device=DEV)
        bad = [
            lambda: fd.fdas_search_device(plan, x.data_ptr() + 4, 1, d_out, d_cnt),
            lambda: fd.fdas_search_device(plan, x, 1, d_out, d_cnt.data_ptr() + 4),
            lambda: fd.fdas_stage_spectrum(plan, x.data_ptr() + 4, spec),
            lambda: fd.fdas_stage_whiten(plan, spec.data_ptr() + 8, spec),
            lambda: fd.fdas_search(plan, x.data_ptr() + 4, 1, np.zeros(info.max_cands, fd.CAND_DTYPE),
                                   np.zeros(1, np.int64)),
        ]
        for call in bad:
            with pytest.raises(fd.FdasError) as e:
                call()
            assert e.value.status == fd.FDAS_ERR_INVALID and "aligned" in str(e.value)
        fd.fdas_search_device(plan, x, 1, d_out, d_cnt)
        torch.cuda.synchronize()
    finally:
        fd.fdas_plan_destroy(plan)


def test_allocation_refusal_is_nomem_and_leaks_nothing(gpu_lib):
    """A plan larger than the device (a 2^24-sample plane of 10001 templates,
    336 GB) is refused with FDAS_ERR_NOMEM: whatever was allocated before the
    refusal is freed, and the refused allocation does not surface as an error
    at a later launch (a small search afterwards works)."""
    fd = gpu_lib
    torch.cuda.synchronize()
    free0, total = torch.cuda.mem_get_info(DEV)
    zmax = 10000
    assert (2 * (zmax // 2) + 1) * (1 << 23) * 4 > total
    with pytest.raises(fd.FdasError) as e:
        fd.fdas_plan_create(1 << 24, zmax, 2, 512, 8192, 16, 6.0, 1 << 16,
                            torch.cuda.current_stream(DEV).cuda_stream)
    assert e.value.status == fd.FDAS_ERR_NOMEM
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info(DEV)
    assert free1 >= free0 - (64 << 20)
    N = 1 << 14
    x = make_series(N, 12, [Chirp(2000.0, 4.0, 14.0, 0.0, 2)])
    plan = plan_on(fd, N, 20, 64, 2048, 4)
    try:
        info = fd.fdas_plan_get_info(plan)
        out = np.zeros(info.max_cands, dtype=fd.CAND_DTYPE)
        cnt = np.zeros(1, dtype=np.int64)
        fd.fdas_search(plan, torch.from_numpy(x).to(DEV), 1, out, cnt)
    finally:
        fd.fdas_plan_destroy(plan)
    assert cnt[0] > 0
