"""Uneven series lengths N = 2^a 3^b 5^c (de-dispersed trials of different
length): the mixed-radix real FFT, the whole path against the oracle, and
batches of uneven trials against single-trial searches."""
import math

import numpy as np
import pytest
import torch

from oracle import fdas_oracle as O
from synthetic import Chirp, make_series

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0") if torch.cuda.is_available() else None


def stream():
    return torch.cuda.current_stream(DEV).cuda_stream


@pytest.mark.parametrize("N", [3 * 4096, 5 * 4096, 15 * 4096, 45 * 4096, 75 * 4096, 3 << 21])
def test_mixed_radix_spectrum_and_whitening(gpu_lib, N):
    fd = gpu_lib
    x = make_series(N, N % 9973, [Chirp(0.31 * N / 2, 12.0, 9.0, 0.2, 2)])
    plan = fd.fdas_plan_create(N, 20, 2, 64, 2048, 1, 6.0, 16, stream())
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
    assert np.max(np.abs(W_gpu - O.whiten(X_orc))) <= 5e-5


def run_search(fd, plan, info, x):
    d_x = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).to(DEV)
    out = np.zeros(info.max_cands, dtype=fd.CAND_DTYPE)
    counts = np.zeros(1, dtype=np.int64)
    fd.fdas_search(plan, d_x, 1, out, counts)
    plane = torch.empty(info.Z * info.nb, dtype=torch.float32, device=DEV)
    fd.fdas_plane_debug(plan, plane)
    torch.cuda.synchronize()
    P = plane.cpu().numpy().reshape(info.Z, info.nb).astype(np.float64)
    return out[:counts[0]], P


def keys(c):
    return {(int(a["r_top"]), int(a["z_idx"]), int(a["h"])) for a in c}


@pytest.mark.parametrize("N", [15 * 4096, 45 * 4096])
def test_search_uneven_length_matches_oracle(gpu_lib, N):
    fd = gpu_lib
    zmax, dz, m, L, nharm = 24, 2, 64, 2048, 8
    x = make_series(N, 17, [Chirp(0.21 * N / 2, 8.0, 9.0, 0.3, 4), Chirp(0.05 * N / 2, -5.0, 7.0, 1.0, 2)])
    plan = fd.fdas_plan_create(N, zmax, dz, m, L, nharm, 6.0, 1 << 18, stream())
    try:
        info = fd.fdas_plan_get_info(plan)
        got, P_gpu = run_search(fd, plan, info, x)
    finally:
        fd.fdas_plan_destroy(plan)
    _, _, P, cands, H = O.search(x, zmax, dz, m, nharm, 6.0)
    assert (np.abs(P_gpu - P) / np.maximum(P, 1.0)).max() <= 1e-4
    T = O.thresholds(nharm)
    want = {(c[0], c[1], c[2]) for c in cands}
    bad = [k for k in keys(got) ^ want if abs(H[k[2]][k[1], k[0]] - T[k[2]]) > 1e-4 * T[k[2]]]
    assert not bad, bad[:5]
    assert want


def test_batch_of_uneven_trials_matches_single_searches(gpu_lib):
    """Each trial gives the same candidates in a batch of uneven lengths as
    through its own plan."""
    fd = gpu_lib
    zmax, dz, m, L, nharm = 30, 2, 128, 2048, 16
    lengths = [1 << 17, 3 << 15, 5 << 14, 1 << 16, 3 << 15]
    xs = [make_series(n, 500 + i, [Chirp(0.17 * n / 2 + 31 * i, 6.0 - 3 * i, 10.0, 0.5, 5)])
          for i, n in enumerate(lengths)]
    maxc = 1 << 16
    single = []
    for x, n in zip(xs, lengths):
        plan = fd.fdas_plan_create(n, zmax, dz, m, L, nharm, 6.0, maxc, stream())
        try:
            info = fd.fdas_plan_get_info(plan)
            got, _ = run_search(fd, plan, info, x)
            single.append(keys(got))
        finally:
            fd.fdas_plan_destroy(plan)
    batch = fd.fdas_batch_create(max(lengths), zmax, dz, m, L, nharm, 6.0, maxc, stream())
    try:
        d_xs = [torch.from_numpy(x).to(DEV) for x in xs]
        d_out = torch.empty(len(xs) * maxc * 16, dtype=torch.uint8, device=DEV)
        d_cnt = torch.zeros(len(xs), dtype=torch.int64, device=DEV)
        fd.fdas_search_batch(batch, d_xs, lengths, d_out, d_cnt)
        torch.cuda.synchronize()
        arr = d_out.cpu().numpy().view(fd.CAND_DTYPE)
        cnt = d_cnt.cpu().numpy()
    finally:
        fd.fdas_batch_destroy(batch)
    for t in range(len(xs)):
        assert single[t]
        assert keys(arr[t * maxc: t * maxc + cnt[t]]) == single[t], t


def test_batch_rejects_longer_series(gpu_lib):
    fd = gpu_lib
    batch = fd.fdas_batch_create(1 << 14, 10, 2, 64, 2048, 1, 6.0, 16, stream())
    try:
        d_x = torch.zeros(1 << 15, dtype=torch.float32, device=DEV)
        d_out = torch.empty(16 * 16, dtype=torch.uint8, device=DEV)
        d_cnt = torch.zeros(1, dtype=torch.int64, device=DEV)
        with pytest.raises(fd.FdasError) as e:
            fd.fdas_search_batch(batch, [d_x], [1 << 15], d_out, d_cnt)
        assert e.value.status == fd.FDAS_ERR_INVALID
    finally:
        fd.fdas_batch_destroy(batch)
