"""Parity of the tensor-core (tcgen05) correlation modes with the FP64 oracle.

Eq. 1 evaluated as a dense product of the 16-bit hi/lo-split templates and
the Hankel-blocked whitened spectrum, float32 accumulation:
  * bf16 hi/lo: each operand carries 16 significant bits and the dropped
    lo*lo product is 2^-16 relative, so |A| is good to ~2^-16 * ||tau|| ||X||
    and |dP| <= 1e-4 * max(P, 1) (the float32 path's tolerance) holds;
  * fp16 hi/lo: 22 bits per operand, so the float32 accumulation of the
    6m products dominates: about sqrt(6m) * 2^-23 relative to |A|^2
    (6.6e-6 at m = 512); the bound is 2e-5.
The maximum error of each case is printed (the per-result error that the
precision variant reports).
"""
import math

import numpy as np
import pytest
import torch

from oracle import fdas_oracle as O
from synthetic import Chirp, make_series

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0") if torch.cuda.is_available() else None
TOL = {1: 1e-4, 2: 2e-5}


def make_plan(fd, N, zmax, m, L, nharm, mode, max_cands=1 << 20):
    stream = torch.cuda.current_stream(DEV).cuda_stream
    plan = fd.fdas_plan_create(N, zmax, 2, m, L, nharm, 6.0, max_cands, stream)
    fd.fdas_plan_set_correlation(plan, mode)
    return plan


def dev_c64(a):
    return torch.from_numpy(np.ascontiguousarray(a.astype(np.complex64))).to(DEV)


@pytest.mark.parametrize("mode", [1, 2])
@pytest.mark.parametrize("N,zmax,m", [
    (1 << 12, 16, 64),        # 4 bin blocks, one row tile, 6 K blocks
    (1 << 14, 20, 64),
    (1 << 15, 100, 256),      # 202 rows: two row tiles (the second ragged)
    (1 << 14, 200, 512),      # zmax=200 templates: four row tiles, 48 K blocks
    (3 << 12, 40, 128),       # uneven length: 12 bin blocks
])
def test_gemm_plane_matches_oracle(gpu_lib, mode, N, zmax, m):
    fd = gpu_lib
    rng = np.random.default_rng(N + zmax + 7 * mode)
    nb = N // 2
    Xw = (rng.standard_normal(nb) + 1j * rng.standard_normal(nb)) / math.sqrt(2)
    Xw[100] += 12.0
    Xw[nb - 3] += 9.0
    Xw = Xw.astype(np.complex64).astype(np.complex128)
    plan = make_plan(fd, N, zmax, m, max(2048, 2 * m), 1, mode)
    try:
        info = fd.fdas_plan_get_info(plan)
        plane = torch.full((info.Z * nb,), -1.0, dtype=torch.float32, device=DEV)
        fd.fdas_stage_plane(plan, dev_c64(Xw), plane)
        torch.cuda.synchronize()
    finally:
        fd.fdas_plan_destroy(plan)
    P_gpu = plane.cpu().numpy().reshape(info.Z, nb).astype(np.float64)
    P_orc = O.power_plane(Xw, O.template_bank(zmax, 2, m))
    rel = np.abs(P_gpu - P_orc) / np.maximum(P_orc, 1.0)
    print(f"mode {mode} N {N} zmax {zmax} m {m}: max |dP|/max(P,1) = {rel.max():.3e}")
    assert rel.max() <= TOL[mode], rel.max()


@pytest.mark.parametrize("mode", [1, 2])
def test_gemm_search_matches_oracle(gpu_lib, mode):
    """Whole search in a tensor-core mode: candidate keys equal the oracle's
    except keys whose oracle sum lies within the tolerance band of T_h."""
    fd = gpu_lib
    N, zmax, m = 1 << 16, 60, 128
    chirps = [Chirp(1234.6, 14.0, 7.0, 0.2, 6), Chirp(9000.2, -30.0, 6.0, 2.0, 4),
              Chirp(20000.0, 3.0, 5.0, 1.0, 8)]
    x = make_series(N, 77, chirps)
    plan = make_plan(fd, N, zmax, m, 2048, 16, mode)
    try:
        info = fd.fdas_plan_get_info(plan)
        d_x = torch.from_numpy(x).to(DEV)
        out = np.zeros(info.max_cands, dtype=fd.CAND_DTYPE)
        cnt = np.zeros(1, dtype=np.int64)
        fd.fdas_search(plan, d_x, 1, out, cnt)
        got = out[:cnt[0]]
        plane = torch.empty(info.Z * info.nb, dtype=torch.float32, device=DEV)
        fd.fdas_plane_debug(plan, plane)
        torch.cuda.synchronize()
    finally:
        fd.fdas_plan_destroy(plan)
    _, _, P, cands, H = O.search(x, zmax, 2, m, 16, 6.0)
    P_gpu = plane.cpu().numpy().reshape(P.shape).astype(np.float64)
    rel = (np.abs(P_gpu - P) / np.maximum(P, 1.0)).max()
    print(f"mode {mode}: plane max |dP|/max(P,1) = {rel:.3e}")
    assert rel <= TOL[mode]
    T = O.thresholds(16)
    want = {(c[0], c[1], c[2]) for c in cands}
    have = {(int(a["r_top"]), int(a["z_idx"]), int(a["h"])) for a in got}
    for (r, j, h) in want ^ have:
        # each of the h terms may be off by TOL * max(P, 1)
        assert abs(H[h][j, r] - T[h]) <= TOL[mode] * (T[h] + h), (r, j, h, H[h][j, r], T[h])
    recall = len(want & have) / max(len(want), 1)
    print(f"mode {mode}: {len(have)} candidates, recall {recall:.6f}")
    assert {16, 8}.issubset({c[2] for c in cands})


def test_gemm_mode_switch_and_rejects(gpu_lib):
    """The mode can be switched back and forth on one plan (same plane as a
    fresh plan); unsupported shapes and modes are rejected."""
    fd = gpu_lib
    N, zmax, m = 1 << 14, 20, 64
    rng = np.random.default_rng(3)
    Xw = (rng.standard_normal(N // 2) + 1j * rng.standard_normal(N // 2)).astype(np.complex64)
    stream = torch.cuda.current_stream(DEV).cuda_stream
    plan = fd.fdas_plan_create(N, zmax, 2, m, 2048, 1, 6.0, 1024, stream)
    try:
        info = fd.fdas_plan_get_info(plan)
        planes = []
        for mode in (1, 0, 2, 1):
            fd.fdas_plan_set_correlation(plan, mode)
            out = torch.empty(info.Z * info.nb, dtype=torch.float32, device=DEV)
            fd.fdas_stage_plane(plan, dev_c64(Xw), out)
            planes.append(out.cpu().numpy())
        assert np.array_equal(planes[0], planes[3])
        assert not np.array_equal(planes[0], planes[1])
        with pytest.raises(fd.FdasError):
            fd.fdas_plan_set_correlation(plan, 7)
    finally:
        fd.fdas_plan_destroy(plan)
    plan = fd.fdas_plan_create(N, zmax, 2, 72, 2048, 1, 6.0, 1024, stream)
    try:
        with pytest.raises(fd.FdasError) as e:
            fd.fdas_plan_set_correlation(plan, 1)   # m % 32 != 0
        assert e.value.status == fd.FDAS_ERR_INVALID
    finally:
        fd.fdas_plan_destroy(plan)


def test_gemm_full_size_sampled(gpu_lib):
    """N = 2^23, zmax = 200, m = 512 in bf16 hi/lo: sampled plane cells
    against direct sums of Eq. 1 on the oracle's whitened spectrum."""
    fd = gpu_lib
    from synthetic import workload
    x, p = workload("cfg2_n2e23_z200", device=DEV)
    plan = make_plan(fd, p["N"], p["zmax"], p["m"], p["L"], p["nharm"], 1, max_cands=1 << 22)
    try:
        info = fd.fdas_plan_get_info(plan)
        d_x = torch.from_numpy(x).to(DEV)
        out = np.zeros(info.max_cands, dtype=fd.CAND_DTYPE)
        cnt = np.zeros(1, dtype=np.int64)
        fd.fdas_search(plan, d_x, 1, out, cnt)
        plane = torch.empty(info.Z * info.nb, dtype=torch.float32, device=DEV)
        fd.fdas_plane_debug(plan, plane)
        torch.cuda.synchronize()
    finally:
        fd.fdas_plan_destroy(plan)
    Xw = O.whiten(O.spectrum(x))
    taus = O.template_bank(p["zmax"], p["dz"], p["m"])
    rng = np.random.default_rng(1)
    nb, Z = info.nb, info.Z
    js = rng.integers(0, Z, 400)
    rs = np.concatenate([rng.integers(0, nb, 390), [0, 1, 511, 512, nb - 512, nb - 1, 4096,
                                                     4095, nb // 2, 7]])
    ref = O.plane_cells(Xw, taus, js, rs)
    gp = plane.view(Z, nb)[torch.from_numpy(js).to(DEV), torch.from_numpy(rs).to(DEV)]
    gp = gp.cpu().numpy().astype(np.float64)
    rel = (np.abs(gp - ref) / np.maximum(ref, 1.0)).max()
    print(f"full size bf16: sampled max |dP|/max(P,1) = {rel:.3e}")
    assert rel <= 1e-4
