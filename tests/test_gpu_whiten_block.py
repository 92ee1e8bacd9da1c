"""Parity of the block-median whitening variant with the FP64 oracle:
the whitened spectrum element by element (max |dXw| <= 5e-5, Xw has unit
rms: a float32 median of float32 powers and one float32 interpolation), and
a whole search in block mode against the oracle's candidate list."""
import math

import numpy as np
import pytest
import torch

from oracle import fdas_oracle as O
from synthetic import Chirp, make_series, workload

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0") if torch.cuda.is_available() else None


@pytest.mark.parametrize("N", [1 << 12, 1 << 15, 3 << 12, 15 << 12, 1 << 20])
def test_block_whitening_matches_oracle(gpu_lib, N):
    fd = gpu_lib
    rng = np.random.default_rng(N)
    nb = N // 2
    # red-ish noise: power rising with k plus a few strong lines
    k = np.arange(nb)
    X = (rng.standard_normal(nb) + 1j * rng.standard_normal(nb)) * np.sqrt(1.0 + 3e-3 * k)
    X[[5, nb // 3, nb - 2]] += 40.0
    X = X.astype(np.complex64)
    stream = torch.cuda.current_stream(DEV).cuda_stream
    plan = fd.fdas_plan_create(N, 4, 2, 64, 2048, 1, 6.0, 16, stream)
    try:
        fd.fdas_plan_set_whitening(plan, fd.FDAS_WHITEN_BLOCK)
        d_x = torch.from_numpy(X).to(DEV)
        d_w = torch.empty_like(d_x)
        fd.fdas_stage_whiten(plan, d_x, d_w)
        torch.cuda.synchronize()
    finally:
        fd.fdas_plan_destroy(plan)
    got = d_w.cpu().numpy().astype(np.complex128)
    want = O.whiten_block(X.astype(np.complex128))
    assert got[0] == 0
    err = np.abs(got - want).max()
    assert err <= 5e-5, err


def test_block_whitening_search_matches_oracle(gpu_lib):
    fd = gpu_lib
    x, p = workload("cfg1_n2e17_z50")
    stream = torch.cuda.current_stream(DEV).cuda_stream
    plan = fd.fdas_plan_create(p["N"], p["zmax"], p["dz"], p["m"], p["L"], p["nharm"],
                               p["sigma"], 1 << 16, stream)
    try:
        fd.fdas_plan_set_whitening(plan, fd.FDAS_WHITEN_BLOCK)
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
    _, _, P, cands, H = O.search(x, p["zmax"], p["dz"], p["m"], p["nharm"], p["sigma"],
                                 whitening="block")
    P_gpu = plane.cpu().numpy().reshape(P.shape).astype(np.float64)
    assert (np.abs(P_gpu - P) / np.maximum(P, 1.0)).max() <= 1e-4
    T = O.thresholds(p["nharm"])
    want = {(c[0], c[1], c[2]) for c in cands}
    have = {(int(a["r_top"]), int(a["z_idx"]), int(a["h"])) for a in out[:cnt[0]]}
    for (r, j, h) in want ^ have:
        assert abs(H[h][j, r] - T[h]) <= 1e-4 * T[h], (r, j, h)
    assert any(abs(r - 10000) <= 1 for (r, j, h) in have)
