"""Half-bin (interbinned) planes on the GPU against the FP64 oracle: the
interleaved plane P[j][2r + e] = |A(r + e/2, z_j)|^2 element by element
(|dP| <= 1e-4 max(P, 1), the float32 path's bar) and a whole search whose
candidates count half bins."""
import math

import numpy as np
import pytest
import torch

from oracle import fdas_oracle as O
from synthetic import Chirp, make_series

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0") if torch.cuda.is_available() else None


@pytest.mark.parametrize("N,zmax,m,L", [
    (1 << 14, 20, 64, 2048),
    (1 << 15, 100, 256, 4096),
    (1 << 14, 200, 512, 8192),     # two segments, ragged tail
    (3 << 12, 30, 128, 2048),      # uneven length
])
def test_half_bin_plane_matches_oracle(gpu_lib, N, zmax, m, L):
    fd = gpu_lib
    rng = np.random.default_rng(N + zmax + 1)
    nb = N // 2
    Xw = (rng.standard_normal(nb) + 1j * rng.standard_normal(nb)) / math.sqrt(2)
    Xw[100] += 12.0
    Xw[nb // 2] += 7.0 * np.exp(0.3j)
    Xw = Xw.astype(np.complex64).astype(np.complex128)
    stream = torch.cuda.current_stream(DEV).cuda_stream
    plan = fd.fdas_plan_create(N, zmax, 2, m, L, 1, 6.0, 16, stream)
    try:
        fd.fdas_plan_set_interbin(plan, 1)
        info = fd.fdas_plan_get_info(plan)
        assert info.plane_floats == info.Z * 2 * nb
        plane = torch.full((info.Z * 2 * nb,), -1.0, dtype=torch.float32, device=DEV)
        d_x = torch.from_numpy(Xw.astype(np.complex64)).to(DEV)
        fd.fdas_stage_plane(plan, d_x, plane)
        torch.cuda.synchronize()
    finally:
        fd.fdas_plan_destroy(plan)
    P_gpu = plane.cpu().numpy().reshape(info.Z, 2 * nb).astype(np.float64)
    P_orc = O.power_plane_interbin(Xw, zmax, 2, m)
    rel = np.abs(P_gpu - P_orc) / np.maximum(P_orc, 1.0)
    assert rel.max() <= 1e-4, rel.max()


def test_half_bin_search_matches_oracle(gpu_lib):
    fd = gpu_lib
    N, zmax, m = 1 << 16, 40, 128
    chirps = [Chirp(3000.5, 10.0, 7.0, 0.3, 4), Chirp(7100.25, -16.0, 8.0, 1.1, 2),
              Chirp(12000.0, 4.0, 6.0, 2.0, 8)]
    x = make_series(N, 91, chirps)
    stream = torch.cuda.current_stream(DEV).cuda_stream
    plan = fd.fdas_plan_create(N, zmax, 2, m, 2048, 8, 6.0, 1 << 15, stream)
    try:
        fd.fdas_plan_set_interbin(plan, 1)
        info = fd.fdas_plan_get_info(plan)
        d_x = torch.from_numpy(x).to(DEV)
        out = np.zeros(info.max_cands, dtype=fd.CAND_DTYPE)
        cnt = np.zeros(1, dtype=np.int64)
        fd.fdas_search(plan, d_x, 1, out, cnt)
        plane = torch.empty(info.Z * 2 * info.nb, dtype=torch.float32, device=DEV)
        fd.fdas_plane_debug(plan, plane)
        torch.cuda.synchronize()
        # back to the integer plane on the same plan
        fd.fdas_plan_set_interbin(plan, 0)
        out0 = np.zeros(info.max_cands, dtype=fd.CAND_DTYPE)
        fd.fdas_search(plan, d_x, 1, out0, cnt)
    finally:
        fd.fdas_plan_destroy(plan)
    _, _, P, cands, H = O.search(x, zmax, 2, m, 8, 6.0, interbin=True)
    P_gpu = plane.cpu().numpy().reshape(P.shape).astype(np.float64)
    assert (np.abs(P_gpu - P) / np.maximum(P, 1.0)).max() <= 1e-4
    T = O.thresholds(8)
    got = out[out["h"] > 0]
    want = {(c[0], c[1], c[2]) for c in cands}
    have = {(int(a["r_top"]), int(a["z_idx"]), int(a["h"])) for a in got}
    for (r, j, h) in want ^ have:
        assert abs(H[h][j, r] - T[h]) <= 1e-4 * T[h], (r, j, h)
    # the half-bin chirp at 3000.5 is found at the odd column 6001
    assert any(c[0] == 6001 and c[2] == 1 for c in cands)
    assert (6001, (10 + 40) // 2, 1) in have
    _, _, _, cands0, H0 = O.search(x, zmax, 2, m, 8, 6.0)
    have0 = {(int(a["r_top"]), int(a["z_idx"]), int(a["h"])) for a in out0[out0["h"] > 0]}
    for (r, j, h) in have0 ^ {(c[0], c[1], c[2]) for c in cands0}:
        assert abs(H0[h][j, r] - T[h]) <= 1e-4 * T[h], (r, j, h)
