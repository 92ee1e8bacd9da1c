"""Failure detection of the bounded device waits (no planted hang): the
tensor-core correlation's pipeline waits are given a limit of one poll, so
the first wait runs out; the kernel must still retire its copies and MMAs,
free its tensor memory and return, the call must report FDAS_ERR_TIMEOUT,
and the same plan must then search correctly with the default limit."""
import numpy as np
import pytest
import torch

from oracle import fdas_oracle as O
from synthetic import Chirp, make_series

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0") if torch.cuda.is_available() else None


@pytest.mark.parametrize("mode", [1, 2])
def test_wait_that_runs_out_reports_timeout_and_the_plan_recovers(gpu_lib, mode):
    fd = gpu_lib
    N, zmax, m, L, nharm = 1 << 14, 20, 64, 2048, 4
    x = make_series(N, 31, [Chirp(2100.3, 6.0, 12.0, 0.5, 3)])
    stream = torch.cuda.current_stream(DEV).cuda_stream
    plan = fd.fdas_plan_create(N, zmax, 2, m, L, nharm, 6.0, 1 << 16, stream)
    try:
        fd.fdas_plan_set_correlation(plan, mode)
        info = fd.fdas_plan_get_info(plan)
        d_x = torch.from_numpy(x).to(DEV)
        out = np.zeros(info.max_cands, dtype=fd.CAND_DTYPE)
        cnt = np.zeros(1, dtype=np.int64)
        fd.fdas_plan_set_wait_limit(plan, 1)
        for _ in range(2):
            with pytest.raises(fd.FdasError) as e:
                fd.fdas_search(plan, d_x, 1, out, cnt)
            assert e.value.status == fd.FDAS_ERR_TIMEOUT
        white = torch.zeros(N, dtype=torch.float32, device=DEV)
        plane = torch.empty(info.Z * info.nb, dtype=torch.float32, device=DEV)
        with pytest.raises(fd.FdasError) as e:
            fd.fdas_stage_plane(plan, white, plane)
        assert e.value.status == fd.FDAS_ERR_TIMEOUT
        torch.cuda.synchronize()             # the context is still usable
        fd.fdas_plan_set_wait_limit(plan, 0)
        fd.fdas_search(plan, d_x, 1, out, cnt)
        fd.fdas_plane_debug(plan, plane)
        torch.cuda.synchronize()
    finally:
        fd.fdas_plan_destroy(plan)
    _, _, P, cands, H = O.search(x, zmax, 2, m, nharm, 6.0)
    P_gpu = plane.cpu().numpy().reshape(P.shape).astype(np.float64)
    tol = {1: 1e-4, 2: 2e-5}[mode]
    assert (np.abs(P_gpu - P) / np.maximum(P, 1.0)).max() <= tol
    T = O.thresholds(nharm)
    have = {(int(c["r_top"]), int(c["z_idx"]), int(c["h"])) for c in out[: cnt[0]]}
    want = {(c[0], c[1], c[2]) for c in cands}
    assert want
    for (r, j, h) in have ^ want:
        assert abs(H[h][j, r] - T[h]) <= tol * (T[h] + h), (r, j, h)
