"""Batches that mix zmax classes and series lengths (the stream of DM trials
of Section 1, each searched over its own acceleration range): one
fdas_search_batch call, direct or as one graph launch, gives every trial the
same sorted candidate list as a single-trial plan of that trial's class and
length, and those lists match the oracle."""
import numpy as np
import pytest
import torch

from oracle import fdas_oracle as O
from synthetic import Chirp, make_series

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0") if torch.cuda.is_available() else None

# zmax -> (template width m, segment length L), the 128/256/512-tap pattern
CLASSES = {50: (128, 2048), 100: (256, 4096), 200: (512, 8192)}
NHARM = 8
MAXC = 1 << 14


def sorted_list(arr):
    a = np.array(arr, dtype=arr.dtype)
    a.sort(order=["h", "r_top", "z_idx"])
    return a


def single_plan_list(fd, x, zmax):
    m, L = CLASSES[zmax]
    stream = torch.cuda.current_stream(DEV).cuda_stream
    plan = fd.fdas_plan_create(len(x), zmax, 2, m, L, NHARM, 6.0, MAXC, stream)
    try:
        out = np.zeros(MAXC, dtype=fd.CAND_DTYPE)
        cnt = np.zeros(1, dtype=np.int64)
        fd.fdas_search(plan, torch.from_numpy(x).to(DEV), 1, out, cnt)
    finally:
        fd.fdas_plan_destroy(plan)
    return out[: cnt[0]]


def trials():
    lengths = [1 << 16, 3 << 14, 5 << 13, 1 << 15, 1 << 16, 3 << 14]
    zmaxes = [200, 50, 100, 200, 100, 50]
    xs = []
    for i, (n, z) in enumerate(zip(lengths, zmaxes)):
        chirps = [Chirp(0.21 * n / 2 + 57 * i, (0.3 - 0.1 * i) * z, 9.0, 0.3 * i, 4)]
        xs.append(make_series(n, 4100 + i, chirps))
    return lengths, zmaxes, xs


def run_batch(fd, batch, xs, lengths, zmaxes):
    d_xs = [torch.from_numpy(x).to(DEV) for x in xs]
    d_out = torch.empty(len(xs) * MAXC * 16, dtype=torch.uint8, device=DEV)
    d_cnt = torch.zeros(len(xs), dtype=torch.int64, device=DEV)
    fd.fdas_search_batch(batch, d_xs, lengths, d_out, d_cnt, zmaxes)
    torch.cuda.synchronize()
    arr = d_out.cpu().numpy().view(fd.CAND_DTYPE)
    cnt = d_cnt.cpu().numpy()
    return [sorted_list(arr[t * MAXC: t * MAXC + cnt[t]]) for t in range(len(xs))], d_xs


@pytest.mark.parametrize("graphs", [0, 1])
def test_mixed_zmax_batch_equals_single_plans(gpu_lib, graphs):
    fd = gpu_lib
    lengths, zmaxes, xs = trials()
    single = [single_plan_list(fd, x, z) for x, z in zip(xs, zmaxes)]
    stream = torch.cuda.Stream(DEV)   # two trial lanes need a non-default stream
    m, L = CLASSES[50]
    # the smallest class first, so that adding the others grows the shared
    # workspaces (and remakes the lane)
    batch = fd.fdas_batch_create(max(lengths), 50, 2, m, L, NHARM, 6.0, MAXC, stream.cuda_stream)
    try:
        for z in (100, 200):
            fd.fdas_batch_add_class(batch, z, *CLASSES[z])
        fd.fdas_batch_set_graphs(batch, graphs)
        got, _ = run_batch(fd, batch, xs, lengths, zmaxes)
        again, _ = run_batch(fd, batch, xs, lengths, zmaxes)   # replay (graphs) or relaunch
        info = fd.fdas_batch_get_info(batch)
    finally:
        fd.fdas_batch_destroy(batch)
    assert info.n_classes == 3
    for t in range(len(xs)):
        assert len(single[t]) > 0
        assert got[t].tobytes() == sorted_list(single[t]).tobytes(), t
        assert again[t].tobytes() == got[t].tobytes(), t
    if graphs:
        assert info.graph_launches == 2 and info.graph_builds >= 1


def test_mixed_zmax_batch_matches_oracle(gpu_lib):
    fd = gpu_lib
    lengths, zmaxes, xs = trials()
    pick = [1, 2, 3]            # one trial of each class
    stream = torch.cuda.Stream(DEV)
    batch = fd.fdas_batch_create(1 << 16, 200, 2, *CLASSES[200], NHARM, 6.0, MAXC,
                                 stream.cuda_stream)
    try:
        for z in (50, 100):
            fd.fdas_batch_add_class(batch, z, *CLASSES[z])
        got, _ = run_batch(fd, batch, [xs[i] for i in pick], [lengths[i] for i in pick],
                           [zmaxes[i] for i in pick])
    finally:
        fd.fdas_batch_destroy(batch)
    T = O.thresholds(NHARM)
    for g, i in zip(got, pick):
        m, _ = CLASSES[zmaxes[i]]
        _, _, _, cands, H = O.search(xs[i], zmaxes[i], 2, m, NHARM, 6.0)
        have = {(int(c["r_top"]), int(c["z_idx"]), int(c["h"])) for c in g}
        want = {(c[0], c[1], c[2]) for c in cands}
        assert want
        for (r, j, h) in have ^ want:
            assert abs(H[h][j, r] - T[h]) <= 1e-4 * T[h], (i, (r, j, h))


def test_batch_class_errors(gpu_lib):
    fd = gpu_lib
    stream = torch.cuda.current_stream(DEV).cuda_stream
    batch = fd.fdas_batch_create(1 << 14, 20, 2, 64, 2048, 1, 6.0, 16, stream)
    try:
        with pytest.raises(fd.FdasError) as e:
            fd.fdas_batch_add_class(batch, 20, 64, 2048)       # one class per zmax
        assert e.value.status == fd.FDAS_ERR_INVALID
        with pytest.raises(fd.FdasError) as e:
            fd.fdas_batch_add_class(batch, 31, 64, 2048)       # dz = 2 must divide zmax
        assert e.value.status == fd.FDAS_ERR_INVALID
        with pytest.raises(fd.FdasError) as e:
            fd.fdas_batch_add_class(batch, 40, 2048, 2048)     # L >= 2 m
        assert e.value.status == fd.FDAS_ERR_INVALID
        d_x = torch.zeros(1 << 14, dtype=torch.float32, device=DEV)
        d_out = torch.empty(16 * 16, dtype=torch.uint8, device=DEV)
        d_cnt = torch.zeros(1, dtype=torch.int64, device=DEV)
        with pytest.raises(fd.FdasError) as e:
            fd.fdas_search_batch(batch, [d_x], [1 << 14], d_out, d_cnt, [40])  # no such class
        assert e.value.status == fd.FDAS_ERR_INVALID
        fd.fdas_batch_add_class(batch, 40, 128, 2048)
        fd.fdas_search_batch(batch, [d_x], [1 << 14], d_out, d_cnt, [40])
        torch.cuda.synchronize()
        assert fd.fdas_batch_get_info(batch).n_classes == 2
    finally:
        fd.fdas_batch_destroy(batch)


@pytest.mark.slow
def test_mixed_zmax_batch_full_size(gpu_lib):
    """The serving shapes at full size: three 2^23-sample trials and one at an
    uneven length, zmax 50 / 100 / 200 / 200, 16 harmonics, through one
    fdas_search_batch call on two lanes: each trial's sorted list is byte for
    byte the list of a single plan of its class."""
    from synthetic import random_chirps, snap_235
    fd = gpu_lib
    maxc = 1 << 20
    n_full = 1 << 23
    rng = np.random.default_rng(21)
    lengths = [n_full, n_full, n_full, snap_235(3.1e6 * 2)]
    zmaxes = [50, 100, 200, 200]
    xs = [make_series(n, 7100 + i, random_chirps(rng, 3, n, z), device=DEV)
          for i, (n, z) in enumerate(zip(lengths, zmaxes))]
    single = []
    stream = torch.cuda.current_stream(DEV).cuda_stream
    for x, z in zip(xs, zmaxes):
        m, L = CLASSES[z]
        plan = fd.fdas_plan_create(len(x), z, 2, m, L, 16, 6.0, maxc, stream)
        try:
            out = np.zeros(maxc, dtype=fd.CAND_DTYPE)
            cnt = np.zeros(1, dtype=np.int64)
            fd.fdas_search(plan, torch.from_numpy(x).to(DEV), 1, out, cnt)
        finally:
            fd.fdas_plan_destroy(plan)
        single.append(sorted_list(out[: cnt[0]]))
    st = torch.cuda.Stream(DEV)
    batch = fd.fdas_batch_create(n_full, 200, 2, *CLASSES[200], 16, 6.0, maxc, st.cuda_stream)
    try:
        for z in (50, 100):
            fd.fdas_batch_add_class(batch, z, *CLASSES[z])
        fd.fdas_batch_set_graphs(batch, 0)
        d_xs = [torch.from_numpy(x).to(DEV) for x in xs]
        d_out = torch.empty(len(xs) * maxc * 16, dtype=torch.uint8, device=DEV)
        d_cnt = torch.zeros(len(xs), dtype=torch.int64, device=DEV)
        fd.fdas_search_batch(batch, d_xs, lengths, d_out, d_cnt, zmaxes)
        torch.cuda.synchronize()
        arr = d_out.cpu().numpy().view(fd.CAND_DTYPE)
        cnt = d_cnt.cpu().numpy()
    finally:
        fd.fdas_batch_destroy(batch)
    for t in range(len(xs)):
        assert len(single[t]) > 0
        got = sorted_list(arr[t * maxc: t * maxc + cnt[t]])
        assert got.tobytes() == single[t].tobytes(), t
