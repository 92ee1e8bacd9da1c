"""Batches of uneven-length DM trials as captured CUDA graphs, and the
segment-length autotuner: a graph replay gives exactly what direct launches
give, a repeated batch replays without capturing again, and a tuned batch
uses the fastest segment length it timed."""
import numpy as np
import pytest
import torch

from synthetic import Chirp, make_series

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0") if torch.cuda.is_available() else None

LENGTHS = [1 << 16, 3 << 13, 5 << 12, 1 << 14, 15 << 12, 1 << 15]
N_MAX = 1 << 16
MAXC = 1 << 14


def series_list():
    xs = []
    for i, n in enumerate(LENGTHS):
        chirps = [Chirp(0.11 * n / 2 + 31 * i, 3.0 * (i % 4) - 4, 9.0, 0.3 * i, 4)]
        xs.append(torch.from_numpy(make_series(n, 500 + i, chirps)).to(DEV))
    torch.cuda.synchronize()
    return xs


def run(fd, batch, xs, stream):
    d_out = torch.zeros(len(xs) * MAXC * 16, dtype=torch.uint8, device=DEV)
    d_cnt = torch.zeros(len(xs), dtype=torch.int64, device=DEV)
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        fd.fdas_search_batch(batch, xs, [x.numel() for x in xs], d_out, d_cnt)
    stream.synchronize()
    return unpack(fd, d_out, d_cnt, len(xs))


def unpack(fd, d_out, d_cnt, n):
    cnt = d_cnt.cpu().numpy()
    raw = d_out.cpu().numpy().view(fd.CAND_DTYPE).reshape(n, MAXC)
    res = []
    for t in range(n):
        c = raw[t, :min(cnt[t], MAXC)].copy()
        c.sort(order=["h", "r_top", "z_idx"])
        res.append((int(cnt[t]), c.tobytes()))
    return res


def test_graph_replay_equals_direct_launches(gpu_lib):
    fd = gpu_lib
    stream = torch.cuda.Stream(DEV)
    xs = series_list()
    batch = fd.fdas_batch_create(N_MAX, 20, 2, 64, 2048, 8, 6.0, MAXC, stream.cuda_stream)
    try:
        fd.fdas_batch_set_graphs(batch, 0)
        direct = run(fd, batch, xs, stream)
        assert fd.fdas_batch_get_info(batch).graphs == 0
        fd.fdas_batch_set_graphs(batch, 1)
        g1 = run(fd, batch, xs, stream)
        g2 = run(fd, batch, xs, stream)
        info = fd.fdas_batch_get_info(batch)
        assert info.graphs == 1
        assert info.graph_launches == 2
        assert g1 == direct and g2 == direct
        assert all(c > 0 for c, _ in direct)
        # same arguments again: a pure replay, no capture
        d_out = torch.zeros(len(xs) * MAXC * 16, dtype=torch.uint8, device=DEV)
        d_cnt = torch.zeros(len(xs), dtype=torch.int64, device=DEV)
        lens = [x.numel() for x in xs]
        torch.cuda.synchronize()
        with torch.cuda.stream(stream):
            fd.fdas_search_batch(batch, xs, lens, d_out, d_cnt)
            builds = fd.fdas_batch_get_info(batch).graph_builds
            d_cnt.zero_()
            fd.fdas_search_batch(batch, xs, lens, d_out, d_cnt)
        stream.synchronize()
        info = fd.fdas_batch_get_info(batch)
        assert info.graph_builds == builds
        assert info.graph_launches == 4
        assert unpack(fd, d_out, d_cnt, len(xs)) == direct
        assert info.n_lengths == len(set(LENGTHS))
    finally:
        fd.fdas_batch_destroy(batch)


def test_tuned_batch_picks_the_fastest_segment(gpu_lib):
    fd = gpu_lib
    stream = torch.cuda.Stream(DEV)
    batch = fd.fdas_batch_create_tuned(N_MAX, 40, 2, 128, 4, 6.0, MAXC, None, stream.cuda_stream)
    try:
        info = fd.fdas_batch_get_info(batch)
        assert info.n_tuned == 6
        assert list(info.tuned_segment[:6]) == [2048, 2048, 4096, 4096, 8192, 8192]
        assert list(info.tuned_hs_block[:6]) == [256, 32] * 3
        ms = list(info.tuned_ms[:6])
        assert all(t > 0 for t in ms)
        best = int(np.argmin(ms))
        assert info.segment == info.tuned_segment[best]
        assert info.hs_block == info.tuned_hs_block[best]
        xs = series_list()
        got = run(fd, batch, xs, stream)
    finally:
        fd.fdas_batch_destroy(batch)
    # a plain batch with the chosen segment length gives the same lists
    ref_batch = fd.fdas_batch_create(N_MAX, 40, 2, 128, info.segment, 4, 6.0, MAXC,
                                     stream.cuda_stream)
    try:
        fd.fdas_batch_set_graphs(ref_batch, 0)
        ref = run(fd, ref_batch, xs, stream)
    finally:
        fd.fdas_batch_destroy(ref_batch)
    assert got == ref


def test_tuner_skips_segments_shorter_than_2m(gpu_lib):
    fd = gpu_lib
    stream = torch.cuda.Stream(DEV)
    probe = torch.from_numpy(make_series(N_MAX, 9, [])).to(DEV)
    torch.cuda.synchronize()
    batch = fd.fdas_batch_create_tuned(N_MAX, 20, 2, 2048, 1, 6.0, 256, probe,
                                       stream.cuda_stream)
    try:
        info = fd.fdas_batch_get_info(batch)
        assert info.n_tuned == 4
        assert list(info.tuned_segment[:4]) == [4096, 4096, 8192, 8192]
        assert info.segment in (4096, 8192)
    finally:
        fd.fdas_batch_destroy(batch)
