"""The serving loop: requests of mixed length and acceleration range, queued
together and served by concurrent slots, give exactly the candidates that a
standalone search of each one gives."""
import numpy as np
import pytest
import torch

from synthetic import Chirp, make_series

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0") if torch.cuda.is_available() else None

CLASSES = {20: (64, 2048), 40: (128, 2048)}


def standalone(fd, x, zmax):
    m, L = CLASSES[zmax]
    n = x.shape[0]
    stream = torch.cuda.current_stream(DEV).cuda_stream
    plan = fd.fdas_plan_create(n, zmax, 2, m, L, 8, 6.0, 1 << 16, stream)
    try:
        info = fd.fdas_plan_get_info(plan)
        d_x = torch.from_numpy(x).to(DEV)
        out = np.zeros(info.max_cands, dtype=fd.CAND_DTYPE)
        cnt = np.zeros(1, dtype=np.int64)
        fd.fdas_search(plan, d_x, 1, out, cnt)
        return out[:cnt[0]], int(cnt[0])
    finally:
        fd.fdas_plan_destroy(plan)


def test_results_alone_equal_results_in_the_mix(gpu_lib):
    from paper_1511_07343_gb300.serve import Server
    fd = gpu_lib
    lengths = [1 << 16, 3 << 14, 1 << 15, 5 << 13, 1 << 16, 3 << 14, 1 << 16, 1 << 15]
    zs = [20, 40, 40, 20, 40, 20, 20, 40]
    xs = [make_series(n, 70 + i, [Chirp(0.13 * n / 2 + 97 * i, 4.0 * (i % 3) - 3, 9.0, 0.1 * i, 4)])
          for i, n in enumerate(lengths)]
    with Server(n_max=1 << 16, n_slots=3, classes=CLASSES, nharm=8, max_cands=1 << 16) as srv:
        futs = [srv.submit(x, z) for x, z in zip(xs, zs)]
        res = [f.result(timeout=300) for f in futs]
        assert srv.stats["admitted"] == len(xs)
    for x, z, r in zip(xs, zs, res):
        ref, cnt = standalone(fd, x, z)
        assert r.count == cnt
        assert cnt > 0
        assert r.candidates.tobytes() == np.sort(ref, order=["h", "r_top", "z_idx"]).tobytes()
        assert r.latency_ms > 0


def test_memory_budget_limits_slots(gpu_lib):
    """Admission by footprint: a budget below one slot's footprint starts no
    slot (submit refuses); a budget of one slot starts exactly one, which
    serves every request of both classes, in batches of up to two."""
    from paper_1511_07343_gb300.serve import Server, batch_footprint
    srv = Server(n_max=1 << 15, n_slots=2, classes=CLASSES, nharm=4, max_cands=1 << 14,
                 hbm_budget=1)
    with pytest.raises(ValueError):
        srv.submit(np.zeros(1 << 15, dtype=np.float32), 20)
    srv.close()
    budget = batch_footprint(1 << 15, CLASSES, 2, 1 << 14, lanes=True)
    with Server(n_max=1 << 15, n_slots=2, classes=CLASSES, nharm=4, max_cands=1 << 14,
                hbm_budget=budget) as srv:
        assert srv.stats["slots"] == 1
        xs = [make_series(1 << 15, 200 + i, [Chirp(3000.0 + 10 * i, 2.0, 12.0, 0.0, 2)])
              for i in range(6)]
        futs = [srv.submit(x, (20, 40)[i % 2]) for i, x in enumerate(xs)]
        res = [f.result(timeout=300) for f in futs]
        assert srv.stats["largest_batch"] <= 2
    assert all(r.count > 0 for r in res)


def test_cancelled_request_does_not_stop_the_server(gpu_lib):
    """Requests cancelled while queued are dropped; every other request is
    served and equals its standalone search."""
    from paper_1511_07343_gb300.serve import Server
    fd = gpu_lib
    xs = [make_series(1 << 15, 600 + i, [Chirp(2500.0 + 40 * i, 3.0, 11.0, 0.2, 3)])
          for i in range(8)]
    with Server(n_max=1 << 15, n_slots=1, classes=CLASSES, nharm=8, max_cands=1 << 16,
                max_batch=2) as srv:
        futs = [srv.submit(x, 20) for x in xs]
        cancelled = [i for i in (3, 5, 6) if futs[i].cancel()]
        res = {i: f.result(timeout=300) for i, f in enumerate(futs) if i not in cancelled}
        assert srv.stats["cancelled"] == len(cancelled)
    for i, r in res.items():
        ref, cnt = standalone(fd, xs[i], 20)
        assert r.count == cnt
        assert r.candidates.tobytes() == np.sort(ref, order=["h", "r_top", "z_idx"]).tobytes()


def test_batch_footprint_bounds_the_batch_device_bytes(gpu_lib):
    from paper_1511_07343_gb300.serve import DEFAULT_CLASSES, batch_footprint
    fd = gpu_lib
    stream = torch.cuda.Stream(DEV)
    n = 1 << 20
    batch = fd.fdas_batch_create(n, 200, 2, 512, 8192, 16, 6.0, 1 << 16, stream.cuda_stream)
    try:
        for z in (50, 100):
            fd.fdas_batch_add_class(batch, z, *DEFAULT_CLASSES[z])
        d_x = torch.zeros(2 * n, dtype=torch.float32, device=DEV)
        d_out = torch.empty(2 * (1 << 16) * 16, dtype=torch.uint8, device=DEV)
        d_cnt = torch.zeros(2, dtype=torch.int64, device=DEV)
        fd.fdas_search_batch(batch, [d_x[:n], d_x[n:]], [n, n], d_out, d_cnt, [50, 200])
        torch.cuda.synchronize()
        info = fd.fdas_batch_get_info(batch)
    finally:
        fd.fdas_batch_destroy(batch)
    est = batch_footprint(n, DEFAULT_CLASSES, 2, 1 << 16, lanes=True)
    assert info.device_bytes <= est <= 1.5 * info.device_bytes, (info.device_bytes, est)


def test_footprint_estimate_bounds_the_plans_device_bytes(gpu_lib):
    from paper_1511_07343_gb300.serve import plan_footprint
    fd = gpu_lib
    stream = torch.cuda.current_stream(DEV).cuda_stream
    for zmax, (m, L) in {50: (128, 2048), 200: (512, 8192)}.items():
        plan = fd.fdas_plan_create(1 << 20, zmax, 2, m, L, 16, 6.0, 1 << 16, stream)
        try:
            info = fd.fdas_plan_get_info(plan)
        finally:
            fd.fdas_plan_destroy(plan)
        est = plan_footprint(1 << 20, zmax, m, L, 2, 1 << 16)
        assert info.device_bytes <= est <= 1.5 * info.device_bytes, (zmax, info.device_bytes, est)
