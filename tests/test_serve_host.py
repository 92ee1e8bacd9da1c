"""Host logic of the serving loop that needs no GPU: the footprint estimate
used for admission and the thread-safe byte budget."""
import threading

import pytest

from paper_1511_07343_gb300.serve import Budget, plan_footprint, DEFAULT_CLASSES


def test_footprint_covers_the_plane_and_grows_with_zmax():
    n = 1 << 23
    sizes = {z: plan_footprint(n, z, m, L) for z, (m, L) in DEFAULT_CLASSES.items()}
    assert sizes[50] < sizes[100] < sizes[200]
    # at least the float32 plane and its 4-bin maxima: 5 bytes per cell
    assert sizes[200] >= 201 * (n // 2) * 5
    assert plan_footprint(n // 2, 200, 512, 8192) < sizes[200]


def test_budget_reserve_release():
    b = Budget(100)
    assert b.try_reserve(60)
    assert not b.try_reserve(41)
    assert b.try_reserve(40)
    b.release(60)
    assert b.reserved == 40
    with pytest.raises(ValueError):
        b.release(41)


def test_budget_is_thread_safe():
    b = Budget(1000)
    got = []

    def worker():
        for _ in range(200):
            if b.try_reserve(7):
                got.append(1)
                b.release(7)

    ts = [threading.Thread(target=worker) for _ in range(8)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    assert b.reserved == 0 and len(got) == 1600
