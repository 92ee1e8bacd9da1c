"""The allocation-free real FFT against the plan-based one.

fdas_spectrum_noalloc serves callers that must not allocate device memory
(a real-time loop with a fixed device footprint, or a host framework that
owns the allocator) and so cannot create a plan. It keeps its scratch in a
fixed device array shared by all calls; this file checks, through the C ABI,
that two calls in a row give the same spectrum as fdas_stage_spectrum and
as the oracle's, and that repeated calls leave the device's free memory
unchanged. It is collected last so that a failure here never hides the other
tests.
"""
import math

import numpy as np
import pytest
import torch

from oracle import fdas_oracle as O
from synthetic import Chirp, make_series

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("logn", [14, 20])
def test_noalloc_spectrum_matches_plan_path(gpu_lib, logn):
    fd = gpu_lib
    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream(dev).cuda_stream
    N = 1 << logn
    plan = fd.fdas_plan_create(N, 10, 2, 64, 2048, 1, 6.0, 16, stream)
    try:
        for call in range(2):  # two calls in a row on the shared scratch
            x = make_series(N, 900 + 10 * logn + call, [Chirp(0.2 * N / 2, 6.0, 10.0, 0.4, 3)])
            d_x = torch.from_numpy(x).to(dev)
            ref = torch.empty(N, dtype=torch.float32, device=dev)
            out = torch.full((N,), float("nan"), dtype=torch.float32, device=dev)
            fd.fdas_stage_spectrum(plan, d_x, ref)
            fd.fdas_spectrum_noalloc(d_x, N, out, stream)
            torch.cuda.synchronize()
            a = ref.cpu().numpy().view(np.complex64).astype(np.complex128)
            b = out.cpu().numpy().view(np.complex64).astype(np.complex128)
            rms = math.sqrt(np.mean(np.abs(a) ** 2))
            assert np.all(np.isfinite(b))
            assert np.max(np.abs(a - b)) <= 2e-5 * rms
            X = O.spectrum(x)
            assert np.max(np.abs(b - X)) <= 2e-5 * math.sqrt(np.mean(np.abs(X) ** 2))
    finally:
        fd.fdas_plan_destroy(plan)


def test_noalloc_rejects_sizes_beyond_its_limit(gpu_lib):
    fd = gpu_lib
    with pytest.raises(fd.FdasError) as e:
        fd.fdas_spectrum_noalloc(256, 1 << 21, 256, 0)   # aligned stand-ins: never touched
    assert e.value.status == fd.FDAS_ERR_INVALID
    assert "2^20" in str(e.value)


def test_noalloc_calls_leave_device_memory_unchanged(gpu_lib):
    """After a first call (which looks up the scratch array's address), more
    calls change neither the device's free memory nor torch's allocations:
    the entry point allocates and frees nothing."""
    fd = gpu_lib
    dev = torch.device("cuda:0")
    stream = torch.cuda.current_stream(dev).cuda_stream
    N = 1 << 18
    d_x = torch.from_numpy(make_series(N, 77, [Chirp(1000.0, 2.0, 9.0, 0.0, 1)])).to(dev)
    out = torch.empty(N, dtype=torch.float32, device=dev)
    fd.fdas_spectrum_noalloc(d_x, N, out, stream)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info(dev)
    alloc0 = torch.cuda.memory_allocated(dev)
    first = out.clone()
    for _ in range(5):
        fd.fdas_spectrum_noalloc(d_x, N, out, stream)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info(dev)
    assert free1 == free0
    assert torch.cuda.memory_allocated(dev) == alloc0 + first.numel() * 4
    assert torch.equal(out, first)


def test_noalloc_rejects_misaligned_pointers(gpu_lib):
    fd = gpu_lib
    dev = torch.device("cuda:0")
    buf = torch.zeros(1 << 13, dtype=torch.float32, device=dev)
    for a, b in ((buf.data_ptr() + 4, buf.data_ptr()), (buf.data_ptr(), buf.data_ptr() + 4)):
        with pytest.raises(fd.FdasError) as e:
            fd.fdas_spectrum_noalloc(a, 1 << 12, b, 0)
        assert e.value.status == fd.FDAS_ERR_INVALID
        assert "aligned" in str(e.value)
