"""CPU-side checks of the C-ABI library: it builds, loads, exports every
symbol the header declares, validates arguments before touching the GPU, and
its float64 Fresnel integrals (the ones the template kernel runs) agree with
scipy's."""
import os
import re

import numpy as np
import pytest
from scipy import special

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1511_07343_gb300 import build as b
    b.build()
    from paper_1511_07343_gb300 import fdas
    fdas.load()
    return fdas


def declared_functions():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^[A-Za-z_][\w\s\*]*?\b(fdas_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("fdas_plan_create", "fdas_plan_destroy", "fdas_search", "fdas_plane_debug",
                     "fdas_strerror"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    import ctypes
    so = ctypes.CDLL(lib.library_path())
    missing = [n for n in declared_functions() if not hasattr(so, n)]
    assert not missing, missing


def test_binding_uses_header_names(lib):
    for n in declared_functions():
        assert hasattr(lib, n), n


@pytest.mark.parametrize("x", list(np.linspace(-30, 30, 241)) + [1.79, 1.8, 1.81, 1e-3, 250.3, -410.7])
def test_host_fresnel_matches_scipy(lib, x):
    c, s = lib.fdas_host_fresnel(float(x))
    S, C = special.fresnel(x)
    assert abs(c - C) < 2e-14 and abs(s - S) < 2e-14, (x, c - C, s - S)


@pytest.mark.parametrize("args", [
    dict(N=3000), dict(N=1 << 11), dict(N=1 << 25), dict(N=7 * 4096), dict(N=3 * 2048), dict(zmax=-2), dict(dz=0), dict(zmax=5, dz=2),
    dict(m=7), dict(m=4), dict(L=1024), dict(L=2048, m=1100), dict(nharm=3), dict(nharm=32),
    dict(sigma=0.0), dict(max_cands=0)])
def test_plan_create_rejects_bad_arguments(lib, args):
    p = dict(N=1 << 14, zmax=20, dz=2, m=64, L=2048, nharm=4, sigma=6.0, max_cands=100)
    p.update(args)
    with pytest.raises(lib.FdasError) as e:
        lib.fdas_plan_create(p["N"], p["zmax"], p["dz"], p["m"], p["L"], p["nharm"], p["sigma"],
                             p["max_cands"])
    assert e.value.status == lib.FDAS_ERR_INVALID


def test_strerror(lib):
    assert lib.fdas_strerror(0) == "ok"
    assert "overflow" in lib.fdas_strerror(lib.FDAS_ERR_OVERFLOW)
    assert lib.fdas_strerror(-99) == "unknown status"


def test_null_arguments_are_rejected(lib):
    import ctypes
    so = lib.load()
    assert so.fdas_search(None, None, 1, None, None) == lib.FDAS_ERR_INVALID
    assert so.fdas_plan_destroy(None) == lib.FDAS_OK
    assert so.fdas_plan_get_info(None, None) == lib.FDAS_ERR_INVALID
    assert so.fdas_host_fresnel(1.0, None, None) == lib.FDAS_ERR_INVALID
    del ctypes


@pytest.mark.parametrize("N", [3 * 4096, 5 * 4096, 15 * 4096, 45 * 4096, 3 << 21])
def test_plan_create_accepts_235_lengths(lib, N):
    """Uneven lengths 2^a 3^b 5^c (a >= 12) pass validation; on a machine
    without a GPU creation then stops at the first device allocation."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("needs a machine without a GPU")
    with pytest.raises(lib.FdasError) as e:
        lib.fdas_plan_create(N, 20, 2, 64, 2048, 4, 6.0, 100)
    assert e.value.status in (lib.FDAS_ERR_NOMEM, lib.FDAS_ERR_CUDA)


def test_newer_entry_points_reject_null_and_bad_arguments(lib):
    """Argument checks of the later entry points run before any device work."""
    import ctypes
    so = lib.load()
    INV = lib.FDAS_ERR_INVALID
    assert so.fdas_plan_set_correlation(None, 1) == INV
    assert so.fdas_plan_set_whitening(None, 1) == INV
    assert so.fdas_plan_set_harmsum_block(None, 32) == INV
    assert so.fdas_plan_set_interbin(None, 1) == INV
    assert so.fdas_plan_set_wait_limit(None, 1) == INV
    assert so.fdas_distill(None, None, None, None, None) == INV
    assert so.fdas_batch_set_graphs(None, 1) == INV
    assert so.fdas_batch_get_info(None, None) == INV
    assert so.fdas_search_batch(None, None, None, None, 1, None, None) == INV
    assert so.fdas_batch_add_class(None, 100, 256, 4096) == INV
    assert so.fdas_batch_destroy(None) == lib.FDAS_OK
    out = ctypes.c_void_p()
    assert so.fdas_batch_create_tuned(None, 1 << 14, 20, 2, 64, 4, 6.0, 16, None, None) == INV
    # an impossible length fails before the tuner touches the device
    assert so.fdas_batch_create_tuned(ctypes.byref(out), 3000, 20, 2, 64, 4, 6.0, 16, None,
                                      None) == INV
    assert out.value is None
    assert so.fdas_spectrum_noalloc(None, 1 << 14, None, None) == INV
    assert so.fdas_stage_plane(None, None, None) == INV


def test_binding_dtypes_match_the_c_structs(lib):
    """The numpy record types and ctypes structures mirror fdas.h."""
    assert lib.CAND_DTYPE.itemsize == 16
    assert lib.PEAK_DTYPE.itemsize == 24
    assert list(lib.PEAK_DTYPE.names) == ["r_top", "z_idx", "h", "power", "sigma", "log10_p"]
    import ctypes
    assert ctypes.sizeof(lib.fdas_batch_info) == 8 + 4 * 4 + 8 * 2 + 4 + 3 * 4 * 8 + 4 + 8
    src = open(os.path.join(ROOT, "include", "fdas.h")).read()
    for field in ("r_top", "z_idx", "power", "sigma", "log10_p", "graph_builds", "tuned_ms"):
        assert field in src


def test_misaligned_device_pointers_are_rejected_before_device_work(lib):
    """A series or spectrum pointer that is not 8-byte aligned (a view at an
    odd float) is an argument error, returned before the GPU is touched (so
    it also holds on this machine without one)."""
    with pytest.raises(lib.FdasError) as e:
        lib.fdas_spectrum_noalloc(0x10004, 1 << 12, 0x20000, 0)
    assert e.value.status == lib.FDAS_ERR_INVALID
    assert "d_series" in str(e.value) and "aligned" in str(e.value)
    with pytest.raises(lib.FdasError) as e:
        lib.fdas_spectrum_noalloc(0x10000, 1 << 12, 0x20004, 0)
    assert e.value.status == lib.FDAS_ERR_INVALID
    assert "d_spectrum" in str(e.value)
    so = lib.load()
    assert so.fdas_batch_create_tuned(None, 1 << 14, 20, 2, 64, 4, 6.0, 16, 0x10004,
                                      None) == lib.FDAS_ERR_INVALID
