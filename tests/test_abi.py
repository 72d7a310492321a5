"""Host-side checks of the C ABI (no GPU needed): the library loads, exports
every entry point include/fmm.h declares, and rejects bad arguments before it
touches the device."""
import ctypes
import subprocess

import pytest

from paper_1206_0115_b300 import build


@pytest.fixture(scope="module")
def F():
    build.build()
    from paper_1206_0115_b300 import fmm
    return fmm


def test_header_symbols_exported(F):
    names = F.exported_symbols_of_header()
    assert len(names) >= 16
    out = subprocess.run(["nm", "-D", "--defined-only", F.LIB_PATH], capture_output=True, text=True,
                         check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    for n in names:
        getattr(F.lib, n)


def test_bad_arguments_rejected_before_device_use(F):
    h = ctypes.c_void_p()
    assert F.lib.fmm_create(0, 5, ctypes.byref(h)) == F.FMM_ERR_ARG
    assert b"height" in F.lib.fmm_last_error(None)
    assert F.lib.fmm_create(4, 1, ctypes.byref(h)) == F.FMM_ERR_ARG
    assert b"order" in F.lib.fmm_last_error(None)
    assert F.lib.fmm_create(12, 5, ctypes.byref(h)) == F.FMM_ERR_ARG
    assert F.lib.fmm_create(4, 11, ctypes.byref(h)) == F.FMM_ERR_ARG
    assert F.lib.fmm_create(4, 5, None) == F.FMM_ERR_ARG
    for fn, args in [("fmm_set_stream", (None, None)), ("fmm_set_precision", (None, 1)),
                     ("fmm_set_particles", (None, 0, None, None)), ("fmm_evaluate", (None, None, None)),
                     ("fmm_get_order", (None, None)), ("fmm_get_box", (None, None)),
                     ("fmm_get_stats", (None, None)), ("fmm_set_timing", (None, 1))]:
        assert getattr(F.lib, fn)(*args) == F.FMM_ERR_ARG, fn
    assert F.lib.fmm_destroy(None) == F.FMM_OK


def test_create_without_device_reports_cuda_error(F):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    h = ctypes.c_void_p()
    assert F.lib.fmm_create(4, 5, ctypes.byref(h)) == F.FMM_ERR_CUDA
    assert h.value is None
    assert b"device" in F.lib.fmm_last_error(None)
