"""Host-side checks of the C ABI (no GPU needed): the library loads, exports
every entry point include/fmm.h declares, and rejects bad arguments before it
touches the device."""
import ctypes
import subprocess

import numpy as np
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


def test_server_request_bytes_formula(F):
    """The admission estimate the header documents: 256 B per particle plus,
    per cell (1.15 x min(n, 8^(h-1)) + 1), 28 x cpad + 4 x 189 x (16 | 32) + 1024."""
    for n, h, p in [(0, 3, 5), (1000, 3, 5), (10**6, 6, 7), (5 * 10**6, 7, 5), (12345, 1, 2)]:
        cpad = (p ** 3 + 1 + 31) // 32 * 32
        cells = int(1.15 * min(n, 8 ** (h - 1))) + 1
        want = 256 * n + cells * (28 * cpad + 4 * 189 * (16 if p <= 5 else 32) + 1024)
        assert F.fmm_server_request_bytes(n, h, p) == want
    assert F.fmm_server_request_bytes(-1, 3, 5) == -1
    assert F.fmm_server_request_bytes(10, 3, 11) == -1


def test_server_config_rejected_before_device_use(F):
    cfg = F.fmm_server_config(0, 1, 1 << 30, 1000, 4, 0)
    s = ctypes.c_void_p()
    assert F.lib.fmm_server_create(ctypes.byref(cfg), ctypes.byref(s)) == F.FMM_ERR_ARG
    for bad in [(2, 7, 1 << 30, 1000, 4, 0), (2, 1, 0, 1000, 4, 0), (2, 1, 1 << 30, 0, 4, 0),
                (2, 1, 1 << 30, 1000, 0, 0), (2, 1, 1 << 30, 1000, 5000, 0), (17, 1, 1 << 30, 1000, 4, 0)]:
        cfg = F.fmm_server_config(*bad)
        assert F.lib.fmm_server_create(ctypes.byref(cfg), ctypes.byref(s)) == F.FMM_ERR_ARG, bad
    assert F.lib.fmm_server_destroy(None) == F.FMM_OK
    assert F.lib.fmm_server_submit(None, 1, 3, 5, None, None, None, None, None) == F.FMM_ERR_ARG


def test_batch_plan_slots_are_aligned_disjoint_cells(F):
    """The batch layout (host only): every problem with particles owns an
    aligned, disjoint range of 8^(h-1) leaf keys -- one cell of the batch
    tree -- larger slots first, the leaf level minimal."""
    from paper_1206_0115_b300 import inputs
    rng_counts, rng_heights, _, _ = inputs.batch_workload(nprob=64, nmax=5e4)
    cases = [
        (rng_counts, rng_heights),
        ([5, 0, 7, 1, 9], [3, 4, 1, 6, 3]),
        ([1], [1]),
        ([10] * 9, [2] * 9),            # 9 slots of 8 keys: needs a leaf level of 2
        ([3, 3], [9, 1]),
        ([3], [10]),                    # one slot of the largest size
    ]
    for counts, heights in cases:
        counts = np.asarray(counts, dtype=np.int64)
        heights = np.asarray(heights, dtype=np.int32)
        key, lev, Lf = F.fmm_batch_plan(counts, heights)
        used = counts > 0
        assert np.all(key[~used] == -1) and np.all(lev[~used] == -1)
        size = 8 ** (heights.astype(np.int64) - 1)
        assert np.all(key[used] % size[used] == 0)                  # aligned: one cell
        assert np.all(lev[used] == Lf - (heights[used] - 1))
        spans = sorted((int(key[k]), int(key[k] + size[k])) for k in np.nonzero(used)[0])
        for (a0, a1), (b0, b1) in zip(spans, spans[1:]):
            assert a1 <= b0                                            # disjoint
        assert spans[-1][1] <= 8 ** Lf
        need = max(int(size[used].sum()), int(size[used].max()))
        assert Lf == 0 or 8 ** (Lf - 1) < need or Lf == int(heights[used].max()) - 1  # minimal
        order = np.argsort(key[used], kind="stable")
        assert np.all(np.diff(heights[used][order]) <= 0)             # larger slots first
    with pytest.raises(F.FMMError):
        F.fmm_batch_plan([1, 1], [10, 10])                             # 2 x 8^9 keys
    with pytest.raises(F.FMMError):
        F.fmm_batch_plan([1], [0])


def test_debug_build_exports_the_same_entry_points(F):
    """The bounds-checking build (FMM_DEBUG) is the same library with checks
    compiled in: it exports every entry point the header declares, says so
    through fmm_debug_build, and the normal build says it is not one."""
    lib = build.build(debug=True)
    out = subprocess.run(["nm", "-D", "--defined-only", lib], capture_output=True, text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    missing = [n for n in F.exported_symbols_of_header() if n not in exported]
    assert not missing, missing
    dbg = ctypes.CDLL(lib)
    assert dbg.fmm_debug_build() == 1
    assert F.lib.fmm_debug_build() == 0
    assert F.lib.fmm_debug_check(None) == F.FMM_ERR_ARG
