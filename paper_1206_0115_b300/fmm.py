"""Python binding of libfmm_b300.so (include/fmm.h), argument marshalling only.

Every function keeps its C name and returns what the C call returns; the
arrays are passed as raw pointers.  Device arrays are torch CUDA tensors
(PyTorch serves only as the device allocator and stream owner here); host
arrays are numpy arrays or CPU tensors.  There is no fallback: importing this
module fails if the shared library is absent, and a failing C call raises
FMMError with the library's message.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# FMM_LIBRARY=debug selects the debug build (bounds checks, fmm_debug_check)
LIB_PATH = os.path.join(HERE, "libfmm_b300_debug.so" if os.environ.get("FMM_LIBRARY") == "debug"
                        else "libfmm_b300.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "fmm.h")

FMM_OK, FMM_ERR_ARG, FMM_ERR_OOM, FMM_ERR_CUDA, FMM_ERR_STATE, FMM_ERR_TIMEOUT = 0, -1, -2, -3, -4, -5
FMM_FP64, FMM_MIXED = 0, 1
FMM_M2L_FULL, FMM_M2L_SVD = 0, 1
FMM_P2P_VARIANTS = 16
FMM_SCHED_CANDIDATES = 8
STATUS_NAMES = {0: "FMM_OK", -1: "FMM_ERR_ARG", -2: "FMM_ERR_OOM", -3: "FMM_ERR_CUDA", -4: "FMM_ERR_STATE",
                -5: "FMM_ERR_TIMEOUT"}

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with paper_1206_0115_b300/build.py "
                      "(the package has no CPU fallback)")

lib = C.CDLL(LIB_PATH)

_vp = C.c_void_p
_SIGS = {
    "fmm_create": [C.c_int, C.c_int, C.POINTER(_vp)],
    "fmm_destroy": [_vp],
    "fmm_set_stream": [_vp, _vp],
    "fmm_set_precision": [_vp, C.c_int],
    "fmm_set_m2l": [_vp, C.c_int, C.c_double],
    "fmm_set_kernel": [_vp, C.c_double, C.c_double],
    "fmm_evaluate_stokes": [_vp, _vp, _vp],
    "fmm_get_svd_ranks": [_vp, _vp],
    "fmm_set_particles": [_vp, C.c_int64, _vp, _vp],
    "fmm_set_batch": [_vp, C.c_int32, _vp, _vp, _vp, _vp],
    "fmm_get_batch_info": [_vp, C.c_int32, _vp, _vp],
    "fmm_batch_plan": [C.c_int32, _vp, _vp, _vp, _vp, _vp],
    "fmm_evaluate": [_vp, _vp, _vp],
    "fmm_get_order": [_vp, _vp],
    "fmm_trim": [_vp],
    "fmm_autotune": [_vp, _vp, _vp],
    "fmm_set_p2p_variant": [_vp, C.c_int],
    "fmm_get_box": [_vp, _vp],
    "fmm_get_level_size": [_vp, C.c_int, _vp],
    "fmm_get_level_keys": [_vp, C.c_int, _vp],
    "fmm_get_level_ranges": [_vp, C.c_int, _vp, _vp],
    "fmm_get_expansion": [_vp, C.c_int, C.c_int, _vp],
    "fmm_get_stats": [_vp, _vp],
    "fmm_get_work": [_vp, _vp],
    "fmm_set_timing": [_vp, C.c_int],
    "fmm_get_stage_times": [_vp, _vp],
    "fmm_get_m2l_kernel_times": [_vp, _vp],
    "fmm_morton_order_noalloc": [C.c_int64, _vp, C.c_int, _vp, _vp, _vp],
    "fmm_measure_fp32_rate": [_vp],
    "fmm_set_wait_limit": [_vp, C.c_double],
    "fmm_get_p2p_bins": [_vp, _vp, _vp],
    "fmm_set_schedule": [_vp, C.c_int],
    "fmm_debug_build": [],
    "fmm_debug_check": [_vp],
    "fmm_get_schedule": [_vp, _vp, _vp],
}
_SIGS.update({
    "fmm_server_create": [_vp, C.POINTER(_vp)],
    "fmm_server_warmup": [_vp, C.c_int],
    "fmm_server_submit": [_vp, C.c_int64, C.c_int, C.c_int, _vp, _vp, _vp, _vp, C.POINTER(C.c_int64)],
    "fmm_server_wait": [_vp, C.c_int64, C.c_double, _vp],
    "fmm_server_stats": [_vp, _vp],
    "fmm_server_destroy": [_vp],
})
for _name, _args in _SIGS.items():
    _f = getattr(lib, _name)
    _f.argtypes = _args
    _f.restype = C.c_int
lib.fmm_last_error.argtypes = [_vp]
lib.fmm_last_error.restype = C.c_char_p
lib.fmm_server_last_error.argtypes = [_vp]
lib.fmm_server_last_error.restype = C.c_char_p
lib.fmm_server_request_bytes.argtypes = [C.c_int64, C.c_int, C.c_int]
lib.fmm_server_request_bytes.restype = C.c_int64


class fmm_server_config(C.Structure):
    _fields_ = [("lanes", C.c_int32), ("precision", C.c_int32), ("hbm_budget_bytes", C.c_int64),
                ("max_batch_particles", C.c_int64), ("max_batch_requests", C.c_int32), ("reserved", C.c_int32)]


class FMMError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


def _check(h, status: int):
    if status != FMM_OK:
        msg = lib.fmm_last_error(h)
        raise FMMError(status, msg.decode() if msg else "")
    return status


def _ptr(a) -> int | None:
    """Raw address of a torch tensor or numpy array (None for None)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("arrays passed to the FMM library must be contiguous")
        return a.data_ptr()
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays passed to the FMM library must be C-contiguous")
        return a.ctypes.data
    raise TypeError(f"unsupported array type {type(a)}")


# ---- the C entry points, same names --------------------------------------------

def fmm_create(height: int, order: int) -> int:
    h = _vp()
    _check(None, lib.fmm_create(height, order, C.byref(h)))
    return h.value


def fmm_destroy(h) -> int:
    return _check(h, lib.fmm_destroy(h))


def fmm_set_stream(h, stream) -> int:
    handle = stream.cuda_stream if hasattr(stream, "cuda_stream") else stream
    return _check(h, lib.fmm_set_stream(h, handle))


def fmm_set_precision(h, precision: int) -> int:
    return _check(h, lib.fmm_set_precision(h, precision))


def fmm_set_kernel(h, s: float, c: float = 0.0) -> int:
    return _check(h, lib.fmm_set_kernel(h, float(s), float(c)))


def fmm_evaluate_stokes(h, f, u) -> int:
    return _check(h, lib.fmm_evaluate_stokes(h, _ptr(f), _ptr(u)))


def fmm_set_m2l(h, method: int, eps: float = 0.0) -> int:
    return _check(h, lib.fmm_set_m2l(h, method, float(eps)))


def fmm_get_svd_ranks(h) -> np.ndarray:
    out = np.zeros(16, dtype=np.int32)
    _check(h, lib.fmm_get_svd_ranks(h, _ptr(out)))
    return out


def fmm_set_particles(h, n: int, xyz, q) -> int:
    return _check(h, lib.fmm_set_particles(h, n, _ptr(xyz), _ptr(q)))


def fmm_set_batch(h, counts, heights, xyz, q) -> int:
    counts = np.ascontiguousarray(counts, dtype=np.int64)
    heights = np.ascontiguousarray(heights, dtype=np.int32)
    if counts.shape != heights.shape or counts.ndim != 1:
        raise ValueError("counts and heights must be 1-D arrays of the same length")
    return _check(h, lib.fmm_set_batch(h, len(counts), _ptr(counts), _ptr(heights), _ptr(xyz), _ptr(q)))


def fmm_batch_plan(counts, heights):
    """Host-only slot layout of a batch: (slot_key[k], slot_level[k], leaf level)."""
    counts = np.ascontiguousarray(counts, dtype=np.int64)
    heights = np.ascontiguousarray(heights, dtype=np.int32)
    key = np.zeros(len(counts), dtype=np.int64)
    lev = np.zeros(len(counts), dtype=np.int64)
    leaf = np.zeros(1, dtype=np.int32)
    _check(None, lib.fmm_batch_plan(len(counts), _ptr(counts), _ptr(heights), _ptr(key), _ptr(lev), _ptr(leaf)))
    return key, lev, int(leaf[0])


def fmm_get_batch_info(h, k: int):
    info = np.zeros(8, dtype=np.int64)
    box = np.zeros(4, dtype=np.float64)
    _check(h, lib.fmm_get_batch_info(h, k, _ptr(info), _ptr(box)))
    return info, box


def fmm_evaluate(h, phi, F) -> int:
    return _check(h, lib.fmm_evaluate(h, _ptr(phi), _ptr(F)))


def fmm_autotune(h):
    """Returns (choice [index, warps, chunk, sources per instruction, unroll],
    mean ms of each P2P variant)."""
    choice = np.zeros(5, dtype=np.int32)
    times = np.zeros(FMM_P2P_VARIANTS, dtype=np.float32)
    _check(h, lib.fmm_autotune(h, _ptr(choice), _ptr(times)))
    return choice, times


def fmm_set_p2p_variant(h, variant: int) -> int:
    return _check(h, lib.fmm_set_p2p_variant(h, variant))


def fmm_trim(h) -> int:
    return _check(h, lib.fmm_trim(h))


def fmm_get_order(h, perm) -> int:
    return _check(h, lib.fmm_get_order(h, _ptr(perm)))


def fmm_get_box(h) -> np.ndarray:
    out = np.zeros(4)
    _check(h, lib.fmm_get_box(h, _ptr(out)))
    return out


def fmm_get_level_size(h, level: int) -> int:
    out = np.zeros(1, dtype=np.int64)
    _check(h, lib.fmm_get_level_size(h, level, _ptr(out)))
    return int(out[0])


def fmm_get_level_keys(h, level: int, keys) -> int:
    return _check(h, lib.fmm_get_level_keys(h, level, _ptr(keys)))


def fmm_get_level_ranges(h, level: int, first, count) -> int:
    return _check(h, lib.fmm_get_level_ranges(h, level, _ptr(first), _ptr(count)))


def fmm_get_expansion(h, level: int, which: int, out) -> int:
    return _check(h, lib.fmm_get_expansion(h, level, which, _ptr(out)))


def fmm_get_stats(h) -> np.ndarray:
    out = np.zeros(8, dtype=np.int64)
    _check(h, lib.fmm_get_stats(h, _ptr(out)))
    return out


def fmm_get_work(h) -> np.ndarray:
    out = np.zeros(16, dtype=np.int64)
    _check(h, lib.fmm_get_work(h, _ptr(out)))
    return out


def fmm_set_timing(h, mode) -> int:
    """0 off, 1 (or True) events in the normal schedule, 2 every stage alone."""
    return _check(h, lib.fmm_set_timing(h, int(mode)))


def fmm_get_stage_times(h) -> np.ndarray:
    out = np.zeros(8, dtype=np.float32)
    _check(h, lib.fmm_get_stage_times(h, _ptr(out)))
    return out


def fmm_get_m2l_kernel_times(h) -> np.ndarray:
    out = np.zeros(2, dtype=np.float32)
    _check(h, lib.fmm_get_m2l_kernel_times(h, _ptr(out)))
    return out


def fmm_get_p2p_bins(h):
    """(out[4]: small shape, large shape, small items, large items; times [2][variants])"""
    out = np.zeros(4, dtype=np.int64)
    times = np.zeros((2, FMM_P2P_VARIANTS), dtype=np.float32)
    _check(h, lib.fmm_get_p2p_bins(h, _ptr(out), _ptr(times)))
    return out, times


def fmm_set_schedule(h, sched: int) -> int:
    return _check(h, lib.fmm_set_schedule(h, int(sched)))


def fmm_get_schedule(h):
    """(schedule, mean evaluation ms of each candidate of the last autotune)"""
    sched = np.zeros(1, dtype=np.int32)
    times = np.zeros(FMM_SCHED_CANDIDATES, dtype=np.float32)
    _check(h, lib.fmm_get_schedule(h, _ptr(sched), _ptr(times)))
    return int(sched[0]), times


def fmm_debug_build() -> bool:
    return bool(lib.fmm_debug_build())


def fmm_debug_check() -> int:
    """The first failed bounds check since the last call (site << 32 | index), 0 if none."""
    out = np.zeros(1, dtype=np.uint64)
    _check(None, lib.fmm_debug_check(_ptr(out)))
    return int(out[0])


def fmm_set_wait_limit(h, seconds: float) -> int:
    return _check(h, lib.fmm_set_wait_limit(h, float(seconds)))


def fmm_measure_fp32_rate() -> np.ndarray:
    """[scalar FMA flop/s, packed f32x2 FMA flop/s, SM count, 0] of the current device."""
    out = np.zeros(4, dtype=np.float64)
    _check(None, lib.fmm_measure_fp32_rate(_ptr(out)))
    return out


def fmm_morton_order_noalloc(n: int, xyz, height: int, keys, perm, stream=None) -> int:
    handle = stream.cuda_stream if hasattr(stream, "cuda_stream") else stream
    return _check(None, lib.fmm_morton_order_noalloc(n, _ptr(xyz), height, _ptr(keys), _ptr(perm), handle))


def _check_server(s, status: int):
    if status != FMM_OK:
        msg = lib.fmm_server_last_error(s) if s else b""
        raise FMMError(status, msg.decode() if msg else "")
    return status


def fmm_server_request_bytes(n: int, height: int, order: int) -> int:
    return int(lib.fmm_server_request_bytes(n, height, order))


def fmm_server_create(lanes: int, precision: int, hbm_budget_bytes: int, max_batch_particles: int,
                      max_batch_requests: int) -> int:
    cfg = fmm_server_config(lanes, precision, hbm_budget_bytes, max_batch_particles, max_batch_requests, 0)
    s = _vp()
    _check_server(None, lib.fmm_server_create(C.byref(cfg), C.byref(s)))
    return s.value


def fmm_server_warmup(s, order: int) -> int:
    return _check_server(s, lib.fmm_server_warmup(s, order))


def fmm_server_submit(s, n: int, height: int, order: int, xyz, q, phi, F) -> int:
    t = C.c_int64(0)
    _check_server(s, lib.fmm_server_submit(s, n, height, order, _ptr(xyz), _ptr(q), _ptr(phi), _ptr(F),
                                           C.byref(t)))
    return t.value


def fmm_server_wait(s, ticket: int, timeout_s: float = -1.0) -> np.ndarray:
    """Blocks (without the GIL) until the request is done; returns its times
    [queue ms, service ms, latency ms, batch size]."""
    times = np.zeros(4, dtype=np.float64)
    _check_server(s, lib.fmm_server_wait(s, ticket, timeout_s, _ptr(times)))
    return times


def fmm_server_stats(s) -> np.ndarray:
    out = np.zeros(13, dtype=np.int64)
    _check_server(s, lib.fmm_server_stats(s, _ptr(out)))
    return out


def fmm_server_destroy(s) -> int:
    return lib.fmm_server_destroy(s)


def fmm_server_last_error(s) -> str:
    m = lib.fmm_server_last_error(s)
    return m.decode() if m else ""


def fmm_last_error(h) -> str:
    m = lib.fmm_last_error(h)
    return m.decode() if m else ""


# ---- convenience wrapper -------------------------------------------------------

class FMM:
    """Owns one handle.  Inputs/outputs are torch tensors (CUDA or CPU) or numpy
    arrays; every step runs in the CUDA library."""

    def __init__(self, height: int, order: int, precision: int = FMM_MIXED, stream=None,
                 m2l: int = FMM_M2L_SVD, svd_eps: float = 0.0, kernel_s: float = 1.0,
                 kernel_c: float = 0.0):
        self.h = fmm_create(height, order)
        self.height, self.order = height, order
        fmm_set_precision(self.h, precision)
        fmm_set_m2l(self.h, m2l, svd_eps)
        if kernel_s != 1.0 or kernel_c != 0.0:
            fmm_set_kernel(self.h, kernel_s, kernel_c)
        if stream is not None:
            fmm_set_stream(self.h, stream)
        self.n = 0

    def close(self):
        if getattr(self, "h", None):
            fmm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_precision(self, precision: int):
        fmm_set_precision(self.h, precision)

    def set_m2l(self, method: int, eps: float = 0.0):
        fmm_set_m2l(self.h, method, eps)

    def set_kernel(self, s: float, c: float = 0.0):
        """Kernel (|x - y|^2 + c^2)^(-s/2) of later evaluations (s = 1, c = 0:
        Laplace)."""
        fmm_set_kernel(self.h, s, c)

    def svd_ranks(self) -> np.ndarray:
        return fmm_get_svd_ranks(self.h)

    def set_particles(self, xyz, q):
        n = int(xyz.shape[0])
        fmm_set_particles(self.h, n, xyz, q)
        self.n = n

    def set_batch(self, counts, heights, xyz, q):
        """Independent problems, particles concatenated in problem order."""
        fmm_set_batch(self.h, counts, heights, xyz, q)
        self.n = int(np.sum(counts))

    def batch_info(self, k: int):
        return fmm_get_batch_info(self.h, k)

    def evaluate(self, phi, F):
        fmm_evaluate(self.h, phi, F)

    def evaluate_stokes(self, f, u):
        """Stokeslet velocities u [n][3] of forces f [n][3] at the particles."""
        fmm_evaluate_stokes(self.h, f, u)

    def order_perm(self, out):
        fmm_get_order(self.h, out)

    def level_size(self, level: int) -> int:
        return fmm_get_level_size(self.h, level)

    def box(self) -> np.ndarray:
        return fmm_get_box(self.h)

    def stats(self) -> np.ndarray:
        return fmm_get_stats(self.h)


def exported_symbols_of_header(path: str = HEADER) -> list[str]:
    """Names of the functions include/fmm.h declares."""
    import re
    text = open(path).read()
    return sorted(set(re.findall(r"^\s*(?:fmm_status|const char\*)\s+(fmm_\w+)\s*\(", text, re.M)))
