"""ctypes front end of the FP64 CPU oracle (oracle.c).

TEST INFRASTRUCTURE ONLY: imported by the tests, by the package's smoke check
and by the benchmark's CPU-baseline leg, never by the product library.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None

_d = C.POINTER(C.c_double)
_i64 = C.POINTER(C.c_int64)
_u64 = C.POINTER(C.c_uint64)
_i32 = C.POINTER(C.c_int32)


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        sig = {
            "ofmm_cheb_nodes": (None, [C.c_int, _d]),
            "ofmm_cheb_S": (C.c_double, [C.c_int, C.c_double, C.c_double]),
            "ofmm_cheb_dS": (C.c_double, [C.c_int, C.c_double, C.c_double]),
            "ofmm_bounding_cube": (None, [C.c_int64, _d, _d, _d]),
            "ofmm_keys": (None, [C.c_int64, _d, _d, C.c_double, C.c_int, _u64]),
            "ofmm_create": (C.c_void_p, [C.c_int64, _d, _d, C.c_int, C.c_int]),
            "ofmm_destroy": (None, [C.c_void_p]),
            "ofmm_box": (None, [C.c_void_p, _d, _d]),
            "ofmm_level_size": (C.c_int64, [C.c_void_p, C.c_int]),
            "ofmm_level_keys": (None, [C.c_void_p, C.c_int, _u64]),
            "ofmm_level_ranges": (None, [C.c_void_p, C.c_int, _i64, _i64]),
            "ofmm_perm": (None, [C.c_void_p, _i64]),
            "ofmm_p2m": (None, [C.c_void_p]),
            "ofmm_m2m": (None, [C.c_void_p]),
            "ofmm_m2l": (None, [C.c_void_p]),
            "ofmm_l2l": (None, [C.c_void_p]),
            "ofmm_l2p": (None, [C.c_void_p, _d, _d]),
            "ofmm_p2p": (None, [C.c_void_p, _d, _d]),
            "ofmm_expansion": (None, [C.c_void_p, C.c_int, C.c_int, _d]),
            "ofmm_evaluate": (None, [C.c_void_p, _d, _d]),
            "ofmm_evaluate_sampled": (None, [C.c_void_p, C.c_int64, _i64, _d, _d]),
            "ofmm_transfer_symmetry": (None, [_i32, _i32, _i32, _i32]),
            "ofmm_canonical_index": (C.c_int, [_i32]),
            "ofmm_node_permutation": (None, [C.c_int, _i32, _i32, _i32]),
            "ofmm_jacobi_svd": (C.c_int, [C.c_int, _d, _d, _d, _d]),
            "ofmm_set_m2l_svd": (C.c_int, [C.c_void_p, C.c_double]),
            "ofmm_svd_rank": (C.c_int, [C.c_void_p, C.c_int]),
            "ofmm_copy_m2l_svd": (C.c_int, [C.c_void_p, C.c_void_p]),
            "ofmm_m2l_apply": (None, [C.c_void_p, _i32, _d, _d]),
            "ofmm_m2l_pair_count": (C.c_int64, [C.c_void_p, C.c_int]),
            "ofmm_coverage": (None, [C.c_void_p, _i32]),
            "ofmm_direct": (None, [C.c_int64, _d, _d, _d, _d]),
            "ofmm_direct_kernel": (None, [C.c_int64, _d, _d, C.c_double, C.c_double, _d, _d]),
            "ofmm_direct_sampled_kernel": (None, [C.c_int64, _d, _d, C.c_double, C.c_double, C.c_int64, _i64, _d, _d]),
            "ofmm_set_kernel": (C.c_int, [C.c_void_p, C.c_double, C.c_double]),
            "ofmm_stokes_direct": (None, [C.c_int64, _d, _d, _d]),
            "ofmm_direct_sampled": (None, [C.c_int64, _d, _d, C.c_int64, _i64, _d, _d]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _p(a: np.ndarray, ct):
    return a.ctypes.data_as(ct)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def cheb_nodes(order: int) -> np.ndarray:
    out = np.zeros(order)
    lib().ofmm_cheb_nodes(order, _p(out, _d))
    return out


def cheb_S(order: int, xbar: float, xi: float) -> float:
    return lib().ofmm_cheb_S(order, xbar, xi)


def cheb_dS(order: int, xbar: float, xi: float) -> float:
    return lib().ofmm_cheb_dS(order, xbar, xi)


def bounding_cube(xyz):
    xyz = _f64(xyz).reshape(-1, 3)
    lo = np.zeros(3)
    w = np.zeros(1)
    lib().ofmm_bounding_cube(xyz.shape[0], _p(xyz, _d), _p(lo, _d), _p(w, _d))
    return lo, float(w[0])


def morton_keys(xyz, lo, width: float, leaf: int) -> np.ndarray:
    xyz = _f64(xyz).reshape(-1, 3)
    lo = _f64(lo)
    keys = np.zeros(xyz.shape[0], dtype=np.uint64)
    lib().ofmm_keys(xyz.shape[0], _p(xyz, _d), _p(lo, _d), width, leaf, _p(keys, _u64))
    return keys


def direct(xyz, q, kernel_s: float = 1.0, kernel_c: float = 0.0):
    """Exact potentials and fields by O(N^2) summation (eq. 1, 2; otherwise
    the kernel (|x - y|^2 + c^2)^(-s/2) and F = -grad phi)."""
    xyz = _f64(xyz).reshape(-1, 3)
    q = _f64(q)
    n = xyz.shape[0]
    phi = np.zeros(n)
    F = np.zeros((n, 3))
    lib().ofmm_direct_kernel(n, _p(xyz, _d), _p(q, _d), float(kernel_s), float(kernel_c), _p(phi, _d), _p(F, _d))
    return phi, F


def direct_sampled(xyz, q, idx, kernel_s: float = 1.0, kernel_c: float = 0.0):
    xyz = _f64(xyz).reshape(-1, 3)
    q = _f64(q)
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    phi = np.zeros(idx.shape[0])
    F = np.zeros((idx.shape[0], 3))
    lib().ofmm_direct_sampled_kernel(xyz.shape[0], _p(xyz, _d), _p(q, _d), float(kernel_s), float(kernel_c), idx.shape[0],
                                     _p(idx, _i64), _p(phi, _d), _p(F, _d))
    return phi, F


def stokes_direct(xyz, f):
    """Stokeslet sums u_i = sum_{k != i} [f_k / r + d (d . f_k) / r^3],
    d = x_i - x_k (the Stokes kernel, unit viscosity factor), by O(N^2)
    summation."""
    xyz = _f64(xyz).reshape(-1, 3)
    f = _f64(f).reshape(-1, 3)
    u = np.zeros_like(xyz)
    lib().ofmm_stokes_direct(xyz.shape[0], _p(xyz, _d), _p(f, _d), _p(u, _d))
    return u


def stokes_fmm(xyz, f, height: int, order: int, svd_eps=None):
    """The Stokeslet sums from four 1/r FMM passes on one tree.  With
    phi^j, F^j = -grad phi^j the 1/r potentials and fields of the charges
    f_j (j = 0, 1, 2) and phi^3, F^3 those of the charges y . f,

        u_i = phi^i + sum_j x_j F^j_i - F^3_i,

    because d (d . f) / r^3 = -grad_x(1/r) ((x . f) - (y . f)).  The identity
    holds for any origin; positions are used as given."""
    xyz = _f64(xyz).reshape(-1, 3)
    f = _f64(f).reshape(-1, 3)
    charges = [f[:, 0], f[:, 1], f[:, 2], (xyz * f).sum(axis=1)]
    phis, Fs = [], []
    for q in charges:
        with OracleFMM(xyz, np.ascontiguousarray(q), height, order, svd_eps=svd_eps) as o:
            ph, F = o.evaluate()
        phis.append(ph)
        Fs.append(F)
    u = np.zeros_like(xyz)
    for i in range(3):
        u[:, i] = phis[i] + sum(xyz[:, j] * Fs[j][:, i] for j in range(3)) - Fs[3][:, i]
    return u


# SVD-compressed M2L (Sec. 2.1.2): cube symmetries, canonical vectors, Jacobi SVD

def canonical_vectors():
    """The 16 canonical transfer vectors (0 <= a <= b <= c <= 3, c >= 2), in
    the order of their index."""
    return [(a, b, c) for a in range(4) for b in range(a, 4) for c in range(b, 4) if c >= 2]


def transfer_symmetry(t):
    """(that, axis, sign) with t_d = sign[d] * that[axis[d]]."""
    ti = np.ascontiguousarray(t, dtype=np.int32)
    that = np.zeros(3, dtype=np.int32)
    axis = np.zeros(3, dtype=np.int32)
    sign = np.zeros(3, dtype=np.int32)
    lib().ofmm_transfer_symmetry(_p(ti, _i32), _p(that, _i32), _p(axis, _i32), _p(sign, _i32))
    return tuple(int(v) for v in that), axis, sign


def canonical_index(that) -> int:
    a = np.ascontiguousarray(that, dtype=np.int32)
    return int(lib().ofmm_canonical_index(_p(a, _i32)))


def node_permutation(order: int, axis, sign) -> np.ndarray:
    axis = np.ascontiguousarray(axis, dtype=np.int32)
    sign = np.ascontiguousarray(sign, dtype=np.int32)
    out = np.zeros(order ** 3, dtype=np.int32)
    lib().ofmm_node_permutation(order, _p(axis, _i32), _p(sign, _i32), _p(out, _i32))
    return out


def jacobi_svd(A):
    """(U, s, V, sweeps) with A = U diag(s) V^T (square A)."""
    A = _f64(A)
    n = A.shape[0]
    U = np.zeros((n, n))
    V = np.zeros((n, n))
    s = np.zeros(n)
    sweeps = lib().ofmm_jacobi_svd(n, _p(A, _d), _p(U, _d), _p(s, _d), _p(V, _d))
    return U, s, V, int(sweeps)


class OracleFMM:
    """One tree of the oracle: box, keys, sort and levels are built on creation.

    svd_eps: None for the full-rank M2L operators; a positive number switches
    M2L to the 16 SVD-compressed operators truncated at s_i >= svd_eps * s_0
    (the paper's pairing is svd_eps = 10^-order).
    """

    def __init__(self, xyz, q, height: int, order: int, svd_eps=None, svd_from=None, kernel_s: float = 1.0,
                 kernel_c: float = 0.0):
        self.xyz = _f64(xyz).reshape(-1, 3)
        self.q = _f64(q)
        self.n = self.xyz.shape[0]
        self.height, self.order = height, order
        self.ncoef = order ** 3
        self._h = lib().ofmm_create(self.n, _p(self.xyz, _d), _p(self.q, _d), height, order)
        if not self._h:
            raise ValueError("oracle rejected the arguments")
        self.kernel_s, self.kernel_c = kernel_s, kernel_c
        if (kernel_s != 1.0 or kernel_c != 0.0) and lib().ofmm_set_kernel(self._h, float(kernel_s),
                                                                           float(kernel_c)) != 0:
            raise ValueError("oracle: kernel outside -2 <= s <= 4, s != 0, c >= 0")
        self.svd_eps = svd_eps
        if svd_from is not None:
            # reuse another tree's compressed operators (they depend on order and eps only)
            self.svd_eps = svd_from.svd_eps
            if lib().ofmm_copy_m2l_svd(self._h, svd_from._h) != 0:
                raise ValueError("oracle: cannot share the compressed operators")
        elif svd_eps is not None and lib().ofmm_set_m2l_svd(self._h, float(svd_eps)) != 0:
            raise ValueError("oracle: the compression needs height >= 3, a homogeneous kernel (c = 0) "
                             "and a converged SVD")

    def svd_ranks(self) -> np.ndarray:
        return np.array([lib().ofmm_svd_rank(self._h, k) for k in range(16)])

    def m2l_apply(self, t, M) -> np.ndarray:
        """(operator of transfer vector t at unit half-width) @ M."""
        ti = np.ascontiguousarray(t, dtype=np.int32)
        M = _f64(M)
        out = np.zeros(self.ncoef)
        lib().ofmm_m2l_apply(self._h, _p(ti, _i32), _p(M, _d), _p(out, _d))
        return out

    def close(self):
        if self._h:
            lib().ofmm_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # tree
    def box(self):
        lo = np.zeros(3)
        w = np.zeros(1)
        lib().ofmm_box(self._h, _p(lo, _d), _p(w, _d))
        return lo, float(w[0])

    def level_size(self, level: int) -> int:
        return int(lib().ofmm_level_size(self._h, level))

    def level_keys(self, level: int) -> np.ndarray:
        out = np.zeros(self.level_size(level), dtype=np.uint64)
        lib().ofmm_level_keys(self._h, level, _p(out, _u64))
        return out

    def level_ranges(self, level: int):
        n = self.level_size(level)
        first = np.zeros(n, dtype=np.int64)
        count = np.zeros(n, dtype=np.int64)
        lib().ofmm_level_ranges(self._h, level, _p(first, _i64), _p(count, _i64))
        return first, count

    def perm(self) -> np.ndarray:
        out = np.zeros(self.n, dtype=np.int64)
        lib().ofmm_perm(self._h, _p(out, _i64))
        return out

    # operators
    def p2m(self):
        lib().ofmm_p2m(self._h)

    def m2m(self):
        lib().ofmm_m2m(self._h)

    def m2l(self):
        lib().ofmm_m2l(self._h)

    def l2l(self):
        lib().ofmm_l2l(self._h)

    def l2p(self):
        phi = np.zeros(self.n)
        F = np.zeros((self.n, 3))
        lib().ofmm_l2p(self._h, _p(phi, _d), _p(F, _d))
        return phi, F

    def p2p(self):
        phi = np.zeros(self.n)
        F = np.zeros((self.n, 3))
        lib().ofmm_p2p(self._h, _p(phi, _d), _p(F, _d))
        return phi, F

    def expansion(self, level: int, which: str) -> np.ndarray:
        out = np.zeros((self.level_size(level), self.ncoef))
        lib().ofmm_expansion(self._h, level, 1 if which == "L" else 0, _p(out, _d))
        return out

    def evaluate(self):
        phi = np.zeros(self.n)
        F = np.zeros((self.n, 3))
        lib().ofmm_evaluate(self._h, _p(phi, _d), _p(F, _d))
        return phi, F

    def evaluate_sampled(self, idx):
        idx = np.ascontiguousarray(idx, dtype=np.int64)
        phi = np.zeros(idx.shape[0])
        F = np.zeros((idx.shape[0], 3))
        lib().ofmm_evaluate_sampled(self._h, idx.shape[0], _p(idx, _i64), _p(phi, _d), _p(F, _d))
        return phi, F

    def m2l_pair_count(self, level: int) -> int:
        return int(lib().ofmm_m2l_pair_count(self._h, level))

    def coverage(self) -> np.ndarray:
        nl = self.level_size(self.height - 1)
        out = np.zeros((nl, nl), dtype=np.int32)
        lib().ofmm_coverage(self._h, _p(out, _i32))
        return out


def rel_l2(x, ref) -> float:
    """||x - ref||_2 / ||ref||_2 over all entries (vectors: over all components)."""
    x = np.asarray(x, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    den = np.sqrt((ref * ref).sum())
    return float(np.sqrt(((x - ref) ** 2).sum()) / den) if den > 0 else float(np.abs(x).max())


def num_threads() -> int:
    v = os.environ.get("OMP_NUM_THREADS")
    return int(v) if v else (os.cpu_count() or 1)
