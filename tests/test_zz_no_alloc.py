"""The allocation-free Morton ordering against the ordinary tree build.

fmm_morton_order_noalloc is meant for callers that cannot allocate device
memory while they run: a serving process whose HBM belongs to a pool it
reserved at start-up, or a plug-in that only receives buffers from its host
application.  Instead of cudaMalloc it uses one fixed array compiled into the
library, shared by every call on a GPU and keeping the previous call's
contents.  Its output must be exactly what fmm_set_particles builds: the same
Morton permutation (fmm_get_order) and, per Morton rank, the key of the
particle's leaf (fmm_get_level_keys of the leaf level, repeated over each
leaf's particles).  Integer results, so the bar is bit equality, and it is
checked on two calls in a row with different sizes and shapes so that stale
contents of the shared array would show.
"""
import ctypes

import numpy as np
import pytest

from paper_1206_0115_b300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1206_0115_b300 import build
    build.build()
    from paper_1206_0115_b300 import fmm
    return fmm


def _reference_order(F, xyz_d, q_d, h):
    import torch
    n = xyz_d.shape[0]
    with F.FMM(h, 3, F.FMM_FP64) as f:
        f.set_particles(xyz_d, q_d)
        perm = torch.empty(n, dtype=torch.int64, device="cuda")
        F.fmm_get_order(f.h, perm)
        nl = f.level_size(h - 1)
        lk = np.zeros(nl, dtype=np.uint64)
        first = np.zeros(nl, dtype=np.int64)
        count = np.zeros(nl, dtype=np.int64)
        F.fmm_get_level_keys(f.h, h - 1, lk)
        F.fmm_get_level_ranges(f.h, h - 1, first, count)
    return perm.cpu().numpy(), np.repeat(lk, count)


def test_noalloc_matches_set_particles_twice(F):
    import torch
    cases = [(200_000, 1, "cube", 6), (37_000, 3, "ellipsoid", 8)]
    for n, seed, dist, h in cases:
        xyz, q = inputs.particles(n, seed, dist, "pos")
        xyz_d = torch.from_numpy(xyz).cuda()
        keys = torch.full((n,), -1, dtype=torch.int64, device="cuda")
        perm = torch.full((n,), -1, dtype=torch.int64, device="cuda")
        st = F.lib.fmm_morton_order_noalloc(n, xyz_d.data_ptr(), h, keys.data_ptr(), perm.data_ptr(), None)
        assert st == F.FMM_OK, F.fmm_last_error(None)
        ref_perm, ref_keys = _reference_order(F, xyz_d, torch.from_numpy(q).cuda(), h)
        assert np.array_equal(perm.cpu().numpy(), ref_perm), (n, dist)
        assert np.array_equal(keys.cpu().numpy().astype(np.uint64), ref_keys), (n, dist)


def test_noalloc_rejects_oversize_and_bad_arguments(F):
    n = (1 << 18) + 1
    st = F.lib.fmm_morton_order_noalloc(n, ctypes.c_void_p(16), 4, ctypes.c_void_p(16), ctypes.c_void_p(16), None)
    assert st == F.FMM_ERR_ARG
    assert "262144" in F.fmm_last_error(None)
    assert F.lib.fmm_morton_order_noalloc(10, None, 4, None, None, None) == F.FMM_ERR_ARG
    assert F.lib.fmm_morton_order_noalloc(10, ctypes.c_void_p(16), 0, ctypes.c_void_p(16), ctypes.c_void_p(16),
                                          None) == F.FMM_ERR_ARG
