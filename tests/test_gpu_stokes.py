"""The Stokes kernel (fmm_evaluate_stokes): Stokeslet velocities from four
1/r passes on one tree.

The oracle is oracle.stokes_fmm (the same four passes through the FP64 CPU
oracle, positions as given) and oracle.stokes_direct (the Stokeslet sums
written out).  Bars: FP64 <= 1e-10 and mixed precision <= 1e-5 relative L2
against the oracle's FMM (same height, order and M2L form); trees of height
<= 2 against the direct sums (FP64 <= 1e-12); the handle's own charges are
restored (a later fmm_evaluate is unchanged, bit for bit).
"""
import functools

import numpy as np
import pytest

import oracle
from paper_1206_0115_b300 import inputs

pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-10
TOL_MIXED = 1e-5


@pytest.fixture(scope="module")
def F():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1206_0115_b300 import build
    build.build()
    from paper_1206_0115_b300 import fmm
    return fmm


@functools.lru_cache(maxsize=None)
def _case(n, seed, dist):
    xyz, q = inputs.particles(n, seed, dist, "sym")
    f = np.stack([inputs.charges(n, seed + 1 + k, "sym", 0) for k in range(3)], axis=1)
    return xyz, q, np.ascontiguousarray(f)


@functools.lru_cache(maxsize=None)
def _oracle(n, seed, dist, h, p, svd):
    xyz, _, f = _case(n, seed, dist)
    return oracle.stokes_fmm(xyz, f, h, p, svd_eps=10.0 ** -p if (svd and h >= 3) else None)


def _gpu(F, xyz, q, f, h, p, precision, m2l, host=False):
    import torch
    n = len(q)
    with F.FMM(h, p, precision, m2l=m2l) as fm:
        fm.set_particles(torch.from_numpy(xyz).cuda(), torch.from_numpy(q).cuda())
        if host:
            u = np.zeros((n, 3))
            fm.evaluate_stokes(f, u)
            return u
        u = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
        fm.evaluate_stokes(torch.from_numpy(f).cuda(), u)
        torch.cuda.synchronize()
        return u.cpu().numpy()


@pytest.mark.parametrize("svd", [True, False], ids=["svd", "full"])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_stokes_matches_the_oracle(F, svd, prec):
    precision = F.FMM_FP64 if prec == "fp64" else F.FMM_MIXED
    tol = TOL_FP64 if prec == "fp64" else TOL_MIXED
    m2l = F.FMM_M2L_SVD if svd else F.FMM_M2L_FULL
    for n, seed, dist, h, p in ((20000, 101, "cube", 4, 5), (30000, 105, "ellipsoid", 5, 6)):
        xyz, q, f = _case(n, seed, dist)
        u = _gpu(F, xyz, q, f, h, p, precision, m2l, host=(dist == "cube"))
        ref = _oracle(n, seed, dist, h, p, svd)
        assert oracle.rel_l2(u, ref) <= tol, (dist, prec, oracle.rel_l2(u, ref))


@pytest.mark.parametrize("h", [1, 2])
def test_stokes_near_field_only_is_the_direct_sum(F, h):
    xyz, q, f = _case(3000, 109, "cube")
    ud = oracle.stokes_direct(xyz, f)
    u = _gpu(F, xyz, q, f, h, 4, F.FMM_FP64, F.FMM_M2L_SVD)
    assert oracle.rel_l2(u, ud) <= 1e-12
    u = _gpu(F, xyz, q, f, h, 4, F.FMM_MIXED, F.FMM_M2L_SVD)
    assert oracle.rel_l2(u, ud) <= TOL_MIXED


def test_stokes_error_against_the_direct_sum_falls_with_order(F):
    xyz, q, f = _case(20000, 113, "cube")
    ud = oracle.stokes_direct(xyz, f)
    errs = []
    for p in (3, 5, 7):
        u = _gpu(F, xyz, q, f, 4, p, F.FMM_MIXED, F.FMM_M2L_SVD)
        eo = oracle.rel_l2(_oracle(20000, 113, "cube", 4, p, True), ud)
        e = oracle.rel_l2(u, ud)
        assert e <= eo + TOL_MIXED, (p, e, eo)
        errs.append(e)
    assert errs[0] > errs[1] > errs[2], errs


def test_stokes_restores_the_charges_and_checks_state(F):
    import torch
    xyz, q, f = _case(20000, 117, "cube")
    n = len(q)
    with F.FMM(4, 5, F.FMM_MIXED) as fm:
        fm.set_particles(torch.from_numpy(xyz).cuda(), torch.from_numpy(q).cuda())
        outs = []
        for k in range(2):
            phi = torch.zeros(n, dtype=torch.float64, device="cuda")
            Fo = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
            fm.evaluate(phi, Fo)
            torch.cuda.synchronize()
            outs.append((phi.cpu().numpy(), Fo.cpu().numpy()))
            if k == 0:
                fm.evaluate_stokes(f, np.zeros((n, 3)))
        assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])
        fm.set_kernel(2.0)
        with pytest.raises(F.FMMError) as e:
            fm.evaluate_stokes(f, np.zeros((n, 3)))
        assert e.value.status == F.FMM_ERR_STATE
    with F.FMM(3, 4, F.FMM_MIXED) as fm:
        with pytest.raises(F.FMMError) as e:
            fm.evaluate_stokes(f, np.zeros((n, 3)))        # no particles
        assert e.value.status == F.FMM_ERR_STATE
        fm.set_batch(np.array([1000, 2000], dtype=np.int64), np.array([3, 4], dtype=np.int32),
                     torch.from_numpy(xyz[:3000].copy()).cuda(), torch.from_numpy(q[:3000].copy()).cuda())
        with pytest.raises(F.FMMError) as e:
            fm.evaluate_stokes(f[:3000].copy(), np.zeros((3000, 3)))
        assert e.value.status == F.FMM_ERR_STATE
