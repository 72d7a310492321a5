"""Failure detection without a fault: a bounded device-side wait that runs out.

Every pipeline wait of the tensor-core M2L kernels is bounded in time.  With
the handle's limit set to 1 ns (fmm_set_wait_limit), the first wait that is
not already satisfied gives up: the kernel raises its error word, waits for
the copies and MMAs it has already issued (with the default 2 s limit),
frees its tensor memory and returns.  The next call on the handle reports
FMM_ERR_TIMEOUT, and the same handle with the default limit, and a fresh
handle, then give results that match the oracle: the CUDA context stays
usable.
"""
import numpy as np
import pytest

import oracle
from paper_1206_0115_b300 import inputs

pytestmark = pytest.mark.gpu

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


def _eval(f, dx, dq):
    import torch
    n = dq.shape[0]
    phi = torch.zeros(n, dtype=torch.float64, device="cuda")
    Fo = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    f.set_particles(dx, dq)
    f.evaluate(phi, Fo)
    torch.cuda.synchronize()
    return phi, Fo


@pytest.mark.parametrize("m2l", ["svd", "full"])
def test_expired_wait_reports_timeout_and_the_context_survives(F, m2l):
    import torch
    xyz, q = inputs.particles(20000, 41, "cube", "sym")
    dx, dq = torch.from_numpy(xyz).cuda(), torch.from_numpy(q).cuda()
    method = F.FMM_M2L_SVD if m2l == "svd" else F.FMM_M2L_FULL
    with oracle.OracleFMM(xyz, q, 4, 5, svd_eps=1e-5 if m2l == "svd" else None) as o:
        rphi, rF = o.evaluate()
    with F.FMM(4, 5, F.FMM_MIXED, m2l=method) as f:
        assert int(f.stats()[4]) in (2, 5)  # the tensor-core M2L runs
        with pytest.raises(F.FMMError) as e:
            F.fmm_set_wait_limit(f.h, 0.0)
        assert e.value.status == F.FMM_ERR_ARG
        F.fmm_set_wait_limit(f.h, 1e-9)
        _eval(f, dx, dq)  # returns after enqueueing; the kernels give up inside
        phi = torch.zeros(len(q), dtype=torch.float64, device="cuda")
        Fo = torch.zeros((len(q), 3), dtype=torch.float64, device="cuda")
        with pytest.raises(F.FMMError) as e:
            f.evaluate(phi, Fo)
        assert e.value.status == F.FMM_ERR_TIMEOUT
        # the same handle, default limit: the flag was cleared and results are right
        F.fmm_set_wait_limit(f.h, 2.0)
        phi, Fo = _eval(f, dx, dq)
        assert oracle.rel_l2(phi.cpu().numpy(), rphi) <= TOL_MIXED
        assert oracle.rel_l2(Fo.cpu().numpy(), rF) <= TOL_MIXED
    with F.FMM(4, 5, F.FMM_MIXED, m2l=method) as g:
        phi, Fo = _eval(g, dx, dq)
        assert oracle.rel_l2(phi.cpu().numpy(), rphi) <= TOL_MIXED
        assert oracle.rel_l2(Fo.cpu().numpy(), rF) <= TOL_MIXED
    assert np.isfinite(torch.ones(4, device="cuda").sum().item())
