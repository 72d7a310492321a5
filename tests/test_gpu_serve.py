"""The solve server (fmm_server_*): continuous batching of independent
requests.

Bars: every request's result equals the same request solved alone through
fmm_set_particles + fmm_evaluate within 1e-6 relative L2 (mixed precision;
only the grouping of the tensor-core partial sums may differ) and matches the
FP64 oracle's FMM within 1e-5; the admission rule never lets the memory
estimate in flight exceed the budget; requests are batched together and
batches run at once on several lanes.
"""
import threading

import numpy as np
import pytest

import oracle
from paper_1206_0115_b300 import inputs

pytestmark = pytest.mark.gpu

TOL_ALONE = 1e-6
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


def _requests(count, seed0, nmin=800, nmax=30000, orders=(4, 5)):
    u = inputs.uniform01(seed0, 2 * count)
    reqs = []
    for k in range(count):
        n = int(10 ** (np.log10(nmin) + u[k] * (np.log10(nmax) - np.log10(nmin))))
        p = orders[int(u[count + k] * len(orders)) % len(orders)]
        s = seed0 + 1 + k
        xyz, q = inputs.particles(n, s, "cube" if s % 2 == 0 else "ellipsoid", "sym")
        reqs.append(dict(xyz=xyz, q=q, h=inputs.batch_height(n, 3, 5), p=p))
    return reqs


def _alone(F, r):
    import torch
    n = len(r["q"])
    with F.FMM(r["h"], r["p"], F.FMM_MIXED) as f:
        f.set_particles(torch.from_numpy(r["xyz"]).cuda(), torch.from_numpy(r["q"]).cuda())
        phi = torch.zeros(n, dtype=torch.float64, device="cuda")
        Fo = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
        f.evaluate(phi, Fo)
        torch.cuda.synchronize()
        return phi.cpu().numpy(), Fo.cpu().numpy()


def _submit(F, s, r):
    n = len(r["q"])
    r["phi"] = np.zeros(n)
    r["F"] = np.zeros((n, 3))
    r["ticket"] = F.fmm_server_submit(s, n, r["h"], r["p"], r["xyz"], r["q"], r["phi"], r["F"])


def test_results_in_the_mix_equal_results_alone(F):
    reqs = _requests(14, 4000)
    s = F.fmm_server_create(2, F.FMM_MIXED, 64 << 30, 200_000, 8)
    try:
        for order in (4, 5):
            F.fmm_server_warmup(s, order)
        for r in reqs:
            _submit(F, s, r)
        times = [F.fmm_server_wait(s, r["ticket"], 120.0) for r in reqs]
        st = F.fmm_server_stats(s)
    finally:
        F.fmm_server_destroy(s)
    assert st[0] == len(reqs) and st[2] == sum(len(r["q"]) for r in reqs)
    assert st[1] < len(reqs), "requests were not batched"
    assert st[5] >= 2
    assert max(t[3] for t in times) >= 2
    for k, r in enumerate(reqs):
        aphi, aF = _alone(F, r)
        assert oracle.rel_l2(r["phi"], aphi) <= TOL_ALONE, k
        assert oracle.rel_l2(r["F"], aF) <= TOL_ALONE, k
    for r in reqs[:3]:
        with oracle.OracleFMM(r["xyz"], r["q"], r["h"], r["p"], svd_eps=10.0 ** -r["p"]) as o:
            rphi, rF = o.evaluate()
        assert oracle.rel_l2(r["phi"], rphi) <= TOL_MIXED
        assert oracle.rel_l2(r["F"], rF) <= TOL_MIXED


def test_arrivals_during_work_overlap_on_lanes(F):
    """Requests submitted by several threads while earlier ones run are
    admitted by free lanes; two batches run at the same time."""
    reqs = _requests(24, 5000, nmin=20000, nmax=120000, orders=(5,))
    s = F.fmm_server_create(3, F.FMM_MIXED, 64 << 30, 150_000, 4)
    try:
        F.fmm_server_warmup(s, 5)

        def producer(part):
            for r in part:
                _submit(F, s, r)
        ths = [threading.Thread(target=producer, args=(reqs[k::4],)) for k in range(4)]
        for t in ths:
            t.start()
        for t in ths:
            t.join()
        for r in reqs:
            F.fmm_server_wait(s, r["ticket"], 300.0)
        st = F.fmm_server_stats(s)
    finally:
        F.fmm_server_destroy(s)
    assert st[0] == len(reqs)
    assert st[4] >= 2, "no two batches ran at once"
    assert st[12] == 0
    for k in (0, 5, 11, 23):
        aphi, aF = _alone(F, reqs[k])
        assert oracle.rel_l2(reqs[k]["phi"], aphi) <= TOL_ALONE, k
        assert oracle.rel_l2(reqs[k]["F"], aF) <= TOL_ALONE, k


def test_admission_respects_the_budget(F):
    reqs = _requests(10, 6000, nmin=5000, nmax=40000, orders=(4,))
    est = [F.fmm_server_request_bytes(len(r["q"]), r["h"], r["p"]) for r in reqs]
    budget = max(est) + min(est)
    s = F.fmm_server_create(4, F.FMM_MIXED, budget, 10_000_000, 64)
    try:
        big = dict(xyz=inputs.cube(400_000, 6999), q=np.ones(400_000), h=6, p=4)
        assert F.fmm_server_request_bytes(400_000, 6, 4) > budget
        with pytest.raises(F.FMMError) as e:
            _submit(F, s, big)
        assert e.value.status == F.FMM_ERR_OOM
        for r in reqs:
            _submit(F, s, r)
        for r in reqs:
            F.fmm_server_wait(s, r["ticket"], 300.0)
        st = F.fmm_server_stats(s)
    finally:
        F.fmm_server_destroy(s)
    assert st[0] == len(reqs)
    assert 0 < st[3] <= budget
    assert st[12] == 0, "an evaluation graph capture failed on a lane"
    aphi, aF = _alone(F, reqs[3])
    assert oracle.rel_l2(reqs[3]["phi"], aphi) <= TOL_ALONE


def test_device_buffers_and_errors(F):
    import torch
    r = _requests(1, 7000, nmin=3000, nmax=3001, orders=(5,))[0]
    n = len(r["q"])
    s = F.fmm_server_create(1, F.FMM_MIXED, 8 << 30, 100_000, 4)
    try:
        x, q = torch.from_numpy(r["xyz"]).cuda(), torch.from_numpy(r["q"]).cuda()
        phi = torch.zeros(n, dtype=torch.float64, device="cuda")
        Fo = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
        t = F.fmm_server_submit(s, n, r["h"], r["p"], x, q, phi, Fo)
        times = F.fmm_server_wait(s, t, 120.0)
        assert times[2] >= times[1] >= 0 and times[3] == 1
        with pytest.raises(F.FMMError):
            F.fmm_server_wait(s, t, 1.0)          # the ticket was released
        with pytest.raises(F.FMMError):
            F.fmm_server_submit(s, n, 0, 5, x, q, phi, Fo)
        bad = r["xyz"].copy()
        bad[0, 0] = np.inf
        rb = dict(xyz=bad, q=r["q"], h=r["h"], p=r["p"])
        _submit(F, s, rb)
        with pytest.raises(F.FMMError) as e:
            F.fmm_server_wait(s, rb["ticket"], 120.0)
        assert e.value.status == F.FMM_ERR_ARG
        # the lane recovers: the next request is served
        r2 = dict(r)
        _submit(F, s, r2)
        F.fmm_server_wait(s, r2["ticket"], 120.0)
    finally:
        F.fmm_server_destroy(s)
    aphi, aF = _alone(F, r)
    assert oracle.rel_l2(phi.cpu().numpy(), aphi) <= TOL_ALONE
    assert oracle.rel_l2(r2["phi"], aphi) <= TOL_ALONE


def test_lanes_create_handles_while_others_capture(F):
    """Four lanes with no warm-up: each creates its handles (and computes the
    compressed operators) on first use while other lanes capture and replay
    their evaluation graphs.  Handle creation is ordered on the handle's own
    stream, with no device-wide synchronisation and no legacy-stream copy, so
    no lane's graph capture fails (a failed capture would fall back to
    launch-by-launch evaluation and be counted in stats[12])."""
    reqs = _requests(32, 8000, nmin=3000, nmax=60000, orders=(3, 4, 5, 6))
    s = F.fmm_server_create(4, F.FMM_MIXED, 64 << 30, 120_000, 4)
    try:
        def producer(part):
            for r in part:
                _submit(F, s, r)
        ths = [threading.Thread(target=producer, args=(reqs[k::4],)) for k in range(4)]
        for t in ths:
            t.start()
        for t in ths:
            t.join()
        for r in reqs:
            F.fmm_server_wait(s, r["ticket"], 300.0)
        st = F.fmm_server_stats(s)
    finally:
        F.fmm_server_destroy(s)
    assert st[0] == len(reqs)
    assert st[12] == 0, "an evaluation graph capture failed while another lane created a handle"
    for k in (0, 9, 18, 31):
        aphi, aF = _alone(F, reqs[k])
        assert oracle.rel_l2(reqs[k]["phi"], aphi) <= TOL_ALONE, k
        assert oracle.rel_l2(reqs[k]["F"], aF) <= TOL_ALONE, k
