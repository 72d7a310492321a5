"""Batched problems (fmm_set_batch): many independent problems in one tree,
each stage one launch for the whole batch.

A batch is, by definition, the independent problems it holds: the oracle is
the FP64 CPU oracle run on each problem alone (same height and order).  Bars,
per problem:
  * tree (root cube, Morton permutation, cell keys and particle / child
    ranges at every level of the problem's own tree): bit-exact;
  * FP64 path: relative L2 error against the oracle's FMM <= 1e-10;
  * mixed path: relative L2 error against the oracle's FMM <= 1e-5, and
    against the same problem solved alone on the GPU <= 1e-6 (the batch changes
    nothing but the grouping of the tensor-core partial sums).
"""
import numpy as np
import pytest

import oracle
from paper_1206_0115_b300 import inputs

pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-10
TOL_MIXED = 1e-5
TOL_ALONE = 1e-6


@pytest.fixture(scope="module")
def F():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1206_0115_b300 import build
    build.build()
    from paper_1206_0115_b300 import fmm
    return fmm


def _mixed_batch():
    """Uneven sizes, both distributions, heights 1..5, an empty problem, a
    single particle and a cluster of coincident points."""
    probs = []
    specs = [(3000, "cube", 4), (17000, "ellipsoid", 5), (0, "cube", 3), (1, "cube", 3), (900, "ellipsoid", 3),
             (5000, "cube", 2), (40, "cube", 1), (12000, "cube", 4), (2500, "ellipsoid", 4)]
    for k, (n, dist, h) in enumerate(specs):
        xyz, q = inputs.particles(n, 500 + k, dist, "pos" if k % 2 else "sym")
        probs.append((xyz, q, h))
    # coincident points and a point on the cube's upper faces
    xyz = np.repeat(np.array([[0.25, 0.5, 0.75]]), 6, axis=0)
    xyz = np.vstack([xyz, inputs.cube(60, 77), [[1.0, 1.0, 1.0]]])
    probs.append((np.ascontiguousarray(xyz), inputs.charges(len(xyz), 78, "pos", 0), 3))
    return probs


def _concat(probs):
    counts = np.array([len(q) for _, q, _ in probs], dtype=np.int64)
    heights = np.array([h for _, _, h in probs], dtype=np.int32)
    xyz = np.ascontiguousarray(np.concatenate([x.reshape(-1, 3) for x, _, _ in probs]))
    q = np.ascontiguousarray(np.concatenate([q for _, q, _ in probs]))
    return counts, heights, xyz, q


def _run_batch(F, probs, p, precision, host=False):
    import torch
    counts, heights, xyz, q = _concat(probs)
    n = len(q)
    with F.FMM(3, p, precision) as f:
        if host:
            f.set_batch(counts, heights, xyz, q)
            phi = np.zeros(n)
            Fo = np.zeros((n, 3))
            f.evaluate(phi, Fo)
        else:
            f.set_batch(counts, heights, torch.from_numpy(xyz).cuda(), torch.from_numpy(q).cuda())
            phi_t = torch.zeros(n, dtype=torch.float64, device="cuda")
            F_t = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
            f.evaluate(phi_t, F_t)
            torch.cuda.synchronize()
            phi, Fo = phi_t.cpu().numpy(), F_t.cpu().numpy()
        infos = [f.batch_info(k) for k in range(len(probs))]
    return phi, Fo, infos


def _split(a, counts):
    return np.split(a, np.cumsum(counts)[:-1])


def _run_alone(F, xyz, q, h, p, precision):
    import torch
    n = len(q)
    with F.FMM(h, p, precision) as f:
        f.set_particles(torch.from_numpy(xyz).cuda(), torch.from_numpy(q).cuda())
        phi = torch.zeros(n, dtype=torch.float64, device="cuda")
        Fo = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
        f.evaluate(phi, Fo)
        torch.cuda.synchronize()
        return phi.cpu().numpy(), Fo.cpu().numpy()


def test_batch_tree_bit_exact(F):
    """Every problem's tree inside the batch equals the oracle's tree of the
    problem alone, shifted by the problem's slot."""
    import torch
    probs = _mixed_batch()
    counts, heights, xyz, q = _concat(probs)
    n = len(q)
    with F.FMM(3, 3, F.FMM_FP64) as f:
        f.set_batch(counts, heights, torch.from_numpy(xyz).cuda(), torch.from_numpy(q).cuda())
        perm = torch.zeros(n, dtype=torch.int64, device="cuda")
        F.fmm_get_order(f.h, perm)
        perm = perm.cpu().numpy()
        Lf = int(f.batch_info(0)[0][4])
        lev = {}
        for l in range(Lf + 1):
            nc = F.fmm_get_level_size(f.h, l)
            keys = np.zeros(nc, dtype=np.uint64)
            first = np.zeros(nc, dtype=np.int64)
            count = np.zeros(nc, dtype=np.int64)
            if nc:
                F.fmm_get_level_keys(f.h, l, keys)
                F.fmm_get_level_ranges(f.h, l, first, count)
            lev[l] = (keys.astype(np.int64), first, count)
        assert np.array_equal(f.box(), [0.0, 0.0, 0.0, 1.0])
        seen = np.zeros(n, dtype=bool)
        for k, (px, pq, h) in enumerate(probs):
            info, box = f.batch_info(k)
            r0, cnt, S, slot, _, hk, i0 = (int(v) for v in info[:7])
            assert cnt == len(pq) and hk == h and i0 == int(np.sum(counts[:k]))
            if cnt == 0:
                assert S == -1
                continue
            L = h - 1
            assert S == Lf - L and slot % (8 ** L) == 0
            with oracle.OracleFMM(px, pq, h, 3) as o:
                olo, ow = o.box()
                assert np.array_equal(box[:3], olo) and box[3] == ow, k
                seg = perm[r0:r0 + cnt]
                assert np.array_equal(seg - i0, o.perm()), k
                seen[seg] = True
                for j in range(h):
                    keys, first, count = lev[S + j]
                    base = slot >> (3 * (L - j))
                    sel = (keys >= base) & (keys < base + 8 ** j)
                    assert np.array_equal(keys[sel] - base, o.level_keys(j).astype(np.int64)), (k, j)
                    ofirst, ocount = o.level_ranges(j)
                    assert np.array_equal(count[sel], ocount), (k, j)
                    if j == L:
                        assert np.array_equal(first[sel] - r0, ofirst), (k, j)
                    else:
                        below = lev[S + j + 1][0]
                        bsel = (below >= (slot >> (3 * (L - j - 1)))) & (below < (slot >> (3 * (L - j - 1))) + 8 ** (j + 1))
                        c0 = int(np.argmax(bsel)) if bsel.any() else 0
                        assert np.array_equal(first[sel] - c0, ofirst), (k, j)
        assert seen.sum() == n


@pytest.mark.parametrize("precision,tol", [(1, TOL_MIXED), (0, TOL_FP64)])
def test_batch_matches_oracle_per_problem(F, precision, tol):
    p = 5
    probs = _mixed_batch()
    counts = [len(q) for _, q, _ in probs]
    phi, Fo, _ = _run_batch(F, probs, p, precision)
    for k, ((px, pq, h), bphi, bF) in enumerate(zip(probs, _split(phi, counts), _split(Fo, counts))):
        if len(pq) == 0:
            continue
        # (trees below height 3 have no M2L, hence no compressed operators)
        with oracle.OracleFMM(px, pq, h, p, svd_eps=10.0 ** -p if h >= 3 else None) as o:
            rphi, rF = o.evaluate()
        if len(pq) == 1:
            assert np.all(bphi == 0.0) and np.all(bF == 0.0)
            continue
        assert oracle.rel_l2(bphi, rphi) <= tol, (k, oracle.rel_l2(bphi, rphi))
        assert oracle.rel_l2(bF, rF) <= tol, (k, oracle.rel_l2(bF, rF))


def test_batch_equals_problems_solved_alone(F):
    p = 5
    probs = _mixed_batch()
    counts = [len(q) for _, q, _ in probs]
    phi, Fo, _ = _run_batch(F, probs, p, 1)
    for k, ((px, pq, h), bphi, bF) in enumerate(zip(probs, _split(phi, counts), _split(Fo, counts))):
        if len(pq) < 2:
            continue
        aphi, aF = _run_alone(F, px, pq, h, p, 1)
        assert oracle.rel_l2(bphi, aphi) <= TOL_ALONE, (k, oracle.rel_l2(bphi, aphi))
        assert oracle.rel_l2(bF, aF) <= TOL_ALONE, (k, oracle.rel_l2(bF, aF))


def test_batch_host_pointers_and_reload(F):
    """Host inputs give the device inputs' results; a handle that held a batch
    solves a single problem like a fresh one."""
    import torch
    p = 4
    probs = _mixed_batch()[:5]
    dphi, dF, _ = _run_batch(F, probs, p, 1)
    hphi, hF, _ = _run_batch(F, probs, p, 1, host=True)
    assert np.array_equal(dphi, hphi) and np.array_equal(dF, hF)
    counts, heights, xyz, q = _concat(probs)
    px, pq, h = probs[1]
    with F.FMM(h, p, 1) as f:
        f.set_batch(counts, heights, xyz, q)
        f.set_particles(torch.from_numpy(px).cuda(), torch.from_numpy(pq).cuda())
        phi = torch.zeros(len(pq), dtype=torch.float64, device="cuda")
        Fo = torch.zeros((len(pq), 3), dtype=torch.float64, device="cuda")
        f.evaluate(phi, Fo)
        torch.cuda.synchronize()
        aphi, aF = _run_alone(F, px, pq, h, p, 1)
        assert np.array_equal(phi.cpu().numpy(), aphi) and np.array_equal(Fo.cpu().numpy(), aF)


def test_batch_rejects_bad_input(F):
    with F.FMM(3, 3, 1) as f:
        x = np.zeros((2, 3))
        q = np.ones(2)
        with pytest.raises(F.FMMError):
            f.set_batch([2], [0], x, q)          # height out of range
        with pytest.raises(F.FMMError):          # negative count
            f.set_batch([-1], [3], x, q)
        with pytest.raises(F.FMMError):          # 2 x 8^9 leaf cells do not fit in 8^9
            f.set_batch([1, 1], [10, 10], x, q)
        bad = x.copy()
        bad[1, 2] = np.nan
        with pytest.raises(F.FMMError):
            f.set_batch([1, 1], [3, 3], bad, q)
        with pytest.raises(F.FMMError):
            F.fmm_get_batch_info(f.h, 5)


@pytest.mark.slow
def test_batched_workload_sampled(F):
    """The 256-problem batched workload (sizes 1e3 .. 2e5, heights 3..6, p = 5,
    mixed) at full size: sampled problems against the oracle, every problem
    against the zero net force of its own direct sum's symmetry."""
    import torch
    counts, heights, xyz, q = inputs.batch_workload()
    n = len(q)
    p = 5
    with F.FMM(3, p, 1) as f:
        f.set_batch(counts, heights, torch.from_numpy(xyz).cuda(), torch.from_numpy(q).cuda())
        phi = torch.zeros(n, dtype=torch.float64, device="cuda")
        Fo = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
        f.evaluate(phi, Fo)
        torch.cuda.synchronize()
        phi, Fo = phi.cpu().numpy(), Fo.cpu().numpy()
    starts = np.concatenate([[0], np.cumsum(counts)])
    for k in (0, 7, 100, int(np.argmax(counts)), int(np.argmin(counts))):
        a, b = starts[k], starts[k + 1]
        with oracle.OracleFMM(xyz[a:b], q[a:b], int(heights[k]), p, svd_eps=10.0 ** -p) as o:
            rphi, rF = o.evaluate()
        assert oracle.rel_l2(phi[a:b], rphi) <= TOL_MIXED, k
        assert oracle.rel_l2(Fo[a:b], rF) <= TOL_MIXED, k


def test_p2p_variants_agree_and_autotune_picks_one(F):
    """Every shape of the mixed P2P kernel gives the same result up to the
    grouping of FP32 partial sums; the autotuner times each occupancy bin
    (leaves of at most 64 particles, larger leaves) in every shape and keeps
    each bin's fastest, and the binned evaluation agrees with the others."""
    import torch
    probs = _mixed_batch()
    counts, heights, xyz, q = _concat(probs)
    n = len(q)
    out = {}
    with F.FMM(3, 5, F.FMM_MIXED) as f:
        f.set_batch(counts, heights, torch.from_numpy(xyz).cuda(), torch.from_numpy(q).cuda())
        phi = torch.zeros(n, dtype=torch.float64, device="cuda")
        Fo = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
        for v in range(F.FMM_P2P_VARIANTS):
            F.fmm_set_p2p_variant(f.h, v)
            f.evaluate(phi, Fo)
            torch.cuda.synchronize()
            out[v] = (phi.cpu().numpy().copy(), Fo.cpu().numpy().copy())
        choice, times = F.fmm_autotune(f.h)
        assert 0 <= choice[0] < F.FMM_P2P_VARIANTS and np.all(times > 0)
        bins, bin_ms = F.fmm_get_p2p_bins(f.h)
        assert bins[2] > 0 and bins[3] > 0, "the batch has small and large leaves"
        sched, sched_ms = F.fmm_get_schedule(f.h)
        assert sched in (0, 1, 2, 3) and sched_ms[0] > 0 and sched_ms[1] > 0
        pick = int(np.argmin(np.where(sched_ms > 0, sched_ms, np.inf)))
        assert sched == pick % 4
        best = []
        for b in range(2):
            timed = bin_ms[b][bin_ms[b] >= 0]
            assert len(timed) == (F.FMM_P2P_VARIANTS - 2 if b == 0 else F.FMM_P2P_VARIANTS)
            ms = np.where(bin_ms[b] >= 0, bin_ms[b], np.inf)
            if pick >= 4:  # the schedule stage kept the fastest non-persistent shapes
                ms[[14, 15]] = np.inf
            best.append(int(np.argmin(ms)))
        # either each bin's fastest shape, or one item shape for both bins
        assert (int(bins[0]), int(bins[1])) == tuple(best) or (int(bins[0]) == int(bins[1]) and int(bins[0]) not in (12, 13))
        assert int(choice[0]) == int(bins[0])
        f.evaluate(phi, Fo)
        torch.cuda.synchronize()
        binned = (phi.cpu().numpy().copy(), Fo.cpu().numpy().copy())
        with pytest.raises(F.FMMError):
            F.fmm_set_p2p_variant(f.h, F.FMM_P2P_VARIANTS)
    for v in range(1, F.FMM_P2P_VARIANTS):
        assert oracle.rel_l2(out[v][0], out[0][0]) <= TOL_ALONE, v
        assert oracle.rel_l2(out[v][1], out[0][1]) <= TOL_ALONE, v
    assert oracle.rel_l2(binned[0], out[0][0]) <= TOL_ALONE
    assert oracle.rel_l2(binned[1], out[0][1]) <= TOL_ALONE


def test_batch_problems_of_very_different_magnitude(F):
    """Two problems whose charges differ by a factor of 1e8 in one batch: each
    matches its own oracle within the mixed bar.  The M2L's FP16 operands are
    scaled per multipole row and per (problem, level), never by a scale that
    one problem's magnitude sets for another; the handle reports the FP16
    form."""
    a = inputs.particles(8000, 801, "cube", "sym")
    b = inputs.particles(12000, 802, "ellipsoid", "pos")
    probs = [(a[0], a[1], 4), (b[0], 1e-8 * b[1], 5)]
    phi, Fo, _ = _run_batch(F, probs, 5, F.FMM_MIXED)
    with F.FMM(3, 5, F.FMM_MIXED) as f:
        import torch
        counts, heights, xyz, q = _concat(probs)
        f.set_batch(counts, heights, torch.from_numpy(xyz).cuda(), torch.from_numpy(q).cuda())
        assert int(f.stats()[5]) == 1
    off = 0
    for x, q, h in probs:
        sl = slice(off, off + len(q))
        off += len(q)
        with oracle.OracleFMM(x, q, h, 5, svd_eps=1e-5) as o:
            rphi, rF = o.evaluate()
        assert oracle.rel_l2(phi[sl], rphi) <= TOL_MIXED
        assert oracle.rel_l2(Fo[sl], rF) <= TOL_MIXED
