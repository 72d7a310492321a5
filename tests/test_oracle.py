"""Pins of the FP64 CPU oracle against what the paper and mathematics fix.

Each test names the property it pins and the paper passage it comes from.  None
of them re-types an oracle formula: they compare against closed forms, hand
values (tests/golden), textbook identities (Lagrange interpolation is unique),
library routines (numpy polynomials, numpy's stable sort), invariants
(Newton's third law, moment conservation, translation/permutation/scale
invariance) and brute force on tiny inputs.
"""
import itertools
from fractions import Fraction

import numpy as np
import pytest
from numpy.polynomial import Polynomial
from numpy.polynomial import chebyshev as npcheb

import oracle
from conftest import read_golden
from paper_1206_0115_b300 import inputs

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


# ---------------------------------------------------------------- Sec. 2.1.1

@pytest.mark.parametrize("p", range(2, 11))
def test_nodes_are_chebyshev_roots(p):
    """Sec. 2.1.1: interpolation points are the roots of T_p (numpy's Chebyshev
    series gives T_p independently), distinct, symmetric and in (-1, 1)."""
    x = oracle.cheb_nodes(p)
    coef = np.zeros(p + 1)
    coef[p] = 1.0
    assert np.abs(npcheb.chebval(x, coef)).max() < 1e-13
    assert np.all(np.diff(x) < 0)
    assert np.array_equal(x, -x[::-1])
    assert np.all(np.abs(x) < 1)


def test_nodes_closed_form():
    assert np.allclose(oracle.cheb_nodes(2), [np.sqrt(0.5), -np.sqrt(0.5)], rtol=0, atol=3e-16)
    assert np.allclose(oracle.cheb_nodes(3), [np.sqrt(3) / 2, 0.0, -np.sqrt(3) / 2], rtol=0, atol=3e-16)


def _lagrange(nodes, m):
    others = np.delete(nodes, m)
    return Polynomial.fromroots(others) / np.prod(nodes[m] - others)


@pytest.mark.parametrize("p", [2, 3, 4, 5, 7, 8, 10])
def test_S_is_the_lagrange_basis(p):
    """Eq. 5 defines S(xbar_m, .) as a polynomial of degree p-1; at the p
    Chebyshev roots the degree-(p-1) interpolant is unique, so S(xbar_m, .) must
    equal the textbook Lagrange basis polynomial of node m.  A dropped term, a
    wrong 1/p or 2/p factor or a wrong T_n would fail here.  The derivative is
    checked against the Lagrange polynomial's derivative."""
    x = oracle.cheb_nodes(p)
    xi = np.linspace(-1.0, 1.0, 37)
    for m in range(p):
        Lm = _lagrange(x, m)
        dLm = Lm.deriv()
        got = np.array([oracle.cheb_S(p, x[m], v) for v in xi])
        dgot = np.array([oracle.cheb_dS(p, x[m], v) for v in xi])
        assert np.abs(got - Lm(xi)).max() < 1e-12
        assert np.abs(dgot - dLm(xi)).max() < 1e-10 * max(1.0, np.abs(dLm(xi)).max())


@pytest.mark.parametrize("p", [3, 5, 7])
def test_S_kronecker_and_partition_of_unity(p):
    """Pin P1: S(xbar_m, xbar_k) = delta_mk and sum_m S(xbar_m, xi) = 1."""
    x = oracle.cheb_nodes(p)
    S = np.array([[oracle.cheb_S(p, x[m], x[k]) for k in range(p)] for m in range(p)])
    assert np.abs(S - np.eye(p)).max() < 1e-14
    for xi in np.linspace(-1, 1, 11):
        assert abs(sum(oracle.cheb_S(p, x[m], xi) for m in range(p)) - 1.0) < 1e-14


# ---------------------------------------------------------------- tree (Sec. 3.2, 4.2)

def test_morton_keys_golden():
    """Hand-interleaved keys (tests/golden/morton_keys.txt), root cube [0,1]^3."""
    for leaf, x, y, z, ix, iy, iz, key in read_golden("morton_keys.txt"):
        got = oracle.morton_keys(np.array([[float(x), float(y), float(z)]]), np.zeros(3), 1.0, int(leaf))
        assert int(got[0]) == int(key), (x, y, z)


def test_bounding_cube():
    xyz = np.array([[0.5, -1.0, 2.0], [1.5, 3.0, 2.25], [0.75, 0.0, 2.0]])
    lo, w = oracle.bounding_cube(xyz)
    assert lo.tolist() == [0.5, -1.0, 2.0] and w == 4.0
    lo, w = oracle.bounding_cube(np.array([[0.25, 0.5, 0.75]]))
    assert lo.tolist() == [0.25, 0.5, 0.75] and w == 1.0   # degenerate cube: side 1


def test_sort_is_stable_and_tree_consistent():
    """The Morton permutation is numpy's stable argsort of the oracle's keys
    (ties keep input order); leaves are the runs of equal keys; each level's
    keys are numpy.unique of the finer level's keys >> 3."""
    xyz, q = inputs.particles(3000, 11, "cube", "pos")
    xyz[100:140] = xyz[7]                                  # coincident points
    with oracle.OracleFMM(xyz, q, 4, 3) as o:
        lo, w = o.box()
        keys = oracle.morton_keys(xyz, lo, w, 3)
        perm = o.perm()
        assert np.array_equal(perm, np.argsort(keys, kind="stable"))
        lk = o.level_keys(3)
        first, count = o.level_ranges(3)
        assert np.array_equal(lk, np.unique(keys))
        assert count.sum() == len(xyz) and np.all(count > 0)
        assert np.array_equal(first, np.concatenate([[0], np.cumsum(count)[:-1]]))
        sk = keys[perm]
        for i in range(len(lk)):
            assert np.all(sk[first[i]:first[i] + count[i]] == lk[i])
        for lev in (2, 1, 0):
            fine = o.level_keys(lev + 1)
            assert np.array_equal(o.level_keys(lev), np.unique(fine >> np.uint64(3)))
            f, c = o.level_ranges(lev)
            assert c.sum() == len(fine)
            for i, k in enumerate(o.level_keys(lev)):
                assert np.all(fine[f[i]:f[i] + c[i]] >> np.uint64(3) == k)


# ---------------------------------------------------------------- direct sum (eq. 1, 2)

def _frac(s):
    return float(sum(Fraction(t) for t in s.split("+")))


def test_direct_golden_two_three_particles():
    rows = read_golden("two_three_particles.txt")
    for case in ("A", "B"):
        rs = [r for r in rows if r[0] == case]
        xyz = np.array([[float(v) for v in r[1:4]] for r in rs])
        q = np.array([float(r[4]) for r in rs])
        phi_ref = np.array([_frac(r[5]) for r in rs])
        F_ref = np.array([[_frac(v) for v in r[6:9]] for r in rs])
        phi, F = oracle.direct(xyz, q)
        assert np.abs(phi - phi_ref).max() < 1e-15
        assert np.abs(F - F_ref).max() < 1e-15


def test_direct_newton_third_law_and_scaling():
    """Pin P8: sum_i q_i F_i = 0 (F_ij = -F_ji); pin P9: x -> 2x gives phi/2 and
    F/4 (1/r is homogeneous of degree -1)."""
    xyz, q = inputs.particles(2000, 5, "cube", "sym")
    phi, F = oracle.direct(xyz, q)
    net = (q[:, None] * F).sum(axis=0)
    assert np.abs(net).max() < 1e-13 * np.abs(q[:, None] * F).sum()
    phi2, F2 = oracle.direct(2.0 * xyz, q)
    assert np.abs(phi2 - phi / 2).max() < 1e-13 * np.abs(phi).max()
    assert np.abs(F2 - F / 4).max() < 1e-13 * np.abs(F).max()
    idx = np.array([0, 17, 1999, 17])
    ps, Fs = oracle.direct_sampled(xyz, q, idx)
    assert np.array_equal(ps, phi[idx]) and np.array_equal(Fs, F[idx])


def test_direct_skips_coincident_pairs():
    xyz = np.array([[0.0, 0.0, 0.0], [0.0, 0.0, 0.0], [1.0, 0.0, 0.0]])
    q = np.array([1.0, 1.0, 1.0])
    phi, F = oracle.direct(xyz, q)
    assert phi.tolist() == [1.0, 1.0, 2.0]
    assert F[2].tolist() == [2.0, 0.0, 0.0]


# ---------------------------------------------------------------- FMM operators

def _centres(o, level):
    lo, w = o.box()
    keys = o.level_keys(level).astype(np.int64)
    ic = np.zeros((len(keys), 3), dtype=np.int64)
    for b in range(level):
        for d in range(3):
            ic[:, d] |= ((keys >> (3 * b + 2 - d)) & 1) << b
    wl = w / 2 ** level
    return lo[None, :] + (ic + 0.5) * wl, wl / 2


@pytest.mark.parametrize("p", [2, 3, 5])
def test_p2m_m2m_reproduce_moments(p):
    """Pins P2 and P3: interpolation at p nodes reproduces every polynomial of
    degree <= p-1 per axis exactly, so for such f the multipole expansion of
    every cell, whether made by P2M (leaf) or by M2M (coarser levels), obeys
    sum_m M_m f(c + a xbar_m) = sum_{j in cell} q_j f(y_j).  Monomials
    x^a y^b z^c with a, b, c < p are tested (charge: a=b=c=0; dipole: one 1)."""
    xyz, q = inputs.particles(4000, 21, "cube", "sym")
    h = 5
    with oracle.OracleFMM(xyz, q, h, p) as o:
        o.p2m()
        o.m2m()
        xbar = oracle.cheb_nodes(p)
        perm = o.perm()
        ys, qs = xyz[perm], q[perm]
        for level in range(2, h):
            ctr, a = _centres(o, level)
            M = o.expansion(level, "M")
            # particles per cell at this level: leaf ranges mapped through ancestors
            lf, lc = o.level_ranges(h - 1)
            lkeys = o.level_keys(h - 1) >> np.uint64(3 * (h - 1 - level))
            ckeys = o.level_keys(level)
            cell_of_leaf = np.searchsorted(ckeys, lkeys)
            rng = np.random.default_rng(level)
            for cell in rng.choice(len(ckeys), size=min(6, len(ckeys)), replace=False):
                sel = np.concatenate([np.arange(lf[i], lf[i] + lc[i]) for i in np.nonzero(cell_of_leaf == cell)[0]])
                nodes = ctr[cell][None, None, None, :] + a * np.stack(np.meshgrid(xbar, xbar, xbar, indexing="ij"), -1)
                nodes = nodes.reshape(-1, 3)
                for e in [(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1), (p - 1, p - 1, p - 1), (p - 1, 0, 1 % p)]:
                    f_nodes = np.prod((nodes - ctr[cell]) ** np.array(e), axis=1)
                    f_parts = np.prod((ys[sel] - ctr[cell]) ** np.array(e), axis=1)
                    lhs = (M[cell] * f_nodes).sum()
                    rhs = (qs[sel] * f_parts).sum()
                    scale = np.abs(M[cell] * f_nodes).sum() + np.abs(qs[sel] * f_parts).sum() + 1e-300
                    assert abs(lhs - rhs) < 1e-12 * scale, (level, cell, e)


@pytest.mark.parametrize("h", [1, 2])
def test_shallow_tree_is_direct_sum(h):
    """Pin P4: with h <= 2 no cell pair is well separated (no M2L at levels
    0, 1), so the FMM is the direct sum."""
    xyz, q = inputs.particles(1500, 9, "cube", "sym")
    pd, Fd = oracle.direct(xyz, q)
    with oracle.OracleFMM(xyz, q, h, 4) as o:
        phi, F = o.evaluate()
    assert np.abs(phi - pd).max() < 1e-12 * np.abs(pd).max()
    assert np.abs(F - Fd).max() < 1e-12 * np.abs(Fd).max()


@pytest.mark.parametrize("h,dist", [(3, "cube"), (4, "cube"), (4, "ellipsoid"), (5, "ellipsoid")])
def test_every_leaf_pair_covered_exactly_once(h, dist):
    """Pin P5 (Sec. 2.1.2, Sec. 3.3): each ordered pair of leaves is handled
    either by P2P (near field) or by exactly one M2L between ancestors."""
    xyz, q = inputs.particles(600 if h < 5 else 1500, 31, dist, "pos")
    with oracle.OracleFMM(xyz, q, h, 2) as o:
        cov = o.coverage()
    assert cov.shape[0] > 8
    assert np.all(cov == 1)


def test_interaction_list_sizes():
    """Sec. 2.1.2 / 3.3 counts (tests/golden/interaction_counts.txt): in a
    full tree an interior cell has 27 near leaves (itself included), 189 far
    cells, and the transfer vectors over all cells number 316."""
    g = {r[0]: int(r[1]) for r in read_golden("interaction_counts.txt")}
    n = 8                                                   # full tree, h = 4
    c = (np.arange(n) + 0.5) / n
    xyz = np.stack(np.meshgrid(c, c, c, indexing="ij"), -1).reshape(-1, 3)
    xyz = np.concatenate([xyz, [[0.0, 0.0, 0.0], [1.0, 1.0, 1.0]]])
    with oracle.OracleFMM(xyz, np.ones(len(xyz)), 4, 2) as o:
        assert o.level_size(3) == 512
        cov = o.coverage()
        keys = o.level_keys(3).astype(np.int64)
    # near-field count of an interior leaf = number of pairs covered by P2P:
    # coverage counts both, so count neighbours geometrically via the tree
    ic = np.zeros((512, 3), dtype=np.int64)
    for b in range(3):
        for d in range(3):
            ic[:, d] |= ((keys >> (3 * b + 2 - d)) & 1) << b
    interior = np.all((ic >= 2) & (ic <= 5), axis=1)
    cheb = np.abs(ic[:, None, :] - ic[None, :, :]).max(axis=2)
    assert np.all((cheb <= 1).sum(axis=1)[interior] == g["near_neighbours_with_self"])
    assert np.all(cov == 1)
    with oracle.OracleFMM(xyz, np.ones(len(xyz)), 4, 2) as o:
        pairs = o.m2l_pair_count(3)
    # interior cells at level 3 whose parents are interior see 189 far cells
    far_interior = (6 * 8 - 8) ** 3 - (3 * 8 - 2) ** 3
    assert pairs == far_interior
    tv = set()
    for i in range(512):
        for j in range(512):
            d = ic[j] - ic[i]
            if np.abs(d).max() >= 2 and np.all(np.abs((ic[j] >> 1) - (ic[i] >> 1)) <= 1):
                tv.add(tuple(d))
    assert len(tv) == g["transfer_vectors"]
    deep = np.all((ic >= 2) & (ic <= 5), axis=1)
    i = int(np.nonzero(deep)[0][0])
    nfar = sum(1 for j in range(512) if np.abs(ic[j] - ic[i]).max() >= 2
               and np.all(np.abs((ic[j] >> 1) - (ic[i] >> 1)) <= 1))
    assert nfar == g["far_field_max"]


def test_m2l_pair_counts_full_tree():
    """Pin P6: the M2L pair count per level of a full tree equals the closed
    form (6n-8)^3 - (3n-2)^3, n = 2^l, and the ratios between levels agree with
    the M2L work shares printed in Sec. 4.3 (work-breakdown figure) to the
    precision of those percentages."""
    rows = read_golden("m2l_work_shares.txt")
    n = 16                                                  # full tree, h = 5
    c = (np.arange(n) + 0.5) / n
    xyz = np.stack(np.meshgrid(c, c, c, indexing="ij"), -1).reshape(-1, 3)
    xyz = np.concatenate([xyz, [[0.0, 0.0, 0.0], [1.0, 1.0, 1.0]]])
    with oracle.OracleFMM(xyz, np.ones(len(xyz)), 5, 2) as o:
        for lev, pairs, _ in rows:
            if int(lev) <= 4:
                assert o.m2l_pair_count(int(lev)) == int(pairs)
    for (l0, p0, s0), (l1, p1, s1) in zip(rows[:-1], rows[1:]):
        closed = int(p1) / int(p0)
        paper = float(s1) / float(s0)
        assert abs(closed / paper - 1) < 0.05, (l0, l1, closed, paper)


@pytest.mark.parametrize("dist", ["cube", "ellipsoid"])
def test_fmm_converges_to_direct_sum(dist):
    """Pin P7 (Sec. 2.1.2, accuracy paragraph): the FMM error against the
    exact sum falls as p rises; for the potential it lies within 100x of the
    paper's 1e-5 / 1e-7 / 1e-9 at p = 3 / 5 / 7 (the paper's figures include
    its SVD step, so only the order of magnitude is comparable)."""
    xyz, q = inputs.particles(6000, 41, dist, "pos")
    pd, Fd = oracle.direct(xyz, q)
    ep, eF = [], []
    for p in range(2, 8):
        with oracle.OracleFMM(xyz, q, 4, p) as o:
            phi, F = o.evaluate()
        ep.append(oracle.rel_l2(phi, pd))
        eF.append(oracle.rel_l2(F, Fd))
    assert all(b < a for a, b in zip(ep, ep[1:])), ep
    assert all(b < a for a, b in zip(eF, eF[1:])), eF
    env = {3: 1e-5, 5: 1e-7, 7: 1e-9}
    for p, e in env.items():
        assert ep[p - 2] < 100 * e, (p, ep[p - 2])


def test_fmm_invariances():
    """Pin P9 and symmetry: scaling all positions by 2 gives phi/2 and F/4
    (homogeneity used by M2L, Sec. 2.1.2, and the 1/a of L2P); translating by
    a vector leaves results unchanged; swapping the x and y axes swaps F's
    components (catches an axis mix-up in any operator)."""
    xyz, q = inputs.particles(5000, 51, "cube", "sym")
    with oracle.OracleFMM(xyz, q, 4, 4) as o:
        phi, F = o.evaluate()
    with oracle.OracleFMM(2.0 * xyz, q, 4, 4) as o:
        phi2, F2 = o.evaluate()
    assert np.abs(phi2 - phi / 2).max() < 1e-12 * np.abs(phi).max()
    assert np.abs(F2 - F / 4).max() < 1e-12 * np.abs(F).max()
    with oracle.OracleFMM(xyz + np.array([0.25, -0.5, 1.0]), q, 4, 4) as o:
        phit, Ft = o.evaluate()
    assert np.abs(phit - phi).max() < 1e-11 * np.abs(phi).max()
    assert np.abs(Ft - F).max() < 1e-11 * np.abs(F).max()
    with oracle.OracleFMM(xyz[:, [1, 0, 2]], q, 4, 4) as o:
        phis, Fs = o.evaluate()
    assert np.abs(phis - phi).max() < 1e-11 * np.abs(phi).max()
    assert np.abs(Fs - F[:, [1, 0, 2]]).max() < 1e-11 * np.abs(F).max()


def test_fmm_net_force_at_fmm_error_level():
    """Pin P8 for the FMM: sum_i q_i F_i vanishes up to the FMM error."""
    xyz, q = inputs.particles(8000, 61, "cube", "pos")
    with oracle.OracleFMM(xyz, q, 4, 6) as o:
        phi, F = o.evaluate()
    pd, Fd = oracle.direct(xyz, q)
    err = oracle.rel_l2(F, Fd)
    net = np.abs((q[:, None] * F).sum(axis=0)).max()
    assert net < 10 * err * np.abs(q[:, None] * F).sum()


def test_sampled_evaluation_matches_full():
    xyz, q = inputs.particles(5000, 71, "ellipsoid", "pos")
    with oracle.OracleFMM(xyz, q, 5, 4) as o:
        phi, F = o.evaluate()
    idx = np.array([0, 3, 999, 4999, 2500, 3])
    with oracle.OracleFMM(xyz, q, 5, 4) as o:
        ps, Fs = o.evaluate_sampled(idx)
    assert np.abs(ps - phi[idx]).max() < 1e-13 * np.abs(phi).max()
    assert np.abs(Fs - F[idx]).max() < 1e-13 * np.abs(F).max()


def test_degenerate_inputs():
    with oracle.OracleFMM(np.zeros((0, 3)), np.zeros(0), 4, 3) as o:
        phi, F = o.evaluate()
        assert phi.shape == (0,)
    with oracle.OracleFMM(np.array([[0.3, 0.2, 0.1]]), np.array([2.0]), 4, 3) as o:
        phi, F = o.evaluate()
        assert phi.tolist() == [0.0] and F.tolist() == [[0.0, 0.0, 0.0]]
    xyz = np.tile([[0.5, 0.5, 0.5]], (10, 1))
    with oracle.OracleFMM(xyz, np.ones(10), 5, 3) as o:
        phi, F = o.evaluate()
        assert np.all(phi == 0.0) and np.all(F == 0.0)
    with pytest.raises(ValueError):
        oracle.OracleFMM(np.array([[np.nan, 0, 0]]), np.ones(1), 4, 3)
    with pytest.raises(ValueError):
        oracle.OracleFMM(np.zeros((1, 3)), np.ones(1), 0, 3)


# ---- SVD-compressed M2L (Sec. 2.1.2, "Improved M2L operator", Table 1) ----

def _far_vectors():
    return [t for t in itertools.product(range(-3, 4), repeat=3) if max(map(abs, t)) >= 2]


def _K_formula(t, p):
    """K_t[m][n] = 1/|2t + xbar_n - xbar_m| (unit half-width), from numpy's
    Chebyshev roots, for checks of the symmetry map only."""
    x = np.polynomial.chebyshev.chebpts1(p)[::-1]
    P = np.array(list(itertools.product(x, x, x)))
    d = 2.0 * np.asarray(t, dtype=float)[None, None, :] + P[None, :, :] - P[:, None, :]
    return 1.0 / np.linalg.norm(d, axis=2)


def test_jacobi_svd_matches_numpy():
    """The oracle's one-sided Jacobi SVD against LAPACK (numpy): singular
    values, reconstruction and orthogonality, on a full-rank matrix and on a
    numerically rank-10 one (the shape of the M2L operators' spectra)."""
    rng = np.random.default_rng(7)
    for A in (rng.standard_normal((40, 40)),
              rng.standard_normal((40, 10)) @ rng.standard_normal((10, 40))):
        U, s, V, sweeps = oracle.jacobi_svd(A)
        assert sweeps > 0
        ref = np.linalg.svd(A, compute_uv=False)
        assert np.abs(s - ref).max() <= 1e-13 * ref[0]
        assert np.all(np.diff(s) <= 0)
        assert np.abs(U @ np.diag(s) @ V.T - A).max() <= 1e-13 * ref[0]
        assert np.abs(V.T @ V - np.eye(40)).max() <= 1e-13
        k = int((s > 1e-10 * s[0]).sum())
        assert np.abs(U[:, :k].T @ U[:, :k] - np.eye(k)).max() <= 1e-12


def test_canonical_vectors_and_symmetry_orbits():
    """Sec. 2.1.2: the 316 transfer vectors are images of 16 under the cube's
    symmetries.  Each t is sign * that[axis] with that sorted, and the number
    of t per canonical vector equals its orbit size under the 48 symmetries
    (brute force)."""
    cv = oracle.canonical_vectors()
    assert len(cv) == 16 and len(set(cv)) == 16
    count = {}
    for t in _far_vectors():
        that, axis, sign = oracle.transfer_symmetry(t)
        assert list(that) == sorted(map(abs, t))
        assert sorted(axis) == [0, 1, 2]
        assert [sign[d] * that[axis[d]] for d in range(3)] == list(t)
        k = oracle.canonical_index(that)
        assert cv[k] == that
        count[k] = count.get(k, 0) + 1
    assert sum(count.values()) == 316
    for k, that in enumerate(cv):
        orbit = {tuple(s[d] * that[perm[d]] for d in range(3))
                 for perm in itertools.permutations(range(3))
                 for s in itertools.product((-1, 1), repeat=3)}
        assert count[k] == len(orbit)


@pytest.mark.parametrize("p", [3, 4])
def test_symmetry_maps_canonical_operators(p):
    """K_t[sigma.m][sigma.n] = K_that[m][n] for every far t: the node map
    of the symmetry is the one under which the operators coincide (a wrong
    axis, sign or direction of the map breaks it)."""
    for t in _far_vectors():
        that, axis, sign = oracle.transfer_symmetry(t)
        sm = oracle.node_permutation(p, axis, sign)
        assert sorted(sm) == list(range(p ** 3))
        Kt, Kc = _K_formula(t, p), _K_formula(that, p)
        assert np.abs(Kt[np.ix_(sm, sm)] - Kc).max() <= 1e-15 * Kc.max()


@pytest.mark.parametrize("p", [4, 5])
def test_compressed_operator_error_bound(p):
    """For every far t, the compressed operator differs from K_t by at most
    the first dropped singular value: |(K~_t - K_t) M| <= eps s_0 |M| (with
    eps = 10^-p, truncation at s_i >= eps s_0); the uncompressed operator is
    K_t itself."""
    eps = 10.0 ** -p
    xyz, q = inputs.particles(500, 3, "cube", "pos")
    rng = np.random.default_rng(p)
    full = oracle.OracleFMM(xyz, q, 3, p)
    comp = oracle.OracleFMM(xyz, q, 3, p, svd_eps=eps)
    try:
        for t in _far_vectors():
            M = rng.standard_normal(p ** 3)
            K = _K_formula(t, p)
            s0 = np.linalg.svd(K, compute_uv=False)[0]
            exact = K @ M
            assert np.abs(full.m2l_apply(t, M) - exact).max() <= 1e-13 * np.abs(exact).max()
            assert np.linalg.norm(comp.m2l_apply(t, M) - exact) <= 1.01 * eps * s0 * np.linalg.norm(M)
    finally:
        full.close()
        comp.close()


def test_svd_ranks_match_table1():
    """Table 1: the weighted rank of the 16 compressed operators (weights =
    how many of the 316 transfer vectors each one serves) with (l, eps) =
    (Acc, 10^-Acc) lies within 5% of the paper's 4.6 / 11.2 / 22.2, and the
    cost ratio 2 l^3 r16 / r316^2 formed with the paper's r316 within 0.05 of
    its last column."""
    xyz, q = inputs.particles(500, 3, "cube", "pos")
    weight = np.zeros(16)
    for t in _far_vectors():
        weight[oracle.canonical_index(oracle.transfer_symmetry(t)[0])] += 1
    for acc, r316, r16, ratio in (map(float, r) for r in read_golden("svd_ranks_table1.txt")):
        p = int(acc)
        with oracle.OracleFMM(xyz, q, 3, p, svd_eps=10.0 ** -p) as o:
            ranks = o.svd_ranks()
        # the ranks equal the count of LAPACK singular values above the threshold
        for k, that in enumerate(oracle.canonical_vectors()):
            s = np.linalg.svd(_K_formula(that, p), compute_uv=False)
            assert ranks[k] == int((s >= 10.0 ** -p * s[0]).sum())
        w = float((weight * ranks).sum() / 316)
        assert abs(w - r16) <= 0.05 * r16, (p, w)
        assert abs(2 * p ** 3 * w / r316 ** 2 - ratio) <= 0.05, (p, w)


@pytest.mark.parametrize("p", [3, 4, 5, 6, 7])
def test_svd_rank_decisions_have_margin(p):
    """No singular value of a canonical operator lies within 1e-6 (relative)
    of the threshold 10^-p s_0, so any accurate SVD (the oracle's Jacobi, the
    CUDA path's) truncates at the same rank."""
    eps = 10.0 ** -p
    for that in oracle.canonical_vectors():
        s = np.linalg.svd(_K_formula(that, p), compute_uv=False)
        assert np.abs(s / s[0] - eps).min() > 1e-6 * eps


def test_svd_fmm_close_to_full_rank_fmm():
    """The compressed M2L changes the FMM result by less than eps_SVD = 10^-p
    (relative L2, phi and F) and leaves its error against the direct sum
    within 10% of the full-rank FMM's."""
    xyz, q = inputs.particles(6000, 41, "cube", "pos")
    pd, Fd = oracle.direct(xyz, q)
    for p in (3, 4, 5, 6):
        with oracle.OracleFMM(xyz, q, 4, p) as o:
            pf, Ff = o.evaluate()
        with oracle.OracleFMM(xyz, q, 4, p, svd_eps=10.0 ** -p) as o:
            ps, Fs = o.evaluate()
        assert oracle.rel_l2(ps, pf) <= 10.0 ** -p and oracle.rel_l2(Fs, Ff) <= 10.0 ** -p
        assert oracle.rel_l2(ps, pd) <= 1.1 * oracle.rel_l2(pf, pd)
        assert oracle.rel_l2(Fs, Fd) <= 1.1 * oracle.rel_l2(Ff, Fd)


def test_svd_sampled_evaluation_matches_full():
    xyz, q = inputs.particles(4000, 52, "ellipsoid", "sym")
    idx = np.arange(0, 4000, 37)
    with oracle.OracleFMM(xyz, q, 5, 4, svd_eps=1e-4) as o:
        phi, F = o.evaluate()
    with oracle.OracleFMM(xyz, q, 5, 4, svd_eps=1e-4) as o:
        ps, Fs = o.evaluate_sampled(idx)
    assert np.abs(ps - phi[idx]).max() <= 1e-12 * np.abs(phi).max()
    assert np.abs(Fs - F[idx]).max() <= 1e-12 * np.abs(F).max()


def test_shared_svd_operators_give_the_same_result():
    """A tree that copies another tree's compressed operators evaluates
    exactly as one that computed its own."""
    xyz, q = inputs.particles(3000, 53, "cube", "sym")
    xyz2, q2 = inputs.particles(64, 1, "cube", "pos")
    with oracle.OracleFMM(xyz2, q2, 3, 4, svd_eps=1e-4) as src, oracle.OracleFMM(xyz, q, 4, 4, svd_eps=1e-4) as a, \
            oracle.OracleFMM(xyz, q, 4, 4, svd_from=src) as b:
        pa, Fa = a.evaluate()
        pb, Fb = b.evaluate()
        assert b.svd_ranks().tolist() == a.svd_ranks().tolist()
    assert np.array_equal(pa, pb) and np.array_equal(Fa, Fb)


# ---- the kernel family |x - y|^-s (fmm_set_kernel; the black-box method needs
# only kernel values).  s = 1 must reproduce the Laplace oracle above exactly;
# the other pins use the mathematics of the family, not its formula.

KERNELS = (0.5, 2.0, 3.0)


def test_kernel_exponent_one_is_the_laplace_oracle():
    xyz, q = inputs.particles(1500, 61, "cube", "sym")
    a = oracle.direct(xyz, q)
    b = oracle.direct(xyz, q, kernel_s=1.0)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    with oracle.OracleFMM(xyz, q, 4, 5) as o:
        ra = o.evaluate()
    with oracle.OracleFMM(xyz, q, 4, 5, kernel_s=1.0) as o:
        rb = o.evaluate()
    assert np.array_equal(ra[0], rb[0]) and np.array_equal(ra[1], rb[1])


@pytest.mark.parametrize("s", KERNELS)
def test_kernel_field_is_minus_gradient_of_potential(s):
    """F_i = -d phi_i / d x_i by central differences of the direct sum."""
    xyz, q = inputs.particles(60, 62, "cube", "sym")
    _, F = oracle.direct(xyz, q, kernel_s=s)
    h = 1e-6
    for i in (0, 17, 59):
        for d in range(3):
            xp, xm = xyz.copy(), xyz.copy()
            xp[i, d] += h
            xm[i, d] -= h
            dphi = (oracle.direct(xp, q, kernel_s=s)[0][i] - oracle.direct(xm, q, kernel_s=s)[0][i]) / (2 * h)
            assert abs(-dphi - F[i, d]) <= 1e-6 * max(1.0, np.abs(F[i]).max()), (i, d)


@pytest.mark.parametrize("s", KERNELS)
def test_kernel_homogeneity_and_newton(s):
    """x -> 2x scales phi by 2^-s and F by 2^-(s+1); sum_i q_i F_i = 0 for
    any radial kernel (pairs cancel)."""
    xyz, q = inputs.particles(800, 63, "cube", "sym")
    p1, F1 = oracle.direct(xyz, q, kernel_s=s)
    p2, F2 = oracle.direct(2.0 * xyz, q, kernel_s=s)
    assert oracle.rel_l2(p2, p1 * 2.0 ** -s) <= 1e-13
    assert oracle.rel_l2(F2, F1 * 2.0 ** -(s + 1)) <= 1e-13
    net = (q[:, None] * F1).sum(axis=0)
    assert np.abs(net).max() <= 1e-12 * np.abs(q[:, None] * F1).sum()
    with oracle.OracleFMM(xyz, q, 4, 5, kernel_s=s) as o:
        pa, Fa = o.evaluate()
    with oracle.OracleFMM(2.0 * xyz, q, 4, 5, kernel_s=s) as o:
        pb, Fb = o.evaluate()
    assert oracle.rel_l2(pb, pa * 2.0 ** -s) <= 1e-12
    assert oracle.rel_l2(Fb, Fa * 2.0 ** -(s + 1)) <= 1e-12


@pytest.mark.parametrize("s", KERNELS)
def test_kernel_fmm_converges_to_the_direct_sum(s):
    """The FMM error against the direct sum falls as p rises, trees of height
    <= 2 are the direct sum, and the compressed operators stay within their
    eps of the full-rank ones."""
    xyz, q = inputs.particles(3000, 64, "cube", "pos")
    pd, Fd = oracle.direct(xyz, q, kernel_s=s)
    errs = []
    for p in (3, 5, 7):
        with oracle.OracleFMM(xyz, q, 4, p, kernel_s=s) as o:
            pf, Ff = o.evaluate()
        errs.append(max(oracle.rel_l2(pf, pd), oracle.rel_l2(Ff, Fd)))
        with oracle.OracleFMM(xyz, q, 4, p, kernel_s=s, svd_eps=10.0 ** -p) as o:
            ps, Fs = o.evaluate()
        assert oracle.rel_l2(ps, pf) <= 10.0 ** -p and oracle.rel_l2(Fs, Ff) <= 10.0 ** (1 - p)
    assert errs[0] > 5 * errs[1] > 25 * errs[2], errs
    assert errs[2] <= 1e-4
    with oracle.OracleFMM(xyz, q, 2, 4, kernel_s=s) as o:
        p2, F2 = o.evaluate()
    assert oracle.rel_l2(p2, pd) <= 1e-14 and oracle.rel_l2(F2, Fd) <= 1e-14


def test_kernel_arguments_out_of_range_rejected():
    xyz, q = inputs.particles(10, 65, "cube", "pos")
    for bad in (0.0, -2.5, 4.5, float("nan")):
        with pytest.raises(ValueError):
            oracle.OracleFMM(xyz, q, 3, 3, kernel_s=bad)
    for bad in (-1.0, float("inf"), float("nan")):
        with pytest.raises(ValueError):
            oracle.OracleFMM(xyz, q, 3, 3, kernel_s=1.0, kernel_c=bad)
    # the compression needs one operator set for all levels (c = 0)
    with pytest.raises(ValueError):
        oracle.OracleFMM(xyz, q, 3, 3, kernel_s=1.0, kernel_c=0.1, svd_eps=1e-3)


# ---- multiquadrics: (|x - y|^2 + c^2)^(-s/2), c > 0 (not homogeneous: one
# operator set per level).  s = -1 multiquadric, s = 1 inverse multiquadric.

MQ = ((1.0, 0.05), (-1.0, 0.05), (2.0, 0.02))


def _quadratic_closed_form(xyz, q, c):
    """s = -2: P = |x - y|^2 + c^2, so with Q = sum q, S = sum q x, T = sum q |x|^2
    (self pair excluded): phi_i = Q |x_i|^2 - 2 x_i . S + T + c^2 (Q - q_i),
    F_i = -grad phi_i = 2 S - 2 Q x_i."""
    Q = q.sum()
    S = (q[:, None] * xyz).sum(axis=0)
    T = (q * (xyz ** 2).sum(axis=1)).sum()
    phi = Q * (xyz ** 2).sum(axis=1) - 2.0 * xyz @ S + T + c * c * (Q - q)
    return phi, 2.0 * S[None, :] - 2.0 * Q * xyz


@pytest.mark.parametrize("c", [0.0, 0.3])
def test_quadratic_kernel_is_reproduced_exactly(c):
    """Chebyshev interpolation of order p >= 3 reproduces quadratics, so the
    FMM of |x - y|^2 + c^2 equals the closed form to rounding at every height
    (per-level operators for c > 0, the scaled unit set for c = 0); a wrong
    level, scale or sign anywhere in the far field breaks this."""
    xyz, q = inputs.particles(2500, 66, "ellipsoid", "sym")
    pc, Fc = _quadratic_closed_form(xyz, q, c)
    pd, Fd = oracle.direct(xyz, q, kernel_s=-2.0, kernel_c=c)
    assert oracle.rel_l2(pd, pc) <= 1e-13 and oracle.rel_l2(Fd, Fc) <= 1e-13
    for h, p in ((4, 3), (5, 4)):
        with oracle.OracleFMM(xyz, q, h, p, kernel_s=-2.0, kernel_c=c) as o:
            pf, Ff = o.evaluate()
        assert oracle.rel_l2(pf, pc) <= 1e-12, (h, p)
        assert oracle.rel_l2(Ff, Fc) <= 1e-12, (h, p)


@pytest.mark.parametrize("s,c", MQ)
def test_multiquadric_field_is_minus_gradient(s, c):
    xyz, q = inputs.particles(60, 67, "cube", "sym")
    _, F = oracle.direct(xyz, q, kernel_s=s, kernel_c=c)
    h = 1e-6
    for i in (0, 31, 59):
        for d in range(3):
            xp, xm = xyz.copy(), xyz.copy()
            xp[i, d] += h
            xm[i, d] -= h
            dphi = (oracle.direct(xp, q, kernel_s=s, kernel_c=c)[0][i]
                    - oracle.direct(xm, q, kernel_s=s, kernel_c=c)[0][i]) / (2 * h)
            assert abs(-dphi - F[i, d]) <= 1e-6 * max(1.0, np.abs(F[i]).max()), (i, d)


@pytest.mark.parametrize("s,c", MQ)
def test_multiquadric_joint_scaling_and_newton(s, c):
    """x -> 2x together with c -> 2c scales phi by 2^-s and F by 2^-(s+1)
    (direct sum and FMM: the tree is the same, every level's operators are
    rebuilt at the new widths); sum_i q_i F_i = 0."""
    xyz, q = inputs.particles(800, 68, "cube", "sym")
    p1, F1 = oracle.direct(xyz, q, kernel_s=s, kernel_c=c)
    p2, F2 = oracle.direct(2.0 * xyz, q, kernel_s=s, kernel_c=2.0 * c)
    assert oracle.rel_l2(p2, p1 * 2.0 ** -s) <= 1e-13
    assert oracle.rel_l2(F2, F1 * 2.0 ** -(s + 1)) <= 1e-13
    net = (q[:, None] * F1).sum(axis=0)
    assert np.abs(net).max() <= 1e-12 * np.abs(q[:, None] * F1).sum()
    with oracle.OracleFMM(xyz, q, 4, 5, kernel_s=s, kernel_c=c) as o:
        pa, Fa = o.evaluate()
    with oracle.OracleFMM(2.0 * xyz, q, 4, 5, kernel_s=s, kernel_c=2.0 * c) as o:
        pb, Fb = o.evaluate()
    assert oracle.rel_l2(pb, pa * 2.0 ** -s) <= 1e-12
    assert oracle.rel_l2(Fb, Fa * 2.0 ** -(s + 1)) <= 1e-12


@pytest.mark.parametrize("s,c", MQ)
def test_multiquadric_fmm_converges_to_the_direct_sum(s, c):
    xyz, q = inputs.particles(3000, 69, "cube", "pos")
    pd, Fd = oracle.direct(xyz, q, kernel_s=s, kernel_c=c)
    errs = []
    for p in (3, 5, 7):
        with oracle.OracleFMM(xyz, q, 4, p, kernel_s=s, kernel_c=c) as o:
            pf, Ff = o.evaluate()
        errs.append(max(oracle.rel_l2(pf, pd), oracle.rel_l2(Ff, Fd)))
    assert errs[0] > 5 * errs[1] > 25 * errs[2], errs
    assert errs[2] <= 1e-4
    with oracle.OracleFMM(xyz, q, 2, 4, kernel_s=s, kernel_c=c) as o:
        p2, F2 = o.evaluate()
    assert oracle.rel_l2(p2, pd) <= 1e-14 and oracle.rel_l2(F2, Fd) <= 1e-14


# ---- the Stokes kernel (Stokeslet, unit viscosity factor):
# u_i = sum_k [f_k / r + d (d . f_k) / r^3], d = x_i - x_k.

def _forces(n, seed):
    return np.stack([inputs.charges(n, seed + k, "sym", 0) for k in range(3)], axis=1)


def test_stokeslet_hand_values():
    # x1 = 0, x2 = (1, 0, 0), f1 = 0, f2 = (1, 2, 3): d = (-1, 0, 0), r = 1,
    # u1 = f2 + d (d . f2) = (1, 2, 3) + (-1, 0, 0)(-1) = (2, 2, 3); u2 = 0
    u = oracle.stokes_direct(np.array([[0.0, 0, 0], [1.0, 0, 0]]), np.array([[0.0, 0, 0], [1.0, 2, 3]]))
    assert np.array_equal(u, np.array([[2.0, 2, 3], [0, 0, 0]]))
    # x2 = (0, 2, 0), f1 = (-1, 0, 2), f2 = (1, 1, 1): r = 2;
    # u1 = f2 / 2 + (0, -2, 0)(-2) / 8 = (0.5, 1.0, 0.5); u2 = f1 / 2 (d . f1 = 0)
    u = oracle.stokes_direct(np.array([[0.0, 0, 0], [0.0, 2, 0]]), np.array([[-1.0, 0, 2], [1.0, 1, 1]]))
    assert np.allclose(u, np.array([[0.5, 1.0, 0.5], [-0.5, 0.0, 1.0]]), rtol=0, atol=1e-15)


def test_stokeslet_field_is_divergence_free_and_reciprocal():
    """Away from the sources the Stokeslet field has zero divergence (probe:
    a particle with zero force, moved by central differences); the kernel is
    symmetric and even, so <f, U g> = <g, U f>."""
    xyz, _ = inputs.particles(50, 94, "cube", "pos")
    f = _forces(50, 95)
    probe = np.array([0.37, 0.52, 0.61])
    h = 1e-4
    div, scale = 0.0, 0.0
    for d in range(3):
        vals = []
        for sgn in (1.0, -1.0):
            x = np.vstack([xyz, probe + sgn * h * np.eye(3)[d]])
            ff = np.vstack([f, np.zeros((1, 3))])
            vals.append(oracle.stokes_direct(x, ff)[-1])
        g = (vals[0] - vals[1]) / (2 * h)
        div += g[d]
        scale += np.abs(g).sum()
    assert abs(div) <= 1e-6 * scale
    g2 = _forces(50, 98)
    a = (f * oracle.stokes_direct(xyz, g2)).sum()
    b = (g2 * oracle.stokes_direct(xyz, f)).sum()
    assert abs(a - b) <= 1e-13 * abs(a)


def test_stokes_from_four_laplace_passes():
    """Trees of height <= 2 make every 1/r pass a direct sum, so the identity
    u_i = phi^i + sum_j x_j F^j_i - F^3_i must give the Stokeslet sum to
    rounding, for any origin (points shifted far from it too); with a far
    field the error falls with the order."""
    xyz, _ = inputs.particles(1500, 96, "cube", "sym")
    f = _forces(1500, 97)
    ud = oracle.stokes_direct(xyz, f)
    for h in (1, 2):
        assert oracle.rel_l2(oracle.stokes_fmm(xyz, f, h, 4), ud) <= 1e-13
    shifted = xyz + np.array([5.0, -3.0, 2.0])
    assert oracle.rel_l2(oracle.stokes_direct(shifted, f), ud) <= 1e-13
    assert oracle.rel_l2(oracle.stokes_fmm(shifted, f, 2, 4), ud) <= 1e-12
    errs = [oracle.rel_l2(oracle.stokes_fmm(xyz, f, 4, p), ud) for p in (3, 5, 7)]
    assert errs[0] > 5 * errs[1] > 25 * errs[2], errs
    assert errs[2] <= 3e-5
