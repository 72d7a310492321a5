"""Seeded synthetic particle sets shared by the CUDA path's tests, the oracle's
tests and the benchmark.

This module only draws numbers; it holds none of the FMM arithmetic. Both the
oracle and the CUDA library receive the arrays it returns as plain inputs.

Generator: SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014), the 64-bit mixing function with the golden
gamma 0x9E3779B97F4A7C15.  Draw k (k = 0, 1, ...) of a stream with seed s is
mix(s + (k + 1) * gamma mod 2^64); a double in [0, 1) is its top 53 bits
times 2^-53.

Workloads follow the paper's synthetic distributions (Sec. 5.4, the flop-rate
study): points uniform in the unit cube, or on a closed surface (the paper
uses the unit sphere; the workloads here use an ellipsoid with semi-axes
0.5, 0.25, 0.125, a flattened version of it that makes leaf occupancy
uneven).  Charges are uniform in (0, 1] or in [-1, 1).
"""
from __future__ import annotations

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Draws offset .. offset+count-1 of the SplitMix64 stream `seed` (uint64)."""
    k = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + k * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Doubles in [0, 1) from the top 53 bits of each SplitMix64 draw."""
    z = splitmix64(seed, count, offset)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def cube(n: int, seed: int) -> np.ndarray:
    """n points uniform in the unit cube, [n][3] float64 (draws 0 .. 3n-1)."""
    return uniform01(seed, 3 * n).reshape(n, 3).copy()


def ellipsoid_surface(n: int, seed: int, axes=(0.5, 0.25, 0.125)) -> np.ndarray:
    """n points on the ellipsoid surface sum((x_d / axes_d)^2) = 1, centred at 0.

    Three normal deviates g per point (Box-Muller on draws 4i .. 4i+3; the
    fourth deviate is dropped) give x = axes * g / |g|: uniform in direction
    from the centre, not uniform in surface area.
    """
    u = uniform01(seed, 4 * n).reshape(n, 4)
    r1 = np.sqrt(-2.0 * np.log1p(-u[:, 0]))
    r2 = np.sqrt(-2.0 * np.log1p(-u[:, 2]))
    g = np.empty((n, 3))
    g[:, 0] = r1 * np.cos(2.0 * np.pi * u[:, 1])
    g[:, 1] = r1 * np.sin(2.0 * np.pi * u[:, 1])
    g[:, 2] = r2 * np.cos(2.0 * np.pi * u[:, 3])
    norm = np.sqrt((g * g).sum(axis=1))
    norm[norm == 0.0] = 1.0
    return g / norm[:, None] * np.asarray(axes, dtype=np.float64)[None, :]


def charges(n: int, seed: int, kind: str, offset: int) -> np.ndarray:
    """n charges from draws offset .. offset+n-1: 'pos' -> (0, 1], 'sym' -> [-1, 1)."""
    u = uniform01(seed, n, offset)
    if kind == "pos":
        return 1.0 - u
    if kind == "sym":
        return 2.0 * u - 1.0
    raise ValueError(f"unknown charge kind {kind!r}")


def particles(n: int, seed: int, dist: str = "cube", qkind: str = "pos"):
    """(xyz [n][3], q [n]) float64 arrays for one synthetic problem.

    dist: 'cube' (positions use draws 0..3n-1, charges 3n..4n-1) or
    'ellipsoid' (positions 0..4n-1, charges 4n..5n-1).
    """
    if dist == "cube":
        xyz = cube(n, seed)
        q = charges(n, seed, qkind, 3 * n)
    elif dist == "ellipsoid":
        xyz = ellipsoid_surface(n, seed)
        q = charges(n, seed, qkind, 4 * n)
    else:
        raise ValueError(f"unknown distribution {dist!r}")
    return np.ascontiguousarray(xyz), np.ascontiguousarray(q)


# Named workloads: (n, height, order, distribution, charges, seed).
WORKLOADS = {
    # 20,000 points in the unit cube, charges in (0, 1], h = 4, p = 5.
    "cube_n20k_h4_p5": dict(n=20_000, height=4, order=5, dist="cube", qkind="pos", seed=1),
    # 1e6 points in the unit cube, charges in [-1, 1), h = 6, p = 7.
    "cube_n1m_h6_p7": dict(n=1_000_000, height=6, order=7, dist="cube", qkind="sym", seed=2),
    # 1.25e6 points on the same ellipsoid, h = 7, p = 7 (about the same particles per leaf
    # as the 1e7-point case one level deeper; a medium-size profiling case).
    "ellipsoid_n1250k_h7_p7": dict(n=1_250_000, height=7, order=7, dist="ellipsoid", qkind="pos", seed=3),
    # 1e7 points on the (0.5, 0.25, 0.125) ellipsoid, charges in (0, 1], h = 8, p = 7.
    "ellipsoid_n10m_h8_p7": dict(n=10_000_000, height=8, order=7, dist="ellipsoid", qkind="pos", seed=3),
}


def workload(name: str):
    """(xyz, q, height, order) for a named workload."""
    w = WORKLOADS[name]
    xyz, q = particles(w["n"], w["seed"], w["dist"], w["qkind"])
    return xyz, q, w["height"], w["order"]


def batch_height(n: int, hmin: int = 3, hmax: int = 6) -> int:
    """Tree height of a batched problem: the smallest leaf level L with
    32 * 8^L >= n (about 32 particles per leaf in the cube), plus one,
    clamped to [hmin, hmax]."""
    L = 0
    while 32 * 8 ** L < n:
        L += 1
    return min(max(1 + L, hmin), hmax)


def batch_workload(nprob: int = 256, seed: int = 999, nmin: float = 1e3, nmax: float = 2e5,
                   hmin: int = 3, hmax: int = 6):
    """Independent problems of uneven size for the batched path.

    Sizes are log-uniform in [nmin, nmax] (draw k of stream `seed` gives
    problem k); problem k uses seed 1000 + k, points uniform in the unit cube
    if that seed is even and on the ellipsoid surface if it is odd, charges in
    (0, 1].  Returns (counts, heights, xyz, q) with the problems' particles
    concatenated in problem order.
    """
    u = uniform01(seed, nprob)
    lo, hi = np.log10(nmin), np.log10(nmax)
    counts = np.floor(10.0 ** (lo + u * (hi - lo))).astype(np.int64)
    heights = np.array([batch_height(int(n), hmin, hmax) for n in counts], dtype=np.int32)
    xs, qs = [], []
    for k, n in enumerate(counts):
        s = 1000 + k
        xyz, q = particles(int(n), s, "cube" if s % 2 == 0 else "ellipsoid", "pos")
        xs.append(xyz)
        qs.append(q)
    return counts, heights, np.ascontiguousarray(np.concatenate(xs)), np.ascontiguousarray(np.concatenate(qs))
