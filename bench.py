#!/usr/bin/env python
"""Throughput of the black-box FMM on B300: particles per second for one full
pass (tree build + evaluation of potentials and forces), mixed precision.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload NAME] [--only-main]

One JSON line on stdout (rank 0).  A step is fmm_set_particles + fmm_evaluate
on device-resident inputs (all hot-path stages: box, Morton keys, sort, tree,
P2M, M2M, M2L, L2L, L2P, P2P, output).  Each step is bracketed by CUDA events
on the library's stream; between steps a 512 MB buffer is rewritten to flush
the 126 MB L2 (outside the events).  `e2e` repeats the step through the same
C calls with pinned host buffers, host<->device copies inside the timed
region.

The line's `value` is the 1e6-point unit cube (h 6, p 7).  With one GPU the
same line also carries, each measured in this run:
  c3        1e7 points on an ellipsoid surface (h 8, p 7), timed the same way;
  c4        256 uneven problems solved as one batch (p 5);
  c5        a Poisson stream of solve requests through the solve server;
  fp64_gpu  the FP64 GPU path on the cube, and speedup_vs_fp64_gpu;
  err_vs_direct (cube and c3)  relative L2 error of the last timed step's
            phi and F against the FP64 direct sum on 2000 seeded targets
            (the CPU oracle, outside the timed region);
  fp32_peak the FP32 FMA rate of this GPU, measured by a throughput kernel
            of the library (the P2P roofline's denominator).
With N > 1 (torchrun) every rank solves its own independent cube (replicas:
the FMM itself is not sharded), value = all particles / the slowest rank's
time, and the line carries the cube only.

--impl reference times the FP64 CPU oracle (the test oracle, as it stands) on
a density-matched bounded sample of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "cube_n1m_h6_p7"
C3_WORKLOAD = "ellipsoid_n10m_h8_p7"
# the same cube under every kernel of fmm_set_kernel and the Stokes path
KERNELS_WORKLOAD = "kernels_cube_n1m_h6_p7"
METRIC = "FMM particles/s at rel.err<=1e-5 vs FP64 direct; P2P/M2L % roofline; p50/p99 ms"
UNIT = "particles/s"
ERR_BAR = 1e-5
ERR_TARGETS = 2000
# Oracle samples.  The cube is timed on the full workload (about 10 s on 16
# cores).  The 1e7-point ellipsoid is timed on a density-matched sample: a
# surface's occupied leaves grow about 4.1x per level, so 600,000 points of
# the same ellipsoid at h = 6 hold the same ~450 particles per occupied leaf
# as 1e7 points at h = 8.  The reference arm's steps use a density-matched
# sample of the cube (N / 8^k at height - k) so that K steps stay within minutes.
CPU_BASELINE_SAMPLES = {
    WORKLOAD: dict(n=1_000_000, height=6, order=7, dist="cube", qkind="sym", seed=2,
                   note="the timed workload itself"),
    C3_WORKLOAD: dict(n=600_000, height=6, order=7, dist="ellipsoid", qkind="pos", seed=3,
                      note="density-matched sample of the 1e7-point ellipsoid: the same ellipsoid and charges, "
                           "~450 particles per occupied leaf as at N=1e7, h=8"),
}
REFERENCE_STEP_SAMPLE = dict(n=15_625, height=4, order=7, dist="cube", qkind="sym", seed=2)

TF32_OVER_BF16 = 1.1 / 2.25     # nominal dense tensor rates (FP16 runs at the BF16 rate)
# FP32 operations of one P2P interaction as the mixed kernel issues them: the
# exact difference (hi_t - hi_s) + (lo_t - lo_s) per axis (9), the squared
# distance (1 multiply + 2 FMA), q/r (1), q/r^3 (2), the potential sum (1)
# and the field sums (3 FMA) = 19; 1/sqrt runs on the MUFU pipe.  A plain
# single-word FP32 difference would need 13.
P2P_FP32_OPS = 19
P2P_FP32_OPS_PLAIN = 13


def m2l_math(stats) -> str:
    """Operand form of the tensor-core M2L (compressed or full-rank
    operators): FP16 hi/lo pairs (the default) or TF32 hi/lo pairs."""
    return "f16x3" if int(stats[4]) in (2, 5) and int(stats[5]) == 1 else "tf32x3"


def tensor_peak(pk, math: str):
    if math == "f16x3":
        return pk["bf16"], f"FP16 = {pk['src']} bf16 (the same dense rate)"
    return pk["bf16"] * TF32_OVER_BF16, f"TF32 = {pk['src']} bf16 x 1.1/2.25"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["mixed", "fp64"], default="mixed")
    ap.add_argument("--m2l", choices=["full", "svd"], default="svd",
                    help="M2L operators: full-rank K_t, or the SVD-compressed canonical operators (eps = 10^-p)")
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--only-main", action="store_true", help="the named workload alone (no c3/c4/c5/fp64 legs)")
    ap.add_argument("--no-cpu-baseline", action="store_true",
                    help="skip the oracle legs (CPU baseline timing and the error check against the direct sum)")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default P2P kernel shape")
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--fp64-steps", type=int, default=3)
    ap.add_argument("--rate", type=float, default=200.0, help="serving: mean requests per second")
    ap.add_argument("--serve-seconds", type=float, default=10.0, help="serving: length of the request stream")
    ap.add_argument("--lanes", type=int, default=2, help="serving: concurrent batches")
    ap.add_argument("--ring-gb", type=int, default=8, help="serving: pinned result ring (GB)")
    ap.add_argument("--max-batch-particles", type=int, default=8_000_000, help="serving: particles per batch")
    return ap.parse_args()


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return dict(hbm=d["hbm_gbs"], bf16=d["bf16_tflops"], bf16_sus=d.get("bf16_tflops_sustained"),
                    sm_max_mhz=d.get("sm_max_mhz", 2032.0), src="measured")
    return dict(hbm=6400.0, bf16=1800.0, bf16_sus=1400.0, sm_max_mhz=2032.0, src="fallback")


def fp32_peak(fmm):
    """The FP32 FMA rate of this GPU, measured in this run by the library's
    throughput kernel (independent FMA chains on every SM, best of three
    launches), scalar and packed (fma.rn.f32x2); the larger is the peak."""
    r = fmm.fmm_measure_fp32_rate()
    flops = float(max(r[0], r[1]))
    return {"tflops": flops / 1e12, "scalar_tflops": float(r[0]) / 1e12, "packed_tflops": float(r[1]) / 1e12,
            "sms": int(r[2]), "ops_per_s": flops / 2.0,
            "source": "measured in this run: fmm_measure_fp32_rate (FMA chains, 8 x 256 threads per SM, "
                      "best of 3 launches); an FMA is 2 flop and 1 FP32 operation"}


class Clocks:
    """nvidia-smi samples (every 200 ms) taken while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.file = tempfile.NamedTemporaryFile(mode="w+", suffix=".csv", delete=False)
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.file, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.file.flush()
        self.file.seek(0)
        rows = [r.split(",") for r in self.file.read().strip().splitlines() if r.strip()]
        os.unlink(self.file.name)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
                for k, nm in enumerate(names):
                    if r[5 + k].strip().lower().startswith("active"):
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def profiled_traffic(kernel_file: str, profile: str, marker: str, start: str = ""):
    """DRAM bytes per launch recorded in a profiles/ summary, or None when the
    kernel source (the text of kernel_file from `start`, or its beginning, up
    to `marker`) has changed since that capture."""
    import hashlib
    import re
    try:
        src = open(os.path.join(ROOT, kernel_file)).read()
        text = open(os.path.join(ROOT, profile)).read()
    except OSError:
        return None
    a = src.find(start) if start else 0
    cut = src.find(marker, max(a, 0))
    if a < 0 or cut < 0:
        return None
    h = hashlib.sha256(src[a:cut].encode()).hexdigest()
    m = re.search(r"kernel-source-sha256: ([0-9a-f]{64})", text)
    t = re.search(r"dram-traffic-bytes-per-launch[^|\n]*\|[ |]*(\d+)", text)
    if not m or not t or m.group(1) != h:
        return None
    return int(t.group(1))


def replica_throughput(n_local: int, steps: int, local_ms: float, device="cpu"):
    """Whole-job throughput of independent replicas: every rank solved `steps`
    problems of n_local particles in local_ms; the job took as long as the
    slowest rank.  Returns (particles per second, max ms over ranks)."""
    max_ms = float(local_ms)
    import torch.distributed as dist
    ws = 1
    if dist.is_available() and dist.is_initialized():
        import torch
        ws = dist.get_world_size()
        t = torch.tensor([max_ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        max_ms = float(t.item())
    return n_local * ws * steps / (max_ms / 1e3), max_ms


def stage_rooflines(n, h, p, ncell, iso, build_ms, pk, precision):
    """HBM rooflines of the stages around M2L and P2P (each timed alone):
    algorithmic bytes per evaluation / stage time against the measured copy
    bandwidth.  Mixed precision: a multipole row is C FP32 hi/lo pairs (8 B
    per coefficient), a local row C + 1 FP32 values."""
    if precision != "mixed" or h < 3:
        return None
    C = p ** 3
    Lf = h - 1
    leaves = ncell[Lf]
    parents = sum(ncell[2:Lf])  # cells of levels 2 .. Lf-1 (M2M outputs, L2L inputs)
    bw = pk["hbm"]
    stages = {
        # P2M: pos32 in, leaf multipoles out; M2M: 8 children in, parent out
        "upward": (16 * n + 8 * C * leaves + 9 * 8 * C * parents, iso[0]),
        # L2L: parent in, 8 children read and written
        "l2l": (4 * (C + 1) * parents + 2 * 8 * 4 * (C + 1) * parents, iso[4]),
        # L2P + output: pos32, near field and permutation in, phi and F (FP64) out, leaf locals in
        "l2p_out": (n * (16 + 16 + 4 + 32) + 4 * (C + 1) * leaves, iso[6]),
        # tree build: coordinates and charges in (twice: cube, keys), 4 radix passes of key + index,
        # gather in Morton order (32 B in, 32 + 16 + 16 + 4 B out), cells
        "set_particles": (n * (32 + 24 + 4 * 16 + 32 + 68) + 20 * sum(ncell), build_ms),
    }
    out = {}
    for k, (b, ms) in stages.items():
        out[k] = {"ms": float(ms), "bytes": int(b), "gbs": b / (ms / 1e3) / 1e9,
                  "frac_of_hbm": b / (ms / 1e3) / 1e9 / bw}
    return out


def m2l_rooflines(fmm, np, stats, work, kt, stage, p, pk, main: bool):
    """(roofline of the dominant M2L kernel, the projection's, tensor-pipe
    counts) from the algorithmic work of fmm_get_work and the kernels' own
    CUDA-event times inside the timed steps."""
    C = p ** 3
    m2l_kind = int(stats[4])
    math = m2l_math(stats)
    mlabel = "3xFP16" if math == "f16x3" else "3xTF32"
    m2l_pairs = int(work[1:12].sum())
    cpad = ((C + 1 + 31) // 32) * 32
    if m2l_kind >= 3:
        # compressed: y = V^T M (2 C r flop) and L += U y (2 C r flop) per pair
        m2l_flop = 4.0 * C * int(work[13])
        m2l_alg = f"4 x {C} x sum of pair ranks {int(work[13])} = {m2l_flop:.4g} flop per evaluation"
    else:
        m2l_flop = 2.0 * C * C * m2l_pairs
        m2l_alg = f"2 x {C}^2 flop x {m2l_pairs} pairs = {m2l_flop:.4g} flop per evaluation"
    fp32_tf = pk["fp32"]["tflops"]
    if m2l_kind in (2, 5):
        peak, peak_note = tensor_peak(pk, math)
        bound = "tensor"
    elif m2l_kind in (1, 4):
        bound, peak, peak_note = "alu", fp32_tf, "FP32 FMA, measured (fmm_measure_fp32_rate)"
    else:
        bound, peak, peak_note = "alu", fp32_tf / 64.0, "FP64 FMA: measured FP32 rate / 64 (nominal ratio)"
    tensor_pipe = None
    roofline_proj = None
    if m2l_kind == 5:
        kernel_name = (f"k_svd_expand16_tc (compressed M2L expansion L += U y, tcgen05, {mlabel}), all levels"
                       if math == "f16x3" else
                       f"k_svd_expand_tc (compressed M2L expansion L += U y, tcgen05, {mlabel}), all levels")
        half_flop = m2l_flop / 2.0
        m2l_ms = float(kt[1])
        achieved = half_flop / (m2l_ms / 1e3) / 1e12
        m2l_alg = (f"2 x {C} x sum of pair ranks {int(work[13])} = {half_flop:.4g} flop per launch "
                   f"(the projection carries as much)")
        # the profile's counters are those of the FP16-operand kernel (k_svd_expand16_tc)
        traffic = (profiled_traffic("paper_1206_0115_b300/csrc/m2l_svd_tc.cu", "profiles/m2l_svd_cube_n1m_h6_p7.md",
                                    "// Unit u -> (group g, tile, column half h)",
                                    "// ---- expansion, FP16 form") if main and math == "f16x3" else None)
        # MMA flop issued (three products per multiply, the padded shapes)
        hw_p = 3 * 2.0 * 128 * cpad * int(work[14])
        hw_e = 3 * 2.0 * 128 * cpad * int(work[15])
        tensor_pipe = {"operands": math,
                       "expansion": {"mma_flop_per_launch": hw_e, "tflops": hw_e / (kt[1] / 1e3) / 1e12,
                                     "frac_of_peak": hw_e / (kt[1] / 1e3) / 1e12 / peak},
                       "projection": {"mma_flop_per_launch": hw_p, "tflops": hw_p / (kt[0] / 1e3) / 1e12,
                                      "frac_of_peak": hw_p / (kt[0] / 1e3) / 1e12 / peak}}
        ach_p = half_flop / (kt[0] / 1e3) / 1e12
        roofline_proj = {"kernel": f"k_svd_proj_tc (compressed M2L projection y = V^T M, tcgen05, {mlabel})",
                         "bound": "tensor", "achieved": ach_p, "peak": peak, "unit": "TFLOP/s",
                         "frac": ach_p / peak, "ms": float(kt[0]), "peak_source": peak_note}
    elif m2l_kind == 2:
        kernel_name = f"k_m2l_tc (full-rank M2L, tcgen05, {mlabel}), all levels"
        m2l_ms = float(kt[1])
        achieved = m2l_flop / (m2l_ms / 1e3) / 1e12
        traffic = (profiled_traffic("paper_1206_0115_b300/csrc/m2l_tc.cu", "profiles/m2l_tc_cube_n1m_h6_p7.md",
                                    "// L_T[m] = (1/a) * sum over the tile's groups") if main else None)
        hw_flop = 3 * 2.0 * 128 * cpad * cpad * int(work[12])
        tensor_pipe = {"operands": math, "mma_flop_per_launch": hw_flop, "tflops": hw_flop / (m2l_ms / 1e3) / 1e12,
                       "frac_of_peak": hw_flop / (m2l_ms / 1e3) / 1e12 / peak}
    else:
        kernel_name = ["k_m2l_simt<double> (FP64 CUDA cores), all levels",
                       "k_m2l_simt<float> (FP32 CUDA cores), all levels", "",
                       "k_m2l_proj + k_m2l_expand <double> (compressed, FP64 CUDA cores), all levels",
                       "k_m2l_proj + k_m2l_expand <float> (compressed, FP32 CUDA cores), all levels"][m2l_kind]
        m2l_ms = float(np.mean(stage[:, 1]))
        achieved = m2l_flop / (m2l_ms / 1e3) / 1e12
        traffic = None
    roof = {"kernel": kernel_name, "bound": bound, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": traffic, "ms": m2l_ms, "algorithmic": m2l_alg,
            "peak_source": peak_note}
    return roof, roofline_proj, tensor_pipe


def p2p_roofline(p2p_pairs: int, p2p_ms: float, pk, kernel: str, traffic=None):
    """The near field against the FP32 pipe: achieved = 20 flop per directed
    interaction (the paper's convention) over the P2P launch time, against
    the FP32 rate measured in this run; also the fraction of the FP32
    operation rate the kernel's 19 issued operations per interaction fill."""
    fp = pk["fp32"]
    ips = p2p_pairs / (p2p_ms / 1e3)
    return {"bound": "alu", "kernel": kernel, "achieved": 20.0 * ips / 1e12, "peak": fp["tflops"],
            "unit": "TFLOP/s", "frac": 20.0 * ips / (fp["tflops"] * 1e12), "traffic": traffic, "ms": p2p_ms,
            "algorithmic": f"20 flop x {p2p_pairs} directed interactions = {20.0 * p2p_pairs:.4g} flop per launch",
            "peak_source": "FP32 FMA rate measured in this run (fp32_peak)",
            "interactions": p2p_pairs, "interactions_per_s": ips,
            "fp32_ops_per_interaction": P2P_FP32_OPS,
            "fp32_pipe_frac": P2P_FP32_OPS * ips / fp["ops_per_s"],
            "fp32_pipe_frac_plain_13": P2P_FP32_OPS_PLAIN * ips / fp["ops_per_s"]}


def dominant(rooflines: dict):
    """The roofline of the kernel with the longest launch time."""
    best = None
    for r in rooflines.values():
        if r is not None and (best is None or r["ms"] > best["ms"]):
            best = r
    return best


def autotune(fmm, h):
    """fmm_autotune: the near field's shape per occupancy bin (leaves of at
    most 64 particles / larger leaves), each bin timed alone in every shape."""
    choice, ttimes = fmm.fmm_autotune(h)
    bins, bin_ms = fmm.fmm_get_p2p_bins(h)
    rep = {"p2p_variant": int(choice[0]), "warps_per_block": int(choice[1]), "chunk": int(choice[2]),
           "sources_per_instruction": int(choice[3]), "unroll": int(choice[4]),
           "variant_ms": [round(float(t), 4) for t in ttimes], "bins": {}}
    for b, name in enumerate(("small_leaves", "large_leaves")):
        rep["bins"][name] = {"items": int(bins[2 + b]), "variant": int(bins[b]),
                             "variant_ms": [round(float(t), 4) for t in bin_ms[b]]}
    sched, sched_ms = fmm.fmm_get_schedule(h)
    names = ("with_expansion", "at_start", "with_projection", "with_projection_2xstages")
    names = list(names) + [n + "_nonpersistent" for n in names]
    # fmm_autotune keeps the fastest candidate (the first on a tie); candidates
    # 4..7 are 0..3 with the near field's non-persistent shapes
    timed = [(float(t), k) for k, t in enumerate(sched_ms) if t >= 0]
    pick = min(timed)[1] if timed else int(sched)
    rep["schedule"] = {"p2p_starts": names[pick], "candidate": pick,
                       "evaluate_ms": {k: round(float(t), 4) for k, t in zip(names, sched_ms)}}
    return rep


def sample_targets(n: int, k: int = ERR_TARGETS, seed: int = 5):
    import numpy as np
    return np.sort(np.random.default_rng(seed).choice(n, size=min(k, n), replace=False))


# ---- the oracle legs ---------------------------------------------------------
# The CPU oracle serves two purposes here, both outside the timed region: the
# CPU baseline (its FMM timed on the host cores) and the accuracy check of
# the timed run's own output against the exact sum on sampled targets.

def oracle_operators(order: int, m2l: str):
    """An oracle tree whose compressed M2L operators later trees reuse (the
    operators depend on the order only, as the GPU path's are computed once
    per handle); None for the full-rank operators."""
    if m2l != "svd":
        return None
    import oracle
    from paper_1206_0115_b300 import inputs
    xyz, q = inputs.particles(64, 1, "cube", "pos")
    return oracle.OracleFMM(xyz, q, 3, order, svd_eps=10.0 ** -order)


def oracle_error_check(xyz, q, outputs: dict, idx):
    """Relative L2 error of each (phi, F) in `outputs` on the targets idx
    against the FP64 direct sum (the oracle's O(N) per target sum)."""
    import oracle
    t0 = time.perf_counter()
    pd, Fd = oracle.direct_sampled(xyz, q, idx)
    t = time.perf_counter() - t0
    res = {}
    for name, (phi, F) in outputs.items():
        ep, eF = oracle.rel_l2(phi[idx], pd), oracle.rel_l2(F[idx], Fd)
        res[name] = {"phi": ep, "F": eF, "targets": int(len(idx)), "bar": ERR_BAR,
                     "within_bar": bool(ep <= ERR_BAR and eF <= ERR_BAR),
                     "reference": f"FP64 direct sum (oracle) over all {len(q)} sources, {t:.1f} s on the host"}
    return res


def cpu_baseline(sample: dict, m2l: str):
    """The FP64 oracle's FMM on `sample` (the timed workload or a stated
    density-matched sample of it), with the same M2L operators."""
    import oracle
    from paper_1206_0115_b300 import inputs
    xyz, q = inputs.particles(sample["n"], sample["seed"], sample["dist"], sample["qkind"])
    ops = oracle_operators(sample["order"], m2l)
    t0 = time.perf_counter()
    with oracle.OracleFMM(xyz, q, sample["height"], sample["order"], svd_from=ops) as o:
        o.evaluate()
    t = time.perf_counter() - t0
    return {"value": sample["n"] / t, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": (f"N={sample['n']} {sample['dist']}, h={sample['height']}, p={sample['order']} "
                       f"({sample['note']}), FP64 oracle FMM ({m2l} M2L operators, computed beforehand) "
                       f"incl. tree build, 1 run, {t:.2f} s")}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    s = REFERENCE_STEP_SAMPLE
    import oracle
    from paper_1206_0115_b300 import inputs
    xyz, q = inputs.particles(s["n"], s["seed"], s["dist"], s["qkind"])

    ops = oracle_operators(s["order"], args.m2l)

    def step():
        with oracle.OracleFMM(xyz, q, s["height"], s["order"], svd_from=ops) as o:
            o.evaluate()

    for _ in range(args.warmup):
        step()
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        step()
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    value = s["n"] * args.steps / tot
    sample = (f"each step: N={s['n']} uniform cube, h={s['height']}, p={s['order']} (same particles per "
              f"leaf as {WORKLOAD}), FP64 oracle FMM ({args.m2l} M2L operators, computed beforehand) "
              f"incl. tree build")
    print(json.dumps({
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
        "config": {"workload": WORKLOAD, "sample": sample},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


# ---- one problem ---------------------------------------------------------------

def measure_single(args, fmm, dev, workload: str, pk, rank: int = 0, main: bool = True):
    """Times `workload` (fmm_set_particles + fmm_evaluate per step) and
    returns (result dict, host inputs, host outputs of the last timed step)."""
    import numpy as np
    import torch

    from paper_1206_0115_b300 import inputs
    ws, _, local = dist_env()
    w = dict(inputs.WORKLOADS[workload])
    xyz_np, q_np = inputs.particles(w["n"], w["seed"] + 1000 * rank, w["dist"], w["qkind"])
    n, h, p = w["n"], w["height"], w["order"]
    prec = fmm.FMM_MIXED if args.precision == "mixed" else fmm.FMM_FP64
    stream = torch.cuda.Stream(device=dev)
    method = fmm.FMM_M2L_SVD if args.m2l == "svd" else fmm.FMM_M2L_FULL
    f = fmm.FMM(h, p, prec, stream=stream, m2l=method)
    xyz = torch.from_numpy(xyz_np).to(dev)
    q = torch.from_numpy(q_np).to(dev)
    phi = torch.empty(n, dtype=torch.float64, device=dev)
    F = torch.empty((n, 3), dtype=torch.float64, device=dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    fmm.fmm_set_timing(f.h, True)

    def step():
        f.set_particles(xyz, q)
        f.evaluate(phi, F)

    torch.cuda.synchronize()
    for _ in range(max(args.warmup, 1)):
        step()
    torch.cuda.synchronize()
    tuned = None
    if not args.no_autotune:
        tuned = autotune(fmm, f.h)
        step()
        torch.cuda.synchronize()
    work = fmm.fmm_get_work(f.h)
    stats = f.stats()
    # stage times with every stage run alone (P2P normally overlaps M2L), for
    # the per-kernel rooflines; outside the timed region
    fmm.fmm_set_timing(f.h, 2)
    iso = []
    for _ in range(3):
        step()
        iso.append(fmm.fmm_get_stage_times(f.h).tolist())
    iso = np.median(np.array(iso), axis=0)
    fmm.fmm_set_timing(f.h, 1)
    step()
    torch.cuda.synchronize()

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    mids = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    stage = []
    ktimes = []
    tc_timed = int(stats[4]) in (2, 5)
    clocks = Clocks(local)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    t_wall = time.perf_counter()
    for k in range(args.steps):
        with torch.cuda.stream(stream):
            flush.fill_(float(k))
        starts[k].record(stream)
        f.set_particles(xyz, q)
        mids[k].record(stream)
        f.evaluate(phi, F)
        ends[k].record(stream)
        stage.append(fmm.fmm_get_stage_times(f.h).tolist())
        if tc_timed:
            ktimes.append(fmm.fmm_get_m2l_kernel_times(f.h).tolist())
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall
    if ws > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    build_ms = float(np.mean([s.elapsed_time(e) for s, e in zip(starts, mids)]))
    value, total_ms = replica_throughput(n, args.steps, sum(ms), device=dev)
    ncell = [fmm.fmm_get_level_size(f.h, l) for l in range(h)]
    out_phi, out_F = phi.cpu().numpy(), F.cpu().numpy()  # the last timed step's results
    stats = f.stats()

    # end to end through the same calls with pinned host buffers
    xyz_h = torch.from_numpy(xyz_np).pin_memory()
    q_h = torch.from_numpy(q_np).pin_memory()
    phi_h = torch.empty(n, dtype=torch.float64).pin_memory()
    F_h = torch.empty((n, 3), dtype=torch.float64).pin_memory()
    e_ms = []
    for k in range(args.e2e_steps + 1 if args.e2e_steps > 0 else 0):
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        f.set_particles(xyz_h, q_h)
        f.evaluate(phi_h, F_h)
        b.record(stream)
        torch.cuda.synchronize()
        if k > 0:
            e_ms.append(a.elapsed_time(b))
    e2e_value = replica_throughput(n, len(e_ms), sum(e_ms), device=dev)[0] if e_ms else None
    f.close()
    del flush

    stage = np.array(stage)
    kt = np.mean(np.array(ktimes), axis=0) if ktimes else None
    roof, roof_proj, tensor_pipe = m2l_rooflines(fmm, np, stats, work, kt, stage, p, pk, main)
    p2p_kernel = ("k_p2p32x2p / k_p2p32x2 / k_p2p32x2c (the near field in the autotuned shapes, run alone)"
                  if tuned else "k_p2p32x2<8,128,4> (the near field, run alone)")
    roof_p2p = p2p_roofline(int(work[0]), float(iso[5]), pk, p2p_kernel,
                            profiled_traffic("paper_1206_0115_b300/csrc/nearfield.cu",
                                             "profiles/p2p_cube_n1m_h6_p7.md", "// ---- the Stokeslet near field")
                            if main else None)
    kernels = {"m2l_expansion": roof, "m2l_projection": roof_proj, "p2p": roof_p2p}
    math = m2l_math(stats)
    res = {
        "value": value, "unit": UNIT, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps,
        "dtype": f"f32+{math}" if args.precision == "mixed" else "f64",
        "config": {"workload": workload, "n": n, "height": h, "order": p, "precision": args.precision,
                   "m2l": args.m2l, "distribution": w["dist"], "charges": w["qkind"], "seed": w["seed"],
                   "l2": "flushed between steps (512 MB rewrite outside the timed events)",
                   "parallelism": "replicas" if ws > 1 else "single"},
        "p50_ms": float(np.percentile(ms, 50)), "p99_ms": float(np.percentile(ms, 99)),
        "set_particles_ms": build_ms,
        "stage_ms": {"upward": float(np.mean(stage[:, 0])), "m2l_all": float(np.mean(stage[:, 1])),
                     "m2l_main": float(np.mean(stage[:, 2])), "m2l_rest": float(np.mean(stage[:, 3])),
                     "l2l": float(np.mean(stage[:, 4])), "p2p": float(np.mean(stage[:, 5])),
                     "l2p_out": float(np.mean(stage[:, 6])), "evaluate": float(np.mean(stage[:, 7]))},
        "stage_ms_isolated": {"upward": float(iso[0]), "m2l_main": float(iso[2]), "m2l_rest": float(iso[3]),
                              "l2l": float(iso[4]), "p2p": float(iso[5]), "l2p_out": float(iso[6])},
        # the kernel with the longest launch time; every one of the three below
        "roofline": dominant(kernels),
        "roofline_m2l_expansion": roof,
        "roofline_m2l_projection": roof_proj,
        "roofline_p2p": roof_p2p,
        "tensor_pipe": tensor_pipe,
        "autotune": tuned,
        "roofline_stages": stage_rooflines(n, h, p, ncell, iso, build_ms, pk, args.precision),
        "gpu_launches": int((stats[0] + stats[1]) * args.steps),
        # evaluations that ran launch by launch after a failed graph capture (0 expected)
        "graph_fallbacks": int(stats[6]),
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(32 * n),
                "d2h_bytes_per_step": int(32 * n), "steps": len(e_ms)},
        "clocks": clk,
        "wall_s": t_wall,
    }
    return res, (xyz_np, q_np), (out_phi, out_F)


def measure_fp64(args, fmm, dev, workload: str):
    """The FP64 GPU path (every stage in FP64 on the GPU, the same M2L
    operators) on `workload`: a few steps after one warm-up (which computes
    the FP64 operators), timed like the mixed path."""
    import numpy as np
    import torch

    from paper_1206_0115_b300 import inputs
    w = dict(inputs.WORKLOADS[workload])
    xyz_np, q_np = inputs.particles(w["n"], w["seed"], w["dist"], w["qkind"])
    n, h, p = w["n"], w["height"], w["order"]
    stream = torch.cuda.Stream(device=dev)
    method = fmm.FMM_M2L_SVD if args.m2l == "svd" else fmm.FMM_M2L_FULL
    xyz = torch.from_numpy(xyz_np).to(dev)
    q = torch.from_numpy(q_np).to(dev)
    phi = torch.empty(n, dtype=torch.float64, device=dev)
    F = torch.empty((n, 3), dtype=torch.float64, device=dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    ms = []
    with fmm.FMM(h, p, fmm.FMM_FP64, stream=stream, m2l=method) as f:
        f.set_particles(xyz, q)
        f.evaluate(phi, F)
        torch.cuda.synchronize()
        for k in range(max(1, args.fp64_steps)):
            with torch.cuda.stream(stream):
                flush.fill_(float(k))
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            f.set_particles(xyz, q)
            f.evaluate(phi, F)
            b.record(stream)
            b.synchronize()
            ms.append(a.elapsed_time(b))
    t = float(np.mean(ms))
    return {"value": n / (t / 1e3), "unit": UNIT, "ms_per_step": t, "steps": len(ms), "dtype": "f64",
            "config": {"workload": workload, "precision": "fp64", "m2l": args.m2l}}, (phi.cpu().numpy(),
                                                                                      F.cpu().numpy())


BATCH_WORKLOAD = "batched_256_p5"


def measure_batched(args, fmm, dev, pk, rank: int = 0):
    """256 independent problems of uneven size (1e3 .. 2e5 particles, heights
    3..6 by size, cube or ellipsoid by seed, p = 5) solved as one batch: a step
    is fmm_set_batch + fmm_evaluate over all of them (one launch per stage)."""
    import numpy as np
    import torch

    from paper_1206_0115_b300 import inputs
    ws, _, local = dist_env()
    p = 5
    counts, heights, xyz_np, q_np = inputs.batch_workload(seed=999 + 1000 * rank)
    n = int(counts.sum())
    prec = fmm.FMM_MIXED if args.precision == "mixed" else fmm.FMM_FP64
    stream = torch.cuda.Stream(device=dev)
    method = fmm.FMM_M2L_SVD if args.m2l == "svd" else fmm.FMM_M2L_FULL
    f = fmm.FMM(3, p, prec, stream=stream, m2l=method)
    xyz = torch.from_numpy(xyz_np).to(dev)
    q = torch.from_numpy(q_np).to(dev)
    phi = torch.empty(n, dtype=torch.float64, device=dev)
    F = torch.empty((n, 3), dtype=torch.float64, device=dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def step():
        f.set_batch(counts, heights, xyz, q)
        f.evaluate(phi, F)

    fmm.fmm_set_timing(f.h, 1)
    torch.cuda.synchronize()
    for _ in range(max(args.warmup, 1)):
        step()
    torch.cuda.synchronize()
    tuned = None
    if not args.no_autotune:
        tuned = autotune(fmm, f.h)
        step()
        torch.cuda.synchronize()
    work = fmm.fmm_get_work(f.h)
    stats = f.stats()
    fmm.fmm_set_timing(f.h, 2)
    iso = []
    for _ in range(3):
        step()
        iso.append(fmm.fmm_get_stage_times(f.h).tolist())
    iso = np.median(np.array(iso), axis=0)
    fmm.fmm_set_timing(f.h, 1)
    step()
    torch.cuda.synchronize()
    tc_timed = int(stats[4]) in (2, 5)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    mids = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ktimes = []
    clocks = Clocks(local)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    for k in range(args.steps):
        with torch.cuda.stream(stream):
            flush.fill_(float(k))
        starts[k].record(stream)
        f.set_batch(counts, heights, xyz, q)
        mids[k].record(stream)
        f.evaluate(phi, F)
        ends[k].record(stream)
        if tc_timed:
            ktimes.append(fmm.fmm_get_m2l_kernel_times(f.h).tolist())
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    ms = [a.elapsed_time(b) for a, b in zip(starts, ends)]
    build_ms = [a.elapsed_time(b) for a, b in zip(starts, mids)]
    value, total_ms = replica_throughput(n, args.steps, sum(ms), device=dev)
    xyz_h = torch.from_numpy(xyz_np).pin_memory()
    q_h = torch.from_numpy(q_np).pin_memory()
    phi_h = torch.empty(n, dtype=torch.float64).pin_memory()
    F_h = torch.empty((n, 3), dtype=torch.float64).pin_memory()
    e_ms = []
    for k in range(args.e2e_steps + 1 if args.e2e_steps > 0 else 0):
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        f.set_batch(counts, heights, xyz_h, q_h)
        f.evaluate(phi_h, F_h)
        b.record(stream)
        torch.cuda.synchronize()
        if k > 0:
            e_ms.append(a.elapsed_time(b))
    e2e_value = replica_throughput(n, len(e_ms), sum(e_ms), device=dev)[0] if e_ms else None
    leaf_level = int(f.batch_info(0)[0][4])
    stats = f.stats()
    f.close()
    del flush
    C = p ** 3
    cpad = ((C + 1 + 31) // 32) * 32
    math = m2l_math(stats)
    mlabel = "3xFP16" if math == "f16x3" else "3xTF32"
    peak, peak_note = tensor_peak(pk, math)
    kt = np.mean(np.array(ktimes), axis=0) if ktimes else None
    half_flop = 2.0 * C * int(work[13])
    kexp = ("k_svd_expand16_tc" if math == "f16x3" else "k_svd_expand_tc")
    kernels = {
        "m2l_expansion": None if kt is None else {
            "kernel": f"{kexp} (compressed M2L expansion, tcgen05, {mlabel}), all problems and levels",
            "bound": "tensor", "achieved": half_flop / (kt[1] / 1e3) / 1e12, "peak": peak, "unit": "TFLOP/s",
            "frac": half_flop / (kt[1] / 1e3) / 1e12 / peak, "traffic": None, "ms": float(kt[1]),
            "algorithmic": f"2 x {C} x sum of pair ranks {int(work[13])} = {half_flop:.4g} flop per launch",
            "peak_source": peak_note},
        "m2l_projection": None if kt is None else {
            "kernel": f"k_svd_proj_tc (compressed M2L projection, tcgen05, {mlabel}), all problems and levels",
            "bound": "tensor", "achieved": half_flop / (kt[0] / 1e3) / 1e12, "peak": peak, "unit": "TFLOP/s",
            "frac": half_flop / (kt[0] / 1e3) / 1e12 / peak, "traffic": None, "ms": float(kt[0]),
            "algorithmic": f"2 x {C} x sum of pair ranks {int(work[13])} = {half_flop:.4g} flop per launch",
            "peak_source": peak_note},
        "p2p": p2p_roofline(int(work[0]), float(iso[5]), pk, "the near field in the autotuned shapes, run alone"),
    }
    res = {
        "value": value, "unit": UNIT, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps,
        "dtype": f"f32+{math}" if args.precision == "mixed" else "f64",
        "config": {"workload": BATCH_WORKLOAD, "problems": int(len(counts)), "n_total": n,
                   "n_min": int(counts.min()), "n_max": int(counts.max()),
                   "heights": {str(hh): int((heights == hh).sum()) for hh in sorted(set(heights.tolist()))},
                   "order": p, "precision": args.precision, "m2l": args.m2l,
                   "distribution": "cube (even seed) / ellipsoid surface (odd seed)", "charges": "pos",
                   "batch_tree_leaf_level": leaf_level,
                   "l2": "flushed between steps (512 MB rewrite outside the timed events)",
                   "parallelism": "replicas" if ws > 1 else "single"},
        "p50_ms": float(np.percentile(ms, 50)), "p99_ms": float(np.percentile(ms, 99)),
        "set_batch_ms": float(np.mean(build_ms)),
        "stage_ms_isolated": {"upward": float(iso[0]), "m2l_main": float(iso[2]), "m2l_rest": float(iso[3]),
                              "l2l": float(iso[4]), "p2p": float(iso[5]), "l2p_out": float(iso[6])},
        "roofline": dominant(kernels),
        "roofline_m2l_expansion": kernels["m2l_expansion"],
        "roofline_m2l_projection": kernels["m2l_projection"],
        "roofline_p2p": kernels["p2p"],
        "tensor_pipe": None if kt is None else {
            "operands": math,
            "expansion_frac_of_peak": 3 * 2.0 * 128 * cpad * int(work[15]) / (kt[1] / 1e3) / 1e12 / peak,
            "projection_frac_of_peak": 3 * 2.0 * 128 * cpad * int(work[14]) / (kt[0] / 1e3) / 1e12 / peak},
        "autotune": tuned,
        "gpu_launches": int((stats[0] + stats[1]) * args.steps),
        "graph_fallbacks": int(stats[6]),
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(32 * n),
                "d2h_bytes_per_step": int(32 * n), "steps": len(e_ms)},
        "clocks": clk,
    }
    return res, (counts, heights, xyz_np, q_np)


def batch_cpu_baseline(args, counts, heights, xyz_np, q_np, p: int = 5):
    """The oracle on a bounded sample of the batch: its first 8 problems, one
    after another."""
    import numpy as np
    import oracle
    st = np.concatenate([[0], np.cumsum(counts)])
    ops = oracle_operators(p, args.m2l)
    t0 = time.perf_counter()
    m = 0
    for k in range(8):
        a, b = st[k], st[k + 1]
        with oracle.OracleFMM(xyz_np[a:b], q_np[a:b], int(heights[k]), p, svd_from=ops) as o:
            o.evaluate()
        m += b - a
    t = time.perf_counter() - t0
    return {"value": m / t, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"problems 0..7 of the batch ({m} particles) one after another, FP64 "
                      f"oracle FMM ({args.m2l} M2L operators, computed beforehand), {t:.2f} s"}


def run_batched(args):
    import torch

    from paper_1206_0115_b300 import build
    build.build()
    from paper_1206_0115_b300 import fmm
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    pk = peaks()
    pk["fp32"] = fp32_peak(fmm)
    res, data = measure_batched(args, fmm, dev, pk, rank)
    if rank == 0:
        line = {"metric": METRIC, "n_gpus": ws, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "data": "synthetic"}
        line.update(res)
        line["fp32_peak"] = pk["fp32"]
        if ws == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = batch_cpu_baseline(args, *data)
        print(json.dumps(line))
    if ws > 1:
        torch.distributed.destroy_process_group()


def run_ours(args):
    import torch

    from paper_1206_0115_b300 import build
    build.build()
    from paper_1206_0115_b300 import fmm

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    pk = peaks()
    pk["fp32"] = fp32_peak(fmm)
    main, (xyz, q), outs = measure_single(args, fmm, dev, args.workload, pk, rank, main=True)
    if rank != 0:
        if ws > 1:
            torch.distributed.destroy_process_group()
        return
    line = {"metric": METRIC, "n_gpus": ws, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "data": "synthetic"}
    line.update(main)
    line["fp32_peak"] = pk["fp32"]
    extras = ws == 1 and not args.only_main and args.workload == WORKLOAD and args.precision == "mixed"
    fp64_out = None
    if extras:
        fp64, fp64_out = measure_fp64(args, fmm, dev, WORKLOAD)
        line["fp64_gpu"] = fp64
        line["speedup_vs_fp64_gpu"] = main["value"] / fp64["value"]
    oracle_ok = ws == 1 and not args.no_cpu_baseline
    if oracle_ok:
        outputs = {"mixed": outs}
        if fp64_out is not None:
            outputs["fp64_gpu"] = fp64_out
        errs = oracle_error_check(xyz, q, outputs, sample_targets(len(q)))
        line["err_vs_direct"] = errs["mixed"]
        if "fp64_gpu" in errs:
            line["fp64_gpu"]["err_vs_direct"] = errs["fp64_gpu"]
    del xyz, q, outs, fp64_out
    if extras:
        c3, (x3, q3), o3 = measure_single(args, fmm, dev, C3_WORKLOAD, pk, rank, main=False)
        if oracle_ok:
            c3["err_vs_direct"] = oracle_error_check(x3, q3, {"mixed": o3}, sample_targets(len(q3)))["mixed"]
            c3["cpu_baseline"] = cpu_baseline(CPU_BASELINE_SAMPLES[C3_WORKLOAD], args.m2l)
        del x3, q3, o3
        line["c3"] = c3
        c4, data4 = measure_batched(args, fmm, dev, pk, rank)
        if oracle_ok:
            c4["cpu_baseline"] = batch_cpu_baseline(args, *data4)
        line["c4"] = c4
        line["c5"] = measure_serving(args, fmm)
    if oracle_ok and args.workload in CPU_BASELINE_SAMPLES:
        line["cpu_baseline"] = cpu_baseline(CPU_BASELINE_SAMPLES[args.workload], args.m2l)
    print(json.dumps(line))
    if ws > 1:
        torch.distributed.destroy_process_group()


SERVE_WORKLOAD = "serving_poisson200"


class Ring:
    """Pinned host arena handed out in arrival order and returned in the same
    order (a FIFO ring); take() blocks while the ring is full."""

    def __init__(self, nbytes: int):
        import threading

        import torch
        self.buf = torch.empty(nbytes // 8, dtype=torch.float64).pin_memory().numpy()
        self.cap = len(self.buf)
        self.head = 0          # next free slot (float64 units)
        self.used = 0
        self.spans = []        # (start, length incl. the padding skipped at the end), FIFO
        self.cv = threading.Condition()

    def take(self, nbytes: int):
        n = nbytes // 8
        if n > self.cap:
            raise ValueError("request larger than the result ring")
        with self.cv:
            while True:
                pad = self.cap - self.head if self.head + n > self.cap else 0
                if self.used + pad + n <= self.cap:
                    break
                self.cv.wait()
            start = 0 if pad else self.head
            self.spans.append(pad + n)
            self.used += pad + n
            self.head = (start + n) % self.cap
            return self.buf[start:start + n]

    def give(self, nbytes: int):
        with self.cv:
            self.used -= self.spans.pop(0)
            self.cv.notify_all()


def measure_serving(args, fmm):
    """Poisson stream of solve requests (mean 200 per second; sizes
    log-uniform in [1e4, 5e6] particles, uniform cube, order 5 or 7 by coin
    flip, height from the size as in the batched workload, capped at 8)
    through the solve server: 2 lanes, 150 GB admission budget.  Requests
    carry host buffers (inputs pinned, outputs in a pinned ring); latency is
    submit to results in host memory."""
    import threading

    import numpy as np
    import torch

    from paper_1206_0115_b300 import inputs

    ws, rank, local = dist_env()
    rate, seconds = args.rate, args.serve_seconds
    nreq = max(1, int(rate * seconds))
    seed = 2_000_000 + 1000 * rank
    u = inputs.uniform01(seed, 3 * nreq)
    gaps = -np.log1p(-u[:nreq]) / rate
    arrivals = np.cumsum(gaps)
    sizes = np.floor(10.0 ** (4.0 + u[nreq:2 * nreq] * (np.log10(5e6) - 4.0))).astype(np.int64)
    orders = np.where(u[2 * nreq:] < 0.5, 5, 7)
    heights = np.array([inputs.batch_height(int(n), 3, 8) for n in sizes])
    # request payloads: prefixes of four base sets of 5e6 points uniform in the
    # unit cube (a prefix of a uniform sample is a uniform sample), charges in (0, 1]
    bases = []
    for b in range(4):
        xyz, q = inputs.particles(5_000_000, seed + 1 + b, "cube", "pos")
        bases.append((torch.from_numpy(xyz).pin_memory(), torch.from_numpy(q).pin_memory()))

    lanes = args.lanes
    budget = 150 << 30
    prec = fmm.FMM_MIXED if args.precision == "mixed" else fmm.FMM_FP64
    s = fmm.fmm_server_create(lanes, prec, budget, args.max_batch_particles, 64)
    try:
        for p in (5, 7):
            fmm.fmm_server_warmup(s, p)

        # result buffers: a pinned ring (requests finish about in arrival order
        # and are collected in that order); a request waits for room
        ring = Ring(args.ring_gb << 30)

        def make(k):
            n = int(sizes[k])
            xyz, q = bases[k % 4]
            out = ring.take(32 * n)
            return dict(n=n, h=int(heights[k]), p=int(orders[k]), xyz=xyz[:n], q=q[:n],
                        phi=out[:n], F=out[n:].reshape(n, 3), ring=32 * n)

        # untimed warm-up traffic: grows the lanes' resident buffers
        warm = [make(k) for k in range(min(nreq, 3 * lanes))]
        for r in warm:
            r["t"] = fmm.fmm_server_submit(s, r["n"], r["h"], r["p"], r["xyz"], r["q"], r["phi"], r["F"])
        for r in warm:
            fmm.fmm_server_wait(s, r["t"])
            ring.give(r["ring"])
        st0 = fmm.fmm_server_stats(s)

        reqs = [None] * nreq
        tickets = [None] * nreq
        submit_err = []
        clocks = Clocks(local)
        clocks.start()
        t0 = time.perf_counter()

        def producer():
            try:
                for k in range(nreq):
                    dt = t0 + arrivals[k] - time.perf_counter()
                    if dt > 0:
                        time.sleep(dt)
                    r = reqs[k] = make(k)
                    tickets[k] = fmm.fmm_server_submit(s, r["n"], r["h"], r["p"], r["xyz"], r["q"], r["phi"], r["F"])
            except Exception as e:  # surfaced below
                submit_err.append(e)

        th = threading.Thread(target=producer)
        th.start()
        times = []
        for k in range(nreq):
            while tickets[k] is None and not submit_err:
                time.sleep(0.0005)
            if submit_err:
                break
            times.append(fmm.fmm_server_wait(s, tickets[k]))
            if k < nreq - 8:
                ring.give(reqs[k]["ring"])  # the last few stay readable for the check below
        th.join()
        t_end = time.perf_counter()
        clk = clocks.stop()
        if submit_err:
            raise submit_err[0]
        st = fmm.fmm_server_stats(s) - st0
        st[3:8] = fmm.fmm_server_stats(s)[3:8]
        span_lanes = lanes * (time.perf_counter() - t0)
    finally:
        fmm.fmm_server_destroy(s)
    times = np.array(times)
    done_at = arrivals + times[:, 2] / 1e3          # completion, seconds after t0
    span = float(done_at.max())
    parts = int(sizes.sum())
    lat = times[:, 2]
    # correctness spot check: the last request of each order against a lone solve
    check = {}
    for p in (5, 7):
        ks = np.nonzero(orders[nreq - 8:] == p)[0] + nreq - 8
        if len(ks) == 0:
            continue
        k = int(ks[-1])
        r = reqs[k]
        with fmm.FMM(r["h"], r["p"], prec) as f:
            f.set_particles(r["xyz"].numpy(), r["q"].numpy())
            phi = np.empty(r["n"])
            Fo = np.empty((r["n"], 3))
            f.evaluate(phi, Fo)
        rel = lambda a, b: float(np.linalg.norm(a - b) / np.linalg.norm(b))
        check[str(p)] = {"request": k, "n": r["n"], "rel_l2_phi_vs_alone": rel(r["phi"], phi),
                         "rel_l2_F_vs_alone": rel(r["F"], Fo)}
    result = {
        "metric": METRIC, "value": parts / span, "unit": UNIT, "n_gpus": 1, "steps": nreq,
        "warmup": len(warm), "ms_per_step": 1e3 * span / nreq, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None,
        # the server's handles take the library's default operand form unless FMM_M2L_MATH=tf32
        "dtype": ("f32+" + ("tf32x3" if os.environ.get("FMM_M2L_MATH") == "tf32" else "f16x3"))
                 if args.precision == "mixed" else "f64", "data": "synthetic",
        "config": {"workload": SERVE_WORKLOAD, "rate_rps": rate, "duration_s": seconds, "requests": nreq,
                   "n_range": [10_000, 5_000_000], "orders": [5, 7], "heights": "3..8 by size",
                   "distribution": "cube", "lanes": lanes, "hbm_budget_bytes": budget,
                   "max_batch_particles": args.max_batch_particles, "max_batch_requests": 64,
                   "payload": "prefixes of 4 seeded 5e6-point cube sets (pinned host); outputs in a pinned host ring",
                   "precision": args.precision, "m2l": "svd"},
        "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
        "latency_ms": {"p50": float(np.percentile(lat, 50)), "p90": float(np.percentile(lat, 90)),
                       "p99": float(np.percentile(lat, 99)), "max": float(lat.max()),
                       "queue_p50": float(np.percentile(times[:, 0], 50)),
                       "queue_p99": float(np.percentile(times[:, 0], 99)),
                       "service_p50": float(np.percentile(times[:, 1], 50))},
        "offered": {"requests_per_s": nreq / float(arrivals[-1]), "particles_per_s": parts / float(arrivals[-1])},
        "sustained": {"requests_per_s": nreq / span, "particles_per_s": parts / span, "span_s": span,
                      "wall_s": t_end - t0},
        "server": {"batches": int(st[1]), "mean_batch_requests": float(nreq / max(1, st[1])),
                   "largest_batch": int(st[5]), "peak_batches_at_once": int(st[4]),
                   "peak_inflight_estimate_bytes": int(st[3]), "device_bytes_held": int(st[7]),
                   "lane_time_s": {"copy_in": st[8] / 1e6, "set_batch": st[9] / 1e6,
                                   "evaluate_and_copy_out": st[10] / 1e6},
                   "lane_busy_frac": float((st[8] + st[9] + st[10]) / 1e6 / span_lanes),
                   "trims": int(st[11])},
        "check_vs_alone": check,
        "e2e": {"value": parts / span, "unit": UNIT, "h2d_bytes_per_step": int(32 * parts / nreq),
                "d2h_bytes_per_step": int(32 * parts / nreq)},
        "clocks": clk,
    }
    return result


def run_serving(args):
    import torch

    from paper_1206_0115_b300 import build
    build.build()
    from paper_1206_0115_b300 import fmm
    _, _, local = dist_env()
    torch.cuda.set_device(local)
    print(json.dumps(measure_serving(args, fmm)))


def run_kernels(args):
    """One step (fmm_set_particles + evaluation) of the 1e6-point cube (h 6,
    p 7, mixed) for each kernel: 1/r (the reference line), |x - y|^-s
    (compressed M2L), multiquadrics (c > 0: full-rank operators per level)
    and Stokes (fmm_evaluate_stokes: four 1/r passes + the direct Stokeslet
    near field).  Each: CUDA events on the library's stream, L2 flushed
    between steps, operators and SVDs built during the warm-up."""
    import numpy as np
    import torch

    from paper_1206_0115_b300 import build, inputs
    build.build()
    from paper_1206_0115_b300 import fmm

    ws, rank, local = dist_env()
    if ws > 1 and rank != 0:
        return
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = dict(inputs.WORKLOADS[WORKLOAD])
    xyz_np, q_np = inputs.particles(w["n"], w["seed"], w["dist"], w["qkind"])
    n, h, p = w["n"], w["height"], w["order"]
    f_np = np.ascontiguousarray(np.stack([inputs.charges(n, 7 + k, "sym", 0) for k in range(3)], axis=1))
    xyz = torch.from_numpy(xyz_np).to(dev)
    q = torch.from_numpy(q_np).to(dev)
    fo = torch.from_numpy(f_np).to(dev)
    phi = torch.empty(n, dtype=torch.float64, device=dev)
    F = torch.empty((n, 3), dtype=torch.float64, device=dev)
    u = torch.empty((n, 3), dtype=torch.float64, device=dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.Stream(device=dev)
    cases = [("laplace 1/r", 1.0, 0.0, fmm.FMM_M2L_SVD, False),
             ("|x-y|^-2", 2.0, 0.0, fmm.FMM_M2L_SVD, False),
             ("|x-y|^-0.5", 0.5, 0.0, fmm.FMM_M2L_SVD, False),
             ("|x-y| (s = -1)", -1.0, 0.0, fmm.FMM_M2L_SVD, False),
             ("inverse multiquadric c = 0.01", 1.0, 0.01, fmm.FMM_M2L_FULL, False),
             ("multiquadric c = 0.01", -1.0, 0.01, fmm.FMM_M2L_FULL, False),
             ("stokes", 1.0, 0.0, fmm.FMM_M2L_SVD, True)]
    out = {}
    clocks = Clocks(local)
    clocks.start()
    for name, ks, kc, m2l, stokes in cases:
        with fmm.FMM(h, p, fmm.FMM_MIXED, stream=stream, m2l=m2l, kernel_s=ks, kernel_c=kc) as hd:
            def step():
                hd.set_particles(xyz, q)
                if stokes:
                    hd.evaluate_stokes(fo, u)
                else:
                    hd.evaluate(phi, F)
            for _ in range(max(args.warmup, 1)):
                step()
            torch.cuda.synchronize()
            ms = []
            for k in range(args.steps):
                with torch.cuda.stream(stream):
                    flush.fill_(float(k))
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                step()
                b.record(stream)
                b.synchronize()
                ms.append(a.elapsed_time(b))
            t = statistics.median(ms)
            out[name] = {"ms_per_step": round(t, 4), "value": round(n / (t * 1e-3), 1),
                         "m2l": "compressed" if m2l == fmm.FMM_M2L_SVD else "full-rank per level"}
    clk = clocks.stop()
    base = out["laplace 1/r"]["ms_per_step"]
    for v in out.values():
        v["relative_to_laplace"] = round(v["ms_per_step"] / base, 3)
    print(json.dumps({"metric": "particles/s per kernel (one step: tree build + evaluation)", "unit": UNIT,
                      "higher_is_better": True, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
                      "dtype": "f32 (mixed: FP32 near field, tensor-core M2L on FP16 hi/lo operands, "
                               "outputs written as FP64)",
                      "data": "synthetic", "config": {"workload": KERNELS_WORKLOAD, "n": n, "height": h,
                                                      "order": p, "precision": "mixed", "l2": "flushed"},
                      "kernels": out, "clocks": clk}))


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == KERNELS_WORKLOAD:
        run_kernels(args)
    elif args.workload == BATCH_WORKLOAD:
        run_batched(args)
    elif args.workload == SERVE_WORKLOAD:
        run_serving(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
