"""The bounds-checking build (libfmm_b300_debug.so, compiled with FMM_DEBUG):
on a cube, a surface and a batch, every near-field shape and both M2L
operand forms run without a failed check, and the results are the same bits
as the normal build's (the checks guard accesses, they change no
arithmetic).  The debug library runs in a child process (FMM_LIBRARY=debug);
this process runs the normal one."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle
from paper_1206_0115_b300 import inputs

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# Evaluates the cases of CASES with the library the environment selects and
# writes every output to OUT (npz); with TUNE, first runs fmm_autotune on each
# mixed case (every near-field shape is launched) and records
# fmm_debug_check after all of it.
CHILD = r"""
import json, os, sys
import numpy as np
import torch
sys.path.insert(0, os.environ["ROOT"])
from paper_1206_0115_b300 import fmm, inputs
cases = json.loads(os.environ["CASES"])
res, tuned = {}, 0
for name, c in cases.items():
    if c["kind"] == "batch":
        probs = [inputs.particles(n, s, d, "pos") for n, s, d in zip(c["n"], c["seeds"], c["dist"])]
        xyz = np.concatenate([p[0] for p in probs]); q = np.concatenate([p[1] for p in probs])
    else:
        xyz, q = inputs.particles(c["n"], c["seed"], c["dist"], "sym")
    n = len(q)
    prec = fmm.FMM_MIXED if c["precision"] == "mixed" else fmm.FMM_FP64
    with fmm.FMM(c["h"], c["p"], prec) as f:
        if c["kind"] == "batch":
            f.set_batch(np.array(c["n"], dtype=np.int64), np.array(c["heights"], dtype=np.int32),
                        torch.from_numpy(xyz).cuda(), torch.from_numpy(q).cuda())
        else:
            f.set_particles(torch.from_numpy(xyz).cuda(), torch.from_numpy(q).cuda())
        if prec == fmm.FMM_MIXED:
            if os.environ.get("TUNE") == "1":
                fmm.fmm_autotune(f.h)
                tuned += 1
            fmm.fmm_set_p2p_variant(f.h, c.get("variant", 0))
            fmm.fmm_set_schedule(f.h, 0)
        phi = torch.zeros(n, dtype=torch.float64, device="cuda")
        F = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
        f.evaluate(phi, F)
        torch.cuda.synchronize()
        res[name + "_phi"] = phi.cpu().numpy(); res[name + "_F"] = F.cpu().numpy()
np.savez(os.environ["OUT"], **res)
print(json.dumps({"debug_build": fmm.fmm_debug_build(), "first_failure": fmm.fmm_debug_check(), "tuned": tuned}))
"""

CASES = {
    "cube_mixed": dict(kind="single", n=20000, seed=7, dist="cube", h=4, p=5, precision="mixed"),
    "cube_mixed_p7": dict(kind="single", n=60000, seed=8, dist="cube", h=5, p=7, precision="mixed", variant=14),
    "cube_fp64": dict(kind="single", n=20000, seed=7, dist="cube", h=4, p=5, precision="fp64"),
    "surface_mixed": dict(kind="single", n=80000, seed=9, dist="ellipsoid", h=5, p=5, precision="mixed",
                          variant=12),
    "batch_mixed": dict(kind="batch", n=[3000, 20000, 9000], seeds=[11, 12, 13],
                        dist=["cube", "ellipsoid", "cube"], heights=[3, 4, 3], h=4, p=5, precision="mixed"),
}


def _run(tmp_path, lib: str, tune: bool):
    out = str(tmp_path / f"{lib}.npz")
    env = dict(os.environ, ROOT=ROOT, CASES=json.dumps(CASES), OUT=out, TUNE="1" if tune else "0")
    if lib == "debug":
        env["FMM_LIBRARY"] = "debug"
    else:
        env.pop("FMM_LIBRARY", None)
    r = subprocess.run([sys.executable, "-c", CHILD], env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    return json.loads(r.stdout.strip().splitlines()[-1]), dict(np.load(out))


@pytest.fixture(scope="module")
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1206_0115_b300 import build
    build.build()
    build.build(debug=True)


def test_debug_build_checks_pass_and_match_the_normal_build(built, tmp_path):
    info, dbg = _run(tmp_path, "debug", tune=True)
    assert info["debug_build"] is True and info["tuned"] == 4
    assert info["first_failure"] == 0, hex(info["first_failure"])
    info_n, ref = _run(tmp_path, "normal", tune=False)
    assert info_n["debug_build"] is False and info_n["first_failure"] == 0
    for k in ref:
        assert np.array_equal(ref[k], dbg[k]), k
    # and the results are the method's (the oracle's FMM, same operators)
    c = CASES["cube_mixed"]
    xyz, q = inputs.particles(c["n"], c["seed"], c["dist"], "sym")
    with oracle.OracleFMM(xyz, q, c["h"], c["p"], svd_eps=10.0 ** -c["p"]) as o:
        rphi, rF = o.evaluate()
    assert oracle.rel_l2(dbg["cube_mixed_phi"], rphi) <= 1e-5
    assert oracle.rel_l2(dbg["cube_mixed_F"], rF) <= 1e-5
    assert oracle.rel_l2(dbg["cube_fp64_phi"], rphi) <= 1e-10
