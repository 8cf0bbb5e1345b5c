"""The bounds-checked build (libll_check.so, -DLL_CHECK): every index a kernel takes from a
sphere or map table is tested before its access, and an index out of its table's range is
reported as LL_EINVAL after the call.  Run through each kernel path (fused and split per-k
work, plane pass on single lanes and on lane pairs, both recursions, both precisions, the
symmetric wedge, a metal), it finds no such index and gives the coefficients of the plain
build."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (name, config, precision, flavour, steps, environment)
CASES = [
    ("small_fp64_ph", "small", "fp64", "ph", 40, {}),
    ("small_fp32_nh", "small", "fp32", "nh", 20, {}),
    ("small_split_fp32", "small", "fp32", "ph", 20, {"LL_SPLIT_PERK": "1"}),
    ("small_split_fp64_nh", "small", "fp64", "nh", 10, {"LL_SPLIT_PERK": "1"}),
    ("small_lane_pairs", "small", "fp32", "ph", 20, {"LL_XY_PAIR": "1", "LL_TUNE": "0"}),
    ("wedge_fp32", "small_ibz", "fp32", "ph", 20, {}),
    ("kb_fp32", "kb", "fp32", "ph", 10, {}),
    ("metal_fp32_nh", "metal", "fp32", "nh", 20, {}),
    ("metal_fp64_ph", "metal", "fp64", "ph", 40, {}),
    ("metal_split_fp32_nh", "metal", "fp32", "nh", 20, {"LL_SPLIT_PERK": "1"}),
]

SCRIPT = r"""
import json, sys
import numpy as np
sys.path.insert(0, {root!r})
import workloads as w
from tests.helpers import chain_from_bundle
cfg, prec, flav, n = {cfg!r}, {prec!r}, {flav!r}, {n}
spec = {{"small": w.config_small, "kb": w.config_kb, "metal": w.config_metal,
         "small_ibz": lambda: w.config_small(True)}}[cfg]()
ch = chain_from_bundle(w.get_bundle(spec), precision=prec, flavour=flav, max_steps=n)
b, g, z = ch.lanczos(n)
print(json.dumps({{"beta": list(map(float, b)), "z": [[float(c.real), float(c.imag)] for c in z]}}))
"""


def _run(lib_path, cfg, prec, flav, n, env_extra):
    env = dict(os.environ, **env_extra)
    if lib_path:
        env["LL_LIBRARY"] = lib_path
    else:
        env.pop("LL_LIBRARY", None)
    code = SCRIPT.format(root=ROOT, cfg=cfg, prec=prec, flav=flav, n=n)
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


@pytest.fixture(scope="module")
def check_lib():
    from paper_2111_06623_gb300.build import build_library
    build_library()
    return build_library(check=True)


@pytest.mark.parametrize("name,cfg,prec,flav,n,env", CASES, ids=[c[0] for c in CASES])
def test_checked_build_finds_no_out_of_range_index(check_lib, name, cfg, prec, flav, n, env):
    got = _run(check_lib, cfg, prec, flav, n, env)        # raises on LL_EINVAL (an index out of range)
    want = _run(None, cfg, prec, flav, n, env)
    tol = 1e-12 if prec == "fp64" else 1e-5
    b0, b1 = np.array(got["beta"]), np.array(want["beta"])
    assert np.max(np.abs(b0 - b1) / np.abs(b1)) < tol
    z0, z1 = np.array(got["z"]), np.array(want["z"])
    assert np.max(np.abs(z0 - z1)) <= tol * np.max(np.abs(z1))
