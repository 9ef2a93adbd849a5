"""The multi-core build of the oracle (the same C source compiled with OpenMP,
used only to time the CPU baseline) computes what the single-threaded build the
tests pin computes: only the order of its FP64 sums differs.  Each build runs
in a child process of its own (the wrapper loads one library per process)."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, sys
import numpy as np
sys.path.insert(0, %(root)r)
import oracle
rng = np.random.default_rng(5)
dims = [60, 45, 30]
nnz = 4000
flat = rng.choice(dims[0] * dims[1] * dims[2], size=nnz, replace=False)
i, rem = np.divmod(flat, dims[1] * dims[2])
j, k = np.divmod(rem, dims[2])
idx = np.stack([i, j, k]).astype(np.int32)
val = rng.random(nnz).astype(np.float32)
R = 6
F = [rng.standard_normal((d, R)) for d in dims]
t = oracle.Tensor(idx, val, dims)
out = {"mttkrp": [oracle.mttkrp(t, m, F).tolist() for m in range(3)]}
st, Fa, lam, fit = oracle.als_sweep(t, F)
out["als"] = [f.tolist() for f in Fa] + [list(lam), fit, st]
st, Fg, alpha, loss, _ = oracle.gd_step(t, F, 0.1)
out["gd"] = [f.tolist() for f in Fg] + [alpha, loss, st]
print(json.dumps(out))
"""


def run_build(lib, threads):
    env = dict(os.environ, DFACTO_ORACLE_LIB=lib, OMP_NUM_THREADS=str(threads))
    res = subprocess.run([sys.executable, "-c", CHILD % {"root": ROOT}], env=env,
                         capture_output=True, text=True, timeout=300, check=True)
    return json.loads(res.stdout.strip().splitlines()[-1])


def rel(a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def test_openmp_build_matches_single_threaded_build():
    sys.path.insert(0, ROOT)
    import oracle
    single = oracle.build()
    try:
        multi = oracle.build(openmp=True)
    except Exception as e:  # pragma: no cover - a toolchain without OpenMP
        pytest.skip("no OpenMP build: %s" % e)
    a = run_build(single, 1)
    b = run_build(multi, 4)
    for m in range(3):
        assert rel(b["mttkrp"][m], a["mttkrp"][m]) <= 1e-13, m
    for m in range(3):
        assert rel(b["als"][m], a["als"][m]) <= 1e-10, m
    assert rel(b["als"][3], a["als"][3]) <= 1e-10
    assert abs(b["als"][4] - a["als"][4]) <= 1e-12 and b["als"][5] == a["als"][5]
    # the accepted step is the same; the factors and objective agree to rounding
    assert b["gd"][3] == a["gd"][3] and b["gd"][5] == a["gd"][5]
    for m in range(3):
        assert rel(b["gd"][m], a["gd"][m]) <= 1e-12, m
    assert abs(b["gd"][4] - a["gd"][4]) <= 1e-12 * abs(a["gd"][4])
