"""The DTS_DEBUG_BOUNDS build (libdts_debug.so, loaded with DTS_DEBUG_BOUNDS=1).

A child process runs the bounds-checked library: its self-test shows that a
failed check comes back as DTS_ERR_INTERNAL (the check touches no memory), and
solves of every form on ragged grids pass every check, with fluences equal to
the normal build's bit for bit (the checks only skip accesses that fail).
"""
import json
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest

from paper_1910_11335_b300 import dts, inputs

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# name, precision, grid, S_N, P_L, batch: every sweep and moment kernel the checks cover
CASES = [
    ("splitbf16_s8", dts.PREC_FP32_SPLITBF16, (13, 11, 9), 8, 3, 4),
    ("tf32_s6", dts.PREC_FP32_TF32, (10, 9, 17), 6, 1, 5),
    ("splitbf16_s4", dts.PREC_FP32_SPLITBF16, (9, 14, 6), 4, 2, 11),
    ("fp32_batched", dts.PREC_FP32, (13, 11, 9), 8, 3, 7),
    ("fp32_single", dts.PREC_FP32, (9, 8, 10), 8, 3, 1),
    ("fp64", dts.PREC_FP64, (9, 8, 10), 4, 1, 2),
]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1910_11335_b300 import build
    build.build()
    build.build(debug_bounds=True)


def _solve(prec, dims, N, L, B):
    w = inputs.small_cone(*dims, n_groups=2, sn_order=N, legendre_order=L, n_sources=B)
    p = dts.problem_from_workload(w, precision=prec, tol=0.0, max_iters=3)
    p.solve(allow_not_converged=True)
    return np.stack([p.fluence(b, dts.TOTAL) for b in range(B)])


def test_debug_bounds_build(tmp_path):
    child = textwrap.dedent(f"""
        import json, sys
        import numpy as np
        sys.path.insert(0, {ROOT!r})
        sys.path.insert(0, {os.path.join(ROOT, 'tests')!r})
        from paper_1910_11335_b300 import dts
        from test_gpu_debug_bounds import CASES, _solve
        assert dts.DEBUG_BOUNDS and dts.LIB_PATH.endswith("libdts_debug.so")
        out = {{"clean": dts.debug_bounds_selftest(False), "planted": dts.debug_bounds_selftest(True)}}
        for name, prec, dims, N, L, B in CASES:
            np.save({str(tmp_path)!r} + "/" + name + ".npy", _solve(prec, dims, N, L, B))
        print(json.dumps(out))
    """)
    env = {**os.environ, "DTS_DEBUG_BOUNDS": "1"}
    r = subprocess.run([sys.executable, "-c", child], env=env, capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0, r.stderr[-3000:]
    out = json.loads(r.stdout.strip().splitlines()[-1])
    assert out["clean"][:2] == [True, dts.DTS_OK]
    is_dbg, status, msg = out["planted"]
    assert is_dbg and status == dts.DTS_ERR_INTERNAL and "bounds check failed" in msg and "site 63" in msg
    assert not dts.DEBUG_BOUNDS
    assert dts.debug_bounds_selftest(True)[:2] == (False, dts.DTS_OK)   # the normal build has no checks
    for name, prec, dims, N, L, B in CASES:
        ref = _solve(prec, dims, N, L, B)
        got = np.load(tmp_path / (name + ".npy"))
        assert np.array_equal(got, ref), name
