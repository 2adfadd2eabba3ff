"""Full-size, converged parity of the three large configurations with the FP64
CPU oracle, through the C ABI.

The oracle needs tens of minutes per configuration at these sizes, so its
converged solutions are stored once by tests/golden/make_fullsize.py (which
calls only the oracle): the fluence at 4096 seeded voxels per group and the
full-field sum, sum of squares and maximum. Here the library's converged
fluence is compared with them:

  - 64^3 heterogeneous cone beam, FP64, all 19 groups, both sides to 1e-12:
    max error over the samples / full-field max <= 1e-10 per group, and the
    full-field sums agree to 1e-10;
  - 128^3 reduced-precision form, groups 0..4 (downscatter only, so exact
    without the later groups), every FP32 form to 1e-6: relative L2 error over
    the samples <= 1e-4 per group and over all five groups;
  - 96^3 batch of 32 sources in the benchmark's launch configuration, every
    FP32 form: sources 0 (19 groups), 8, 16 and 24 (groups 0..5), relative L2
    <= 1e-4 per (source, group) and per solve.
"""
import os

import numpy as np
import pytest

from paper_1910_11335_b300 import dts, inputs
from parity_util import TOL_FP32_L2, TOL_FP64

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
FP32_FORMS = [dts.PREC_FP32, dts.PREC_FP32_SPLITBF16, dts.PREC_FP32_TF32]
FP32_IDS = ["fp32", "splitbf16", "tf32"]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1910_11335_b300 import build
    build.build()


def load(name):
    path = os.path.join(GOLDEN, f"fullsize_{name}.npz")
    if not os.path.exists(path):
        pytest.fail(f"{path} is missing: run tests/golden/make_fullsize.py {name}")
    z = np.load(path)
    runs = []
    for i in range(int(z["n_runs"])):
        runs.append({k[len(f"r{i}_"):]: z[k] for k in z.files if k.startswith(f"r{i}_")})
    return runs


def sampled_errors(fluence, ref, key):
    """(max error / full max, sampled relative L2) per group of a [G][V] fluence."""
    idx = ref["idx"]
    a = fluence[: int(ref["n_groups"]), idx]
    b = ref[f"{key}_samples"]
    rmax = np.abs(a - b).max(axis=1) / ref[f"{key}_max"]
    rl2 = np.linalg.norm(a - b, axis=1) / np.linalg.norm(b, axis=1)
    overall = float(np.linalg.norm(a - b) / np.linalg.norm(b))
    return rmax, rl2, overall


def test_fullsize_hetero64_fp64_converged():
    (ref,) = load("hetero64")
    w = inputs.hetero_64()
    p = dts.problem_from_workload(w, precision=dts.PREC_FP64, tol=float(ref["tol"]), max_iters=5000)
    st = p.solve()
    assert st.converged == 1
    its = p.iterations()[0]
    assert np.all(np.abs(its - ref["iters"]) <= 1), (its, ref["iters"])
    for key, comp in (("collided", dts.COLLIDED), ("total", dts.TOTAL)):
        f = p.fluence(0, comp)
        rmax, _, _ = sampled_errors(f, ref, key)
        print(f"hetero64 fp64 {key}: max sampled rel-max error {rmax.max():.3e}")
        assert np.all(rmax <= TOL_FP64), rmax
        sums = f.sum(axis=1)
        assert np.all(np.abs(sums - ref[f"{key}_sum"]) <= TOL_FP64 * np.abs(ref[f"{key}_sum"]))
        assert np.allclose(np.abs(f).max(axis=1), ref[f"{key}_max"], rtol=TOL_FP64, atol=0)


@pytest.mark.parametrize("prec", FP32_FORMS, ids=FP32_IDS)
def test_fullsize_precision128(prec):
    (ref,) = load("precision128")
    G = int(ref["n_groups"])
    w = inputs.first_groups(inputs.precision_128(), G)
    p = dts.problem_from_workload(w, precision=prec, tol=1e-6, max_iters=1000, tile=(8, 4, 4))
    st = p.solve()
    assert st.converged == 1
    for key, comp in (("collided", dts.COLLIDED), ("total", dts.TOTAL)):
        f = p.fluence(0, comp)
        _, rl2, overall = sampled_errors(f, ref, key)
        print(f"precision128 prec={prec} {key}: per-group rel L2 {np.array2string(rl2, precision=2)} "
              f"overall {overall:.3e}")
        assert np.all(rl2 <= TOL_FP32_L2), rl2
        assert overall <= TOL_FP32_L2
        rel = np.abs(f.sum(axis=1) - ref[f"{key}_sum"]) / np.abs(ref[f"{key}_sum"])
        assert np.all(rel <= TOL_FP32_L2), rel


@pytest.mark.parametrize("prec", FP32_FORMS, ids=FP32_IDS)
def test_fullsize_batch96(prec):
    runs = load("batch96")
    w = inputs.batch_96()
    p = dts.problem_from_workload(w, precision=prec, tol=1e-6, max_iters=1000, tile=(8, 4, 4))
    st = p.solve()
    assert st.converged == 1 and st.sweeps > 32 * 19
    for ref in runs:
        b = int(ref["source"])
        for key, comp in (("collided", dts.COLLIDED), ("total", dts.TOTAL)):
            f = p.fluence(b, comp)
            _, rl2, overall = sampled_errors(f, ref, key)
            print(f"batch96 prec={prec} source {b} {key}: worst group rel L2 {rl2.max():.3e}, "
                  f"solve {overall:.3e}")
            assert np.all(rl2 <= TOL_FP32_L2), (b, rl2)
            assert overall <= TOL_FP32_L2
