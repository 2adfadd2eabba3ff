"""dts_solve_many: several problems (disjoint source sets of one scan, each on
its own stream) solved together, one problem's moment kernels running beside
another's sweep. Each problem's work is that of dts_solve on it alone, and a
source's arithmetic does not depend on the batch it sits in, so the results
equal a one-batch solve of all the sources bit for bit; the parts are also
checked against the FP64 oracle.
"""
import numpy as np
import pytest

from paper_1910_11335_b300 import dts, inputs
from parity_util import TOL_FP32_L2, rel_l2, rel_max

pytestmark = pytest.mark.gpu

FORMS = [dts.PREC_FP64, dts.PREC_FP32, dts.PREC_FP32_SPLITBF16, dts.PREC_FP32_TF32]
FORM_IDS = ["fp64", "fp32", "splitbf16", "tf32"]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1910_11335_b300 import build
    build.build()


def _parts(w, prec, runs, tol, max_iters, same_stream=False):
    import torch
    streams = [torch.cuda.Stream() for _ in runs]
    if same_stream:
        streams = [streams[0]] * len(runs)
    ps = [dts.problem_from_workload(w, precision=prec, tol=tol, max_iters=max_iters, tile=(8, 4, 4),
                                    stream=s.cuda_stream, sources=r) for r, s in zip(runs, streams)]
    return ps, streams


def _tol(prec):
    return 1e-8 if prec == dts.PREC_FP64 else 1e-6


@pytest.mark.parametrize("prec", FORMS, ids=FORM_IDS)
def test_solve_many_equals_one_batch(prec):
    """Converged solves (sources stop at different iterations): fluence, iteration
    counts, residuals and balance of every source equal the one-batch solve's."""
    w = inputs.small_cone(13, 11, 9, n_groups=3, sn_order=8, legendre_order=3, n_sources=7)
    # members 2, 4 and 6: volumetric sources in one material each (they converge at other counts)
    rng = np.random.default_rng(4)
    mat = w.mat_id.reshape(-1)
    for b, m in zip((2, 4, 6), (0, 1, 2)):
        q = np.zeros((3, w.n_voxels))
        idx = np.flatnonzero(mat == m)
        q[:, rng.choice(idx, min(20, idx.size), replace=False)] = 1.0
        w.sources[b] = inputs.Source(kind=0, q=q)
    one = dts.problem_from_workload(w, precision=prec, tol=_tol(prec), max_iters=300, tile=(8, 4, 4))
    st1 = one.solve(allow_not_converged=True)
    runs = dts.source_parts(7, 2, 8)
    assert [len(r) for r in runs] == [3, 4]
    ps, _streams = _parts(w, prec, runs, _tol(prec), 300)
    sts = dts.solve_many(ps, allow_not_converged=True)
    assert sum(s.updates for s in sts) == st1.updates
    assert sum(s.sweeps for s in sts) == st1.sweeps
    it1, res1, bal1 = one.iterations(), one.residuals(), one.balance()
    assert len(set(it1[:, 0])) > 1 or len(set(it1[:, 1])) > 1   # members stop at different counts
    for p, run in zip(ps, runs):
        its, res, bal = p.iterations(), p.residuals(), p.balance()
        for b, k in enumerate(run):
            assert np.array_equal(p.fluence(b, dts.TOTAL), one.fluence(k, dts.TOTAL)), k
            assert np.array_equal(its[b], it1[k]) and np.array_equal(res[b], res1[k]), k
            assert np.array_equal(bal[b], bal1[k]), k


@pytest.mark.parametrize("prec", [dts.PREC_FP64, dts.PREC_FP32_SPLITBF16], ids=["fp64", "splitbf16"])
def test_solve_many_parts_vs_oracle(ora, prec):
    """Three parts (ragged grid, S8 P3) at fixed iteration counts against the oracle."""
    w = inputs.small_cone(10, 9, 17, n_groups=2, sn_order=8, legendre_order=3, n_sources=8)
    runs = dts.source_parts(8, 3, 8)
    assert len(runs) == 3
    ps, _streams = _parts(w, prec, runs, 0.0, 4)
    sts = dts.solve_many(ps, allow_not_converged=True)
    assert all(s.sweeps == len(r) * 2 * 4 for s, r in zip(sts, runs))
    for p, run in zip(ps, runs):
        b = len(run) - 1
        r = ora.solve(w, run[b], tol=0.0, max_iters=4, n_threads=8)
        got = p.fluence(b, dts.COLLIDED)
        for g in range(w.n_groups):
            if prec == dts.PREC_FP64:
                assert rel_max(got[g], r.collided[g]) <= 1e-10, (run[b], g)
            else:
                assert rel_l2(got[g], r.collided[g]) <= TOL_FP32_L2, (run[b], g)


def test_solve_many_one_stream_and_one_problem():
    """Problems sharing one stream (no overlap) and a single problem give the same results."""
    w = inputs.small_cone(9, 8, 8, n_groups=2, sn_order=8, legendre_order=3, n_sources=4)
    one = dts.problem_from_workload(w, precision=dts.PREC_FP32_SPLITBF16, tol=1e-6, max_iters=200,
                                    tile=(8, 4, 4))
    one.solve(allow_not_converged=True)
    runs = dts.source_parts(4, 2, 8)
    ps, _streams = _parts(w, dts.PREC_FP32_SPLITBF16, runs, 1e-6, 200, same_stream=True)
    dts.solve_many(ps, allow_not_converged=True)
    for p, run in zip(ps, runs):
        for b, k in enumerate(run):
            assert np.array_equal(p.fluence(b, dts.TOTAL), one.fluence(k, dts.TOTAL))
    (st,) = dts.solve_many([one], allow_not_converged=True)
    assert st.sweeps > 0


def test_solve_many_not_converged_finishes_every_problem():
    """One part capped below convergence: DTS_ERR_NOT_CONVERGED after every part finished."""
    w = inputs.small_cone(9, 8, 8, n_groups=2, sn_order=8, legendre_order=3, n_sources=6)
    runs = dts.source_parts(6, 2, 8)
    ps, _streams = _parts(w, dts.PREC_FP32, runs, 1e-6, 300)
    capped = dts.problem_from_workload(w, precision=dts.PREC_FP32, tol=1e-6, max_iters=2, tile=(8, 4, 4),
                                       sources=runs[1])
    with pytest.raises(dts.DTSError) as e:
        dts.solve_many([ps[0], capped])
    assert e.value.status == dts.DTS_ERR_NOT_CONVERGED
    sts = dts.solve_many([ps[0], capped], allow_not_converged=True)
    assert sts[0].converged == 1 and sts[1].converged == 0
    assert (capped.iterations() == 2).all()
    ref = dts.problem_from_workload(w, precision=dts.PREC_FP32, tol=1e-6, max_iters=300, tile=(8, 4, 4),
                                    sources=runs[0])
    ref.solve()
    for b in range(len(runs[0])):
        assert np.array_equal(ps[0].fluence(b, dts.TOTAL), ref.fluence(b, dts.TOTAL))


def test_solve_many_argument_errors():
    w = inputs.small_cone(8, 8, 8, n_groups=1, sn_order=4, legendre_order=1, n_sources=2)
    p = dts.problem_from_workload(w, precision=dts.PREC_FP32, tol=1e-6, max_iters=50)
    with pytest.raises(dts.DTSError) as e:
        dts.solve_many([p, p])
    assert e.value.status == dts.DTS_ERR_INVALID_ARG and "twice" in str(e.value)
    with pytest.raises(dts.DTSError) as e:
        dts.solve_many([])
    assert e.value.status == dts.DTS_ERR_INVALID_ARG
    q = dts.Problem(nx=8, ny=8, nz=8, dx=1.0, dy=1.0, dz=1.0, n_groups=1, sn_order=4, legendre_order=1,
                    batch=1, precision=dts.PREC_FP32)
    with pytest.raises(dts.DTSError) as e:
        dts.solve_many([p, q])
    assert e.value.status == dts.DTS_ERR_STATE
