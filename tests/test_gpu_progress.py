"""Per-iteration progress callback (dts_set_iteration_callback): one call per
source iteration with every member's residual, NaN once a member has stopped,
consistent with the final iteration counts and residuals of the solve."""
import numpy as np
import pytest

from paper_1910_11335_b300 import dts, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1910_11335_b300 import build
    build.build()


def _workload():
    w = inputs.small_cone(12, 11, 10, n_groups=2, sn_order=8, legendre_order=3, n_sources=4)
    mat = w.mat_id.reshape(-1)
    q = np.zeros((2, w.n_voxels))
    q[:, np.flatnonzero(mat == 1)[:10]] = 1.0
    w.sources[3] = inputs.Source(kind=0, q=q)   # converges at other counts than the cones
    return w


def _check_log(log, p, G, B):
    its, res = p.iterations(), p.residuals()
    for g in range(G):
        entries = [(it, r) for gg, it, r in log if gg == g]
        assert [it for it, _ in entries] == list(range(1, its[:, g].max() + 1))
        for b in range(B):
            n = its[b, g]
            assert entries[n - 1][1][b] == res[b, g]
            assert all(np.isfinite(r[b]) for _, r in entries[:n])
            assert all(np.isnan(r[b]) for _, r in entries[n:])


@pytest.mark.parametrize("prec", [dts.PREC_FP64, dts.PREC_FP32_SPLITBF16], ids=["fp64", "splitbf16"])
def test_iteration_callback(prec):
    w = _workload()
    p = dts.problem_from_workload(w, precision=prec, tol=1e-6, max_iters=300)
    log = []
    p.on_iteration(lambda g, it, r: log.append((g, it, r)))
    p.solve()
    its = p.iterations()
    assert len(set(its[:, 0])) > 1 or len(set(its[:, 1])) > 1
    _check_log(log, p, 2, 4)
    n = len(log)
    p.on_iteration(None)
    p.solve()
    assert len(log) == n


def test_iteration_callback_with_solve_many():
    import torch
    w = _workload()
    runs = dts.source_parts(4, 2, 8)
    streams = [torch.cuda.Stream() for _ in runs]
    ps = [dts.problem_from_workload(w, precision=dts.PREC_FP32, tol=1e-6, max_iters=300, sources=r,
                                    stream=s.cuda_stream) for r, s in zip(runs, streams)]
    logs = [[], []]
    for p, lg in zip(ps, logs):
        p.on_iteration(lambda g, it, r, lg=lg: lg.append((g, it, r)))
    dts.solve_many(ps)
    for p, lg, run in zip(ps, logs, runs):
        _check_log(lg, p, 2, len(run))
