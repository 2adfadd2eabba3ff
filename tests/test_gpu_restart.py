"""Restart from saved moments (dts_set_initial_guess).

A converged solve's collided moments, given back as the initial guess, make
the next solve stop after one iteration per group with the same fluence; a
member without a guess, and a cleared guess, leave the solve bit for bit as it
was; and a guess is checked against the oracle's converged fluence.
"""
import numpy as np
import pytest

from paper_1910_11335_b300 import dts, inputs
from parity_util import TOL_FP32_L2, rel_l2, rel_max

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1910_11335_b300 import build
    build.build()


def _moments(p, b, G):
    return np.stack([p.moments(b, g) for g in range(G)])   # [G][K][V]


@pytest.mark.parametrize("prec,tol,close", [(dts.PREC_FP64, 1e-9, 1e-8), (dts.PREC_FP32, 1e-6, 2e-5),
                                            (dts.PREC_FP32_SPLITBF16, 1e-6, 2e-5)],
                         ids=["fp64", "fp32", "splitbf16"])
def test_restart_from_converged_moments(prec, tol, close):
    w = inputs.small_cone(12, 11, 10, n_groups=3, sn_order=8, legendre_order=3, n_sources=4)
    G = w.n_groups
    a = dts.problem_from_workload(w, precision=prec, tol=tol, max_iters=400, keep_moments=True)
    a.solve()
    its_a = a.iterations()
    assert its_a.min() > 3
    b = dts.problem_from_workload(w, precision=prec, tol=tol, max_iters=400, keep_moments=True)
    for m in (0, 1, 2):   # member 3 keeps the default start
        b.set_initial_guess(m, _moments(a, m, G))
    b.solve()
    its_b = b.iterations()
    assert (its_b[:3] <= 2).all(), its_b
    assert np.array_equal(its_b[3], its_a[3])
    assert np.array_equal(b.fluence(3, dts.TOTAL), a.fluence(3, dts.TOTAL))
    for m in (0, 1, 2):
        fa, fb = a.fluence(m, dts.COLLIDED), b.fluence(m, dts.COLLIDED)
        for g in range(G):
            assert rel_max(fb[g], fa[g]) <= close, (m, g)
    # cleared: the solve is the default one again, bit for bit
    for m in (0, 1, 2):
        b.set_initial_guess(m, None)
    b.solve()
    assert np.array_equal(b.iterations(), its_a)
    for m in range(4):
        assert np.array_equal(b.fluence(m, dts.TOTAL), a.fluence(m, dts.TOTAL))


def test_restart_matches_oracle(ora):
    """A guess from a loosely converged solve, then tight tolerance: the oracle's converged fluence."""
    w = inputs.small_cone(10, 9, 8, n_groups=2, sn_order=4, legendre_order=1, n_sources=1)
    a = dts.problem_from_workload(w, precision=dts.PREC_FP64, tol=1e-3, max_iters=400, keep_moments=True)
    a.solve()
    b = dts.problem_from_workload(w, precision=dts.PREC_FP64, tol=1e-10, max_iters=400)
    b.set_initial_guess(0, _moments(a, 0, 2))
    b.solve()
    r = ora.solve(w, 0, tol=1e-12, max_iters=1000, n_threads=8)
    tot = b.fluence(0, dts.TOTAL)
    for g in range(2):
        assert rel_max(tot[g], r.total[g]) <= 1e-8, g


def test_restart_arguments():
    w = inputs.small_cone(8, 8, 8, n_groups=2, sn_order=4, legendre_order=1, n_sources=2)
    p = dts.problem_from_workload(w, precision=dts.PREC_FP32, tol=1e-6, max_iters=50)
    G, K, V = 2, 4, 512
    with pytest.raises(dts.DTSError) as e:
        p.set_initial_guess(0, np.zeros(G * K * V - 1))
    assert e.value.status == dts.DTS_ERR_INVALID_ARG
    bad = np.zeros((G, K, V))
    bad[1, 2, 3] = np.nan
    with pytest.raises(dts.DTSError) as e:
        p.set_initial_guess(1, bad)
    assert e.value.status == dts.DTS_ERR_INVALID_ARG
    with pytest.raises(dts.DTSError) as e:
        p.set_initial_guess(2, np.zeros((G, K, V)))
    assert e.value.status == dts.DTS_ERR_INVALID_ARG
    p.set_initial_guess(0, None)   # clearing without a guess is fine
