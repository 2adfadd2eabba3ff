"""Failure paths, with no device fault, hang or trap: an out-of-memory device
allocation (injected on the host) turns into DTS_ERR_OOM, the failed call
releases what it had allocated, and the library keeps working afterwards; a
bounded device wait made to run out (a byte count no copy delivers) turns into
DTS_ERR_TIMEOUT after about a second, and the problem then solves correctly."""
import numpy as np
import pytest

from paper_1910_11335_b300 import dts, inputs
from parity_util import TOL_FP64, rel_max

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("after", [0, 3, 12])
def test_injected_allocation_failure_is_oom_and_leaks_nothing(ora, after):
    import torch
    w = inputs.small_cone(9, 8, 7, n_groups=2, sn_order=4, legendre_order=1)
    dts.problem_from_workload(w, tol=0.0, max_iters=2).close()   # warm the context and the library
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    dts.debug_fail_allocation(after)
    try:
        with pytest.raises(dts.DTSError) as e:
            dts.problem_from_workload(w, tol=0.0, max_iters=2)
    finally:
        dts.debug_fail_allocation(-1)
    assert e.value.status == dts.DTS_ERR_OOM
    assert "injected" in str(e.value)
    torch.cuda.synchronize()
    assert abs(torch.cuda.mem_get_info()[0] - free0) < (4 << 20)
    p = dts.problem_from_workload(w, tol=0.0, max_iters=3)   # the next call is unaffected
    p.solve()
    r = ora.solve(w, tol=0.0, max_iters=3)
    assert rel_max(p.fluence(0, dts.TOTAL), r.total) <= TOL_FP64


def test_bounded_wait_runs_out_and_the_problem_recovers():
    import time
    w = inputs.small_cone(10, 9, 8, n_groups=2, sn_order=8, legendre_order=3, n_sources=2)
    ref = dts.problem_from_workload(w, precision=dts.PREC_FP32_SPLITBF16, tol=0.0, max_iters=3)
    ref.solve(allow_not_converged=True)
    p = dts.problem_from_workload(w, precision=dts.PREC_FP32_SPLITBF16, tol=0.0, max_iters=3)
    p.debug_poison_wait(True)
    t0 = time.perf_counter()
    with pytest.raises(dts.DTSError) as e:
        p.solve()
    dt = time.perf_counter() - t0
    assert e.value.status == dts.DTS_ERR_TIMEOUT and "bounded wait" in str(e.value)
    assert dt < 30.0, dt   # each wait ends by its bound (about a second)
    p.debug_poison_wait(False)
    p.solve(allow_not_converged=True)
    for b in range(2):
        assert np.array_equal(p.fluence(b, dts.TOTAL), ref.fluence(b, dts.TOTAL))
    q = dts.problem_from_workload(w, precision=dts.PREC_FP32, tol=0.0, max_iters=1)
    with pytest.raises(dts.DTSError) as e:
        q.debug_poison_wait(True)
    assert e.value.status == dts.DTS_ERR_STATE


def test_sweep_face_wait_runs_out_and_the_problem_recovers():
    """The sweep's bounded face-copy wait made to run out (dts_debug_poison_wait on = 2): every tile's
    first wait expects 16 bytes more than its copies bring, gives up after about a second, the warp
    waits (bounded) for the copies it did issue and leaves the tile, and the solve returns
    DTS_ERR_TIMEOUT; without the hook the problem solves bit for bit as before. On an 8^3 grid of
    8x4x4 tiles the inner tiles have real y- and z-face copies in flight when their wait gives up."""
    import time
    w = inputs.small_cone(8, 8, 8, n_groups=1, sn_order=8, legendre_order=3, n_sources=2)
    ref = dts.problem_from_workload(w, precision=dts.PREC_FP32_SPLITBF16, tol=0.0, max_iters=2)
    ref.solve(allow_not_converged=True)
    p = dts.problem_from_workload(w, precision=dts.PREC_FP32_SPLITBF16, tol=0.0, max_iters=2)
    p.solve(allow_not_converged=True)   # graphs captured without the hook first
    p.debug_poison_wait(True, sweep=True)
    t0 = time.perf_counter()
    with pytest.raises(dts.DTSError) as e:
        p.solve()
    dt = time.perf_counter() - t0
    assert e.value.status == dts.DTS_ERR_TIMEOUT and "bounded wait" in str(e.value)
    assert dt < 30.0, dt
    p.debug_poison_wait(False)
    p.solve(allow_not_converged=True)
    for b in range(2):
        assert np.array_equal(p.fluence(b, dts.TOTAL), ref.fluence(b, dts.TOTAL))
    with pytest.raises(dts.DTSError) as e:
        dts._check(dts.lib().dts_debug_poison_wait(p._h, 3), p._h)
    assert e.value.status == dts.DTS_ERR_INVALID_ARG


def test_injected_failures_in_output_and_restart_setup():
    """An allocation failing halfway through dts_set_host_output (its second staging slot) or
    dts_set_initial_guess (the guess after its staging T): DTS_ERR_OOM, and the problem still
    solves as before and takes the call when it is made again."""
    w = inputs.small_cone(9, 8, 7, n_groups=2, sn_order=8, legendre_order=3, n_sources=2)
    G, V = w.n_groups, w.n_voxels
    p = dts.problem_from_workload(w, precision=dts.PREC_FP32_SPLITBF16, tol=0.0, max_iters=2)
    p.solve(allow_not_converged=True)
    ref = [p.fluence(b, dts.TOTAL) for b in range(2)]
    host = np.full(2 * G * V, np.nan)
    for call in (lambda: p.set_host_output(dts.TOTAL, host),
                 lambda: p.set_initial_guess(0, np.zeros((G, 16, V)))):
        dts.debug_fail_allocation(1)
        try:
            with pytest.raises(dts.DTSError) as e:
                call()
        finally:
            dts.debug_fail_allocation(-1)
        assert e.value.status == dts.DTS_ERR_OOM
        p.solve(allow_not_converged=True)
        for b in range(2):
            assert np.array_equal(p.fluence(b, dts.TOTAL), ref[b])
    p.set_host_output(dts.TOTAL, host)
    p.solve(allow_not_converged=True)
    for b in range(2):
        assert np.array_equal(host.reshape(2, G, V)[b], ref[b])
