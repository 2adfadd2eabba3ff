"""Device-resident source iteration (dts_set_device_loop): each group's source
iterations run as one CUDA-graph launch (a WHILE node whose body is one
iteration plus a control kernel that takes the convergence decisions on the
device). The same kernels run in the same order on the same data, so every
result equals the host-driven loop's bit for bit: fluence, iteration counts,
residuals, balance terms and the solve's counts (the device loop launches one
control kernel more per iteration). Members stopping at different
iterations, the FP32 forms' stagnation stop, the iteration cap, several problems
together, the callback fallback and a bounded wait that runs out are covered;
one case is also checked against the FP64 oracle directly."""
import numpy as np
import pytest

from paper_1910_11335_b300 import dts, inputs
from parity_util import TOL_FP32_L2, TOL_FP64, rel_l2, rel_max

pytestmark = pytest.mark.gpu

FORMS = [dts.PREC_FP64, dts.PREC_FP32, dts.PREC_FP32_SPLITBF16, dts.PREC_FP32_TF32]
FORM_IDS = ["fp64", "fp32", "splitbf16", "tf32"]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1910_11335_b300 import build
    build.build()


def _mixed_workload(n_sources=7):
    """Cone sources and, on members 2, 4, 6, volumetric sources in one material each:
    the members converge at different iteration counts."""
    w = inputs.small_cone(13, 11, 9, n_groups=3, sn_order=8, legendre_order=3, n_sources=n_sources)
    rng = np.random.default_rng(4)
    mat = w.mat_id.reshape(-1)
    for b, m in zip((2, 4, 6), (0, 1, 2)):
        if b >= n_sources:
            break
        q = np.zeros((3, w.n_voxels))
        idx = np.flatnonzero(mat == m)
        q[:, rng.choice(idx, min(20, idx.size), replace=False)] = 1.0
        w.sources[b] = inputs.Source(kind=0, q=q)
    return w


def _same(a, b, B):
    """Every member's results and the solve's counts are equal bit for bit."""
    pa, sa = a
    pb, sb = b
    for f in ("updates", "sweeps", "sweep_launches", "converged", "max_residual"):
        assert getattr(sa, f) == getattr(sb, f), f
    # the device loop launches one control kernel per iteration of each group's loop
    trips = int(pa.iterations().max(axis=0).sum())
    assert sb.launches == sa.launches + trips, (sa.launches, sb.launches, trips)
    assert np.array_equal(pa.iterations(), pb.iterations())
    assert np.array_equal(pa.residuals(), pb.residuals())
    assert np.array_equal(pa.balance(), pb.balance())
    for k in range(B):
        assert np.array_equal(pa.fluence(k, dts.TOTAL), pb.fluence(k, dts.TOTAL)), k
        assert np.array_equal(pa.fluence(k, dts.COLLIDED), pb.fluence(k, dts.COLLIDED)), k


def _pair(w, prec, tol, max_iters, **kw):
    host = dts.problem_from_workload(w, precision=prec, tol=tol, max_iters=max_iters, tile=(8, 4, 4), **kw)
    dev = dts.problem_from_workload(w, precision=prec, tol=tol, max_iters=max_iters, tile=(8, 4, 4),
                                    device_loop=True, **kw)
    sh = host.solve(allow_not_converged=True)
    sd = dev.solve(allow_not_converged=True)
    return (host, sh), (dev, sd)


@pytest.mark.parametrize("prec", FORMS, ids=FORM_IDS)
def test_device_loop_equals_host_loop(prec):
    """Converged solves whose members stop at different iterations."""
    w = _mixed_workload()
    tol = 1e-8 if prec == dts.PREC_FP64 else 1e-6
    h, d = _pair(w, prec, tol, 300)
    it = h[0].iterations()
    assert len(set(it[:, 0])) > 1 or len(set(it[:, 1])) > 1   # members stop at different counts
    _same(h, d, len(w.sources))
    assert d[1].sweep_ms == 0.0 and d[1].reduce_ms == 0.0 and h[1].sweep_ms > 0.0
    # a second solve of the same problem (the loop graph and its state are reused)
    d2 = d[0].solve(allow_not_converged=True)
    _same(h, (d[0], d2), len(w.sources))


@pytest.mark.parametrize("prec", [dts.PREC_FP32, dts.PREC_FP32_SPLITBF16], ids=["fp32", "splitbf16"])
def test_device_loop_stagnation_stop(prec):
    """A tol below the FP32 forms' rounding floor: members stop when their residual has not
    improved by 1 % in 10 iterations, at the same iteration as on the host."""
    w = _mixed_workload(4)
    h, d = _pair(w, prec, 1e-12, 400)
    assert (h[0].iterations() < 400).any()   # the stagnation stop fired
    assert h[1].converged == 0
    _same(h, d, 4)


def test_device_loop_iteration_cap():
    """tol = 0: every member runs exactly max_iters iterations in every group."""
    w = _mixed_workload(3)
    h, d = _pair(w, dts.PREC_FP32_SPLITBF16, 0.0, 5)
    assert (d[0].iterations() == 5).all()
    _same(h, d, 3)


def test_device_loop_vs_oracle(ora):
    """FP64, ragged tiles, S4 P1, 3 groups at equal iteration counts: the device loop's result
    against the oracle (1e-10 relative max per group)."""
    w = inputs.small_cone(13, 11, 9, n_groups=3, sn_order=4, legendre_order=1)
    p = dts.problem_from_workload(w, precision=dts.PREC_FP64, tol=0.0, max_iters=4, device_loop=True)
    st = p.solve(allow_not_converged=True)
    assert st.sweeps == 3 * 4
    r = ora.solve(w, 0, tol=0.0, max_iters=4, n_threads=8)
    got = p.fluence(0, dts.TOTAL)
    for g in range(w.n_groups):
        assert rel_max(got[g], r.total[g]) <= TOL_FP64, g
    q = dts.problem_from_workload(w, precision=dts.PREC_FP32_SPLITBF16, tol=0.0, max_iters=4, device_loop=True)
    q.solve(allow_not_converged=True)
    got = q.fluence(0, dts.TOTAL)
    for g in range(w.n_groups):
        assert rel_l2(got[g], r.total[g]) <= TOL_FP32_L2, g


def test_device_loop_solve_many_mixed():
    """Three parts solved together, two with the device loop and one with the host loop: each
    equals the one-batch host-loop solve of the same sources."""
    import torch
    w = _mixed_workload()
    prec = dts.PREC_FP32_SPLITBF16
    one = dts.problem_from_workload(w, precision=prec, tol=1e-6, max_iters=300, tile=(8, 4, 4))
    st1 = one.solve(allow_not_converged=True)
    runs = dts.source_parts(7, 3, 8)
    streams = [torch.cuda.Stream() for _ in runs]
    ps = [dts.problem_from_workload(w, precision=prec, tol=1e-6, max_iters=300, tile=(8, 4, 4),
                                    stream=s.cuda_stream, sources=r, device_loop=(i != 1))
          for i, (r, s) in enumerate(zip(runs, streams))]
    sts = dts.solve_many(ps, allow_not_converged=True)
    assert sum(s.updates for s in sts) == st1.updates
    assert sum(s.sweeps for s in sts) == st1.sweeps
    it1, res1, bal1 = one.iterations(), one.residuals(), one.balance()
    for p, run in zip(ps, runs):
        its, res, bal = p.iterations(), p.residuals(), p.balance()
        for b, k in enumerate(run):
            assert np.array_equal(p.fluence(b, dts.TOTAL), one.fluence(k, dts.TOTAL)), k
            assert np.array_equal(its[b], it1[k]) and np.array_equal(res[b], res1[k]), k
            assert np.array_equal(bal[b], bal1[k]), k


def test_device_loop_streamed_output_and_callback_fallback():
    """The streamed output works with the device loop; a problem with an iteration callback keeps
    the host loop (the callback is called, and the phase timings are measured)."""
    w = _mixed_workload(3)
    G, V = w.n_groups, w.n_voxels
    h, d = _pair(w, dts.PREC_FP32_SPLITBF16, 1e-6, 200)
    host = np.full(3 * G * V, np.nan)
    d[0].set_host_output(dts.TOTAL, host)
    d[0].solve(allow_not_converged=True)
    host = host.reshape(3, G, V)
    for b in range(3):
        assert np.array_equal(host[b], h[0].fluence(b, dts.TOTAL))
    seen = []
    d[0].on_iteration(lambda g, it, res: seen.append((g, it)))
    st = d[0].solve(allow_not_converged=True)
    assert len(seen) == int(h[0].iterations().max(axis=0).sum()) and st.sweep_ms > 0.0
    d[0].on_iteration(None)
    st = d[0].solve(allow_not_converged=True)
    assert st.sweep_ms == 0.0
    for b in range(3):
        assert np.array_equal(d[0].fluence(b, dts.TOTAL), h[0].fluence(b, dts.TOTAL))
    d[0].set_device_loop(False)   # back to the host loop
    st = d[0].solve(allow_not_converged=True)
    assert st.sweep_ms > 0.0


def test_device_loop_bounded_wait_runs_out():
    """A bounded wait of the tensor-core moment kernel made to run out: the loop stops at the
    iteration that met it, the solve returns DTS_ERR_TIMEOUT, and the problem then solves as before."""
    import time
    w = inputs.small_cone(10, 9, 8, n_groups=2, sn_order=8, legendre_order=3, n_sources=2)
    ref = dts.problem_from_workload(w, precision=dts.PREC_FP32_SPLITBF16, tol=0.0, max_iters=3)
    ref.solve(allow_not_converged=True)
    p = dts.problem_from_workload(w, precision=dts.PREC_FP32_SPLITBF16, tol=0.0, max_iters=3, device_loop=True)
    p.debug_poison_wait(True)
    t0 = time.perf_counter()
    with pytest.raises(dts.DTSError) as e:
        p.solve()
    dt = time.perf_counter() - t0
    assert e.value.status == dts.DTS_ERR_TIMEOUT and "bounded wait" in str(e.value)
    assert dt < 30.0, dt
    assert (p.iterations() == 1).all()   # each group's loop stopped after its first iteration
    p.debug_poison_wait(False)
    p.solve(allow_not_converged=True)
    for b in range(2):
        assert np.array_equal(p.fluence(b, dts.TOTAL), ref.fluence(b, dts.TOTAL))


@pytest.mark.parametrize("prec", [dts.PREC_FP64, dts.PREC_FP32_SPLITBF16], ids=["fp64", "splitbf16"])
def test_device_loop_restart_from_saved_moments(prec):
    """An initial guess (dts_set_initial_guess) on some members: the device loop starts from it as the
    host loop does (same counts, residuals and fluence bit for bit), and a converged guess stops after
    at most two iterations per group."""
    w = _mixed_workload(4)
    G = w.n_groups
    tol = 1e-8 if prec == dts.PREC_FP64 else 1e-6
    a = dts.problem_from_workload(w, precision=prec, tol=tol, max_iters=300, tile=(8, 4, 4), keep_moments=True)
    a.solve(allow_not_converged=True)
    guess = {m: np.stack([a.moments(m, g) for g in range(G)]) for m in (0, 2)}
    h, d = _pair(w, prec, tol, 300, keep_moments=True)   # default starts first
    for p, _ in (h, d):
        for m, mom in guess.items():
            p.set_initial_guess(m, mom)
    sh = h[0].solve(allow_not_converged=True)
    sd = d[0].solve(allow_not_converged=True)
    _same((h[0], sh), (d[0], sd), 4)
    assert (d[0].iterations()[[0, 2]] <= 2).all()
