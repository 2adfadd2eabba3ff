"""Streamed output (dts_set_host_output): each group's fluence copied to host
memory on a second stream while the later groups solve. The host arrays equal
dts_get_scalar_fluence bit for bit, for every component, in page-locked and
pageable memory, one problem or several solved together."""
import numpy as np
import pytest

from paper_1910_11335_b300 import dts, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1910_11335_b300 import build
    build.build()


def _pinned(n):
    import torch
    return torch.empty(n, dtype=torch.float64).pin_memory().numpy()


@pytest.mark.parametrize("prec", [dts.PREC_FP64, dts.PREC_FP32, dts.PREC_FP32_SPLITBF16],
                         ids=["fp64", "fp32", "splitbf16"])
def test_streamed_output_equals_the_getter(prec):
    w = inputs.small_cone(12, 11, 10, n_groups=4, sn_order=8, legendre_order=3, n_sources=3)
    G, V, B = w.n_groups, w.n_voxels, w.batch
    p = dts.problem_from_workload(w, precision=prec, tol=1e-6, max_iters=200)
    for comp, pinned in ((dts.TOTAL, True), (dts.COLLIDED, False), (dts.UNCOLLIDED, True)):
        host = _pinned(B * G * V) if pinned else np.empty(B * G * V)
        host[:] = np.nan
        p.set_host_output(comp, host)
        p.solve()
        got = host.reshape(B, G, V)
        for b in range(B):
            assert np.array_equal(got[b], p.fluence(b, comp)), (comp, b)
    # off: a later solve leaves the array alone
    p.set_host_output(dts.TOTAL, None)
    host[:] = np.nan
    p.solve()
    assert np.isnan(host).all()


def test_streamed_output_with_solve_many():
    import torch
    w = inputs.small_cone(11, 10, 9, n_groups=3, sn_order=8, legendre_order=3, n_sources=6)
    G, V = w.n_groups, w.n_voxels
    one = dts.problem_from_workload(w, precision=dts.PREC_FP32_SPLITBF16, tol=1e-6, max_iters=200,
                                    tile=(8, 4, 4))
    one.solve()
    runs = dts.source_parts(6, 2, 8)
    streams = [torch.cuda.Stream() for _ in runs]
    ps = [dts.problem_from_workload(w, precision=dts.PREC_FP32_SPLITBF16, tol=1e-6, max_iters=200,
                                    tile=(8, 4, 4), stream=s.cuda_stream, sources=r) for r, s in zip(runs, streams)]
    hosts = [_pinned(len(r) * G * V) for r in runs]
    for p, h in zip(ps, hosts):
        p.set_host_output(dts.TOTAL, h)
    for _ in range(2):   # the staging slots are reused across solves
        for h in hosts:
            h[:] = np.nan
        dts.solve_many(ps)
        for run, h in zip(runs, hosts):
            got = h.reshape(len(run), G, V)
            for b, k in enumerate(run):
                assert np.array_equal(got[b], one.fluence(k, dts.TOTAL)), k


def test_streamed_output_arguments():
    w = inputs.small_cone(8, 8, 8, n_groups=2, sn_order=4, legendre_order=1, n_sources=2)
    p = dts.problem_from_workload(w, precision=dts.PREC_FP32, tol=1e-6, max_iters=50)
    with pytest.raises(dts.DTSError) as e:
        p.set_host_output(dts.TOTAL, np.empty(2 * 2 * 512 - 1))
    assert e.value.status == dts.DTS_ERR_INVALID_ARG
    with pytest.raises(dts.DTSError) as e:
        p.set_host_output(7, np.empty(2 * 2 * 512))
    assert e.value.status == dts.DTS_ERR_INVALID_ARG
    with pytest.raises(ValueError):
        p.set_host_output(dts.TOTAL, np.empty(2 * 2 * 512, dtype=np.float32))
