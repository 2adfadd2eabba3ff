"""Several cone beams summed into one source (dts_set_source_cones): against
the oracle's combined source, by linearity against single-cone GPU solves, in
an FP32 batch next to ordinary members, and its error paths."""
import copy

import numpy as np
import pytest

from paper_1910_11335_b300 import dts, inputs
from parity_util import TOL_FP32_L2, TOL_FP64, rel_l2, rel_max

pytestmark = pytest.mark.gpu


def test_combined_cones_fp64_vs_oracle(ora):
    base = inputs.small_cone(9, 8, 7, n_groups=3, sn_order=4, legendre_order=2)
    w = inputs.combined_cones(base, n_cones=4)
    r = ora.solve(w, 0, tol=0.0, max_iters=5, n_threads=8)
    p = dts.problem_from_workload(w, tol=0.0, max_iters=5, keep_moments=True)
    p.solve(allow_not_converged=True)
    assert rel_max(p.fluence(0, dts.UNCOLLIDED), r.phi_u) <= 1e-13
    for g in range(w.n_groups):
        m = p.moments(0, g)
        for k in range(m.shape[0]):
            assert rel_max(m[k], r.phi_c[g, k]) <= TOL_FP64, (g, k)


def test_combined_cones_uncollided_is_the_sum():
    """Eq. 4 is linear in the source: the combined uncollided fluence is the sum
    of the single-cone ones. (The collided fluence is not, because the
    negative-flux fixup fires near the beam edges; it is checked against the
    oracle's combined source, whose combination is pinned by linearity of the
    fixup-free scheme on the CPU.)"""
    base = inputs.small_cone(8, 7, 6, n_groups=2, sn_order=4, legendre_order=1)
    w = inputs.combined_cones(base, n_cones=3)
    p = dts.problem_from_workload(w, tol=0.0, max_iters=2)
    p.solve(allow_not_converged=True)
    comb = p.fluence(0, dts.UNCOLLIDED)
    acc = np.zeros_like(comb)
    for c in w.sources[0].cones:
        one = copy.copy(base)
        one.sources = [c]
        q = dts.problem_from_workload(one, tol=0.0, max_iters=2)
        q.solve(allow_not_converged=True)
        acc += q.fluence(0, dts.UNCOLLIDED)
    assert np.abs(acc).max() > 0
    assert rel_max(comb, acc) <= 1e-13


@pytest.mark.parametrize("tile", [(8, 4, 4), (8, 4, 8)])
def test_combined_cones_fp32_batch_with_single_cones(ora, tile):
    base = inputs.small_cone(10, 9, 8, n_groups=2, sn_order=8, legendre_order=3, n_sources=2)
    comb = inputs.combined_cones(base, n_cones=5).sources[0]
    w = copy.copy(base)
    w.sources = [base.sources[0], comb, base.sources[1], comb]
    p = dts.problem_from_workload(w, precision=dts.PREC_FP32, tol=0.0, max_iters=4, tile=tile)
    st = p.solve(allow_not_converged=True)
    assert (st.tile_x, st.tile_y, st.tile_z) == tile
    for b in (0, 1):
        r = ora.solve(w, b, tol=0.0, max_iters=4, n_threads=8)
        col = p.fluence(b, dts.COLLIDED)
        assert rel_max(p.fluence(b, dts.UNCOLLIDED), r.phi_u) <= 1e-12
        for g in range(w.n_groups):
            assert rel_l2(col[g], r.collided[g]) <= TOL_FP32_L2, (b, g)
    assert np.array_equal(p.fluence(1, dts.TOTAL), p.fluence(3, dts.TOTAL))


def test_combined_cones_adjoint_refused_and_reset(ora):
    base = inputs.small_cone(6, 5, 4, n_groups=2, sn_order=4, legendre_order=1)
    w = inputs.combined_cones(base, n_cones=2)
    p = dts.problem_from_workload(w, tol=0.0, max_iters=3, keep_moments=True)
    p.solve(allow_not_converged=True)
    with pytest.raises(dts.DTSError) as e:
        p.adjoint(0, np.zeros((2, w.n_voxels)))
    assert e.value.status == dts.DTS_ERR_STATE
    # the member goes back to one cone: the solve matches the single-cone oracle
    p.set_source(0, base.sources[0])
    p.solve(allow_not_converged=True)
    r = ora.solve(base, 0, tol=0.0, max_iters=3, n_threads=8)
    assert rel_max(p.fluence(0, dts.UNCOLLIDED), r.phi_u) <= 1e-13
    assert rel_max(p.fluence(0, dts.COLLIDED)[1], r.collided[1]) <= TOL_FP64
    # every cone must be a point / cone source
    bad = copy.copy(w.sources[0])
    bad.cones = [inputs.Source(kind=0, spectrum=np.ones(w.n_groups))]
    with pytest.raises(dts.DTSError) as e:
        p.set_source(0, bad)
    assert e.value.status == dts.DTS_ERR_INVALID_ARG
