"""dts_get_dose against the oracle's fluence-to-dose conversion."""
import numpy as np
import pytest

from paper_1910_11335_b300 import dts, inputs
from parity_util import TOL_FP64, rel_max

pytestmark = pytest.mark.gpu


def test_dose_matches_oracle(ora):
    w = inputs.small_cone(9, 8, 7, n_groups=3, sn_order=4, legendre_order=1, n_sources=2)
    mu, e = inputs.dose_coefficients(w)
    p = dts.problem_from_workload(w, tol=0.0, max_iters=4)
    p.solve(allow_not_converged=True)
    mat = w.mat_id.reshape(-1)
    for b in range(2):
        for comp in (dts.UNCOLLIDED, dts.COLLIDED, dts.TOTAL):
            phi = p.fluence(b, comp)
            d = p.dose(b, mu, e, comp)
            assert np.abs(d).max() > 0
            # the conversion alone: the oracle's definition on the GPU's own fluence
            assert rel_max(d, ora.dose(phi, mat, mu, e)) <= 1e-14
        # end to end against the oracle's solve
        r = ora.solve(w, b, tol=0.0, max_iters=4, n_threads=8)
        assert rel_max(p.dose(b, mu, e, dts.TOTAL), ora.dose(r.phi_u + r.collided, mat, mu, e)) <= TOL_FP64


def test_dose_errors():
    w = inputs.small_cone(6, 5, 4, n_groups=2, sn_order=4, legendre_order=0)
    mu, e = inputs.dose_coefficients(w)
    p = dts.problem_from_workload(w, tol=0.0, max_iters=2)
    with pytest.raises(dts.DTSError) as ex:
        p.dose(0, mu, e)
    assert ex.value.status == dts.DTS_ERR_STATE
    p.solve(allow_not_converged=True)
    bad = mu.copy()
    bad[0, 0] = -1.0
    with pytest.raises(dts.DTSError) as ex:
        p.dose(0, bad, e)
    assert ex.value.status == dts.DTS_ERR_INVALID_ARG
