"""A downscatter band wider than the FP32 push kernels' four-group ring pass:
every group scatters into every lower group (Eq. 2's group sum with W = G - 1
= 6). The angular-flux forms (FP32 batches with 8K > N_d, and both tensor-core
forms) push the group's moments in several passes; every form is compared with
the FP64 oracle."""
import numpy as np
import pytest

from paper_1910_11335_b300 import dts, inputs
from parity_util import TOL_FP32_L2, rel_l2, rel_max

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1910_11335_b300 import build
    build.build()


def _wide_band(n_sources):
    w = inputs.small_cone(11, 10, 9, n_groups=7, sn_order=8, legendre_order=3, n_sources=n_sources)
    ss = w.sigma_s.copy()   # [n_mat][L+1][G_from][G_to]
    G = w.n_groups
    for gf in range(G):
        for gt in range(gf + 1, G):
            if ss[:, 0, gf, gt].max() == 0.0:   # add the far downscatter the band left out
                near = ss[:, :, gf, min(gf + 1, G - 1)]
                ss[:, :, gf, gt] = 0.02 * near / (gt - gf)
    w.sigma_s = ss
    return w


@pytest.mark.parametrize("prec", [dts.PREC_FP64, dts.PREC_FP32, dts.PREC_FP32_SPLITBF16, dts.PREC_FP32_TF32],
                         ids=["fp64", "fp32", "splitbf16", "tf32"])
def test_wide_downscatter_band_vs_oracle(ora, prec):
    w = _wide_band(4)
    assert (w.sigma_s[:, 0, 0, 6] > 0).all()   # group 0 reaches group 6: band width 6
    p = dts.problem_from_workload(w, precision=prec, tol=0.0, max_iters=3)
    p.solve(allow_not_converged=True)
    for b in (0, 3):
        r = ora.solve(w, b, tol=0.0, max_iters=3, n_threads=8)
        col = p.fluence(b, dts.COLLIDED)
        for g in range(w.n_groups):
            if prec == dts.PREC_FP64:
                assert rel_max(col[g], r.collided[g]) <= 1e-10, (b, g)
            else:
                assert rel_l2(col[g], r.collided[g]) <= TOL_FP32_L2, (b, g)
