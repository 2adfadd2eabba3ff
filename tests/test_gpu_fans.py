"""Fan-beam and multi-fan sources against the oracle, and the option grid of
S_N order x Legendre order (S2..S8, P0..P2) in FP64."""
import copy
import math

import numpy as np
import pytest

from paper_1910_11335_b300 import dts, inputs
from parity_util import TOL_FP32_L2, TOL_FP64, rel_l2, rel_max

pytestmark = pytest.mark.gpu


def _with(w, srcs):
    t = copy.copy(w)
    t.sources = list(srcs)
    return t


def _fp64_parity(ora, w, iters=4):
    p = dts.problem_from_workload(w, tol=0.0, max_iters=iters, keep_moments=True)
    p.solve(allow_not_converged=True)
    for b in range(len(w.sources)):
        r = ora.solve(w, b, tol=0.0, max_iters=iters, n_threads=8)
        assert rel_max(p.fluence(b, dts.UNCOLLIDED), r.phi_u) <= 1e-13, b
        for g in range(w.n_groups):
            m = p.moments(b, g)
            floor = 1e-12 * np.max(np.abs(r.phi_c[g, 0]))
            for k in range(m.shape[0]):
                if np.max(np.abs(r.phi_c[g, k])) <= floor:
                    # a moment the quadrature makes vanish (S2: mu^2 = eta^2 = xi^2 = 1/3 zeroes the l = 2,
                    # m = 0 and cos 2phi moments); both sides must be rounding noise of the scalar moment
                    assert np.max(np.abs(m[k])) <= floor, (b, g, k)
                else:
                    assert rel_max(m[k], r.phi_c[g, k]) <= TOL_FP64, (b, g, k)


def test_fan_beam_fp64_vs_oracle(ora):
    base = inputs.small_cone(10, 9, 8, n_groups=2, sn_order=4, legendre_order=2)
    fans = inputs.fan_sources(base.sources[0].spectrum, 3, half_azimuth=math.radians(17.0),
                              half_polar=math.radians(9.0))
    w = _with(base, fans)
    _fp64_parity(ora, w)
    r = ora.solve(w, 0, tol=0.0, max_iters=1, n_threads=8)
    assert (r.phi_u > 0).any() and (r.phi_u == 0).any()   # a beam, not the whole grid


def test_multi_fan_fp64_vs_oracle(ora):
    base = inputs.small_cone(9, 8, 7, n_groups=2, sn_order=4, legendre_order=1)
    _fp64_parity(ora, inputs.combined_fans(base, n_fans=5, half_azimuth=math.radians(21.0),
                                           half_polar=math.radians(6.0)))


def test_fan_beams_fp32_batch(ora):
    base = inputs.small_cone(10, 9, 8, n_groups=2, sn_order=8, legendre_order=3)
    fans = inputs.fan_sources(base.sources[0].spectrum, 4, half_azimuth=math.radians(19.0),
                              half_polar=math.radians(7.0))
    w = _with(base, fans)
    p = dts.problem_from_workload(w, precision=dts.PREC_FP32, tol=0.0, max_iters=4, tile=(8, 4, 4))
    p.solve(allow_not_converged=True)
    for b in (0, 3):
        r = ora.solve(w, b, tol=0.0, max_iters=4, n_threads=8)
        assert rel_max(p.fluence(b, dts.UNCOLLIDED), r.phi_u) <= 1e-12
        col = p.fluence(b, dts.COLLIDED)
        for g in range(w.n_groups):
            assert rel_l2(col[g], r.collided[g]) <= TOL_FP32_L2, (b, g)


def test_fan_validation():
    base = inputs.small_cone(6, 5, 4, n_groups=1, sn_order=2, legendre_order=0)
    p = dts.problem_from_workload(base, tol=0.0, max_iters=1)
    good = inputs.fan_sources(base.sources[0].spectrum, 1)[0]
    for change in ({"normal": good.axis}, {"half_polar": 2.0}, {"half_azimuth": 0.0}, {"aperture": 2}):
        bad = copy.copy(good)
        for k, v in change.items():
            setattr(bad, k, v)
        with pytest.raises(dts.DTSError) as e:
            p.set_source(0, bad)
        assert e.value.status == dts.DTS_ERR_INVALID_ARG, change


@pytest.mark.parametrize("N", [2, 4, 6, 8])
@pytest.mark.parametrize("L", [0, 1, 2])
def test_option_grid_fp64(ora, N, L):
    w = inputs.small_cone(7, 6, 5, n_groups=2, sn_order=N, legendre_order=L)
    _fp64_parity(ora, w, iters=3)
