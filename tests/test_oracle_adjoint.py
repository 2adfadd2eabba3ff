"""Pins of the oracle's discrete adjoint against central finite differences of
the oracle's forward solve (which shares nothing with the adjoint code except
the cell solve it differentiates). Loss: L = sum_g sum_v a^g(v) phi_total^g(v)."""
import numpy as np
import pytest

from paper_1910_11335_b300 import inputs


def _loss(ora, w, a, st, ss):
    w2 = inputs.Workload(**{**w.__dict__})
    w2.scale_t, w2.scale_s = st, ss
    r = ora.solve(w2, tol=1e-14, max_iters=4000)
    return float((a * r.total).sum())


@pytest.mark.parametrize("kind", ["cone", "thick_volumetric"])
def test_adjoint_matches_central_differences(ora, kind):
    if kind == "cone":
        w = inputs.small_cone(5, 4, 6, n_groups=3, sn_order=4, legendre_order=1, tol=1e-14)
    else:
        w = inputs.random_volumetric(4, 5, 3, n_groups=2, sn_order=4, legendre_order=2,
                                     seed_index=71, thin=False)
    rng = np.random.default_rng(3)
    a = rng.uniform(0.0, 1.0, size=(w.n_groups, w.n_voxels))
    gt, gs, _ = ora.adjoint(w, a, tol=1e-14, max_iters=4000)
    if kind == "thick_volumetric":
        assert np.any(ora.solve(w, tol=1e-14, max_iters=4000).fixups > 0)
    one = np.ones(w.n_voxels)
    h = 1e-6
    scale = max(np.abs(gt).max(), np.abs(gs).max())
    for v in rng.choice(w.n_voxels, 8, replace=False):
        e = np.zeros(w.n_voxels)
        e[v] = h
        fdt = (_loss(ora, w, a, one + e, one) - _loss(ora, w, a, one - e, one)) / (2 * h)
        fds = (_loss(ora, w, a, one, one + e) - _loss(ora, w, a, one, one - e)) / (2 * h)
        assert abs(fdt - gt[v]) <= 1e-6 * abs(gt[v]) + 1e-8 * scale, (v, fdt, gt[v])
        assert abs(fds - gs[v]) <= 1e-6 * abs(gs[v]) + 1e-8 * scale, (v, fds, gs[v])


def test_adjoint_is_linear_in_the_loss_weights(ora):
    w = inputs.small_cone(4, 5, 4, n_groups=2, sn_order=2, legendre_order=1, tol=1e-13)
    rng = np.random.default_rng(8)
    a1, a2 = rng.uniform(size=(2, w.n_groups, w.n_voxels))
    g1 = ora.adjoint(w, a1, tol=1e-14, max_iters=4000)
    g2 = ora.adjoint(w, a2, tol=1e-14, max_iters=4000)
    g3 = ora.adjoint(w, 2.0 * a1 - 0.5 * a2, tol=1e-14, max_iters=4000)
    for x, y, z in zip(g1, g2, g3):
        assert np.allclose(z, 2.0 * x - 0.5 * y, rtol=1e-10, atol=1e-14 * np.abs(x).max())
