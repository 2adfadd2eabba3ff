"""Combined multi-cone source (several cone beams summed into one source, the
paper's CT mode) in the oracle, pinned by the linearity of the method: with
the plain diamond-difference scheme (no fixup, a linear map from source to
fluence) the combined solve equals the sum of the single-cone solves."""
import numpy as np

from paper_1910_11335_b300 import inputs


def test_combined_cones_equal_sum_of_single_cones(ora):
    base = inputs.small_cone(7, 6, 5, n_groups=3, sn_order=4, legendre_order=2)
    w = inputs.combined_cones(base, n_cones=4)
    comb = ora.solve(w, 0, tol=0.0, max_iters=6, n_threads=4, fixup=False)
    cu = np.zeros_like(comb.phi_u)
    cc = np.zeros_like(comb.phi_c)
    for c in w.sources[0].cones:
        one = inputs.with_sources(base, [0])
        one.sources = [c]
        r = ora.solve(one, 0, tol=0.0, max_iters=6, n_threads=4, fixup=False)
        cu += r.phi_u
        cc += r.phi_c
    assert np.abs(cu).max() > 0 and np.abs(cc).max() > 0
    assert np.abs(comb.phi_u - cu).max() <= 1e-13 * np.abs(cu).max()
    for g in range(w.n_groups):
        for k in range(cc.shape[1]):
            ref = np.abs(cc[g, k]).max()
            assert np.abs(comb.phi_c[g, k] - cc[g, k]).max() <= 1e-12 * max(ref, 1e-300), (g, k)


def test_cones_cover_the_ring(ora):
    # four cones at 90 degree steps light four different sides of the phantom
    base = inputs.small_cone(8, 8, 5, n_groups=1, sn_order=2, legendre_order=0)
    w = inputs.combined_cones(base, n_cones=4)
    r = ora.solve(w, 0, tol=0.0, max_iters=1, n_threads=4)
    u = r.phi_u[0].reshape(w.nz, w.ny, w.nx)
    mid = u[w.nz // 2]
    sides = [mid[0, :].sum(), mid[-1, :].sum(), mid[:, 0].sum(), mid[:, -1].sum()]
    assert min(sides) > 0.2 * max(sides)
