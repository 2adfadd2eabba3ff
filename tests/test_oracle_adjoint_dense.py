"""Pin of the oracle's discrete adjoint by a dense transpose solve (no GPU).

On a tiny grid whose cells are thin enough that the negative-flux fixup never
fires, the converged solve is the solution x of one linear system A x = b (all
groups at once, tests/dense_ref.py). For L = sum_g sum_v a_g(v) phi_g(v) = c.x,
the adjoint lambda solves A^T lambda = c, and a parameter theta that enters A
only gives dL/dtheta = -lambda . (dA/dtheta) x. For the per-voxel multipliers:
  dL/dscale_t(v)  = -sum_{g,n} lambda_{g,v,n} sigma_t^g(v) psi_c(g,v,n)
  dL/dscale_s(v)  = +sum_{g,n} lambda_{g,v,n} sum_{g'<=g} sum_n' K^{g'->g}_{nn'}(v) psi_c(g',v,n')
  dL/dsigma_t^g(v) = -sum_n lambda_{g,v,n} psi_c(g,v,n)
The oracle's adjoint (ora_adjoint: reverse sweeps of its own source
iteration, no matrix) must give the same numbers. The volumetric source
(kind 0) does not depend on the cross sections, so b drops out."""
import numpy as np
import pytest

from paper_1910_11335_b300 import inputs


@pytest.mark.parametrize("dims,N,L,G,seed", [((3, 3, 2), 4, 1, 2, 601), ((2, 3, 2), 2, 2, 3, 602)])
def test_oracle_adjoint_matches_dense_transpose(ora, dims, N, L, G, seed):
    from dense_ref import dense_system
    w = inputs.random_volumetric(*dims, n_groups=G, sn_order=N, legendre_order=L, seed_index=seed)
    # a uniform source in thin cells: the flux varies slowly along every flight path, no outflow goes
    # negative, and the fixup's active set is empty (the oracle's adjoint keeps it fixed)
    w.sources[0].q[:] = 1.0
    r = ora.solve(w, tol=1e-15, max_iters=600)
    assert np.all(r.fixups == 0)
    mu, eta, xi, wt = ora.quadrature(N)
    A, b, idx, Kb, sig_t = dense_system(w, (mu, eta, xi, wt))
    V, nd = w.n_voxels, len(wt)
    x = np.linalg.solve(A, b)
    psi = x.reshape(G, V, nd, 4)[:, :, :, 0]
    # the dense solution is the oracle's converged solve
    phi = psi @ wt
    for g in range(G):
        assert np.max(np.abs(phi[g] - r.collided[g])) <= 1e-11 * np.max(np.abs(phi[g]))
    rng = np.random.default_rng(seed)
    a = rng.uniform(0.0, 1.0, size=(G, V))
    c = np.zeros_like(b)
    c.reshape(G, V, nd, 4)[:, :, :, 0] = a[:, :, None] * wt[None, None, :]
    lam = np.linalg.solve(A.T, c).reshape(G, V, nd, 4)[:, :, :, 0]
    gt_d = -np.einsum("gvn,vg,gvn->v", lam, sig_t, psi)
    gs_d = np.zeros(V)
    for g in range(G):
        for gp in range(g + 1):
            gs_d += np.einsum("vn,vnm,vm->v", lam[g], Kb[:, gp, g], psi[gp])
    gg_d = -np.einsum("gvn,gvn->gv", lam, psi)
    gt, gs, gg = ora.adjoint(w, a, tol=1e-15, max_iters=600)
    scale = max(np.abs(gt_d).max(), np.abs(gs_d).max())
    # measured about 2e-16 of the scale on both cases
    assert np.max(np.abs(gt - gt_d)) <= 1e-12 * scale
    assert np.max(np.abs(gs - gs_d)) <= 1e-12 * scale
    assert np.max(np.abs(gg - gg_d)) <= 1e-12 * np.abs(gg_d).max()
    # a mistake a test of this kind must catch: the in-group scattering term left out of dL/dscale_s
    no_ingroup = gs_d - sum(np.einsum("vn,vnm,vm->v", lam[g], Kb[:, g, g], psi[g]) for g in range(G))
    assert np.max(np.abs(gs - no_ingroup)) > 1e-3 * scale
