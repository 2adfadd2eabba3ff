"""Dense direct solve of the discrete S_N / diamond-difference system (test helper).

An independent route to the same discrete solution the source iteration
converges to: instead of sweeping and iterating, it assembles every equation
of Eq. 2 on a tiny grid -- for each cell and direction the diamond-difference
cell balance plus the three closures psi_c = (psi_in + psi_out)/2 -- with the
scattering kernel written in direction space through Legendre polynomials,
    K_{nn'} = sum_l (2l+1)/(4 pi) sigma_{s,l} P_l(Omega_n . Omega_n') w_n',
(no spherical harmonics, no moments), and solves it with LU. Vacuum
boundaries: an in-face on the grid boundary is zero. The system is linear,
so it is compared with the oracle run with its negative-flux fixup switched
off; the fixup itself is pinned cell by cell and by conservation.
"""
from __future__ import annotations

import numpy as np
from numpy.polynomial import legendre as npleg


def _pl(l, x):
    c = np.zeros(l + 1)
    c[l] = 1.0
    return npleg.legval(x, c)


def dense_solve(w, quad, source_dirs=None, phi_u=None, omega_u=None):
    """Solve all groups of workload w (one source) by dense LU.

    quad = (mu, eta, xi, wt). Volumetric sources (kind 0) give an isotropic
    s_n = q/(4 pi); for a kind-1 source pass phi_u[G][V] and omega_u[V][3] and
    the first-collision source is formed as
    sum_{g'<=g} sum_l (2l+1)/(4 pi) sigma_{s,l}^{g'->g} phi_u^{g'} P_l(Omega_n . Omega_u).
    Returns psi_c[G][V][nd] and the scalar fluence phi[G][V].
    """
    mu, eta, xi, wt = quad
    nd, G, V = len(wt), w.n_groups, w.n_voxels
    nx, ny, nz = w.nx, w.ny, w.nz
    L = w.legendre_order
    omega = np.stack([mu, eta, xi], axis=1)
    cosmat = omega @ omega.T
    Pl = np.stack([_pl(l, cosmat) for l in range(L + 1)])           # [L+1][nd][nd]
    mat = w.mat_id.reshape(-1)
    sig_t = w.sigma_t[mat]                                           # [V][G]
    sig_s = w.sigma_s[mat]                                           # [V][L+1][G][G]
    if w.scale_t is not None:
        sig_t = sig_t * w.scale_t.reshape(-1)[:, None]
    if w.scale_s is not None:
        sig_s = sig_s * w.scale_s.reshape(-1)[:, None, None, None]
    a = np.stack([2 * np.abs(mu) / w.dx, 2 * np.abs(eta) / w.dy, 2 * np.abs(xi) / w.dz], axis=1)
    src = w.sources[0]

    def vid(i, j, k):
        return (k * ny + j) * nx + i

    def kernel(v, gf, gt):
        # K[n][n'] = sum_l (2l+1)/(4pi) sigma_{s,l}^{gf->gt}(v) P_l(cos) w_n'
        out = np.zeros((nd, nd))
        for l in range(L + 1):
            out += (2 * l + 1) / (4 * np.pi) * sig_s[v, l, gf, gt] * Pl[l]
        return out * wt[None, :]

    psi_all = np.zeros((G, V, nd))
    nunk = V * nd * 4
    for g in range(G):
        A = np.zeros((nunk, nunk))
        b = np.zeros(nunk)

        def u(v, n, t):
            return (v * nd + n) * 4 + t

        for k in range(nz):
            for j in range(ny):
                for i in range(nx):
                    v = vid(i, j, k)
                    Kvv = kernel(v, g, g)
                    # fixed source per direction
                    s = np.zeros(nd)
                    if src.kind == 0:
                        s += src.q[g, v] / (4 * np.pi)
                    else:
                        cu = omega @ omega_u[v]
                        for gp in range(g + 1):
                            for l in range(L + 1):
                                s += (2 * l + 1) / (4 * np.pi) * sig_s[v, l, gp, g] * phi_u[gp, v] * _pl(l, cu)
                    for gp in range(g):
                        s += kernel(v, gp, g) @ psi_all[gp, v]
                    for n in range(nd):
                        r = u(v, n, 0)
                        # balance row
                        A[r, u(v, n, 0)] += sig_t[v, g]
                        A[r, [u(v, m, 0) for m in range(nd)]] -= Kvv[n]
                        b[r] = s[n]
                        sgn = (np.sign(mu[n]), np.sign(eta[n]), np.sign(xi[n]))
                        up = [(i - int(sgn[0]), j, k), (i, j - int(sgn[1]), k), (i, j, k - int(sgn[2]))]
                        for d in range(3):
                            A[r, u(v, n, 1 + d)] += 0.5 * a[n, d]
                            ii, jj, kk = up[d]
                            inside = 0 <= ii < nx and 0 <= jj < ny and 0 <= kk < nz
                            # closure row: 2 psi_c - psi_in - psi_out = 0
                            rc = u(v, n, 1 + d)
                            A[rc, u(v, n, 0)] += 2.0
                            A[rc, u(v, n, 1 + d)] -= 1.0
                            if inside:
                                vu = vid(ii, jj, kk)
                                A[r, u(vu, n, 1 + d)] -= 0.5 * a[n, d]
                                A[rc, u(vu, n, 1 + d)] -= 1.0
        x = np.linalg.solve(A, b)
        psi_all[g] = x.reshape(V, nd, 4)[:, :, 0]
    phi = psi_all @ wt
    return psi_all, phi


def dense_system(w, quad):
    """The whole multigroup system of workload w (one volumetric source, kind 0)
    as ONE dense matrix: unknowns (g, v, n, t), t = 0 the cell-average flux and
    t = 1..3 the x, y, z outflow; per (g, v, n) the balance row
        sigma_t psi_c + sum_d a_d/2 (psi_out,d - psi_in,d)
            - sum_{g' <= g} sum_n' K^{g'->g}_{n n'} psi_c(g', n') = q/(4 pi)
    (downscatter as blocks below the diagonal) and the three closures
    2 psi_c - psi_in,d - psi_out,d = 0. Returns (A, b, idx) with idx(g, v, n, t)
    the unknown's index, plus the per-cell kernel blocks K[v][g'][g] ([nd][nd])
    and sigma_t[V][G], so that derivatives of A with respect to per-voxel
    multipliers of sigma_t and sigma_s can be written down directly."""
    mu, eta, xi, wt = quad
    nd, G, V = len(wt), w.n_groups, w.n_voxels
    nx, ny, nz = w.nx, w.ny, w.nz
    L = w.legendre_order
    omega = np.stack([mu, eta, xi], axis=1)
    Pl = np.stack([_pl(l, omega @ omega.T) for l in range(L + 1)])
    mat = w.mat_id.reshape(-1)
    sig_t = w.sigma_t[mat].copy()
    sig_s = w.sigma_s[mat].copy()
    a = np.stack([2 * np.abs(mu) / w.dx, 2 * np.abs(eta) / w.dy, 2 * np.abs(xi) / w.dz], axis=1)
    src = w.sources[0]
    assert src.kind == 0

    def idx(g, v, n, t):
        return ((g * V + v) * nd + n) * 4 + t

    Kb = np.zeros((V, G, G, nd, nd))
    for v in range(V):
        for gf in range(G):
            for gt in range(gf, G):
                for l in range(L + 1):
                    Kb[v, gf, gt] += (2 * l + 1) / (4 * np.pi) * sig_s[v, l, gf, gt] * Pl[l]
                Kb[v, gf, gt] *= wt[None, :]
    nunk = G * V * nd * 4
    A = np.zeros((nunk, nunk))
    b = np.zeros(nunk)
    for g in range(G):
        for k in range(nz):
            for j in range(ny):
                for i in range(nx):
                    v = (k * ny + j) * nx + i
                    for n in range(nd):
                        r = idx(g, v, n, 0)
                        A[r, r] += sig_t[v, g]
                        for gp in range(g + 1):
                            A[r, [idx(gp, v, m, 0) for m in range(nd)]] -= Kb[v, gp, g, n]
                        b[r] = src.q[g, v] / (4 * np.pi)
                        step = (int(np.sign(mu[n])), int(np.sign(eta[n])), int(np.sign(xi[n])))
                        up = [(i - step[0], j, k), (i, j - step[1], k), (i, j, k - step[2])]
                        for d in range(3):
                            A[r, idx(g, v, n, 1 + d)] += 0.5 * a[n, d]
                            rc = idx(g, v, n, 1 + d)
                            A[rc, r] += 2.0
                            A[rc, rc] -= 1.0
                            ii, jj, kk = up[d]
                            if 0 <= ii < nx and 0 <= jj < ny and 0 <= kk < nz:
                                vu = (kk * ny + jj) * nx + ii
                                A[r, idx(g, vu, n, 1 + d)] -= 0.5 * a[n, d]
                                A[rc, idx(g, vu, n, 1 + d)] -= 1.0
    return A, b, idx, Kb, sig_t
