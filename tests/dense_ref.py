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
