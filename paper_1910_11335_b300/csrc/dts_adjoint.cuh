// dts_adjoint.cuh -- FP64 discrete adjoint of the converged S_N solve.
//
// For L with dL/dphi_total given per group and voxel, the gradients with
// respect to per-voxel multipliers of sigma_t and sigma_s follow from the
// transposed system, group by group from low energy to high (the transposed
// downscatter runs upward):
//   1. the forward sweep of group g is recomputed from the converged moments
//      and records each cell's flux psi_n and fixup set (which faces the
//      set-to-zero fixup zeroed);
//   2. the adjoint source iteration u = M^T H^T D^T (s + sigma_s^{gg} u), with
//      H^T the transposed diamond-difference sweep: cells in reverse order,
//      faces carrying zeta = 2 dL/d(out-face) / a_d, and per cell
//        chi = (y + sum_{d not in F} a_d zeta_d) / (sigma + sum_{d not in F} a_d),
//        zeta upstream = 2 chi - zeta_d (d not in F), chi (d in F);
//   3. dL/dsigma_t^g = -sum_n chi_n psi_n per cell, the scatter terms from u and
//      the forward moments, and the uncollided part through the ray trace.
// The reduction kernel of the forward solve serves the adjoint iteration
// unchanged (u = octant sum, w = s + sigma_s u).
#pragma once
#include "dts_kernels.cuh"

namespace dts {

struct AdjSweepParams {
    SweepParams<double> s;     // B = 1; M and Dt swapped for the adjoint mode
    double* rec_psi;           // [nd][NC] recorded cell-centre flux
    unsigned char* rec_mask;   // [nd][NC] recorded fixup sets
    double* cpart;             // [8][NC] per-octant sum_n chi_n psi_n
    int NC;
};

__device__ __forceinline__ double dd_cell_record(double q, double sig, double ax, double ay, double az,
                                                 double ix, double iy, double iz, double& ox,
                                                 double& oy, double& oz, unsigned char& mask)
{
    double psi = (q + ax * ix + ay * iy + az * iz) / (sig + ax + ay + az);
    ox = 2.0 * psi - ix;
    oy = 2.0 * psi - iy;
    oz = 2.0 * psi - iz;
    bool fx = false, fy = false, fz = false;
    if (ox < 0.0 || oy < 0.0 || oz < 0.0) {
#pragma unroll 1
        for (int pass = 0; pass < 3; ++pass) {
            const bool nx = !fx && ox < 0.0, ny = !fy && oy < 0.0, nz = !fz && oz < 0.0;
            if (!(nx || ny || nz)) break;
            fx |= nx;
            fy |= ny;
            fz |= nz;
            const double num = q + (fx ? 0.5 * ax : ax) * ix + (fy ? 0.5 * ay : ay) * iy +
                               (fz ? 0.5 * az : az) * iz;
            const double den = sig + (fx ? 0.0 : ax) + (fy ? 0.0 : ay) + (fz ? 0.0 : az);
            psi = num / den;
            ox = fx ? 0.0 : 2.0 * psi - ix;
            oy = fy ? 0.0 : 2.0 * psi - iy;
            oz = fz ? 0.0 : 2.0 * psi - iz;
        }
    }
    mask = (unsigned char)((fx ? 1 : 0) | (fy ? 2 : 0) | (fz ? 4 : 0));
    return psi;
}

// MODE 1: forward sweep that records psi and the fixup sets.
// MODE 2: transposed sweep (reverse traversal of each direction).
template <int NDO, int K, int MODE>
__global__ void __launch_bounds__(kSweepThreads, 2) k_sweep_adj(const AdjSweepParams ap, const int stage)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const SweepParams<double>& p = ap.s;
    const int TX = p.TX, TY = p.TY, TZ = p.TZ, TV = p.TV;
    const int s0 = p.stage_off[stage], cnt = p.stage_off[stage + 1] - s0;
    const int tl = blockIdx.x % cnt;
    const int oct = blockIdx.x / cnt;                  // direction octant (coefficients)
    const int trav = MODE == 2 ? (oct ^ 7) : oct;      // octant of the traversal order
    const unsigned pk = p.stage_tiles[s0 + tl];
    const int ta = pk & 1023, tb = (pk >> 10) & 1023, tc = (pk >> 20) & 1023;
    const bool negx = trav & 1, negy = trav & 2, negz = trav & 4;
    const int tx = negx ? p.NTx - 1 - ta : ta;
    const int ty = negy ? p.NTy - 1 - tb : tb;
    const int tz = negz ? p.NTz - 1 - tc : tc;
    const int tile = (tz * p.NTy + ty) * p.NTx + tx;
    const int fxn = TY * TZ, fyn = TX * TZ, fzn = TX * TY;

    double* Qs = reinterpret_cast<double*>(smem);
    double* fx = Qs + NDO * TV;
    double* fy = fx + NDO * fxn;
    double* fz = fy + NDO * fyn;
    double* sg = fz + NDO * fzn;
    double* Ms = sg + TV;
    double* Ds = Ms + NDO * K;
    double* As = Ds + NDO * K;

    const int tid = threadIdx.x, nth = blockDim.x;
    const int n0 = oct * NDO;
    for (int i = tid; i < NDO * K; i += nth) {
        Ms[i] = p.M[n0 * K + i];
        Ds[(i % K) * NDO + i / K] = p.Dt[n0 * K + i];
    }
    for (int i = tid; i < NDO * 3; i += nth) As[(i / 3) * 4 + i % 3] = p.A[n0 * 3 + i];
    double* gx = p.xf + ((size_t)oct * (p.NTy * p.NTz) + (tz * p.NTy + ty)) * (size_t)(NDO * fxn);
    double* gy = p.yf + ((size_t)oct * (p.NTx * p.NTz) + (tz * p.NTx + tx)) * (size_t)(NDO * fyn);
    double* gz = p.zf + ((size_t)oct * (p.NTx * p.NTy) + (ty * p.NTx + tx)) * (size_t)(NDO * fzn);
    for (int i = tid; i < NDO * fxn; i += nth) fx[i] = ta > 0 ? gx[i] : 0.0;
    for (int i = tid; i < NDO * fyn; i += nth) fy[i] = tb > 0 ? gy[i] : 0.0;
    for (int i = tid; i < NDO * fzn; i += nth) fz[i] = tc > 0 ? gz[i] : 0.0;
    __syncthreads();

    // phase A: angular source of each direction from the moments
    const double* Tt = p.T + (size_t)tile * (K * TV);
    const double* st = p.sigt + (size_t)tile * TV;
#pragma unroll 1
    for (int c = tid; c < TV; c += nth) {
        double t[K];
#pragma unroll
        for (int k = 0; k < K; ++k) t[k] = Tt[k * TV + c];
        sg[c] = st[c];
#pragma unroll 1
        for (int d = 0; d < NDO; ++d) {
            double q = 0.0;
#pragma unroll
            for (int k = 0; k < K; ++k) q = fma(Ms[d * K + k], t[k], q);
            Qs[d * TV + c] = q;
        }
    }
    __syncthreads();

    // phase B: sub-sweeps in the traversal order
    const int gx0 = tx * TX, gy0 = ty * TY, gz0 = tz * TZ;
    for (int s = 0; s < p.nsub; ++s) {
        const int o0 = p.diag_off[s], cs = p.diag_off[s + 1] - o0;
        const int items = cs * NDO;
        for (int it = tid; it < items; it += nth) {
            const int d = it / cs, e = it - d * cs;
            const unsigned pc = p.diag_cells[o0 + e];
            const int lx = pc & 255, ly = (pc >> 8) & 255, lz = (pc >> 16) & 255;
            const int sx = negx ? TX - 1 - lx : lx;
            const int sy = negy ? TY - 1 - ly : ly;
            const int sz = negz ? TZ - 1 - lz : lz;
            const int c = (sz * TY + sy) * TX + sx;
            double* px = fx + d * fxn + sz * TY + sy;
            double* py = fy + d * fyn + sz * TX + sx;
            double* pz = fz + d * fzn + sy * TX + sx;
            const size_t rec = (size_t)(n0 + d) * ap.NC + (size_t)tile * TV + c;
            if (gx0 + sx >= p.nx || gy0 + sy >= p.ny || gz0 + sz >= p.nz) {
                *px = 0.0;
                *py = 0.0;
                *pz = 0.0;
                Qs[d * TV + c] = 0.0;
                continue;
            }
            const double ax = As[d * 4], ay = As[d * 4 + 1], az = As[d * 4 + 2];
            if (MODE == 1) {
                double ox, oy, oz;
                unsigned char mk;
                const double psi = dd_cell_record(Qs[d * TV + c], sg[c], ax, ay, az, *px, *py, *pz,
                                                  ox, oy, oz, mk);
                *px = ox;
                *py = oy;
                *pz = oz;
                Qs[d * TV + c] = psi;
                ap.rec_psi[rec] = psi;
                ap.rec_mask[rec] = mk;
            } else {
                const unsigned char mk = ap.rec_mask[rec];
                const double zx = *px, zy = *py, zz = *pz;
                double num = Qs[d * TV + c], den = sg[c];
                if (!(mk & 1)) { num += ax * zx; den += ax; }
                if (!(mk & 2)) { num += ay * zy; den += ay; }
                if (!(mk & 4)) { num += az * zz; den += az; }
                const double chi = num / den;
                *px = (mk & 1) ? chi : 2.0 * chi - zx;
                *py = (mk & 2) ? chi : 2.0 * chi - zy;
                *pz = (mk & 4) ? chi : 2.0 * chi - zz;
                Qs[d * TV + c] = chi;
            }
        }
        __syncthreads();
    }

    // phase C: octant partial of the moments (adjoint: u_k = sum_n M[n][k] chi_n)
    double* out = p.part + ((size_t)oct * p.NT + tile) * (size_t)(K * TV);
#pragma unroll 1
    for (int c = tid; c < TV; c += nth) {
        double ps[NDO];
#pragma unroll
        for (int d = 0; d < NDO; ++d) ps[d] = Qs[d * TV + c];
#pragma unroll 1
        for (int k = 0; k < K; ++k) {
            double acc = 0.0;
#pragma unroll
            for (int d = 0; d < NDO; ++d) acc = fma(Ds[k * NDO + d], ps[d], acc);
            out[k * TV + c] = acc;
        }
        if (MODE == 2) {
            double cp = 0.0;
            const size_t ct = (size_t)tile * TV + c;
#pragma unroll
            for (int d = 0; d < NDO; ++d) cp += ps[d] * ap.rec_psi[(size_t)(n0 + d) * ap.NC + ct];
            ap.cpart[(size_t)oct * ap.NC + ct] = cp;
        }
    }
    for (int i = tid; i < NDO * fxn; i += nth) gx[i] = fx[i];
    for (int i = tid; i < NDO * fyn; i += nth) gy[i] = fy[i];
    for (int i = tid; i < NDO * fzn; i += nth) gz[i] = fz[i];
}

struct AdjCellParams {
    CellParams c;
    int b, V;
    const double* src;     // [B][8]
    const double* unc;     // [B][G][V]
    const double* mom;     // [B][G][K][V]
    const double* q;       // [B][G][V] or null
    const double* a;       // [G][V] dL/dphi_total
    double* S;             // adjoint source ring [W+1][NT][K][TV]
    size_t Sstride;
    int W;
};

// unit direction of flight of the uncollided photons at a voxel centre
__device__ inline void omega_u(const double* s, const double* C, double* om)
{
    const double d0 = C[0] - s[1], d1 = C[1] - s[2], d2 = C[2] - s[3];
    const double r = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
    om[0] = d0 / r;
    om[1] = d1 / r;
    om[2] = d2 / r;
}

// converged source of group g: T_k = q_k + sum_{g' <= g} sigma_s^{g'->g} (phi_c,k^{g'} + phi_u^{g'} Y_k)
__global__ void k_adj_source_T(const AdjCellParams p, int g, double* T)
{
    const int ct = blockIdx.x * blockDim.x + threadIdx.x;
    const CellParams& c = p.c;
    if (ct >= c.NC) return;
    const int tile = ct / c.TV, cc = ct - tile * c.TV;
    double* Tt = T + (size_t)tile * (c.K * c.TV) + cc;
    const int m = c.mat_t[ct];
    if (m < 0) {
        for (int k = 0; k < c.K; ++k) Tt[(size_t)k * c.TV] = 0.0;
        return;
    }
    double C[3], om[3], Y[16];
    const int v = tiled_to_natural(c, ct, C);
    const double* s = p.src + (size_t)p.b * 8;
    const int kind = (int)s[0];
    if (kind == 1) {
        omega_u(s, C, om);
        sh_eval(c.L, om[0], om[1], om[2], Y);
    }
    const double ss = c.scale_s_t ? c.scale_s_t[ct] : 1.0;
    for (int k = 0; k < c.K; ++k) {
        const int l = l_of_k(k);
        double t = (kind == 0 && k == 0) ? p.q[((size_t)p.b * c.G + g) * p.V + v] : 0.0;
        for (int gp = 0; gp <= g; ++gp) {
            const double sg = c.sigma_s[(((size_t)m * (c.L + 1) + l) * c.G + gp) * c.G + g] * ss;
            if (kind == 1) t += sg * p.unc[((size_t)p.b * c.G + gp) * p.V + v] * Y[k];
            t += sg * p.mom[(((size_t)p.b * c.G + gp) * c.K + k) * p.V + v];
        }
        Tt[(size_t)k * c.TV] = t;
    }
}

// adjoint source of group g (before contributions of the groups below it): a^g e_0
__global__ void k_adj_source_init(const AdjCellParams p, int g, int slot)
{
    const int ct = blockIdx.x * blockDim.x + threadIdx.x;
    const CellParams& c = p.c;
    if (ct >= c.NC) return;
    const int tile = ct / c.TV, cc = ct - tile * c.TV;
    double* S = p.S + (size_t)slot * p.Sstride + (size_t)tile * (c.K * c.TV) + cc;
    const int m = c.mat_t[ct];
    const int v = m >= 0 ? tiled_to_natural(c, ct, nullptr) : 0;
    S[0] = m >= 0 ? p.a[(size_t)g * p.V + v] : 0.0;
    for (int k = 1; k < c.K; ++k) S[(size_t)k * c.TV] = 0.0;
}

struct AdjGradParams {
    AdjCellParams a;
    const double* part;    // [8][NT][K][TV] adjoint octant partials (u)
    const double* cpart;   // [8][NC]
    double* gt;            // [V] dL/dscale_t
    double* gs;            // [V] dL/dscale_s
    double* gsig;          // [G][V] dL/dsigma_t^g (collided part)
    double* dphiu;         // [G][V] dL/dphi_u through the first-collision source
};

// gradients of group g and the transposed downscatter into the lower groups
__global__ void k_adj_grad(const AdjGradParams gp_, int g)
{
    const int ct = blockIdx.x * blockDim.x + threadIdx.x;
    const AdjCellParams& p = gp_.a;
    const CellParams& c = p.c;
    if (ct >= c.NC) return;
    const int m = c.mat_t[ct];
    if (m < 0) return;
    const int tile = ct / c.TV, cc = ct - tile * c.TV;
    double C[3], om[3], Y[16];
    const int v = tiled_to_natural(c, ct, C);
    const double* s = p.src + (size_t)p.b * 8;
    const int kind = (int)s[0];
    if (kind == 1) {
        omega_u(s, C, om);
        sh_eval(c.L, om[0], om[1], om[2], Y);
    }
    const double ss = c.scale_s_t ? c.scale_s_t[ct] : 1.0;
    const size_t pstride = (size_t)c.NT * c.K * c.TV;
    double cp = 0.0;
    for (int o = 0; o < 8; ++o) cp += gp_.cpart[(size_t)o * c.NC + ct];
    const double gst = -cp;
    gp_.gsig[(size_t)g * p.V + v] = gst;
    gp_.gt[v] += c.sigma_t[(size_t)m * c.G + g] * gst;
    double gss = 0.0;
    const int W1 = p.W + 1;
    for (int k = 0; k < c.K; ++k) {
        const int l = l_of_k(k);
        const size_t ik = (size_t)tile * (c.K * c.TV) + (size_t)k * c.TV + cc;
        double uk = 0.0;
        for (int o = 0; o < 8; ++o) uk += gp_.part[o * pstride + ik];
        for (int gq = 0; gq <= g; ++gq) {
            const double tab = c.sigma_s[(((size_t)m * (c.L + 1) + l) * c.G + gq) * c.G + g];
            double src = p.mom[(((size_t)p.b * c.G + gq) * c.K + k) * p.V + v];
            if (kind == 1) {
                const double phu = p.unc[((size_t)p.b * c.G + gq) * p.V + v];
                src += phu * Y[k];
                gp_.dphiu[(size_t)gq * p.V + v] += uk * tab * ss * Y[k];
            }
            gss += tab * uk * src;
        }
        for (int gq = max(0, g - p.W); gq < g; ++gq) {
            const double tab = c.sigma_s[(((size_t)m * (c.L + 1) + l) * c.G + gq) * c.G + g];
            if (tab != 0.0) p.S[(size_t)(gq % W1) * p.Sstride + ik] += tab * ss * uk;
        }
    }
    gp_.gs[v] += gss;
}

// uncollided part: dL/dtau^g(v) = -phi_u^g(v) (a^g(v) + dL/dphi_u^g(v)) spread back
// along the ray from the source to the centre of v (tau = sum ell sigma_t)
__global__ void k_adj_ray(const RayParams rp, const double* a, const double* dphiu, int b, double* gt)
{
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= rp.V) return;
    const double* s = rp.src + (size_t)b * 8;
    if (s[0] != 1.0) return;
    const double* unc = rp.unc + (size_t)b * rp.G * rp.V;
    bool any = false;
    for (int g = 0; g < rp.G; ++g) any |= unc[(size_t)g * rp.V + v] != 0.0;
    if (!any) return;
    const int ci[3] = {v % rp.nx, (v / rp.nx) % rp.ny, v / (rp.nx * rp.ny)};
    const int n[3] = {rp.nx, rp.ny, rp.nz};
    const double lo[3] = {rp.x0, rp.y0, rp.z0}, h[3] = {rp.dx, rp.dy, rp.dz};
    double P[3], d[3];
    for (int ax = 0; ax < 3; ++ax) {
        P[ax] = s[1 + ax];
        d[ax] = lo[ax] + (ci[ax] + 0.5) * h[ax] - P[ax];
    }
    const double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    double a_in = 0.0;
    for (int ax = 0; ax < 3; ++ax)
        if (d[ax] != 0.0) {
            const double t0 = (lo[ax] - P[ax]) / d[ax], t1 = (lo[ax] + n[ax] * h[ax] - P[ax]) / d[ax];
            a_in = fmax(a_in, fmin(t0, t1));
        }
    int idx[3], step[3];
    double tnext[3];
    for (int ax = 0; ax < 3; ++ax) {
        if (d[ax] == 0.0) {
            idx[ax] = ci[ax];
            step[ax] = 0;
            tnext[ax] = 2.0;
            continue;
        }
        int id = (int)floor((P[ax] + a_in * d[ax] - lo[ax]) / h[ax]);
        id = id < 0 ? 0 : (id >= n[ax] ? n[ax] - 1 : id);
        idx[ax] = id;
        step[ax] = d[ax] > 0.0 ? 1 : -1;
        tnext[ax] = (lo[ax] + (id + (d[ax] > 0.0 ? 1 : 0)) * h[ax] - P[ax]) / d[ax];
    }
    double acur = a_in;
    const int max_steps = rp.nx + rp.ny + rp.nz + 3;
    for (int it = 0; it < max_steps; ++it) {
        int ax = 0;
        if (tnext[1] < tnext[ax]) ax = 1;
        if (tnext[2] < tnext[ax]) ax = 2;
        const double a1 = fmin(tnext[ax], 1.0);
        const double seg = (a1 - acur) * r;
        if (seg > 0.0) {
            const int vv = (idx[2] * rp.ny + idx[1]) * rp.nx + idx[0];
            const double* sgm = rp.sigma_t + (size_t)rp.mat[vv] * rp.G;
            double acc = 0.0;
            for (int g = 0; g < rp.G; ++g) {
                const double e = -unc[(size_t)g * rp.V + v] *
                                 (a[(size_t)g * rp.V + v] + dphiu[(size_t)g * rp.V + v]);
                acc += e * seg * sgm[g];
            }
            atomicAdd(&gt[vv], acc);
        }
        if (a1 >= 1.0) break;
        acur = a1;
        idx[ax] += step[ax];
        if (idx[ax] < 0 || idx[ax] >= n[ax]) break;
        tnext[ax] = (lo[ax] + (idx[ax] + (step[ax] > 0 ? 1 : 0)) * h[ax] - P[ax]) / d[ax];
    }
}

}  // namespace dts
