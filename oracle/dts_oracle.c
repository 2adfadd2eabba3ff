/*
 * dts_oracle.c -- plain FP64 CPU oracle for the DOCTORS multigroup S_N
 * source-iteration solve (arxiv 1910.11335).
 *
 * TEST INFRASTRUCTURE ONLY. This file is used by the test suite, by the
 * smoke check and by the CPU-baseline leg of the benchmark, to decide whether
 * the CUDA library is right. The product never links, imports or calls it, and
 * it shares no code, header, table or helper with the CUDA library.
 *
 * What it computes, in the paper's order and notation:
 *   - Eq. 2: the multigroup, discrete-direction transport equation on a voxel
 *     grid with vacuum boundaries, solved by source iteration (Sec. II.C:
 *     "solves ... iteratively"), groups from high energy (g = 0) to low
 *     (downscatter only), diamond difference in space (Sec. IV).
 *   - Eq. 3: the scalar fluence as the quadrature sum over the N(N+2)
 *     level-symmetric directions (Sec. II.E lists S2..S8 = 8/24/48/80).
 *   - Eqs. 4-7: the first-collision split; the uncollided fluence of a point
 *     source is ray traced (Sec. II.B) and its first-collision source drives
 *     the collided solve.
 *   - Eqs. 8-22 and Table 1: the sub-sweep (wavefront) counts and members.
 *
 * Readings taken where the paper is silent or garbled (Eq. 2 is printed with
 * the wrong sums): the scatter kernel is expanded in Legendre moments with
 * sigma_s(mu0) = sum_l (2l+1)/(4 pi) sigma_{s,l} P_l(mu0); real spherical
 * harmonics with the addition-theorem normalisation carry the moments; the
 * diamond-difference cell solve gets a set-to-zero negative-flux fixup with
 * rebalance; the residual is the relative L2 change of the scalar fluence;
 * the uncollided fluence is the voxel-centre point value; the level-symmetric
 * mu_1 values are the textbook ones (S4 from its fourth-moment condition).
 *
 * Deliberately plain: triple loops in upwind order, one direction at a time,
 * no blocking or reordering. Octants may run on separate OpenMP threads, each
 * with its own moment partial; partials are summed in fixed order 0..7, so the
 * result does not depend on the thread count.
 *
 * parity unpinned: whole-solve fluence values (the paper prints no numbers);
 * everything else is pinned by the tests (see tests/test_oracle_*.py).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORA_PI 3.14159265358979323846

/* ------------------------------------------------------------------------- */
/* Level-symmetric quadrature (Sec. II.E: S2/S4/S6/S8 = 8/24/48/80 directions) */
/* ------------------------------------------------------------------------- */

/* Direction cosine levels mu_i, i = 1..N/2:
 * mu_i^2 = mu_1^2 + (i-1) * 2 (1 - 3 mu_1^2) / (N - 2). */
static int ora_levels(int N, double *lev)
{
    double mu1;
    int h = N / 2, i;
    switch (N) {
    case 2: mu1 = sqrt(1.0 / 3.0); break;
    /* S4: mu_1 solves the octant fourth-moment condition
     * (2 mu_1^4 + (1 - 2 mu_1^2)^2) / 3 = 1/5. */
    case 4: mu1 = sqrt((2.0 - sqrt(1.6)) / 6.0); break;
    case 6: mu1 = 0.2666355; break;   /* textbook LS tables */
    case 8: mu1 = 0.2182179; break;
    default: return -1;
    }
    for (i = 0; i < h; ++i)
        lev[i] = (h == 1) ? mu1 : sqrt(mu1 * mu1 + i * 2.0 * (1.0 - 3.0 * mu1 * mu1) / (N - 2));
    return h;
}

/* Dense Gaussian elimination with partial pivoting (tiny systems). */
static int ora_gauss(int n, double *A, double *b)
{
    int i, j, k;
    for (k = 0; k < n; ++k) {
        int p = k;
        for (i = k + 1; i < n; ++i)
            if (fabs(A[i * n + k]) > fabs(A[p * n + k])) p = i;
        if (A[p * n + k] == 0.0) return -1;
        if (p != k) {
            for (j = 0; j < n; ++j) { double t = A[k * n + j]; A[k * n + j] = A[p * n + j]; A[p * n + j] = t; }
            { double t = b[k]; b[k] = b[p]; b[p] = t; }
        }
        for (i = k + 1; i < n; ++i) {
            double f = A[i * n + k] / A[k * n + k];
            for (j = k; j < n; ++j) A[i * n + j] -= f * A[k * n + j];
            b[i] -= f * b[k];
        }
    }
    for (i = n - 1; i >= 0; --i) {
        double s = b[i];
        for (j = i + 1; j < n; ++j) s -= A[i * n + j] * b[j];
        b[i] = s / A[i * n + i];
    }
    return 0;
}

/*
 * Level-symmetric S_N set. Per octant the points are the level triples
 * (a, b, c) with a + b + c = N/2 - 1, Omega = (mu_a, mu_b, mu_c), listed in
 * lexicographic (a, b, c) order. Points that are permutations of each other
 * share a weight; the class weights solve the even-moment conditions
 * sum_octant w mu_x^(2k) = 1/(2k+1) for k in {0, 2, 3} (as many as there are
 * classes; k = 1 holds by symmetry), normalised to 1 per octant, then scaled
 * by pi/2 so the full set sums to 4 pi. Octant o = sx + 2 sy + 4 sz, a set bit
 * meaning a negative cosine. Returns the direction count or -1.
 */
int ora_quadrature(int N, double *mu, double *eta, double *xi, double *w)
{
    double lev[4];
    int h = ora_levels(N, lev);
    int pa[10], pb[10], pc[10], cls[10], key[10][3];
    int np = 0, ncls = 0, a, b, p, c, o, r;
    static const int ks[3] = {0, 2, 3};
    double A[9], rhs[3];
    if (h < 0) return -1;
    for (a = 0; a < h; ++a)
        for (b = 0; b < h - a; ++b) {
            int cc = h - 1 - a - b, s[3] = {a, b, cc}, t;
            /* sort the triple to find its permutation class */
            if (s[0] > s[1]) { t = s[0]; s[0] = s[1]; s[1] = t; }
            if (s[1] > s[2]) { t = s[1]; s[1] = s[2]; s[2] = t; }
            if (s[0] > s[1]) { t = s[0]; s[0] = s[1]; s[1] = t; }
            for (c = 0; c < ncls; ++c)
                if (key[c][0] == s[0] && key[c][1] == s[1] && key[c][2] == s[2]) break;
            if (c == ncls) { key[c][0] = s[0]; key[c][1] = s[1]; key[c][2] = s[2]; ++ncls; }
            pa[np] = a; pb[np] = b; pc[np] = cc; cls[np] = c; ++np;
        }
    for (r = 0; r < ncls; ++r) {
        for (c = 0; c < ncls; ++c) A[r * ncls + c] = 0.0;
        for (p = 0; p < np; ++p) A[r * ncls + cls[p]] += pow(lev[pa[p]], 2.0 * ks[r]);
        rhs[r] = 1.0 / (2.0 * ks[r] + 1.0);
    }
    if (ora_gauss(ncls, A, rhs) != 0) return -1;
    for (o = 0; o < 8; ++o) {
        double sx = (o & 1) ? -1.0 : 1.0, sy = (o & 2) ? -1.0 : 1.0, sz = (o & 4) ? -1.0 : 1.0;
        for (p = 0; p < np; ++p) {
            int n = o * np + p;
            mu[n] = sx * lev[pa[p]];
            eta[n] = sy * lev[pb[p]];
            xi[n] = sz * lev[pc[p]];
            w[n] = rhs[cls[p]] * (ORA_PI / 2.0);
        }
    }
    return 8 * np;
}

/* ------------------------------------------------------------------------- */
/* Real spherical harmonics (Legendre-moment scattering, Fig. 7 / Sec. II.E)  */
/* ------------------------------------------------------------------------- */

/* Associated Legendre P_l^m(x), m >= 0, without the Condon-Shortley phase. */
double ora_assoc_legendre(int l, int m, double x)
{
    double pmm = 1.0, s = sqrt((1.0 - x) * (1.0 + x)), f = 1.0, pm1, pll = 0.0;
    int i, ll;
    for (i = 1; i <= m; ++i) { pmm *= f * s; f += 2.0; }
    if (l == m) return pmm;
    pm1 = x * (2 * m + 1) * pmm;
    if (l == m + 1) return pm1;
    for (ll = m + 2; ll <= l; ++ll) {
        pll = (x * (2 * ll - 1) * pm1 - (ll + m - 1) * pmm) / (ll - m);
        pmm = pm1;
        pm1 = pll;
    }
    return pll;
}

/* Y_lm with sum_m Y_lm(O) Y_lm(O') = P_l(O . O'): Y_l0 = P_l(xi);
 * Y_l,+-m = sqrt(2 (l-m)!/(l+m)!) P_l^m(xi) {cos, sin}(m phi), phi = atan2(eta, mu). */
double ora_real_sh(int l, int m, double mu, double eta, double xi)
{
    int am = m < 0 ? -m : m, i;
    double P = ora_assoc_legendre(l, am, xi), ratio = 1.0, phi;
    if (m == 0) return P;
    for (i = l - am + 1; i <= l + am; ++i) ratio /= (double)i;
    phi = atan2(eta, mu);
    return sqrt(2.0 * ratio) * P * (m > 0 ? cos(am * phi) : sin(am * phi));
}

/* ------------------------------------------------------------------------- */
/* Sub-sweeps (Sec. II.B, Eqs. 8-22, Table 1)                                 */
/* ------------------------------------------------------------------------- */

static long tri(long d) { return d * (d + 1) / 2; }
static long pos0(long v) { return v > 0 ? v : 0; }

/* Eq. 9: P = C_s - L_x - L_y - L_z + G_xy + G_yz + G_xz with Eqs. 10-22. */
long ora_subsweep_size(int nx, int ny, int nz, int S)
{
    long Cs = (long)(S + 1) * (S + 2) / 2;
    long Lx = tri(pos0(S + 1 - nx)), Ly = tri(pos0(S + 1 - ny)), Lz = tri(pos0(S + 1 - nz));
    long Gxy = tri(pos0(S + 1 - nx - ny)), Gyz = tri(pos0(S + 1 - ny - nz));
    long Gxz = tri(pos0(S + 1 - nx - nz));
    return Cs - Lx - Ly - Lz + Gxy + Gyz + Gxz;
}

/* Members of sub-sweep S (i_x + i_y + i_z = S under Eq. 8), i_x descending then
 * i_y descending, as Table 1 lists them. Writes triples, returns the count. */
long ora_subsweep_cells(int nx, int ny, int nz, int S, int32_t *out)
{
    long n = 0;
    int ix, iy, iz;
    for (ix = nx - 1; ix >= 0; --ix)
        for (iy = ny - 1; iy >= 0; --iy) {
            iz = S - ix - iy;
            if (iz < 0 || iz >= nz) continue;
            if (out) { out[3 * n] = ix; out[3 * n + 1] = iy; out[3 * n + 2] = iz; }
            ++n;
        }
    return n;
}

/* ------------------------------------------------------------------------- */
/* Problem description                                                        */
/* ------------------------------------------------------------------------- */

typedef struct {
    int nx, ny, nz;
    double dx, dy, dz, x0, y0, z0;
    int G, N, L, n_mat;
    const double *sigma_t;   /* [n_mat][G] */
    const double *sigma_s;   /* [n_mat][L+1][G_from][G_to] */
    const int32_t *mat;      /* [nz][ny][nx] */
    const double *scale_t;   /* [V] or NULL */
    const double *scale_s;   /* [V] or NULL */
    double tol;
    int max_iters;
    int n_threads;
    int fixup;               /* 1: set-to-zero fixup (the solver's scheme); 0: plain DD */
} ora_problem;

typedef struct {
    int kind;                /* 0 volumetric, 1 point / cone, 2 sum of point / cone sources */
    const double *q;         /* kind 0: [G][V] photons/cm^3 */
    double pos[3], axis[3], half_angle;
    const double *spectrum;  /* kind 1: [G] */
    int n_cones;             /* kind 2: number of cones */
    const double *cone_geo;  /* kind 2: [n_cones][13] pos, axis, half-angle, aperture, normal,
                                half azimuth, half polar */
    const double *cone_spec; /* kind 2: [n_cones][G] */
    int aperture;            /* kind 1: 0 cone (half_angle), 1 fan (the next three fields) */
    double normal[3];        /* fan: normal of the fan plane (not parallel to axis) */
    double half_azimuth;     /* fan: half the azimuthal angle subtended, in the fan plane */
    double half_polar;       /* fan: half the polar angle subtended, out of the fan plane */
} ora_source;

/* Whether the unit direction u from the source lies in its beam (Sec. II.C
 * source types). Cone: angle(u, axis) <= half_angle. Fan: in the frame of the
 * central ray a, the fan-plane normal n (made orthogonal to a) and t = n x a,
 * the elevation asin(u.n) and the azimuth atan2(u.t, u.a) lie within the half
 * polar and half azimuthal angles. */
static int ora_in_beam(const ora_source *s, const double u[3])
{
    double a[3], n[3], t[3], an, nn, na, ua, un, ut;
    int i;
    an = sqrt(s->axis[0] * s->axis[0] + s->axis[1] * s->axis[1] + s->axis[2] * s->axis[2]);
    for (i = 0; i < 3; ++i) a[i] = s->axis[i] / an;
    if (s->aperture != 1) {
        if (s->half_angle >= ORA_PI) return 1;
        return u[0] * a[0] + u[1] * a[1] + u[2] * a[2] >= cos(s->half_angle);
    }
    na = s->normal[0] * a[0] + s->normal[1] * a[1] + s->normal[2] * a[2];
    for (i = 0; i < 3; ++i) n[i] = s->normal[i] - na * a[i];
    nn = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
    for (i = 0; i < 3; ++i) n[i] /= nn;
    t[0] = n[1] * a[2] - n[2] * a[1];
    t[1] = n[2] * a[0] - n[0] * a[2];
    t[2] = n[0] * a[1] - n[1] * a[0];
    ua = u[0] * a[0] + u[1] * a[1] + u[2] * a[2];
    un = u[0] * n[0] + u[1] * n[1] + u[2] * n[2];
    ut = u[0] * t[0] + u[1] * t[1] + u[2] * t[2];
    return fabs(un) <= sin(s->half_polar) && fabs(atan2(ut, ua)) <= s->half_azimuth;
}

typedef struct {
    double *phi_u;      /* [G][V] uncollided fluence (kind 1), may be NULL */
    double *phi_c;      /* [G][K][V] collided moments */
    int32_t *iters;     /* [G] */
    double *resid;      /* [G] final residual */
    double *src;        /* [G] sum_v V_c T_00 of the last sweep */
    double *absorb;     /* [G] sum_v V_c sigma_t phi_00 of the last sweep */
    double *leak;       /* [G] boundary leakage of the last sweep */
    int64_t *fixups;    /* [G] cells where the fixup fired, summed over sweeps */
} ora_result;

static double ora_sigt(const ora_problem *p, int v, int g)
{
    double s = p->sigma_t[p->mat[v] * p->G + g];
    return p->scale_t ? s * p->scale_t[v] : s;
}

static double ora_sigs(const ora_problem *p, int v, int l, int gf, int gt)
{
    double s = p->sigma_s[(((size_t)p->mat[v] * (p->L + 1) + l) * p->G + gf) * p->G + gt];
    return p->scale_s ? s * p->scale_s[v] : s;
}

/* ------------------------------------------------------------------------- */
/* Uncollided fluence (Eq. 4 with no scatter term, ray traced, Sec. II.B)     */
/* ------------------------------------------------------------------------- */

static int ora_cmp(const void *a, const void *b)
{
    double x = *(const double *)a, y = *(const double *)b;
    return (x > y) - (x < y);
}

/* Siddon-style segment list from P to C: every plane crossing of the grid
 * gives a parameter alpha in (0,1); sorted, consecutive alphas bound a
 * segment whose midpoint names its voxel. Outside the grid is vacuum.
 * Writes voxel ids and lengths; returns the segment count. */
static int ora_segments(const ora_problem *p, const double P[3], const double C[3],
                        double *alpha, int *seg_v, double *seg_len)
{
    int dims[3] = {p->nx, p->ny, p->nz}, ax, i, n = 0, ns = 0;
    double lo[3] = {p->x0, p->y0, p->z0}, h[3] = {p->dx, p->dy, p->dz}, d[3], len;
    for (ax = 0; ax < 3; ++ax) d[ax] = C[ax] - P[ax];
    len = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    alpha[n++] = 0.0;
    alpha[n++] = 1.0;
    for (ax = 0; ax < 3; ++ax) {
        if (d[ax] == 0.0) continue;
        for (i = 0; i <= dims[ax]; ++i) {
            double a = (lo[ax] + i * h[ax] - P[ax]) / d[ax];
            if (a > 0.0 && a < 1.0) alpha[n++] = a;
        }
    }
    qsort(alpha, n, sizeof(double), ora_cmp);
    for (i = 0; i + 1 < n; ++i) {
        double a0 = alpha[i], a1 = alpha[i + 1], am, q[3];
        int idx[3], inside = 1;
        if (!(a1 > a0)) continue;
        am = 0.5 * (a0 + a1);
        for (ax = 0; ax < 3; ++ax) {
            q[ax] = P[ax] + am * d[ax];
            idx[ax] = (int)floor((q[ax] - lo[ax]) / h[ax]);
            if (idx[ax] < 0 || idx[ax] >= dims[ax]) inside = 0;
        }
        if (!inside) continue;
        seg_v[ns] = (idx[2] * p->ny + idx[1]) * p->nx + idx[0];
        seg_len[ns] = (a1 - a0) * len;
        ++ns;
    }
    return ns;
}

static int ora_max_alphas(const ora_problem *p) { return p->nx + p->ny + p->nz + 8; }

/* Uncollided fluence at the centre of voxel v for every group:
 * phi_u^g = spectrum_g exp(-tau^g) / (4 pi r^2) inside the cone, 0 outside,
 * tau^g = sum over segments of sigma_t^g * length. Also returns the unit
 * direction of flight Omega_u = (C - P)/r. */
int ora_uncollided_voxel(const ora_problem *p, const ora_source *s, int v,
                         double *phi_u_g, double *omega_u)
{
    int i = v % p->nx, j = (v / p->nx) % p->ny, k = v / (p->nx * p->ny), g, ns, t;
    int na = ora_max_alphas(p);
    double C[3], d[3], r2, r;
    double *alpha = (double *)malloc(sizeof(double) * na);
    int *sv = (int *)malloc(sizeof(int) * na);
    double *sl = (double *)malloc(sizeof(double) * na);
    if (!alpha || !sv || !sl) { free(alpha); free(sv); free(sl); return -1; }
    C[0] = p->x0 + (i + 0.5) * p->dx;
    C[1] = p->y0 + (j + 0.5) * p->dy;
    C[2] = p->z0 + (k + 0.5) * p->dz;
    for (t = 0; t < 3; ++t) d[t] = C[t] - s->pos[t];
    r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    r = sqrt(r2);
    for (t = 0; t < 3; ++t) omega_u[t] = d[t] / r;
    if (!ora_in_beam(s, omega_u)) {
        for (g = 0; g < p->G; ++g) phi_u_g[g] = 0.0;
    } else {
        ns = ora_segments(p, s->pos, C, alpha, sv, sl);
        for (g = 0; g < p->G; ++g) {
            double tau = 0.0;
            for (t = 0; t < ns; ++t) tau += ora_sigt(p, sv[t], g) * sl[t];
            phi_u_g[g] = s->spectrum[g] * exp(-tau) / (4.0 * ORA_PI * r2);
        }
    }
    free(alpha); free(sv); free(sl);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Diamond-difference cell solve with set-to-zero fixup (Sec. IV)             */
/* ------------------------------------------------------------------------- */

/*
 * One cell, one direction. a[d] = 2 |Omega_d| / Delta_d. Diamond difference
 * closes each dimension with psi_c = (psi_in + psi_out)/2, which with the cell
 * balance sum_d (a_d/2)(psi_out - psi_in) + sigma_t psi_c = q gives
 *     psi_c = (q + sum_d a_d psi_in_d) / (sigma_t + sum_d a_d).
 * If an outgoing value 2 psi_c - psi_in_d is negative it is set to zero and
 * dropped from the closure; the balance then gives
 *     psi_c = (q + sum_{d in F} (a_d/2) psi_in_d + sum_{d not in F} a_d psi_in_d)
 *             / (sigma_t + sum_{d not in F} a_d),
 * repeated until no new negative appears (all negatives of a pass are zeroed
 * together). Returns psi_c; writes out[3]; *nfix counts the passes taken.
 */
static double ora_dd_cell_mask(double q, double sig, const double a[3], const double in[3],
                               double out[3], int *nfix, unsigned char *mask);

double ora_dd_cell(double q, double sig, const double a[3], const double in[3],
                   double out[3], int *nfix)
{
    return ora_dd_cell_mask(q, sig, a, in, out, nfix, NULL);
}

/* the same cell solve, also reporting the fixup set (bit d = face d zeroed) */
static double ora_dd_cell_mask(double q, double sig, const double a[3], const double in[3],
                               double out[3], int *nfix, unsigned char *mask)
{
    int fixed[3] = {0, 0, 0}, d, passes = 0;
    double psi = (q + a[0] * in[0] + a[1] * in[1] + a[2] * in[2]) / (sig + a[0] + a[1] + a[2]);
    for (d = 0; d < 3; ++d) out[d] = 2.0 * psi - in[d];
    for (;;) {
        int any = 0;
        double num = q, den = sig;
        for (d = 0; d < 3; ++d)
            if (!fixed[d] && out[d] < 0.0) { fixed[d] = 1; any = 1; }
        if (!any) break;
        ++passes;
        for (d = 0; d < 3; ++d) {
            if (fixed[d]) num += 0.5 * a[d] * in[d];
            else { num += a[d] * in[d]; den += a[d]; }
        }
        psi = num / den;
        for (d = 0; d < 3; ++d) out[d] = fixed[d] ? 0.0 : 2.0 * psi - in[d];
    }
    if (nfix) *nfix = passes;
    if (mask) *mask = (unsigned char)(fixed[0] | fixed[1] << 1 | fixed[2] << 2);
    return psi;
}

/*
 * Sweep one direction over the whole grid in upwind order (z outer, y, x
 * inner, each running along the sign of its cosine). Q[V] is the angular
 * source of this direction, sigt[V] the total cross section; every boundary
 * face on the inflow side carries the uniform value `inflow` (0 for vacuum;
 * the non-zero hook exists for the pure-absorber tests). Writes the
 * cell-centre angular flux psi[V]; returns the leakage
 * sum over outflow boundary faces of |Omega_d| A_d psi_out in *leak and the
 * number of fixup cells in *nfix.
 */
void ora_sweep_dir(const ora_problem *p, const double *sigt, double mu, double eta, double xi,
                   const double *Q, double inflow, double *psi, double *leak, int64_t *nfix)
{
    int nx = p->nx, ny = p->ny, nz = p->nz, ii, jj, kk;
    double a[3] = {2.0 * fabs(mu) / p->dx, 2.0 * fabs(eta) / p->dy, 2.0 * fabs(xi) / p->dz};
    double *fx = (double *)malloc(sizeof(double) * ny * nz);  /* x-face of line (j,k) */
    double *fy = (double *)malloc(sizeof(double) * nx * nz);  /* y-face of line (i,k) */
    double *fz = (double *)malloc(sizeof(double) * nx * ny);  /* z-face of line (i,j) */
    double L = 0.0;
    int64_t nf = 0;
    for (ii = 0; ii < ny * nz; ++ii) fx[ii] = inflow;
    for (ii = 0; ii < nx * nz; ++ii) fy[ii] = inflow;
    for (ii = 0; ii < nx * ny; ++ii) fz[ii] = inflow;
    for (kk = 0; kk < nz; ++kk) {
        int k = xi > 0 ? kk : nz - 1 - kk;
        for (jj = 0; jj < ny; ++jj) {
            int j = eta > 0 ? jj : ny - 1 - jj;
            for (ii = 0; ii < nx; ++ii) {
                int i = mu > 0 ? ii : nx - 1 - ii, v = (k * ny + j) * nx + i, np;
                double in[3] = {fx[k * ny + j], fy[k * nx + i], fz[j * nx + i]}, out[3];
                if (p->fixup) {
                    psi[v] = ora_dd_cell(Q[v], sigt[v], a, in, out, &np);
                } else {
                    int d;
                    psi[v] = (Q[v] + a[0] * in[0] + a[1] * in[1] + a[2] * in[2]) /
                             (sigt[v] + a[0] + a[1] + a[2]);
                    for (d = 0; d < 3; ++d) out[d] = 2.0 * psi[v] - in[d];
                    np = 0;
                }
                if (np) ++nf;
                fx[k * ny + j] = out[0];
                fy[k * nx + i] = out[1];
                fz[j * nx + i] = out[2];
            }
        }
    }
    /* after the sweep every face slot holds the value leaving the grid */
    for (ii = 0; ii < ny * nz; ++ii) L += fabs(mu) * p->dy * p->dz * fx[ii];
    for (ii = 0; ii < nx * nz; ++ii) L += fabs(eta) * p->dx * p->dz * fy[ii];
    for (ii = 0; ii < nx * ny; ++ii) L += fabs(xi) * p->dx * p->dy * fz[ii];
    *leak = L;
    *nfix = nf;
    free(fx); free(fy); free(fz);
}

/* ------------------------------------------------------------------------- */
/* Source iteration (Eqs. 2, 3, 5-7)                                         */
/* ------------------------------------------------------------------------- */

int ora_solve(const ora_problem *p, const ora_source *s, ora_result *res)
{
    const int V = p->nx * p->ny * p->nz, G = p->G, L = p->L, K = (L + 1) * (L + 1);
    const double vol = p->dx * p->dy * p->dz;
    int nd, n, k, g, v, l, m, it, o;
    double mu[80], eta[80], xi[80], w[80];
    double *Y, *D, *M, *phi_u, *omu, *F, *phi, *T, *sigt, *sigs, *part, *leak_o, *uy = NULL;
    int64_t *fix_o;
    int npo, nthreads = p->n_threads > 0 ? p->n_threads : 1;

    nd = ora_quadrature(p->N, mu, eta, xi, w);
    if (nd < 0 || V <= 0 || G <= 0 || L < 0) return -1;
    npo = nd / 8;
    Y = (double *)malloc(sizeof(double) * K * nd);
    D = (double *)malloc(sizeof(double) * K * nd);
    M = (double *)malloc(sizeof(double) * K * nd);
    phi_u = (double *)calloc((size_t)G * V, sizeof(double));
    omu = (double *)calloc((size_t)3 * V, sizeof(double));
    F = (double *)malloc(sizeof(double) * (size_t)K * V);
    phi = (double *)malloc(sizeof(double) * (size_t)K * V);
    T = (double *)malloc(sizeof(double) * (size_t)K * V);
    sigt = (double *)malloc(sizeof(double) * (size_t)V);
    sigs = (double *)malloc(sizeof(double) * (size_t)(L + 1) * V);
    part = (double *)malloc(sizeof(double) * (size_t)8 * K * V);
    leak_o = (double *)malloc(sizeof(double) * 8);
    fix_o = (int64_t *)malloc(sizeof(int64_t) * 8);
    if (!Y || !D || !M || !phi_u || !omu || !F || !phi || !T || !sigt || !sigs || !part) return -2;

    /* moment operators: phi_lm = sum_n w_n Y_lm(O_n) psi_n (Eq. 3 for l = 0);
     * Q_n = sum_lm (2l+1)/(4 pi) T_lm Y_lm(O_n) */
    for (l = 0; l <= L; ++l)
        for (m = -l; m <= l; ++m) {
            k = l * l + l + m;
            for (n = 0; n < nd; ++n) {
                Y[k * nd + n] = ora_real_sh(l, m, mu[n], eta[n], xi[n]);
                D[k * nd + n] = w[n] * Y[k * nd + n];
                M[k * nd + n] = (2.0 * l + 1.0) / (4.0 * ORA_PI) * Y[k * nd + n];
            }
        }

    /* Eq. 4: uncollided fluence of a point source, ray traced */
    if (s->kind == 1) {
        double *pg = (double *)malloc(sizeof(double) * G);
        for (v = 0; v < V; ++v) {
            ora_uncollided_voxel(p, s, v, pg, &omu[3 * v]);
            for (g = 0; g < G; ++g) phi_u[(size_t)g * V + v] = pg[g];
        }
        free(pg);
    }
    /* several cones summed into one source (the CT mode of Sec. II.E): the
     * uncollided fluence is the sum of the cones' and the first-collision
     * source needs, per group and moment, sum_c phi_u,c Y_lm(Omega_c) */
    if (s->kind == 2) {
        double *pg = (double *)malloc(sizeof(double) * G), om[3];
        int c;
        uy = (double *)calloc((size_t)G * K * V, sizeof(double));
        for (c = 0; c < s->n_cones; ++c) {
            ora_source one;
            memset(&one, 0, sizeof one);
            one.kind = 1;
            for (l = 0; l < 3; ++l) {
                one.pos[l] = s->cone_geo[13 * c + l];
                one.axis[l] = s->cone_geo[13 * c + 3 + l];
            }
            one.half_angle = s->cone_geo[13 * c + 6];
            one.aperture = (int)s->cone_geo[13 * c + 7];
            for (l = 0; l < 3; ++l) one.normal[l] = s->cone_geo[13 * c + 8 + l];
            one.half_azimuth = s->cone_geo[13 * c + 11];
            one.half_polar = s->cone_geo[13 * c + 12];
            one.spectrum = s->cone_spec + (size_t)c * G;
            for (v = 0; v < V; ++v) {
                ora_uncollided_voxel(p, &one, v, pg, om);
                for (g = 0; g < G; ++g) {
                    phi_u[(size_t)g * V + v] += pg[g];
                    for (l = 0; l <= L; ++l)
                        for (m = -l; m <= l; ++m)
                            uy[((size_t)g * K + l * l + l + m) * V + v] += pg[g] * ora_real_sh(l, m, om[0], om[1], om[2]);
                }
            }
        }
        free(pg);
    }
    if (res->phi_u) memcpy(res->phi_u, phi_u, sizeof(double) * (size_t)G * V);

    for (g = 0; g < G; ++g) {
        int64_t nfix_g = 0;
        /* fixed source of group g: external / first-collision source (Eq. 5)
         * plus downscatter from the converged collided moments of g' < g */
        for (k = 0; k < K; ++k) {
            l = (int)floor(sqrt((double)k) + 1e-9);
            while (l * l > k) --l;
            while ((l + 1) * (l + 1) <= k) ++l;
            m = k - l * l - l;
            for (v = 0; v < V; ++v) {
                double f = 0.0;
                int gp;
                if (s->kind == 0) {
                    if (k == 0) f = s->q[(size_t)g * V + v];
                } else if (s->kind == 2) {
                    for (gp = 0; gp <= g; ++gp)
                        f += ora_sigs(p, v, l, gp, g) * uy[((size_t)gp * K + k) * V + v];
                } else {
                    double y = ora_real_sh(l, m, omu[3 * v], omu[3 * v + 1], omu[3 * v + 2]);
                    for (gp = 0; gp <= g; ++gp)
                        f += ora_sigs(p, v, l, gp, g) * phi_u[(size_t)gp * V + v] * y;
                }
                for (gp = 0; gp < g; ++gp)
                    f += ora_sigs(p, v, l, gp, g) * res->phi_c[((size_t)gp * K + k) * V + v];
                F[(size_t)k * V + v] = f;
            }
        }
        for (v = 0; v < V; ++v) {
            sigt[v] = ora_sigt(p, v, g);
            for (l = 0; l <= L; ++l) sigs[(size_t)l * V + v] = ora_sigs(p, v, l, g, g);
        }
        for (v = 0; v < K * V; ++v) phi[v] = 0.0;

        for (it = 1; it <= p->max_iters; ++it) {
            double dn = 0.0, nn = 0.0, r, src = 0.0, ab = 0.0, lk = 0.0;
            /* scatter source: T_lm = F_lm + sigma_{s,l}^{g->g} phi_lm */
            for (k = 0; k < K; ++k) {
                l = 0;
                while ((l + 1) * (l + 1) <= k) ++l;
                for (v = 0; v < V; ++v)
                    T[(size_t)k * V + v] = F[(size_t)k * V + v] + sigs[(size_t)l * V + v] * phi[(size_t)k * V + v];
            }
            /* sweep every direction; each octant accumulates its own partial */
#pragma omp parallel for num_threads(nthreads) schedule(static) private(n, k, v)
            for (o = 0; o < 8; ++o) {
                double *Q = (double *)malloc(sizeof(double) * V);
                double *psi = (double *)malloc(sizeof(double) * V);
                double *po = part + (size_t)o * K * V, lko = 0.0;
                int64_t fo = 0;
                for (v = 0; v < K * V; ++v) po[v] = 0.0;
                for (n = o * npo; n < (o + 1) * npo; ++n) {
                    double ln;
                    int64_t fn;
                    for (v = 0; v < V; ++v) {
                        double q = 0.0;
                        for (k = 0; k < K; ++k) q += M[k * nd + n] * T[(size_t)k * V + v];
                        Q[v] = q;
                    }
                    ora_sweep_dir(p, sigt, mu[n], eta[n], xi[n], Q, 0.0, psi, &ln, &fn);
                    lko += w[n] * ln;
                    fo += fn;
                    for (k = 0; k < K; ++k)
                        for (v = 0; v < V; ++v) po[(size_t)k * V + v] += D[k * nd + n] * psi[v];
                }
                leak_o[o] = lko;
                fix_o[o] = fo;
                free(Q); free(psi);
            }
            /* Eq. 3 (and its higher moments): sum the octant partials in order */
            for (v = 0; v < K * V; ++v) {
                double acc = 0.0;
                for (o = 0; o < 8; ++o) acc += part[(size_t)o * K * V + v];
                T[v] = acc;  /* T now holds the new moments */
            }
            for (o = 0; o < 8; ++o) { lk += leak_o[o]; nfix_g += fix_o[o]; }
            for (v = 0; v < V; ++v) {
                double dnew = T[v], dold = phi[v];
                dn += (dnew - dold) * (dnew - dold);
                nn += dnew * dnew;
                ab += vol * sigt[v] * dnew;
                src += vol * (F[v] + sigs[v] * dold);
            }
            r = nn > 0.0 ? sqrt(dn / nn) : 0.0;
            memcpy(phi, T, sizeof(double) * (size_t)K * V);
            if (res->iters) res->iters[g] = it;
            if (res->resid) res->resid[g] = r;
            if (res->src) res->src[g] = src;
            if (res->absorb) res->absorb[g] = ab;
            if (res->leak) res->leak[g] = lk;
            if (r < p->tol) break;
        }
        if (res->fixups) res->fixups[g] = nfix_g;
        memcpy(res->phi_c + (size_t)g * K * V, phi, sizeof(double) * (size_t)K * V);
    }
    free(Y); free(D); free(M); free(phi_u); free(omu); free(F); free(phi); free(T); free(uy);
    free(sigt); free(sigs); free(part); free(leak_o); free(fix_o);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Discrete adjoint of the converged solve (gradients of a linear functional) */
/* ------------------------------------------------------------------------- */

/* Forward sweep of one direction that also records each cell's fixup set
 * (bit d set = face d zeroed) and its cell-centre flux. */
static void ora_sweep_dir_record(const ora_problem *p, const double *sigt, double mu, double eta,
                                 double xi, const double *Q, double *psi, unsigned char *fixset)
{
    int nx = p->nx, ny = p->ny, nz = p->nz, ii, jj, kk;
    double a[3] = {2.0 * fabs(mu) / p->dx, 2.0 * fabs(eta) / p->dy, 2.0 * fabs(xi) / p->dz};
    double *fx = (double *)calloc((size_t)ny * nz, sizeof(double));
    double *fy = (double *)calloc((size_t)nx * nz, sizeof(double));
    double *fz = (double *)calloc((size_t)nx * ny, sizeof(double));
    for (kk = 0; kk < nz; ++kk) {
        int k = xi > 0 ? kk : nz - 1 - kk;
        for (jj = 0; jj < ny; ++jj) {
            int j = eta > 0 ? jj : ny - 1 - jj;
            for (ii = 0; ii < nx; ++ii) {
                int i = mu > 0 ? ii : nx - 1 - ii, v = (k * ny + j) * nx + i, np;
                double in[3] = {fx[k * ny + j], fy[k * nx + i], fz[j * nx + i]}, out[3];
                psi[v] = ora_dd_cell_mask(Q[v], sigt[v], a, in, out, &np, &fixset[v]);
                fx[k * ny + j] = out[0];
                fy[k * nx + i] = out[1];
                fz[j * nx + i] = out[2];
            }
        }
    }
    free(fx); free(fy); free(fz);
}

/* Transpose of the recorded sweep: cells in the reverse of the forward
 * order; y[V] = dL/dpsi (direct), faces carry zeta = 2 (dL/d out-face) / a_d.
 * Per cell, with F the recorded fixup set:
 *   chi = (y + sum_{d not in F} a_d zeta_d) / (sigma + sum_{d not in F} a_d)
 *   zeta passed upstream = 2 chi - zeta_d (d not in F), chi (d in F).
 * chi = dL/dQ for the cell. */
static void ora_sweep_dir_adjoint(const ora_problem *p, const double *sigt, double mu, double eta,
                                  double xi, const double *y, const unsigned char *fixset, double *chi)
{
    int nx = p->nx, ny = p->ny, nz = p->nz, ii, jj, kk;
    double a[3] = {2.0 * fabs(mu) / p->dx, 2.0 * fabs(eta) / p->dy, 2.0 * fabs(xi) / p->dz};
    double *fx = (double *)calloc((size_t)ny * nz, sizeof(double));
    double *fy = (double *)calloc((size_t)nx * nz, sizeof(double));
    double *fz = (double *)calloc((size_t)nx * ny, sizeof(double));
    for (kk = 0; kk < nz; ++kk) {
        int k = xi > 0 ? nz - 1 - kk : kk;
        for (jj = 0; jj < ny; ++jj) {
            int j = eta > 0 ? ny - 1 - jj : jj;
            for (ii = 0; ii < nx; ++ii) {
                int i = mu > 0 ? nx - 1 - ii : ii, v = (k * ny + j) * nx + i, d;
                double z[3] = {fx[k * ny + j], fy[k * nx + i], fz[j * nx + i]};
                double num = y[v], den = sigt[v], c;
                for (d = 0; d < 3; ++d)
                    if (!(fixset[v] >> d & 1u)) { num += a[d] * z[d]; den += a[d]; }
                c = num / den;
                chi[v] = c;
                for (d = 0; d < 3; ++d) z[d] = (fixset[v] >> d & 1u) ? c : 2.0 * c - z[d];
                fx[k * ny + j] = z[0];
                fy[k * nx + i] = z[1];
                fz[j * nx + i] = z[2];
            }
        }
    }
    free(fx); free(fy); free(fz);
}

static int ora_l_of_k(int k)
{
    int l = 0;
    while ((l + 1) * (l + 1) <= k) ++l;
    return l;
}

/*
 * Gradient of L = sum_g sum_v a^g(v) phi_total^g(v) (a = dL_dphi, [G][V]) with
 * respect to the per-voxel multipliers scale_t and scale_s, at the solution of
 * ora_solve (Eqs. 2-7 with the readings above). The discrete adjoint of the
 * converged system: groups run G-1 -> 0; for each, the forward sweep is
 * recomputed from the converged moments to record psi and the fixup sets;
 * the adjoint source s = a e_0 + sum_{g2 > g} sigma_s^{g->g2} u^{g2} is
 * iterated with u = M^T H^T D^T (s + sigma_s^{gg} u) to p->tol; then
 *   dL/dsigma_t^g(v) = -sum_n chi_n psi_n,
 *   dL/dsigma_{s,l}^{g'->g}(v) = sum_{k in l} u_k (phi_c,k^{g'} + phi_u^{g'} Y_k(Omega_u)),
 *   dL/dphi_u^{g'} += sum_g sum_k u^g_k sigma_{s,l}^{g'->g} Y_k(Omega_u),
 * and the uncollided part goes back through the ray trace:
 *   dL/dtau^{g'}(v) = -phi_u^{g'}(v) dL/dphi_u^{g'}(v), tau = sum ell sigma_t.
 * dsig_t_g [G][V] (may be NULL) receives dL/dsigma_t^g(v) of the collided part.
 * Returns 0 on success.
 */
int ora_adjoint(const ora_problem *p, const ora_source *s, const double *dL_dphi,
                double *dL_dscale_t, double *dL_dscale_s, double *dsig_t_g)
{
    if (s->kind == 2) return -3;   /* the adjoint covers volumetric and single-cone sources */
    const int V = p->nx * p->ny * p->nz, G = p->G, L = p->L, K = (L + 1) * (L + 1);
    int nd, n, k, g, gp, v, it, l;
    double mu[80], eta[80], xi[80], w[80];
    double *Y, *D, *M, *omu, *Yu, *phic, *phiu, *T, *sigt, *psi, *u, *unew, *wv, *y, *chi, *sadj, *dphiu;
    unsigned char *fix;
    ora_result r;
    nd = ora_quadrature(p->N, mu, eta, xi, w);
    if (nd < 0) return -1;
    Y = (double *)malloc(sizeof(double) * K * nd);
    D = (double *)malloc(sizeof(double) * K * nd);
    M = (double *)malloc(sizeof(double) * K * nd);
    for (l = 0; l <= L; ++l)
        for (k = l * l; k < (l + 1) * (l + 1); ++k)
            for (n = 0; n < nd; ++n) {
                Y[k * nd + n] = ora_real_sh(l, k - l * l - l, mu[n], eta[n], xi[n]);
                D[k * nd + n] = w[n] * Y[k * nd + n];
                M[k * nd + n] = (2.0 * l + 1.0) / (4.0 * ORA_PI) * Y[k * nd + n];
            }
    phic = (double *)calloc((size_t)G * K * V, sizeof(double));
    phiu = (double *)calloc((size_t)G * V, sizeof(double));
    memset(&r, 0, sizeof r);
    r.phi_u = phiu;
    r.phi_c = phic;
    if (ora_solve(p, s, &r) != 0) return -2;
    omu = (double *)calloc((size_t)3 * V, sizeof(double));
    Yu = (double *)calloc((size_t)K * V, sizeof(double));
    if (s->kind == 1) {
        double *pg = (double *)malloc(sizeof(double) * G);
        for (v = 0; v < V; ++v) {
            ora_uncollided_voxel(p, s, v, pg, &omu[3 * v]);
            for (l = 0; l <= L; ++l)
                for (k = l * l; k < (l + 1) * (l + 1); ++k)
                    Yu[(size_t)k * V + v] = ora_real_sh(l, k - l * l - l, omu[3 * v], omu[3 * v + 1], omu[3 * v + 2]);
        }
        free(pg);
    }
    T = (double *)malloc(sizeof(double) * (size_t)K * V);
    sigt = (double *)malloc(sizeof(double) * V);
    psi = (double *)malloc(sizeof(double) * (size_t)nd * V);
    fix = (unsigned char *)malloc((size_t)nd * V);
    u = (double *)malloc(sizeof(double) * (size_t)K * V);
    unew = (double *)malloc(sizeof(double) * (size_t)K * V);
    wv = (double *)malloc(sizeof(double) * (size_t)K * V);
    y = (double *)malloc(sizeof(double) * V);
    chi = (double *)malloc(sizeof(double) * (size_t)nd * V);
    sadj = (double *)calloc((size_t)G * K * V, sizeof(double));   /* adjoint sources per group */
    dphiu = (double *)calloc((size_t)G * V, sizeof(double));
    for (v = 0; v < V; ++v) { dL_dscale_t[v] = 0.0; dL_dscale_s[v] = 0.0; }
    for (g = 0; g < G; ++g)
        for (v = 0; v < V; ++v) sadj[(size_t)g * K * V + v] = dL_dphi[(size_t)g * V + v];

    for (g = G - 1; g >= 0; --g) {
        /* converged source of group g: T = q + downscatter + in-group scatter */
        for (v = 0; v < V; ++v) sigt[v] = ora_sigt(p, v, g);
        for (k = 0; k < K; ++k) {
            l = ora_l_of_k(k);
            for (v = 0; v < V; ++v) {
                double t = (s->kind == 0 && k == 0) ? s->q[(size_t)g * V + v] : 0.0;
                for (gp = 0; gp <= g; ++gp) {
                    double sg = ora_sigs(p, v, l, gp, g);
                    if (s->kind == 1) t += sg * phiu[(size_t)gp * V + v] * Yu[(size_t)k * V + v];
                    t += sg * phic[((size_t)gp * K + k) * V + v];
                }
                T[(size_t)k * V + v] = t;
            }
        }
        /* record psi and the fixup sets of the converged sweep */
        for (n = 0; n < nd; ++n) {
            double *Q = unew;   /* scratch */
            for (v = 0; v < V; ++v) {
                double q = 0.0;
                for (k = 0; k < K; ++k) q += M[k * nd + n] * T[(size_t)k * V + v];
                Q[v] = q;
            }
            ora_sweep_dir_record(p, sigt, mu[n], eta[n], xi[n], Q, psi + (size_t)n * V, fix + (size_t)n * V);
        }
        /* adjoint source iteration */
        for (v = 0; v < K * V; ++v) u[v] = 0.0;
        for (it = 1; it <= p->max_iters; ++it) {
            double dn = 0.0, nn = 0.0;
            for (k = 0; k < K; ++k) {
                l = ora_l_of_k(k);
                for (v = 0; v < V; ++v)
                    wv[(size_t)k * V + v] = sadj[((size_t)g * K + k) * V + v] + ora_sigs(p, v, l, g, g) * u[(size_t)k * V + v];
            }
            for (v = 0; v < K * V; ++v) unew[v] = 0.0;
            for (n = 0; n < nd; ++n) {
                for (v = 0; v < V; ++v) {
                    double t = 0.0;
                    for (k = 0; k < K; ++k) t += D[k * nd + n] * wv[(size_t)k * V + v];
                    y[v] = t;
                }
                ora_sweep_dir_adjoint(p, sigt, mu[n], eta[n], xi[n], y, fix + (size_t)n * V, chi + (size_t)n * V);
                for (k = 0; k < K; ++k)
                    for (v = 0; v < V; ++v) unew[(size_t)k * V + v] += M[k * nd + n] * chi[(size_t)n * V + v];
            }
            for (v = 0; v < V; ++v) {
                double d = unew[v] - u[v];
                dn += d * d;
                nn += unew[v] * unew[v];
            }
            memcpy(u, unew, sizeof(double) * (size_t)K * V);
            if (!(nn > 0.0) || sqrt(dn / nn) < p->tol) break;
        }
        /* gradients of group g */
        for (v = 0; v < V; ++v) {
            const int m = p->mat[v];
            const double ss = p->scale_s ? p->scale_s[v] : 1.0;
            double gst = 0.0, gss = 0.0;
            for (n = 0; n < nd; ++n) gst -= chi[(size_t)n * V + v] * psi[(size_t)n * V + v];
            if (dsig_t_g) dsig_t_g[(size_t)g * V + v] = gst;
            dL_dscale_t[v] += p->sigma_t[m * G + g] * gst;
            for (k = 0; k < K; ++k) {
                const double uk = u[(size_t)k * V + v];
                l = ora_l_of_k(k);
                for (gp = 0; gp <= g; ++gp) {
                    const double tab = p->sigma_s[(((size_t)m * (L + 1) + l) * G + gp) * G + g];
                    double src = phic[((size_t)gp * K + k) * V + v];
                    if (s->kind == 1) {
                        src += phiu[(size_t)gp * V + v] * Yu[(size_t)k * V + v];
                        dphiu[(size_t)gp * V + v] += uk * tab * ss * Yu[(size_t)k * V + v];
                    }
                    gss += tab * uk * src;
                }
                /* adjoint downscatter into the lower groups */
                for (gp = 0; gp < g; ++gp)
                    sadj[((size_t)gp * K + k) * V + v] += ora_sigs(p, v, l, gp, g) * uk;
            }
            dL_dscale_s[v] += gss;
        }
    }
    /* uncollided fluence: back through the ray trace */
    if (s->kind == 1) {
        int na = ora_max_alphas(p), ns, t;
        double *alpha = (double *)malloc(sizeof(double) * na), *sl = (double *)malloc(sizeof(double) * na);
        int *sv = (int *)malloc(sizeof(int) * na);
        for (v = 0; v < V; ++v) {
            int i = v % p->nx, j = (v / p->nx) % p->ny, kz = v / (p->nx * p->ny);
            double C[3] = {p->x0 + (i + 0.5) * p->dx, p->y0 + (j + 0.5) * p->dy, p->z0 + (kz + 0.5) * p->dz};
            int any = 0;
            for (g = 0; g < G; ++g) any |= phiu[(size_t)g * V + v] != 0.0;
            if (!any) continue;
            ns = ora_segments(p, s->pos, C, alpha, sv, sl);
            for (t = 0; t < ns; ++t) {
                const int vp = sv[t], m = p->mat[vp];
                double acc = 0.0;
                for (g = 0; g < G; ++g) {
                    const double e = -phiu[(size_t)g * V + v] *
                                     (dL_dphi[(size_t)g * V + v] + dphiu[(size_t)g * V + v]);
                    acc += e * sl[t] * p->sigma_t[m * G + g];
                }
                dL_dscale_t[vp] += acc;
            }
        }
        free(alpha); free(sl); free(sv);
    }
    free(Y); free(D); free(M); free(phic); free(phiu); free(omu); free(Yu); free(T); free(sigt);
    free(psi); free(fix); free(u); free(unew); free(wv); free(y); free(chi); free(sadj); free(dphiu);
    return 0;
}

int ora_has_openmp(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 0;
#endif
}
