/*
 * dts.h -- C ABI of the B300 discrete-ordinates (S_N) photon-transport solver.
 *
 * The library solves the multigroup, discrete-direction linear Boltzmann
 * equation on a voxel grid (Eq. 2 of Norris, Wagstaff & Liu, "DOCTORS",
 * arxiv 1910.11335) with vacuum boundaries (Sec. II.A) by source iteration:
 * energy groups run from high energy (group 0) to low, because scattering only
 * moves photons down in energy; inside a group every octant is swept along
 * i+j+k wavefronts (Sec. II.B, Eqs. 8-22) with all of its level-symmetric
 * directions (Sec. II.E: S2/S4/S6/S8) in flight, using diamond difference
 * (Sec. IV) with a set-to-zero negative-flux fixup; the sweep is fed by a
 * Legendre-moment scatter source and reduced to scalar fluence by the
 * quadrature of Eq. 3. Point and cone-beam sources use the first-collision
 * split of Eqs. 4-7: the uncollided fluence is ray traced and its first
 * collisions drive the collided solve.
 *
 * Conventions (every entry point):
 *   - Voxel arrays are [nz][ny][nx] with x fastest; V = nx*ny*nz.
 *   - Group arrays put group 0 at the highest energy.
 *   - Every call returns a dts_status and never throws. On failure the
 *     problem keeps a message readable with dts_last_error(problem); failures
 *     of dts_create_problem leave it in dts_last_error(NULL) (per thread).
 *   - The caller owns every buffer it passes in or out. Input arrays are
 *     copied before the call returns. Host pointers must stay valid only for
 *     the duration of the call (except the buffer of dts_set_host_output,
 *     which later solves write into).
 *   - All device work is ordered on the stream given in dts_problem_desc
 *     (or an internal stream when that is NULL). One problem must be used by
 *     one host thread at a time. Distinct problems are independent.
 *   - Pointers named *_is_device select device (1) or host (0) memory.
 */
#ifndef DTS_H
#define DTS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dts_problem dts_problem;   /* opaque, owned by the library */

typedef enum {
    DTS_OK = 0,
    DTS_ERR_INVALID_ARG = 1,    /* a size, pointer or value is out of range */
    DTS_ERR_STATE = 2,          /* call order violated (e.g. solve before set_*) */
    DTS_ERR_OOM = 3,            /* device or host allocation failed */
    DTS_ERR_CUDA = 4,           /* a CUDA runtime call failed */
    DTS_ERR_NOT_CONVERGED = 5,  /* max_iters reached above tol; results are usable */
    DTS_ERR_TIMEOUT = 6,        /* a bounded device wait gave up (tensor-core forms: the moment
                                   kernel's waits on its copies and MMAs, the sweep's on its face copies) */
    DTS_ERR_INTERNAL = 7        /* a device-side consistency check failed */
} dts_status;

/* Arithmetic of the sweep and of the moment<->direction contractions.
 * FP64: everything in FP64.
 * FP32: sweep, scatter-source contraction and per-octant moment partials in
 *       FP32 on the CUDA cores; the Eq. 3 octant sum of the scalar flux, the
 *       residual and the balance in FP64.
 * FP32_SPLITBF16: FP32 sweep; the scatter-source contraction of Eq. 2,
 *       Q_n = sum_k M[n][k] T_k over the K Legendre moments, runs on the
 *       tensor cores as a [cells x K] x [K x directions] product with both
 *       operands split into bf16 high and low parts (hi.hi + hi.lo + lo.hi,
 *       accumulated in FP32; ~1e-5 relative per term); each source iteration
 *       materialises Q (one FP32 value per cell and direction) and the sweep
 *       reads it. Eq. 3 moments from the FP32 angular fluxes, scalar flux,
 *       residual and balance as in FP32.
 * FP32_TF32: as FP32_SPLITBF16 with tf32 high and low parts (TF32 tensor
 *       cores, three products; ~2^-21 relative per term).
 * The two tensor-core forms need the 8 x 4 x 4 tile (the default for them). */
typedef enum {
    DTS_PREC_FP64 = 0,
    DTS_PREC_FP32 = 1,
    DTS_PREC_FP32_SPLITBF16 = 2,
    DTS_PREC_FP32_TF32 = 3
} dts_precision;

typedef enum {
    DTS_COMP_UNCOLLIDED = 0,    /* ray-traced uncollided fluence (Eq. 4) */
    DTS_COMP_COLLIDED = 1,      /* source-iteration fluence (Eqs. 6-7) */
    DTS_COMP_TOTAL = 2          /* uncollided + collided (Sec. II.A) */
} dts_component;

typedef struct {
    int nx, ny, nz;             /* voxels per axis, each >= 1 */
    double dx, dy, dz;          /* voxel pitch in cm, > 0 */
    double x0, y0, z0;          /* low corner of the grid in cm */
    int n_groups;               /* G >= 1 */
    int sn_order;               /* level-symmetric order N in {2,4,6,8}: N(N+2) directions */
    int legendre_order;         /* scattering order L in 0..3: K = (L+1)^2 moments */
    int batch;                  /* B >= 1 independent sources solved together */
    dts_precision precision;
    double tol;                 /* stop a (source, group) when the relative L2 change of
                                   its scalar fluence drops below tol; 0 runs max_iters */
    int max_iters;              /* source iterations per group, >= 1 */
    void *cuda_stream;          /* cudaStream_t to order work on, or NULL */
    int device;                 /* CUDA device ordinal */
    int tile_x, tile_y, tile_z; /* wavefront tile in voxels (each 1..64); all 0 = default */
    int keep_moments;           /* 1: keep all K collided moments of every group */
} dts_problem_desc;

typedef struct {
    int kind;                   /* 0: isotropic volumetric source; 1: point / cone beam */
    const double *q;            /* kind 0: [G][V] photons/cm^3 (total over 4 pi), host */
    double pos[3];              /* kind 1: source position, cm (outside or inside the grid) */
    double axis[3];             /* kind 1: cone axis (any non-zero length) */
    double half_angle;          /* kind 1: cone half-angle in radians, (0, pi]; pi = isotropic */
    const double *spectrum;     /* kind 1: [G] photons per source particle, host */
    int aperture;               /* kind 1: 0 cone beam (half_angle), 1 fan beam (the fields below) */
    double normal[3];           /* fan: normal of the fan plane, not parallel to axis */
    double half_azimuth;        /* fan: half the azimuthal angle subtended in the fan plane, (0, pi] */
    double half_polar;          /* fan: half the polar angle subtended out of the plane, (0, pi/2] */
} dts_source;

typedef struct {
    int64_t updates;            /* cell-direction-group updates executed: sum over executed
                                   sweeps of V * N(N+2) */
    int64_t sweeps;             /* executed (source, group, iteration) sweeps */
    double max_residual;        /* largest final residual over sources and groups */
    double solve_ms;            /* device time of dts_solve, CUDA events on the stream */
    double sweep_ms;            /* device time of the wavefront sweep launches (all stages);
                                   0 when the iterations ran as a device-resident loop */
    double reduce_ms;           /* device time of the Eq. 3 reduction + residual launches;
                                   0 when the iterations ran as a device-resident loop */
    int64_t launches;           /* kernels launched by this solve */
    int converged;              /* 1 when every (source, group) reached tol */
    int tile_x, tile_y, tile_z; /* wavefront tile used */
    int64_t sweep_launches;     /* wavefront-stage kernel launches of this solve */
} dts_solve_stats;

/*
 * Create a problem: validates desc, builds the quadrature (Sec. II.E) and the
 * wavefront schedule (Eqs. 8-22, applied to tiles), and allocates every
 * device buffer the solve needs (FP64 fluence outputs [B][G][V] for the
 * uncollided and collided parts, per-octant moment partials, fixed-source
 * ring, face buffers). Errors: DTS_ERR_INVALID_ARG for a bad desc,
 * DTS_ERR_OOM, DTS_ERR_CUDA. *out is NULL on failure.
 */
dts_status dts_create_problem(const dts_problem_desc *desc, dts_problem **out);

/*
 * Materials (Sec. II.C: voxel phantom of material ids; multigroup library of
 * total and Legendre scattering cross sections).
 *   sigma_t [n_mat][G]          total cross section, 1/cm, finite and > 0
 *   sigma_s [n_mat][L+1][G][G]  [l][g_from][g_to] Legendre moments in the
 *                               convention sigma_s(mu0) = sum_l (2l+1)/(4 pi)
 *                               sigma_{s,l} P_l(mu0); must be zero for
 *                               g_to < g_from (downscatter only)
 *   mat_id  [V]                 material index per voxel, in [0, n_mat)
 *   scale_t, scale_s [V]        optional per-voxel multipliers (> 0) of
 *                               sigma_t and of every sigma_s entry; NULL = 1
 * All pointers are host memory. Errors: DTS_ERR_INVALID_ARG.
 */
dts_status dts_set_materials(dts_problem *p, int n_mat, const double *sigma_t,
                             const double *sigma_s, const int32_t *mat_id,
                             const double *scale_t, const double *scale_s);

/*
 * Source of batch member batch_index (Sec. II.C source tab; Eqs. 4-5).
 * kind 0: volumetric isotropic source q[G][V]; the uncollided component is
 *         then zero and the collided component holds the whole fluence.
 * kind 1: point source at pos emitting spectrum[g] photons per source particle
 *         isotropically into its beam (Sec. II.C source types): a cone
 *         |angle(r - pos, axis)| <= half_angle (aperture 0), or a fan
 *         (aperture 1): with a = axis, n = normal made orthogonal to a and
 *         t = n x a, the direction u = (r - pos)/|r - pos| is in the beam when
 *         |asin(u.n)| <= half_polar and |atan2(u.t, u.a)| <= half_azimuth
 *         (the paper's theta and phi are the full angles, 2 half_polar and
 *         2 half_azimuth).
 * Errors: DTS_ERR_INVALID_ARG (index, kind, NULL or non-finite data).
 */
dts_status dts_set_source(dts_problem *p, int batch_index, const dts_source *src);

/*
 * Several cone beams summed into one source for batch member batch_index (the
 * CT mode of Sec. II.E and the results section: 16 cones around the phantom
 * in one solve). cones[0..n_cones-1] are kind-1 sources (host memory, copied).
 * By linearity the uncollided fluence is the sum of the cones' (Eq. 4 per
 * cone) and the first-collision source (Eq. 5) the sum of theirs, which the
 * solver forms as sum_g' sigma_s,l(g'->g) U_lm^g' with
 * U_lm^g(v) = sum_c phi_u,c^g(v) Y_lm(Omega_c(v)) (one extra [G][K][V] FP64
 * array per such member). At most 8 materials. The adjoint
 * (dts_solve_adjoint) covers kind 0 and kind 1 only. A later dts_set_source
 * on the member replaces the cones.
 * Errors: DTS_ERR_INVALID_ARG (index, n_cones outside 1..4096, a cone that is
 * not kind 1 or has NULL / non-finite data), DTS_ERR_OOM.
 */
dts_status dts_set_source_cones(dts_problem *p, int batch_index, int n_cones,
                                const dts_source *cones);

/*
 * Solve every batch member: ray trace (Eq. 4), first-collision source (Eq. 5),
 * then for g = 0..G-1 source iteration to tol (Eqs. 2-3, 6-7) followed by the
 * downscatter into later groups. Blocks until the results are on the device.
 * stats may be NULL. Errors: DTS_ERR_STATE if materials or any source are
 * missing; DTS_ERR_NOT_CONVERGED if some (source, group) stopped at max_iters
 * with tol > 0 (results and stats are still filled); DTS_ERR_CUDA.
 */
dts_status dts_solve(dts_problem *p, dts_solve_stats *stats);

/*
 * Streamed output: during every later solve of p (dts_solve or
 * dts_solve_many), component comp of each member's scalar fluence (as
 * dts_get_scalar_fluence gives it, bit for bit) is copied into
 * host[b][g][v] (B x G x V doubles, [nz][ny][nx] voxels) group by group: when
 * group g has converged and pushed its downscatter, its values are gathered
 * on the device and copied to the host on a second stream while the solve
 * goes on with the later groups, so the copies overlap the solve; the solve
 * returns when the last group's copy has landed. Page-locked host memory
 * (cudaHostAlloc or cudaHostRegister) lets the copies run asynchronously;
 * pageable memory works but is copied synchronously. host must stay valid
 * and untouched by the caller while a solve runs; NULL turns the stream off.
 * The first call allocates two staging slots of B x V doubles on the device.
 * Errors: DTS_ERR_INVALID_ARG (p NULL, comp, len < B*G*V), DTS_ERR_OOM,
 * DTS_ERR_CUDA.
 */
dts_status dts_set_host_output(dts_problem *p, dts_component comp, double *host, size_t len);

/*
 * Restart from saved moments: member batch_index's source iteration in every
 * group g starts from moments[g][k][v] (G x K x V doubles, natural voxel order,
 * the collided moments dts_get_moments returns; host or device memory per
 * is_device, copied) instead of from zero. The group's first sweep then sees
 * T = F + sigma_s phi_guess (the scatter term of Eq. 2 evaluated on the
 * guess), and its first residual measures the change from the guess, so a
 * converged guess stops after one iteration. moments NULL clears the member's
 * guess (zeros, which is exactly the default start). The guess holds for every
 * later solve of p until cleared; the first call allocates B*G*K*V doubles on
 * the device (and, in the tensor-core forms, the group's first T as FP32).
 * Errors: DTS_ERR_INVALID_ARG (index, len < G*K*V, a non-finite host value),
 * DTS_ERR_OOM, DTS_ERR_CUDA.
 */
dts_status dts_set_initial_guess(dts_problem *p, int batch_index, const double *moments, size_t len,
                                 int is_device);

/*
 * Per-iteration progress (the paper's progressive display of the iteration,
 * Sec. II.C): after every source iteration of a solve of p (dts_solve or
 * dts_solve_many) the library calls fn(user, group, iteration, residuals,
 * batch) on the solving thread. residuals[b] is member b's relative L2 change
 * of its scalar fluence in that iteration (the convergence measure of tol), or
 * NaN for a member that had stopped before it; the array lives for the call
 * only. iteration counts from 1 in every group. fn must not call the library
 * on p. fn NULL turns the callback off. Errors: DTS_ERR_INVALID_ARG (p NULL).
 */
typedef void (*dts_iteration_fn)(void *user, int group, int iteration, const double *residuals,
                                 int batch);
dts_status dts_set_iteration_callback(dts_problem *p, dts_iteration_fn fn, void *user);

/*
 * Device-resident source iteration (the group loop of Eq. 2, Sec. II.A:
 * source iteration of each group to convergence, groups high to low). With
 * on != 0, every later solve of p (dts_solve or dts_solve_many) runs each
 * group's source iterations as ONE launch of a CUDA graph: a WHILE node whose
 * body is one iteration (all wavefront stages of the sweep, the Eq. 3
 * reduction, the residual) followed by a one-block control kernel that makes,
 * on the device, the decisions the host loop makes after every iteration (a
 * member stops below tol or, in the FP32 forms, after 10 iterations without a
 * 1 % improvement; the group ends when no member iterates or at max_iters, or
 * when a bounded wait of the tensor-core forms has given up). The host then
 * enqueues a whole solve without waiting on any iteration. The same kernels run
 * in the same order on the same data, so results, iteration counts, residuals
 * and balance terms equal those of the host loop bit for bit. Differences: the
 * stats' sweep_ms and reduce_ms are 0 (no per-phase timing inside the loop);
 * a timed-out wait (DTS_ERR_TIMEOUT) is reported when the solve finishes, not
 * after the iteration that met it; no per-iteration NVTX range. A problem with
 * an iteration callback (dts_set_iteration_callback), and every problem in the
 * bounds-checked build, keeps the host loop. The first call with on != 0
 * allocates the loop state on the device (about (12 + 36 G) bytes per member);
 * on = 0 returns to the host loop. Errors: DTS_ERR_INVALID_ARG (p NULL),
 * DTS_ERR_OOM.
 */
dts_status dts_set_device_loop(dts_problem *p, int on);

/*
 * Solve n problems together, each as dts_solve would: typically disjoint
 * source sets of one scan (independent CT projections, Sec. II.E), each
 * problem with its own batch and stream. The host polls the problems and
 * enqueues each problem's next source iteration (sweep, Eqs. 6-7 over the
 * tile wavefront of Eq. 9; then the Eq. 3 reduction and scatter-source
 * formation) as soon as its previous one is complete, so the problems' sweeps
 * and moment kernels overlap on the GPU: the sweep is bound by instruction
 * issue and latency, the moment kernel by HBM. The work and results of each
 * problem are those of dts_solve on it alone, bit for bit; only the overlap
 * differs. Problems sharing one stream get no overlap. Blocks until every
 * problem is solved.
 * problems: n distinct problems on one device (host array, not kept); stats:
 * NULL or n structs, stats[i] filled as dts_solve fills it for problems[i]
 * (its sweep and reduce times are its own, measured while it shared the GPU).
 * Errors: DTS_ERR_INVALID_ARG (NULL, n < 1, a repeated problem, different
 * devices); DTS_ERR_STATE (as dts_solve, on that problem); a CUDA, OOM or
 * TIMEOUT error of one problem stops the scheduling, waits for every
 * problem's stream and is returned; DTS_ERR_NOT_CONVERGED when some problem
 * stopped above tol, after all of them have finished (the others' results
 * are complete). The message of every failure is in dts_last_error(NULL).
 */
dts_status dts_solve_many(dts_problem *const *problems, int n, dts_solve_stats *stats);

/*
 * Copy one component of the scalar fluence of batch member batch_index into
 * out[G][V] (photons/cm^2 per source particle). out_len counts doubles and
 * must be >= G*V. Device copies are ordered on the problem's stream; host
 * copies complete before return. Errors: DTS_ERR_STATE before a solve,
 * DTS_ERR_INVALID_ARG.
 */
dts_status dts_get_scalar_fluence(dts_problem *p, int batch_index, dts_component comp,
                                  double *out, size_t out_len, int out_is_device);

/*
 * Absorbed dose per source particle (Gy) of batch member batch_index from the
 * scalar fluence of component comp: the post-processing module's conversion
 * of photon fluence to absorbed dose (Sec. II.C), in the collision-kerma form
 * since no electrons are transported (Sec. IV):
 *   D(v) = c * sum_g phi_g(v) E_g (mu_en/rho)_g(mat(v)),  c = 1 MeV/g = 1.602176634e-10 Gy,
 * groups summed in order. mu_en_rho [n_mat][G] (cm^2/g) and energy_mev [G]
 * (MeV) are host arrays; out [V] natural order (x fastest), host memory or
 * device memory (out_is_device), written on the problem's stream and
 * synchronised. Errors: DTS_ERR_STATE (no solve), DTS_ERR_INVALID_ARG (index,
 * component, NULL, out_len < V, negative or non-finite coefficients).
 */
dts_status dts_get_dose(dts_problem *p, int batch_index, dts_component comp, const double *mu_en_rho,
                        const double *energy_mev, double *out, size_t out_len, int out_is_device);

/*
 * All K = (L+1)^2 collided flux moments of one group, out[K][V], ordered
 * k = l*l + l + m with real spherical harmonics normalised so that
 * sum_m Y_lm(a) Y_lm(b) = P_l(a.b); k = 0 is the Eq. 3 scalar fluence.
 * Needs desc.keep_moments = 1 (else DTS_ERR_STATE).
 */
dts_status dts_get_moments(dts_problem *p, int batch_index, int group, double *out,
                           size_t out_len, int out_is_device);

/*
 * Discrete adjoint of the converged solve of batch member batch_index
 * (differentiation form; the paper has no adjoint -- it is the gradient of the
 * Eq. 2-7 solution). Given dL/dphi_total [G][V] (the gradient of a scalar loss
 * with respect to the total scalar fluence of every group and voxel), writes
 *   dL_dscale_t [V]  dL/d(multiplier of sigma_t in voxel v), all groups
 *   dL_dscale_s [V]  dL/d(multiplier of every sigma_s entry in voxel v)
 *   dL_dsigma_t [G][V] dL/dsigma_t^g(v) of the collided part (NULL = skip)
 * Groups run from low energy to high; each recomputes its forward sweep from
 * the kept moments (recording fluxes and fixup sets, which stay fixed), then
 * iterates the transposed source iteration to tol / max_iters; the uncollided
 * part is differentiated through the ray trace. Needs DTS_PREC_FP64,
 * keep_moments = 1 and a completed dts_solve (else DTS_ERR_STATE).
 * ptrs_are_device selects device (1) or host (0) memory for all four arrays.
 */
dts_status dts_solve_adjoint(dts_problem *p, int batch_index, const double *dL_dphi,
                             double *dL_dscale_t, double *dL_dscale_s, double *dL_dsigma_t,
                             int ptrs_are_device);

/* Adjoint source iterations per group [G] of the last dts_solve_adjoint. */
dts_status dts_get_adjoint_iterations(dts_problem *p, int32_t *out, size_t out_len);

/* Per (source, group) results of the last solve, host arrays:
 *   iterations [B][G]; residuals [B][G] (final relative L2 change);
 *   balance [B][G][3] = (sum_v V T_00, sum_v V sigma_t phi_00, leakage) of the
 *   last sweep, whose difference is zero up to rounding (particle balance). */
dts_status dts_get_iterations(dts_problem *p, int32_t *out, size_t out_len);
dts_status dts_get_residuals(dts_problem *p, double *out, size_t out_len);
dts_status dts_get_balance(dts_problem *p, double *out, size_t out_len);

/* Message of the last failed call on p (or of the calling thread when p is
 * NULL). Never NULL; valid until the next call on p. */
const char *dts_last_error(const dts_problem *p);

/* Releases every device and host resource of p. NULL is a no-op. */
void dts_destroy_problem(dts_problem *p);

/* Name of a status code. */
const char *dts_status_string(dts_status s);

/* ABI version, incremented on incompatible changes. */
int dts_version(void);

/* Test hook for the out-of-memory path (host-side fault injection; the paper
 * has no counterpart): the device allocation that follows `after` further
 * successful ones in this process fails once as if the device were full, so
 * the call making it returns DTS_ERR_OOM with "injected" in its message and
 * releases everything it had allocated (dts_create_problem leaves *out NULL).
 * after < 0 disarms the hook. No device work. */
void dts_debug_fail_allocation(int after);

/*
 * Host-side helpers (no device work; usable without a GPU).
 * dts_quadrature: the level-symmetric set the solver uses (Sec. II.E), with
 *   octant o = sx + 2 sy + 4 sz (a set bit = negative cosine) holding
 *   directions o*N(N+2)/8 .. ; arrays of >= 80 doubles; *n_dirs = N(N+2).
 * dts_moment_tables: the moment operator D[K][nd] (phi_k = sum_n D[k][n]
 *   psi_n; D[0][n] = w_n is Eq. 3) and the source operator M[nd][K]
 *   (Q_n = sum_k M[n][k] T_k).
 * dts_subsweep_size: Eq. 9, the number of voxels of an nx x ny x nz box with
 *   i_x + i_y + i_z = S (Eqs. 8, 10-22); the solver applies it to tiles.
 */
dts_status dts_quadrature(int sn_order, double *mu, double *eta, double *xi, double *w,
                          int *n_dirs);

/*
 * Wavefront tile chosen by measurement (the batching pattern's autotuner; the
 * paper sweeps one sub-sweep of Eqs. 8-22 per launch and has no tiles). For
 * the shape in *desc (grid, S_N order, Legendre order, precision, device, up
 * to 16 sources) each candidate tile that fits -- 8x4x4 (FP32 batched
 * kernel), 8x4x8, 4x4x8, 16x4x8, 8x8x4, 8x8x8, 4x4x4 -- times two source
 * iterations of a probe problem (one group, homogeneous scatterer, unit
 * volumetric source) and the highest rate of updates per second of sweep plus
 * Eq. 3 reduction time wins. Writes desc->tile_x/y/z; *best_updates_per_s
 * (may be NULL) gets that probe rate.
 * Results are cached per process and, when a cache file is named (below), on
 * disk: a hit returns the stored tile and rate without probing. Runs on the
 * device; allocates and frees probe problems. Errors: DTS_ERR_INVALID_ARG,
 * DTS_ERR_CUDA.
 */
dts_status dts_tune_tile(dts_problem_desc *desc, double *best_updates_per_s);

/*
 * Name the tuner's cache file for this process (path copied; NULL or "" turns
 * the file off); until this is called the environment variable DTS_TUNE_CACHE
 * names it. dts_tune_tile looks a shape up there after its per-process cache
 * and appends each new result as one text line
 *   dts-tune-v1 <device name, blanks as '_'> <SM count> nx ny nz N L
 *               <probe batch = min(batch, 16)> <precision> tx ty tz <rate>
 * (a later line for the same key wins; lines that do not parse are ignored; a
 * file that cannot be read or written is skipped). Host only; always DTS_OK.
 */
dts_status dts_tune_cache_file(const char *path);

/*
 * The DTS_DEBUG_BOUNDS build (libdts_debug.so, compiled with
 * -DDTS_DEBUG_BOUNDS): before the batched sweep, the tensor-core moment
 * kernel, the angular-flux moment kernel and the residual kernel touch a
 * region of a global buffer, they check the region's end against the
 * buffer's allocated size; a region that does not fit is skipped and recorded
 * in a device error word, and the solve returns DTS_ERR_INTERNAL with the
 * kernel and site in its message after the iteration. This call checks that
 * machinery: *is_debug_build (may be NULL) is 1 in the debug build, 0
 * otherwise; in the debug build a one-thread kernel evaluates one bounds
 * check, failing when plant != 0 (it touches no memory either way), and the
 * call returns DTS_ERR_INTERNAL with the message in dts_last_error(NULL) when
 * the check failed, DTS_OK when it passed. The normal build returns DTS_OK
 * without device work.
 */
dts_status dts_debug_bounds_selftest(int plant, int *is_debug_build);

/*
 * Failure-path test hook of the tensor-core forms, whose kernels wait on
 * mbarriers: the moment kernel for its bulk copies and tensor-core results,
 * the sweep for the bulk copies of its face blocks. Every such wait is
 * bounded: it gives up after about a second, the kernel records the failure in
 * a device error word and returns (the moment kernel leaves its item loop with
 * no copy or MMA in flight and frees its tensor memory; the sweep's warp waits,
 * again bounded, for its face copies and leaves its tile), and the solve
 * returns DTS_ERR_TIMEOUT after that iteration (with the device-resident loop:
 * when the solve finishes). With on = 1 every later solve of p makes the moment
 * kernel's flux-stage waits expect 16 bytes that no copy delivers; with on = 2
 * the sweep's first face wait of every tile does (the sweep's captured graphs
 * are made again with that byte count). The waits then run out -- no fault, no
 * trap: they end by their bound. on = 0 restores normal operation, and the
 * problem solves correctly again. Errors: DTS_ERR_INVALID_ARG (p NULL, on not
 * 0, 1 or 2), DTS_ERR_STATE (not a tensor-core form), DTS_ERR_CUDA.
 */
dts_status dts_debug_poison_wait(dts_problem *p, int on);
dts_status dts_moment_tables(int sn_order, int legendre_order, double *D, double *M);
long long dts_subsweep_size(int nx, int ny, int nz, int S);

/*
 * One FP64 source iteration of a single group with no memory allocation.
 * The paper has no counterpart: this exists for callers that cannot allocate
 * device memory when they need a sweep -- code running inside a fixed,
 * caller-managed memory pool, or hosts that forbid further cudaMalloc/cudaFree
 * (those calls also synchronise the device). Everything the sweep needs
 * besides the caller's inputs and outputs lives in one static device array of
 * DTS_NOALLOC_SCRATCH_BYTES bytes that every GPU loading this library reserves
 * until the process exits.
 *
 * Computes phi_k = sum_n D[k][n] psi_n for all K = (L+1)^2 moments, where psi_n
 * is the diamond-difference sweep (set-to-zero fixup, vacuum boundaries) of
 * direction n of the S_N set with angular source Q_n = sum_k M[n][k] T_k
 * (dts_moment_tables gives D and M). This is what dts_solve does in each
 * source iteration, for one group and one source.
 *   src_moments [K][V] device, T_k per voxel (x fastest)
 *   sigma_t     [V]    device, total cross section per voxel, > 0
 *   phi         [K][V] device output
 *   cuda_stream        stream to enqueue on (NULL = legacy default stream)
 * Timing: the first call on a device looks up the device address of the
 * scratch array (with that device current); make that first call before any
 * stream capture. The schedule and direction tables of a call's shape (grid,
 * pitch, S_N and Legendre order) are kept at the start of the array: a call
 * whose shape differs from the previous call's on that device first waits
 * until the device is idle and then copies its tables from host memory
 * (blocking); a call repeating the shape copies nothing, enqueues its kernels
 * on cuda_stream and returns without waiting -- phi is ready when the stream
 * reaches it.
 * Sharing: calls on one device share its array, so two calls on one device
 * whose work is not ordered on one stream race and give wrong results; calls
 * on different devices use different arrays and never race.
 * Errors: DTS_ERR_INVALID_ARG for bad sizes or when the grid needs more
 * scratch than DTS_NOALLOC_SCRATCH_BYTES (about 1.2 KB per voxel at L = 3,
 * 80 bytes at L = 0; message in dts_last_error(NULL)); DTS_ERR_CUDA.
 */
#define DTS_NOALLOC_SCRATCH_BYTES (64u * 1024u * 1024u)
dts_status dts_sweep_once_noalloc(int nx, int ny, int nz, double dx, double dy, double dz,
                                  int sn_order, int legendre_order, const double *src_moments,
                                  const double *sigma_t, double *phi, void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* DTS_H */
