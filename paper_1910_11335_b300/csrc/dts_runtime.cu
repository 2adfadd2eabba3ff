// dts_runtime.cu -- host runtime and C ABI of the B300 S_N solver (include/dts.h).
//
// The runtime owns the device buffers of a problem, the wavefront schedule
// (tile stages of Eq. 9 applied to tiles, and the intra-tile sub-sweeps), the
// group loop (high energy to low), the source-iteration loop with its
// convergence control, and a CUDA graph holding one iteration (all tile
// stages of the sweep, the Eq. 3 reduction and the residual), replayed for
// every iteration of every group.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <array>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <tuple>
#include <string>
#include <vector>

#include "../../include/dts.h"
#include "dts_kernels.cuh"
#include "dts_adjoint.cuh"
#include "dts_tc.cuh"
#include "dts_tc_launch.h"

using namespace dts;

namespace {

thread_local std::string g_thread_error = "no error";

struct DevGuard {
    int prev = -1;
    explicit DevGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DevGuard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

}  // namespace

// lets other translation units of the library report a thread's last error
__attribute__((visibility("hidden"))) void dts_internal_set_thread_error(const char* msg)
{
    g_thread_error = msg;
}

struct dts_problem {
    dts_problem_desc d{};
    std::string err = "no error";
    dts_iteration_fn on_iter = nullptr;   // per-iteration progress callback and its argument
    void* on_iter_user = nullptr;
    double* guess = nullptr;              // initial guess [B][G][K][V] (dts_set_initial_guess), or null
    void* guess_T = nullptr;              // tensor-core forms: the group's first T [B][NT][K][TV] (FP32)
    // streamed output (dts_set_host_output): component host_comp of each finished group copied into
    // host_out[b][g][v] on copy_stream, through two device staging slots of [B][V] doubles
    double* host_out = nullptr;
    int host_comp = 0;
    cudaStream_t copy_stream = nullptr;
    double* out_stage[2] = {nullptr, nullptr};
    cudaEvent_t ev_staged[2] = {nullptr, nullptr}, ev_copied[2] = {nullptr, nullptr};
    bool copied_pending[2] = {false, false};
    int V = 0, G = 0, L = 0, K = 0, nd = 0, ndo = 0, B = 0;
    int TX = 0, TY = 0, TZ = 0, TV = 0, NTx = 0, NTy = 0, NTz = 0, NT = 0, NC = 0;
    int n_stages = 0, nsub = 0, n_mat = 0, W = 0, nblk = 0, n_sm = 148;
    int line_warps = 2;               // warps per CTA of the line sweep kernel
    bool fp64 = true;
    bool psi_mode = false;   // batched FP32 sweep writes angular fluxes; moments formed by k_reduce_psi
    // tensor-core forms: k_moments_q turns the angular fluxes into the next per-direction source Q
    // (scatter-source contraction on tcgen05), which the batched sweep reads
    bool q_mode = false;
    int q_kind = 0;                   // 0 split BF16, 1 TF32
    int q_grid = 0;                   // persistent CTAs of k_moments_q
    void* Qbuf = nullptr;             // [B][8][NT][N_d/8][TV] FP32
    float* Mop = nullptr;             // operator parts M' = 4 pi M, [2][NP][16]
    float* Dop = nullptr;             // Eq. 3 operator parts D, [2][16][N_d] (N_d a multiple of 16)
    int* dev_err = nullptr;           // device error word of the bounded waits
    int* dev_poison = nullptr;        // dts_debug_poison_wait's flag of the moment kernel (tensor-core forms)
    unsigned poison_sweep_tx = 0;     // dts_debug_poison_wait: bytes no copy delivers, added to the sweep's face wait
    int* h_err = nullptr;             // pinned copy, read after every iteration
    size_t rsz = 8;                   // sizeof(R)
    std::vector<int> stage_off_h;     // [n_stages+1]
    std::vector<double> mu, eta, xi, w;
    std::vector<double> sigma_s_h;    // kept for the band width
    // device buffers
    std::vector<void*> allocs;
    std::map<const void*, size_t> alloc_bytes;   // size of every live allocation (bounds checks)
    unsigned *stage_tiles = nullptr, *diag_cells = nullptr;
    int *stage_off = nullptr, *diag_off = nullptr;
    void *Mt = nullptr, *Dt = nullptr, *At = nullptr;
    double* Lw = nullptr;
    double *sigma_t = nullptr, *sigma_s = nullptr;
    float* sigma_s_f = nullptr;       // FP32 copy of sigma_s for FP32 forms
    int *mat_t = nullptr, *mat_nat = nullptr;
    double *scale_t_t = nullptr, *scale_s_t = nullptr, *scale_t_nat = nullptr;
    void* F = nullptr;                // fixed-source ring, sweep precision
    double *phi00 = nullptr, *sigt64 = nullptr, *sigs0 = nullptr;
    void* sigs = nullptr;             // [L+1][NC] in-group scatter, sweep precision
    void *T = nullptr, *part = nullptr, *xf = nullptr, *yf = nullptr, *zf = nullptr, *sigt_r = nullptr;
    double *unc = nullptr, *col = nullptr, *mom = nullptr, *q = nullptr, *tmp = nullptr;
    double *src = nullptr, *spec = nullptr, *leak = nullptr, *blk = nullptr, *status = nullptr;
    // combined multi-cone sources (kind 2): per member its cones (host copies), device
    // tables [B][cone_cap][8] / [B][cone_cap][G], and a row of U per such member
    std::vector<double> fan_h;        // [B][8] beam aperture of kind-1 members (0 cone, 1 fan + its angles)
    double* fan = nullptr;
    std::vector<std::vector<double>> cone_geo_h, cone_spec_h;
    std::vector<int> cone_n_h, uslot_h;
    int cone_cap = 0, n_uslots = 0;
    double *cone_geo = nullptr, *cone_spec = nullptr, *U = nullptr;
    int *cone_n = nullptr, *uslot = nullptr;
    int *active = nullptr, *ctl = nullptr;
    size_t Fstride = 0;
    int F_W = -1;
    // host state
    double* h_status = nullptr;       // pinned [B][4]
    int* h_active = nullptr;          // pinned [B]
    std::vector<double> src_h;        // [B][8]
    std::vector<double> spec_h;       // [B][G]
    std::vector<int> src_set;
    bool materials_set = false, solved = false;
    std::vector<int32_t> iters;       // [B][G]
    std::vector<double> resid;        // [B][G]
    std::vector<double> balance;      // [B][G][3]
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaGraphExec_t graph = nullptr, graph_red = nullptr;
    // device-resident source iteration (dts_set_device_loop): per group one launch of graph_loop, a
    // WHILE node whose body is the sweep, the moment graph and k_loop_control; the loop state lives
    // in one allocation (loop_mem)
    bool device_loop = false, recording_loop = false;
    cudaGraphExec_t graph_loop = nullptr;
    cudaGraphConditionalHandle loop_h = 0;
    void* loop_mem = nullptr;
    int *loop_it = nullptr, *loop_last = nullptr, *loop_iters = nullptr;
    double *loop_best = nullptr, *loop_resid = nullptr, *loop_bal = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    cudaEvent_t eva = nullptr, evb = nullptr, evc = nullptr;   // around the two graph replays
    // adjoint buffers (allocated by the first dts_solve_adjoint, B = 1)
    bool adj_ready = false;
    int adj_W = -1;
    double *adj_T = nullptr, *adj_part = nullptr, *adj_xf = nullptr, *adj_yf = nullptr,
           *adj_zf = nullptr, *adj_psi = nullptr, *adj_cpart = nullptr, *adj_S = nullptr,
           *adj_u00 = nullptr, *adj_a = nullptr, *adj_gt = nullptr, *adj_gs = nullptr,
           *adj_gsig = nullptr, *adj_dphiu = nullptr, *adj_blk = nullptr, *adj_status = nullptr,
           *adj_leak = nullptr;
    unsigned char* adj_mask = nullptr;
    int *adj_active = nullptr, *adj_ctl = nullptr;
    std::vector<int32_t> adj_iters;   // [G]
    int graph_launches = 0;           // kernels per graph replay
};

namespace {

dts_status fail(dts_problem* p, dts_status s, const std::string& msg)
{
    if (p) p->err = msg;
    else g_thread_error = msg;
    return s;
}

#define CK(call)                                                                              \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return fail(p, e_ == cudaErrorMemoryAllocation ? DTS_ERR_OOM : DTS_ERR_CUDA,      \
                        std::string(#call) + ": " + cudaGetErrorString(e_));                  \
    } while (0)

#define TRY(expr)                          \
    do {                                   \
        dts_status s_ = (expr);            \
        if (s_ != DTS_OK) return s_;       \
    } while (0)

// host-side fault injection (dts_debug_fail_allocation): successful device allocations still to
// pass before one fails as out-of-memory; negative = disarmed
std::atomic<long long> g_fail_alloc_after{-1};

dts_status dalloc(dts_problem* p, void** ptr, size_t bytes)
{
    *ptr = nullptr;
    if (bytes == 0) bytes = 16;
    for (long long n = g_fail_alloc_after.load(); n >= 0;) {
        if (g_fail_alloc_after.compare_exchange_weak(n, n - 1)) {
            if (n == 0) {
                char buf[160];
                snprintf(buf, sizeof buf, "cudaMalloc(%zu bytes): injected allocation failure "
                                          "(dts_debug_fail_allocation)", bytes);
                return fail(p, DTS_ERR_OOM, buf);
            }
            break;
        }
    }
    cudaError_t e = cudaMalloc(ptr, bytes);
    if (e != cudaSuccess) {
        *ptr = nullptr;
        cudaGetLastError();
        char buf[160];
        snprintf(buf, sizeof buf, "cudaMalloc(%zu bytes): %s", bytes, cudaGetErrorString(e));
        return fail(p, e == cudaErrorMemoryAllocation ? DTS_ERR_OOM : DTS_ERR_CUDA, buf);
    }
    p->allocs.push_back(*ptr);
    p->alloc_bytes[*ptr] = bytes;
    return DTS_OK;
}

template <typename T>
dts_status dalloc_t(dts_problem* p, T** ptr, size_t count)
{
    return dalloc(p, reinterpret_cast<void**>(ptr), count * sizeof(T));
}

void dfree(dts_problem* p, void* ptr)
{
    if (!ptr) return;
    auto it = std::find(p->allocs.begin(), p->allocs.end(), ptr);
    if (it != p->allocs.end()) p->allocs.erase(it);
    p->alloc_bytes.erase(ptr);
    cudaFree(ptr);
}

// element count of a buffer allocated by dalloc (0 for a null or foreign pointer); the kernels'
// parameters carry these for the checks of the DTS_DEBUG_BOUNDS build
template <typename T>
size_t count_of(const dts_problem* p, const void* ptr)
{
    auto it = p->alloc_bytes.find(ptr);
    return it == p->alloc_bytes.end() ? 0 : it->second / sizeof(T);
}

#ifdef DTS_DEBUG_BOUNDS
// the first failed bounds check of this unit's kernels or the tensor-core unit's, read and
// cleared (0: none); called with the solve's kernels complete
unsigned long long take_bounds_word()
{
    unsigned long long w = 0, z = 0;
    cudaMemcpyFromSymbol(&w, bounds_word, sizeof w);
    cudaMemcpyToSymbol(bounds_word, &z, sizeof z);
    const unsigned long long w2 = dts_internal_tc_bounds_take();
    return w ? w : w2;
}

std::string bounds_message(unsigned long long w)
{
    const unsigned site = (unsigned)(w >> 48);
    const char* where = site <= 10   ? "k_sweep_batch"
                        : site < 30  ? "k_moments_q"
                        : site < 40  ? "k_reduce_psi"
                        : site < 63  ? "k_resid_final"
                                     : "dts_debug_bounds_selftest";
    char buf[160];
    snprintf(buf, sizeof buf, "bounds check failed in %s: site %u, region end %llu beyond its buffer", where,
             site, (unsigned long long)(w & 0xffffffffffffull));
    return buf;
}
#endif

bool isfin(double x) { return std::isfinite(x); }

// ---------------------------------------------------------------------------
// level-symmetric quadrature (Sec. II.E), octant-major
// ---------------------------------------------------------------------------
double det3(const double m[3][3])
{
    return m[0][0] * (m[1][1] * m[2][2] - m[1][2] * m[2][1]) -
           m[0][1] * (m[1][0] * m[2][2] - m[1][2] * m[2][0]) +
           m[0][2] * (m[1][0] * m[2][1] - m[1][1] * m[2][0]);
}

bool ls_set(int N, std::vector<double>& mu, std::vector<double>& eta, std::vector<double>& xi,
            std::vector<double>& w)
{
    double m1sq;
    if (N == 2) m1sq = 1.0 / 3.0;
    else if (N == 4) m1sq = (4.0 - std::sqrt(6.4)) / 12.0;   // root of 6x^2 - 4x + 0.4 = 0
    else if (N == 6) m1sq = 0.2666355 * 0.2666355;
    else if (N == 8) m1sq = 0.2182179 * 0.2182179;
    else return false;
    const int h = N / 2;
    std::vector<double> lev(h);
    for (int i = 0; i < h; ++i)
        lev[i] = std::sqrt(h == 1 ? m1sq : m1sq + 2.0 * i * (1.0 - 3.0 * m1sq) / (N - 2));
    struct Pt { int a, b, c, cls; };
    std::vector<Pt> pts;
    std::vector<std::vector<int>> classes;
    for (int a = 0; a < h; ++a)
        for (int b = 0; a + b < h; ++b) {
            int c = h - 1 - a - b;
            std::vector<int> key = {a, b, c};
            std::sort(key.begin(), key.end());
            int cls = -1;
            for (size_t i = 0; i < classes.size(); ++i)
                if (classes[i] == key) cls = (int)i;
            if (cls < 0) {
                classes.push_back(key);
                cls = (int)classes.size() - 1;
            }
            pts.push_back({a, b, c, cls});
        }
    const int nc = (int)classes.size();
    const int ks[3] = {0, 2, 3};
    // even-moment matching, octant-normalised: sum_c w_c sum_{p in c} mu_x^(2k) = 1/(2k+1)
    double A[3][3] = {{0}}, r[3] = {0};
    for (int e = 0; e < nc; ++e) {
        for (const Pt& pt : pts) A[e][pt.cls] += std::pow(lev[pt.a], 2.0 * ks[e]);
        r[e] = 1.0 / (2.0 * ks[e] + 1.0);
    }
    double wc[3] = {0};
    if (nc == 1) {
        wc[0] = r[0] / A[0][0];
    } else {
        double M[3][3];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) M[i][j] = (i < nc && j < nc) ? A[i][j] : (i == j ? 1.0 : 0.0);
        const double dt = det3(M);
        if (dt == 0.0) return false;
        for (int c = 0; c < nc; ++c) {   // Cramer's rule
            double Mc[3][3];
            std::memcpy(Mc, M, sizeof M);
            for (int i = 0; i < nc; ++i) Mc[i][c] = r[i];
            wc[c] = det3(Mc) / dt;
        }
    }
    const int npo = (int)pts.size();
    mu.assign(8 * npo, 0.0);
    eta.assign(8 * npo, 0.0);
    xi.assign(8 * npo, 0.0);
    w.assign(8 * npo, 0.0);
    const double octant_weight = std::acos(-1.0) / 2.0;   // each octant carries pi/2
    for (int o = 0; o < 8; ++o)
        for (int i = 0; i < npo; ++i) {
            const int n = o * npo + i;
            mu[n] = (o & 1 ? -1.0 : 1.0) * lev[pts[i].a];
            eta[n] = (o & 2 ? -1.0 : 1.0) * lev[pts[i].b];
            xi[n] = (o & 4 ? -1.0 : 1.0) * lev[pts[i].c];
            w[n] = wc[pts[i].cls] * octant_weight;
        }
    return true;
}

// D[k][n] = w_n Y_k(O_n); M[n][k] = (2l+1)/(4 pi) Y_k(O_n)
void moment_tables(int L, const std::vector<double>& mu, const std::vector<double>& eta,
                   const std::vector<double>& xi, const std::vector<double>& w,
                   std::vector<double>& D, std::vector<double>& M)
{
    const int nd = (int)w.size(), K = (L + 1) * (L + 1);
    D.assign((size_t)K * nd, 0.0);
    M.assign((size_t)nd * K, 0.0);
    for (int n = 0; n < nd; ++n) {
        double Y[16];
        sh_eval(L, mu[n], eta[n], xi[n], Y);
        for (int k = 0; k < K; ++k) {
            D[(size_t)k * nd + n] = w[n] * Y[k];
            M[(size_t)n * K + k] = (2.0 * l_of_k(k) + 1.0) / (4.0 * kPi) * Y[k];
        }
    }
}

long long eq9(int nx, int ny, int nz, int S)
{
    auto t = [](long long d) { return d > 0 ? d * (d + 1) / 2 : 0LL; };
    return (long long)(S + 1) * (S + 2) / 2 - t(S + 1 - nx) - t(S + 1 - ny) - t(S + 1 - nz) +
           t(S + 1 - nx - ny) + t(S + 1 - ny - nz) + t(S + 1 - nx - nz);
}

// ---------------------------------------------------------------------------
// kernel dispatch on (precision, directions per octant, moments)
// ---------------------------------------------------------------------------
template <typename R>
using SweepFn = void (*)(const SweepParams<R>, int);
template <typename R>
using RedFn = void (*)(const RedParams<R>);

template <typename R, int NDO>
SweepFn<R> sweep_fn_k(int K)
{
    switch (K) {
    case 1: return k_sweep_stage<R, NDO, 1>;
    case 4: return k_sweep_stage<R, NDO, 4>;
    case 9: return k_sweep_stage<R, NDO, 9>;
    case 16: return k_sweep_stage<R, NDO, 16>;
    }
    return nullptr;
}

template <typename R>
SweepFn<R> sweep_fn_generic(int ndo, int K)
{
    switch (ndo) {
    case 1: return sweep_fn_k<R, 1>(K);
    case 3: return sweep_fn_k<R, 3>(K);
    case 6: return sweep_fn_k<R, 6>(K);
    case 10: return sweep_fn_k<R, 10>(K);
    }
    return nullptr;
}

template <typename R, int NDO, int TY, int TZ>
SweepFn<R> lines_fn_k(int K)
{
    switch (K) {
    case 1: return k_sweep_lines<R, NDO, 1, TY, TZ>;
    case 4: return k_sweep_lines<R, NDO, 4, TY, TZ>;
    case 9: return k_sweep_lines<R, NDO, 9, TY, TZ>;
    case 16: return k_sweep_lines<R, NDO, 16, TY, TZ>;
    }
    return nullptr;
}

template <typename R, int TY, int TZ>
SweepFn<R> lines_fn(int ndo, int K)
{
    switch (ndo) {
    case 1: return lines_fn_k<R, 1, TY, TZ>(K);
    case 3: return lines_fn_k<R, 3, TY, TZ>(K);
    case 6: return lines_fn_k<R, 6, TY, TZ>(K);
    case 10: return lines_fn_k<R, 10, TY, TZ>(K);
    }
    return nullptr;
}

// tiles of exactly 32 x-lines (4 x 8 or 8 x 4) take the warp-synchronous
// kernel; every other tile shape the generic sub-sweep kernel
bool line_tile(const dts_problem* p)
{
    return (p->TY == 4 && p->TZ == 8) || (p->TY == 8 && p->TZ == 4);
}

// FP32 problems with 8 x 4 x 4 or 4 x 4 x 4 tiles take the batched kernel
// (lanes = source x direction pairs)
bool batch_tile(const dts_problem* p)
{
    return !p->fp64 && p->TY == 4 && p->TZ == 4 && (p->TX == 8 || p->TX == 4);
}

// sources per warp of the batched kernels (lanes = source x direction pairs)
int batch_sources_per_warp(const dts_problem* p) { return 32 / p->ndo; }

// the direct-output form pays N_d angular fluxes per cell instead of 8 K octant
// partials, so it is taken where that is less traffic (e.g. S8 with P3)
bool psi_form(const dts_problem* p) { return batch_tile(p) && 8 * p->K > p->nd; }

using BatchFn = void (*)(const SweepParams<float>, int, int, const CUtensorMap);

template <int NDO, int BX, bool PSI>
BatchFn batch_fn_k(int K)
{
    switch (K) {
    case 1: return k_sweep_batch<NDO, 1, BX, PSI>;
    case 4: return k_sweep_batch<NDO, 4, BX, PSI>;
    case 9: return k_sweep_batch<NDO, 9, BX, PSI>;
    case 16: return k_sweep_batch<NDO, 16, BX, PSI>;
    }
    return nullptr;
}

template <int NDO, int BX, bool PSI>
size_t batch_smem_k(int K)
{
    switch (K) {
    case 1: return sweep_batch_smem<NDO, 1, BX, PSI>();
    case 4: return sweep_batch_smem<NDO, 4, BX, PSI>();
    case 9: return sweep_batch_smem<NDO, 9, BX, PSI>();
    case 16: return sweep_batch_smem<NDO, 16, BX, PSI>();
    }
    return 0;
}

template <int BX, bool PSI>
size_t batch_smem_x(int ndo, int K)
{
    switch (ndo) {
    case 1: return batch_smem_k<1, BX, PSI>(K);
    case 3: return batch_smem_k<3, BX, PSI>(K);
    case 6: return batch_smem_k<6, BX, PSI>(K);
    case 10: return batch_smem_k<10, BX, PSI>(K);
    }
    return 0;
}

template <int BX, bool PSI>
BatchFn batch_fn_x(int ndo, int K)
{
    switch (ndo) {
    case 1: return batch_fn_k<1, BX, PSI>(K);
    case 3: return batch_fn_k<3, BX, PSI>(K);
    case 6: return batch_fn_k<6, BX, PSI>(K);
    case 10: return batch_fn_k<10, BX, PSI>(K);
    }
    return nullptr;
}

BatchFn batch_fn(const dts_problem* p)
{
    if (p->q_mode) return dts_internal_qsweep_fn(p->ndo);
    if (p->psi_mode) return p->TX == 8 ? batch_fn_x<8, true>(p->ndo, p->K) : batch_fn_x<4, true>(p->ndo, p->K);
    return p->TX == 8 ? batch_fn_x<8, false>(p->ndo, p->K) : batch_fn_x<4, false>(p->ndo, p->K);
}

using RedPsiFn = void (*)(const RedParams<float>, const float*);
using PushPsiFn = void (*)(const PushParams<float>, int, const float*, int, int);

template <int NDO>
void psi_fns_k(int K, RedPsiFn& r, PushPsiFn& u)
{
    switch (K) {
    case 1: r = k_reduce_psi<NDO, 1>; u = k_push_psi<NDO, 1>; return;
    case 4: r = k_reduce_psi<NDO, 4>; u = k_push_psi<NDO, 4>; return;
    case 9: r = k_reduce_psi<NDO, 9>; u = k_push_psi<NDO, 9>; return;
    case 16: r = k_reduce_psi<NDO, 16>; u = k_push_psi<NDO, 16>; return;
    }
    r = nullptr;
    u = nullptr;
}

void psi_fns(const dts_problem* p, RedPsiFn& r, PushPsiFn& u)
{
    r = nullptr;
    u = nullptr;
    switch (p->ndo) {
    case 1: psi_fns_k<1>(p->K, r, u); return;
    case 3: psi_fns_k<3>(p->K, r, u); return;
    case 6: psi_fns_k<6>(p->K, r, u); return;
    case 10: psi_fns_k<10>(p->K, r, u); return;
    }
}


template <typename R>
SweepFn<R> sweep_fn(const dts_problem* p)
{
    if (line_tile(p))
        return p->TY == 4 ? lines_fn<R, 4, 8>(p->ndo, p->K) : lines_fn<R, 8, 4>(p->ndo, p->K);
    return sweep_fn_generic<R>(p->ndo, p->K);
}

template <typename R>
RedFn<R> reduce_fn(int K)
{
    switch (K) {
    case 1: return k_reduce<R, 1>;
    case 4: return k_reduce<R, 4>;
    case 9: return k_reduce<R, 9>;
    case 16: return k_reduce<R, 16>;
    }
    return nullptr;
}

RedFn<float> reduce4_fn(int K)
{
    switch (K) {
    case 1: return k_reduce4<1>;
    case 4: return k_reduce4<4>;
    case 9: return k_reduce4<9>;
    case 16: return k_reduce4<16>;
    }
    return nullptr;
}

size_t sweep_smem(const dts_problem* p)
{
    if (batch_tile(p)) {
        if (p->q_mode) return dts_internal_qsweep_smem(p->ndo);
        if (p->psi_mode) return p->TX == 8 ? batch_smem_x<8, true>(p->ndo, p->K) : batch_smem_x<4, true>(p->ndo, p->K);
        return p->TX == 8 ? batch_smem_x<8, false>(p->ndo, p->K) : batch_smem_x<4, false>(p->ndo, p->K);
    }
    const int xfaces = line_tile(p) ? 32 : p->TY * p->TZ;
    const size_t n = (size_t)p->ndo * p->TV +
                     (size_t)p->ndo * (xfaces + p->TX * p->TZ + p->TX * p->TY) + p->TV +
                     2 * p->ndo * p->K + 4 * p->ndo;
    size_t bytes = (n * p->rsz + 15) & ~size_t(15);
    return bytes + sizeof(double) * (3 * p->ndo + 32);
}

// threads per sweep CTA: the generic kernel uses 256; the line kernel one
// warp per run of directions (2 warps unless the octant has fewer directions)
int sweep_threads(const dts_problem* p)
{
    if (batch_tile(p)) return 32;
    if (!line_tile(p)) return kSweepThreads;
    const int nw = std::max(1, std::min(p->line_warps, p->ndo));
    return 32 * nw;
}

CellParams cell_params(const dts_problem* p)
{
    CellParams c;
    c.NC = p->NC; c.TV = p->TV; c.TX = p->TX; c.TY = p->TY; c.TZ = p->TZ;
    c.NTx = p->NTx; c.NTy = p->NTy; c.nx = p->d.nx; c.ny = p->d.ny; c.nz = p->d.nz;
    c.G = p->G; c.L = p->L; c.B = p->B; c.K = p->K; c.NT = p->NT;
    c.dx = p->d.dx; c.dy = p->d.dy; c.dz = p->d.dz;
    c.x0 = p->d.x0; c.y0 = p->d.y0; c.z0 = p->d.z0;
    c.mat_t = p->mat_t; c.scale_t_t = p->scale_t_t; c.scale_s_t = p->scale_s_t;
    c.sigma_t = p->sigma_t; c.sigma_s = p->sigma_s;
    return c;
}

// arguments of k_moments_q: init = 1 forms Q = M F of the group's fixed source (phi = 0)
QParams q_params(const dts_problem* p, int init)
{
    QParams q{};
    q.B = p->B; q.NT = p->NT; q.TV = p->TV; q.NC = p->NC; q.nitems = p->B * p->NT; q.init = init;
    q.psi = (const float*)p->part; q.Q = (float*)p->Qbuf; q.phi00 = p->phi00;
    q.F = (const float*)p->F; q.Fstride = p->Fstride; q.ctl = p->ctl;
    q.sigs = (const float*)p->sigs; q.sigt = (const float*)p->sigt_r; q.mat_t = p->mat_t;
    q.active = p->active; q.Dt = (const float*)p->Dt; q.Mop = p->Mop; q.Dop = p->Dop;
    q.vol = p->d.dx * p->d.dy * p->d.dz; q.blk = p->blk; q.err = p->dev_err; q.poison = p->dev_poison;
    q.n_psi = count_of<float>(p, p->part); q.n_Q = count_of<float>(p, p->Qbuf);
    q.n_phi00 = count_of<double>(p, p->phi00); q.n_F = count_of<float>(p, p->F);
    q.n_sigs = count_of<float>(p, p->sigs); q.n_blk = count_of<double>(p, p->blk);
    return q;
}

// cuTensorMapEncodeTiled from the driver, looked up once (the library links only the runtime)
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static const PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            f = nullptr;
        return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
    }();
    return fn;
}

// The Q-input sweep's tensor map of Q [B][8][NT][NDO][TV] (FP32): 4-D {TV, NDO, 8 NT, B} (octant and
// tile merged: their strides are uniform), box {TX, NDO, 1, sources per warp}, zeros outside
dts_status encode_qmap(dts_problem* p, CUtensorMap* map)
{
    const PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return fail(p, DTS_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
    const cuuint64_t row = (cuuint64_t)p->TV * sizeof(float);
    const cuuint64_t dim[4] = {(cuuint64_t)p->TV, (cuuint64_t)p->ndo, 8ull * (cuuint64_t)p->NT, (cuuint64_t)p->B};
    const cuuint64_t stride[3] = {row, row * p->ndo, row * p->ndo * 8ull * (cuuint64_t)p->NT};
    const cuuint32_t box[4] = {(cuuint32_t)p->TX, (cuuint32_t)p->ndo, 1u, (cuuint32_t)batch_sources_per_warp(p)};
    const cuuint32_t estr[4] = {1u, 1u, 1u, 1u};
    const CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, p->Qbuf, dim, stride, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(p, DTS_ERR_CUDA, "cuTensorMapEncodeTiled of Q: error " + std::to_string((int)r));
    return DTS_OK;
}

template <typename R>
dts_status record_sweep(dts_problem* p)
{
    SweepParams<R> sp;
    sp.nx = p->d.nx; sp.ny = p->d.ny; sp.nz = p->d.nz;
    sp.TX = p->TX; sp.TY = p->TY; sp.TZ = p->TZ; sp.TV = p->TV;
    sp.NTx = p->NTx; sp.NTy = p->NTy; sp.NTz = p->NTz; sp.NT = p->NT;
    sp.B = p->B; sp.nsub = p->nsub;
    sp.stage_tiles = p->stage_tiles; sp.stage_off = p->stage_off;
    sp.diag_cells = p->diag_cells; sp.diag_off = p->diag_off;
    sp.M = (const R*)p->Mt; sp.Dt = (const R*)p->Dt; sp.A = (const R*)p->At; sp.Lw = p->Lw;
    sp.T = (const R*)(p->q_mode ? p->Qbuf : p->T); sp.sigt = (const R*)p->sigt_r; sp.part = (R*)p->part;
    sp.xf = (R*)p->xf; sp.yf = (R*)p->yf; sp.zf = (R*)p->zf;
    sp.active = p->active; sp.leak = p->leak;
    sp.n_stage_tiles = count_of<unsigned>(p, p->stage_tiles); sp.n_T = count_of<R>(p, sp.T);
    sp.n_sigt = count_of<R>(p, p->sigt_r); sp.n_part = count_of<R>(p, p->part);
    sp.n_xf = count_of<R>(p, p->xf); sp.n_yf = count_of<R>(p, p->yf); sp.n_zf = count_of<R>(p, p->zf);
    sp.n_leak = count_of<double>(p, p->leak);
    sp.err = p->q_mode ? p->dev_err : nullptr;
    sp.poison_tx = p->q_mode ? p->poison_sweep_tx : 0u;
    const size_t smem = sweep_smem(p);
    if constexpr (sizeof(R) == 4) {
        if (batch_tile(p)) {   // the batched kernel takes the stage's (first tile, count) directly
            CUtensorMap qmap{};   // read by the Q-input form only
            if (p->q_mode) TRY(encode_qmap(p, &qmap));
            BatchFn bf = batch_fn(p);
            if (!bf) return fail(p, DTS_ERR_INTERNAL, "no sweep kernel for this (S_N, P_L)");
            const unsigned groups = (unsigned)((p->B + batch_sources_per_warp(p) - 1) / batch_sources_per_warp(p));
            for (int s = 0; s < p->n_stages; ++s) {
                const int s0 = p->stage_off_h[s], cnt = p->stage_off_h[s + 1] - s0;
                bf<<<(unsigned)cnt * 8u * groups, 32, smem, p->stream>>>(sp, s0, cnt, qmap);
            }
            return DTS_OK;
        }
    }
    SweepFn<R> sf = sweep_fn<R>(p);
    if (!sf) return fail(p, DTS_ERR_INTERNAL, "no sweep kernel for this (S_N, P_L)");
    const int nthr = sweep_threads(p);
    for (int s = 0; s < p->n_stages; ++s) {
        const int cnt = p->stage_off_h[s + 1] - p->stage_off_h[s];
        const unsigned groups = batch_tile(p) ? (unsigned)((p->B + batch_sources_per_warp(p) - 1) /
                                                           batch_sources_per_warp(p))
                                              : (unsigned)p->B;
        const unsigned grid = (unsigned)cnt * 8u * groups;
        sf<<<grid, nthr, smem, p->stream>>>(sp, s);
    }
    return DTS_OK;
}

template <typename R>
dts_status record_reduce(dts_problem* p)
{
    RedParams<R> rp;
    rp.B = p->B; rp.NT = p->NT; rp.TV = p->TV; rp.NC = p->NC;
    rp.part = (const R*)p->part; rp.phi00 = p->phi00; rp.T = (R*)p->T; rp.F = (const R*)p->F;
    rp.Fstride = p->Fstride; rp.ctl = p->ctl; rp.sigs = (const R*)p->sigs; rp.sigs0 = p->sigs0;
    rp.sigt64 = p->sigt64; rp.sigt = (const R*)p->sigt_r;
    rp.mat_t = p->mat_t; rp.active = p->active; rp.vol = p->d.dx * p->d.dy * p->d.dz;
    rp.blk = p->blk;
#ifdef DTS_DEBUG_BOUNDS
    rp.n_part = count_of<R>(p, p->part); rp.n_T = count_of<R>(p, p->T); rp.n_F = count_of<R>(p, p->F);
    rp.n_phi00 = count_of<double>(p, p->phi00); rp.n_sigs = count_of<R>(p, p->sigs);
    rp.n_blk = count_of<double>(p, p->blk);
#endif
    int nblk = p->nblk;
    if constexpr (sizeof(R) == 4) {
        if (p->q_mode) {        // moments from the angular fluxes, then Q = M T on the tensor cores
            nblk = p->NT;
            CK(dts_internal_q_launch(p->ndo, p->K, p->q_kind, q_params(p, 0), p->q_grid, p->stream));
        } else if (p->psi_mode) {      // moments from the angular fluxes, two cells per thread
            nblk = (p->NC / 2 + kRedThreads - 1) / kRedThreads;
            RedPsiFn rf;
            PushPsiFn uf;
            psi_fns(p, rf, uf);
            rf<<<dim3(nblk, p->B), kRedThreads, 0, p->stream>>>(rp, (const float*)p->Dt);
        } else if (p->TV % 4 == 0) {   // four cells per thread
            nblk = (p->NC / 4 + kRedThreads - 1) / kRedThreads;
            RedFn<float> rf4 = reduce4_fn(p->K);
            rf4<<<dim3(nblk, p->B), kRedThreads, 0, p->stream>>>(rp);
        } else {
            reduce_fn<R>(p->K)<<<dim3(nblk, p->B), kRedThreads, 0, p->stream>>>(rp);
        }
    } else {
        reduce_fn<R>(p->K)<<<dim3(nblk, p->B), kRedThreads, 0, p->stream>>>(rp);
    }
    k_resid_final<<<p->B, 1024, 0, p->stream>>>(p->blk, nblk, p->leak, 8 * p->NT, p->status,
                                                count_of<double>(p, p->blk), count_of<double>(p, p->leak),
                                                count_of<double>(p, p->status));
    p->graph_launches = p->n_stages + 2;
    if (p->recording_loop) return DTS_OK;   // the device-resident loop reads the status on the device
    CK(cudaMemcpyAsync(p->h_status, p->status, sizeof(double) * 4 * p->B, cudaMemcpyDeviceToHost,
                       p->stream));
    if (p->q_mode) CK(cudaMemcpyAsync(p->h_err, p->dev_err, sizeof(int), cudaMemcpyDeviceToHost, p->stream));
    return DTS_OK;
}

dts_status capture(dts_problem* p, dts_status (*rec)(dts_problem*), cudaGraphExec_t* out)
{
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(p->stream, cudaStreamCaptureModeThreadLocal));
    dts_status s = rec(p);
    cudaError_t ec = cudaStreamEndCapture(p->stream, &g);
    if (s != DTS_OK) {
        if (g) cudaGraphDestroy(g);
        return s;
    }
    if (ec != cudaSuccess) return fail(p, DTS_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(ec));
    ec = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    if (ec != cudaSuccess) return fail(p, DTS_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(ec));
    return DTS_OK;
}

// one source iteration = two graphs (all tile stages of the sweep; the Eq. 3
// reduction, residual and status copy), so that CUDA events recorded between
// the two replays time the sweep and the reduction separately
dts_status build_graph(dts_problem* p)
{
    if (p->graph) return DTS_OK;
    // kernels with more than 48 KB of dynamic shared memory need the opt-in
    const size_t smem = sweep_smem(p);
    cudaError_t e;
    if (p->fp64) e = cudaFuncSetAttribute(sweep_fn<double>(p),
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    else if (batch_tile(p)) e = cudaFuncSetAttribute(batch_fn(p),
                                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    else e = cudaFuncSetAttribute(sweep_fn<float>(p),
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return fail(p, DTS_ERR_CUDA, std::string("sweep smem attribute: ") + cudaGetErrorString(e));
    TRY(capture(p, p->fp64 ? record_sweep<double> : record_sweep<float>, &p->graph));
    TRY(capture(p, p->fp64 ? record_reduce<double> : record_reduce<float>, &p->graph_red));
    return DTS_OK;
}

LoopParams loop_params(const dts_problem* p)
{
    LoopParams q;
    q.B = p->B; q.G = p->G; q.max_iters = p->d.max_iters; q.fp32_stop = p->fp64 ? 0 : 1;
    q.tol = p->d.tol; q.status = p->status; q.active = p->active; q.ctl = p->ctl;
    q.it = p->loop_it; q.last_improve = p->loop_last; q.best = p->loop_best;
    q.iters = p->loop_iters; q.resid = p->loop_resid; q.balance = p->loop_bal;
    q.err = p->q_mode ? p->dev_err : nullptr; q.h = p->loop_h;
    return q;
}

// the body of the device-resident loop: one source iteration (the kernels of both graphs, without the
// status copies to the host) and the convergence control that sets the WHILE node's condition
dts_status record_loop_body(dts_problem* p)
{
    p->recording_loop = true;
    dts_status s = p->fp64 ? record_sweep<double>(p) : record_sweep<float>(p);
    if (s == DTS_OK) s = p->fp64 ? record_reduce<double>(p) : record_reduce<float>(p);
    p->recording_loop = false;
    TRY(s);
    k_loop_control<<<1, kLoopThreads, 0, p->stream>>>(loop_params(p));
    CK(cudaGetLastError());
    return DTS_OK;
}

// graph_loop: one WHILE node (condition 1 at every launch, so the body runs at least once); the
// body's k_loop_control clears it when the group stops. It stops after max_iters iterations at most.
dts_status build_loop_graph(dts_problem* p)
{
    if (p->graph_loop) return DTS_OK;
    TRY(build_graph(p));   // the sweep kernel's shared-memory attribute
    cudaGraph_t g = nullptr;
    CK(cudaGraphCreate(&g, 0));
    auto bail = [&](cudaError_t e, const char* what) {
        cudaGraphDestroy(g);
        return fail(p, DTS_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
    };
    cudaError_t e = cudaGraphConditionalHandleCreate(&p->loop_h, g, 1, cudaGraphCondAssignDefault);
    if (e != cudaSuccess) return bail(e, "cudaGraphConditionalHandleCreate");
    cudaGraphNodeParams np{};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = p->loop_h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np);
    if (e != cudaSuccess) return bail(e, "cudaGraphAddNode (while)");
    cudaGraph_t body = np.conditional.phGraph_out[0];
    e = cudaStreamBeginCaptureToGraph(p->stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return bail(e, "cudaStreamBeginCaptureToGraph");
    const dts_status s = record_loop_body(p);
    e = cudaStreamEndCapture(p->stream, &body);
    if (s != DTS_OK) {
        cudaGraphDestroy(g);
        return s;
    }
    if (e != cudaSuccess) return bail(e, "loop body capture");
    e = cudaGraphInstantiate(&p->graph_loop, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        p->graph_loop = nullptr;
        return fail(p, DTS_ERR_CUDA, std::string("loop graph instantiate: ") + cudaGetErrorString(e));
    }
    return DTS_OK;
}

// fixed-source ring: (W+1) slots of [B][NT][K][TV] doubles
dts_status ensure_ring(dts_problem* p)
{
    if (p->F && p->F_W == p->W) return DTS_OK;
    if (p->graph) {
        cudaGraphExecDestroy(p->graph);
        p->graph = nullptr;
    }
    if (p->graph_red) {
        cudaGraphExecDestroy(p->graph_red);
        p->graph_red = nullptr;
    }
    if (p->graph_loop) {
        cudaGraphExecDestroy(p->graph_loop);
        p->graph_loop = nullptr;
    }
    dfree(p, p->F);
    p->F = nullptr;
    p->Fstride = (size_t)p->B * p->NC * p->K;
    TRY(dalloc(p, &p->F, p->Fstride * (p->W + 1) * p->rsz));
    p->F_W = p->W;
    return DTS_OK;
}

template <typename R>
void launch_group_xs(dts_problem* p, int g)
{
    const int nb = (p->NC + 255) / 256;
    k_group_xs<R><<<nb, 256, 0, p->stream>>>(cell_params(p), g, (R*)p->sigt_r, p->sigt64, (R*)p->sigs,
                                             p->sigs0);
}

// T = F of the group's ring slot (phi = 0 before the first sweep): one device-to-device copy; with an
// initial guess, T = F + sigma_s phi_guess and phi = phi_guess (tensor-core forms: Q = M T)
template <typename R>
dts_status launch_group_init(dts_problem* p, int g, int slot)
{
    if (p->guess) {   // restart: T = F + sigma_s phi_guess, residual measured against the guess
        R* T = p->q_mode ? (R*)p->guess_T : (R*)p->T;
        k_guess_source<R><<<dim3((p->NC + 255) / 256, p->B), 256, 0, p->stream>>>(
            cell_params(p), p->guess, g, (const R*)p->F + (size_t)slot * p->Fstride, (const R*)p->sigs, T,
            p->phi00, p->V);
        CK(cudaGetLastError());
        if (p->q_mode) {   // Q = M T on the tensor cores, T in place of the fixed source
            QParams q = q_params(p, 1);
            q.F = (const float*)p->guess_T;
            q.Fstride = 0;
            q.n_F = count_of<float>(p, p->guess_T);
            CK(dts_internal_q_launch(p->ndo, p->K, p->q_kind, q, p->q_grid, p->stream));
        }
        return DTS_OK;
    }
    if (p->q_mode) {   // Q = M F on the tensor cores
        CK(dts_internal_q_launch(p->ndo, p->K, p->q_kind, q_params(p, 1), p->q_grid, p->stream));
        return DTS_OK;
    }
    const size_t total = (size_t)p->B * p->NC * p->K;
    CK(cudaMemcpyAsync(p->T, (const R*)p->F + (size_t)slot * p->Fstride, total * sizeof(R), cudaMemcpyDeviceToDevice,
                       p->stream));
    return DTS_OK;
}

template <typename R>
void launch_fixed_source(dts_problem* p, int gt, int slot)
{
    SrcParams<R> sp;
    sp.c = cell_params(p);
    sp.src = p->src; sp.unc = p->unc; sp.q = p->q; sp.F = (R*)p->F; sp.Fstride = p->Fstride;
    sp.V = p->V; sp.W = p->W; sp.sigma_s_f = p->sigma_s_f; sp.U = p->U; sp.uslot = p->uslot;
    k_fixed_source<R><<<dim3((p->NC + 255) / 256, p->B), 256, 0, p->stream>>>(sp, gt, slot);
}

template <typename R>
void launch_push(dts_problem* p, int g)
{
    PushParams<R> pp;
    pp.c = cell_params(p);
    pp.part = (const R*)p->part; pp.F = (R*)p->F; pp.Fstride = p->Fstride; pp.W = p->W; pp.V = p->V;
    pp.col = p->col; pp.mom = p->d.keep_moments ? p->mom : nullptr;
    pp.sigma_s_f = p->sigma_s_f;
    if constexpr (sizeof(R) == 4) {
        if (p->psi_mode) {   // the moments from the angular fluxes; kPushRing lower groups per pass
            RedPsiFn rf;
            PushPsiFn uf;
            psi_fns(p, rf, uf);
            // the tensor-core forms' sweep stores odd octants' angular fluxes in their own x order
            for (int w0 = 0; w0 == 0 || w0 < p->W; w0 += kPushRing)
                uf<<<dim3((p->NC / 2 + 255) / 256, p->B), 256, 0, p->stream>>>(pp, g, (const float*)p->Dt,
                                                                              p->q_mode ? 1 : 0, w0);
            return;
        }
        if (p->TX % 4 == 0 && p->W <= 4) {
            using PushFn = void (*)(const PushParams<float>, int);
            const PushFn f = p->K == 1 ? k_push4<1> : p->K == 4 ? k_push4<4> : p->K == 9 ? k_push4<9> : k_push4<16>;
            f<<<dim3((p->NC / 4 + 255) / 256, p->B), 256, 0, p->stream>>>(pp, g);
            return;
        }
    }
    k_push<R><<<dim3((p->NC + 255) / 256, p->B), 256, 0, p->stream>>>(pp, g);
}

// Streamed output of group g (dts_set_host_output): the group's component of every member gathered on
// the solve's stream into staging slot g & 1, then copied to host_out[b][g][:] on the copy stream while
// the solve goes on with the next groups; a slot is reused once its previous copy has landed.
dts_status stream_group_output(dts_problem* p, int g)
{
    if (!p->host_out) return DTS_OK;
    const int slot = g & 1;
    const size_t V = (size_t)p->V, G = (size_t)p->G;
    if (p->copied_pending[slot]) CK(cudaStreamWaitEvent(p->stream, p->ev_copied[slot], 0));
    k_gather_component<<<dim3((unsigned)((V + 255) / 256), p->B), 256, 0, p->stream>>>(
        p->unc, p->col, p->host_comp, g, (int)G, (int)V, p->out_stage[slot]);
    CK(cudaGetLastError());
    CK(cudaEventRecord(p->ev_staged[slot], p->stream));
    CK(cudaStreamWaitEvent(p->copy_stream, p->ev_staged[slot], 0));
    CK(cudaMemcpy2DAsync(p->host_out + (size_t)g * V, G * V * sizeof(double), p->out_stage[slot],
                         V * sizeof(double), V * sizeof(double), (size_t)p->B, cudaMemcpyDeviceToHost,
                         p->copy_stream));
    CK(cudaEventRecord(p->ev_copied[slot], p->copy_stream));
    p->copied_pending[slot] = true;
    return DTS_OK;
}

// One solve as a sequence of steps, so that several problems can be interleaved
// (dts_solve_many): start, then per group begin_group, (launch_iteration,
// complete_iteration) until the group's members stop, end_group; then finish.
// NVTX ranges are start/end ranges (not a push/pop stack), since the steps of
// interleaved problems do not nest.
// the device-resident loop serves a solve when it is switched on and no per-iteration callback is set;
// the bounds-checked build reads its check word on the host after every iteration, so it keeps the host loop
bool use_device_loop(const dts_problem* p)
{
#ifdef DTS_DEBUG_BOUNDS
    return false;
#else
    return p->device_loop && !p->on_iter && p->loop_mem && p->B <= kLoopMaxMembers;
#endif
}

struct SolveRun {
    dts_problem* p;
    const bool dev;   // the group's source iterations run as one graph launch (dts_set_device_loop)
    int B, G, W1;
    int g = 0, it = 0, n_active = 0;
    int64_t updates = 0, sweeps = 0, sweep_launches = 0, launches = 0;
    double max_res = 0.0, sweep_ms = 0.0, reduce_ms = 0.0;
    bool all_conv = true, done = false;
    int64_t u_per_sweep;
    std::vector<double> best, last_improve;
    nvtxRangeId_t r_solve = 0, r_group = 0, r_iter = 0;

    explicit SolveRun(dts_problem* pp)
        : p(pp), dev(use_device_loop(pp)), B(pp->B), G(pp->G), W1(pp->W + 1),
          u_per_sweep((int64_t)pp->V * pp->nd), best(pp->B),
          last_improve(pp->B)
    {
    }
    ~SolveRun()
    {
        // on every way out (an error included) no copy into the caller's host array is left in flight
        if (p->host_out && p->copy_stream) cudaStreamSynchronize(p->copy_stream);
        if (r_iter) nvtxRangeEnd(r_iter);
        if (r_group) nvtxRangeEnd(r_group);
        if (r_solve) nvtxRangeEnd(r_solve);
    }
    SolveRun(const SolveRun&) = delete;
    SolveRun& operator=(const SolveRun&) = delete;

    // graphs, the first-collision source of every group (A1), the first groups' fixed sources
    dts_status start()
    {
        r_solve = nvtxRangeStartA("dts_solve");
#ifdef DTS_DEBUG_BOUNDS
        take_bounds_word();   // a word left by an earlier failure is not this solve's
#endif
        TRY(ensure_ring(p));
        TRY(build_graph(p));
        if (dev) TRY(build_loop_graph(p));
        if (p->q_mode) {
            CK(cudaMemsetAsync(p->dev_err, 0, sizeof(int), p->stream));
            *p->h_err = 0;
        }
        CK(cudaEventRecord(p->ev0, p->stream));
        {
            RayParams rp;
            rp.nx = p->d.nx; rp.ny = p->d.ny; rp.nz = p->d.nz; rp.V = p->V; rp.G = G;
            rp.dx = p->d.dx; rp.dy = p->d.dy; rp.dz = p->d.dz;
            rp.x0 = p->d.x0; rp.y0 = p->d.y0; rp.z0 = p->d.z0;
            rp.mat = p->mat_nat; rp.scale_t = p->scale_t_nat; rp.sigma_t = p->sigma_t;
            rp.src = p->src; rp.spec = p->spec; rp.unc = p->unc; rp.n_mat = p->n_mat; rp.fan = p->fan;
            if (p->n_mat <= kRayMats) {
                k_raytrace_mat<<<dim3((p->V + kRayThreads - 1) / kRayThreads, B), kRayThreads, 0, p->stream>>>(rp);
            } else {
                for (int g0 = 0; g0 < G; g0 += kRayGroups)
                    k_raytrace<<<dim3((p->V + 127) / 128, B), 128, 0, p->stream>>>(rp, g0);
            }
            if (p->n_uslots > 0) {   // members with several cones
                if (p->n_mat > kRayMats)
                    return fail(p, DTS_ERR_INVALID_ARG, "combined cone sources need at most 8 materials");
                ConeParams cp;
                cp.geo = p->cone_geo; cp.spec = p->cone_spec; cp.n_cones = p->cone_n; cp.slot = p->uslot;
                cp.U = p->U; cp.cap = p->cone_cap; cp.K = p->K; cp.L = p->L;
                k_raytrace_cones<<<dim3((p->V + kRayThreads - 1) / kRayThreads, B), kRayThreads, 0, p->stream>>>(rp, cp);
            }
            CK(cudaGetLastError());
        }
        for (int gg = 0; gg < std::min(G, W1); ++gg) {
            if (p->fp64) launch_fixed_source<double>(p, gg, gg % W1);
            else launch_fixed_source<float>(p, gg, gg % W1);
        }
        launches = (p->n_mat <= kRayMats ? 1 : (G + kRayGroups - 1) / kRayGroups) + std::min(G, W1);
        g = 0;
        return begin_group();
    }

    // group g: its cross sections, every member active again, the group's first source
    dts_status begin_group()
    {
        char gname[32];
        snprintf(gname, sizeof gname, "group %d", g);
        r_group = nvtxRangeStartA(gname);
        const int slot = g % W1;
        if (dev) {   // the same set-up on the device: control values, flags, loop state
            k_loop_begin<<<1, kLoopThreads, 0, p->stream>>>(loop_params(p), g, slot);
        } else {
            k_set_ctl<<<1, 1, 0, p->stream>>>(p->ctl, g, slot);
        }
        CK(cudaMemsetAsync(p->phi00, 0, sizeof(double) * B * p->NC, p->stream));
        if (!dev) {
            for (int b = 0; b < B; ++b) {
                p->h_active[b] = 1;
                p->iters[(size_t)b * G + g] = 0;
                best[b] = INFINITY;
                last_improve[b] = 0;
            }
            // every member is active again before the group's first source is formed (the
            // tensor-core forms' Q = M F skips inactive members)
            CK(cudaMemcpyAsync(p->active, p->h_active, sizeof(int) * B, cudaMemcpyHostToDevice, p->stream));
        }
        if (p->fp64) {
            launch_group_xs<double>(p, g);
            TRY(launch_group_init<double>(p, g, slot));
        } else {
            launch_group_xs<float>(p, g);
            TRY(launch_group_init<float>(p, g, slot));
        }
        CK(cudaGetLastError());
        // set_ctl, group_xs; the group's first source: a copy, or a kernel in the tensor-core forms, plus
        // the guess kernel when there is an initial guess
        launches += 2 + (p->q_mode ? 1 : 0) + (p->guess ? 1 : 0);
        n_active = B;
        it = 0;
        return DTS_OK;
    }

    // the group goes on while a member iterates and the iteration cap is not reached
    bool group_iterating() const { return n_active > 0 && it < p->d.max_iters; }

    // device-resident loop: all of the group's source iterations as one graph launch; the host
    // learns their counts, residuals and balance when the solve finishes
    dts_status launch_group_loop()
    {
        CK(cudaGraphLaunch(p->graph_loop, p->stream));
        n_active = 0;
        return DTS_OK;
    }

    // one source iteration (the sweep graph, then the moment graph) enqueued
    dts_status launch_iteration()
    {
        ++it;
        r_iter = nvtxRangeStartA("source iteration");
        CK(cudaEventRecord(p->eva, p->stream));
        CK(cudaGraphLaunch(p->graph, p->stream));
        CK(cudaEventRecord(p->evb, p->stream));
        CK(cudaGraphLaunch(p->graph_red, p->stream));
        CK(cudaEventRecord(p->evc, p->stream));
        return DTS_OK;
    }

    // waits for the launched iteration, records each member's residual and balance, and
    // retires the members that stopped (A7)
    dts_status complete_iteration()
    {
        CK(cudaEventSynchronize(p->evc));
        nvtxRangeEnd(r_iter);
        r_iter = 0;
        if (p->q_mode && *p->h_err)
            return fail(p, DTS_ERR_TIMEOUT, "k_moments_q: a bounded wait on a bulk copy or the tensor cores gave up");
#ifdef DTS_DEBUG_BOUNDS
        if (const unsigned long long w = take_bounds_word()) return fail(p, DTS_ERR_INTERNAL, bounds_message(w));
#endif
        launches += p->graph_launches;
        sweep_launches += p->n_stages;
        {
            float a = 0.f, b2 = 0.f;
            CK(cudaEventElapsedTime(&a, p->eva, p->evb));
            CK(cudaEventElapsedTime(&b2, p->evb, p->evc));
            sweep_ms += a;
            reduce_ms += b2;
        }
        bool changed = false;
        for (int b = 0; b < B; ++b) {
            if (!p->h_active[b]) continue;
            const double* s = p->h_status + 4 * b;
            const size_t bg = (size_t)b * G + g;
            p->iters[bg] = it;
            p->resid[bg] = s[0];
            p->balance[bg * 3 + 0] = s[1];
            p->balance[bg * 3 + 1] = s[2];
            p->balance[bg * 3 + 2] = s[3];
            updates += u_per_sweep;
            ++sweeps;
            bool stop = p->d.tol > 0.0 && s[0] < p->d.tol;
            if (!stop && !p->fp64 && p->d.tol > 0.0) {
                // FP32 forms: stop when the residual has stagnated at the rounding floor
                if (s[0] < 0.99 * best[b]) {
                    best[b] = s[0];
                    last_improve[b] = it;
                } else if (it - last_improve[b] >= 10) {
                    stop = true;
                }
            }
            if (stop) {
                p->h_active[b] = 0;
                --n_active;
                changed = true;
            }
        }
        if (changed && n_active > 0)
            CK(cudaMemcpyAsync(p->active, p->h_active, sizeof(int) * B, cudaMemcpyHostToDevice, p->stream));
        if (p->on_iter) {
            // this iteration's residual of every member, NaN where the member had stopped before it
            std::vector<double> res(B, std::nan(""));
            for (int b = 0; b < B; ++b)
                if (p->iters[(size_t)b * G + g] == it) res[b] = p->resid[(size_t)b * G + g];
            p->on_iter(p->on_iter_user, g, it, res.data(), B);
        }
        return DTS_OK;
    }

    // the group's downscatter into the ring (A2) and a later group's fixed source; then the
    // next group, or the end of the solve
    dts_status end_group()
    {
        for (int b = 0; !dev && b < B; ++b) {   // device-resident loop: in finish()
            const size_t bg = (size_t)b * G + g;
            max_res = std::max(max_res, p->resid[bg]);
            if (p->d.tol > 0.0 && !(p->resid[bg] < p->d.tol)) all_conv = false;
        }
        const int slot = g % W1;
        if (p->fp64) launch_push<double>(p, g);
        else launch_push<float>(p, g);
        TRY(stream_group_output(p, g));
        // the downscatter push: one kernel, or one pass per kPushRing lower groups from angular fluxes
        launches += (p->psi_mode && !p->fp64) ? std::max(1, (p->W + kPushRing - 1) / kPushRing) : 1;
        if (g + W1 < G) {
            if (p->fp64) launch_fixed_source<double>(p, g + W1, slot);
            else launch_fixed_source<float>(p, g + W1, slot);
            ++launches;
        }
        CK(cudaGetLastError());
        nvtxRangeEnd(r_group);
        r_group = 0;
        if (++g < G) return begin_group();
        done = true;
        return DTS_OK;
    }

    // device-resident loop, once the solve's work is complete: the per-(member, group) iteration
    // counts, residuals and balance terms, and from them the counts the host loop keeps as it goes
    dts_status collect_device_loop()
    {
        const size_t BG = (size_t)B * G;
        CK(cudaMemcpyAsync(p->iters.data(), p->loop_iters, sizeof(int32_t) * BG, cudaMemcpyDeviceToHost,
                           p->stream));
        CK(cudaMemcpyAsync(p->resid.data(), p->loop_resid, sizeof(double) * BG, cudaMemcpyDeviceToHost,
                           p->stream));
        CK(cudaMemcpyAsync(p->balance.data(), p->loop_bal, sizeof(double) * 3 * BG, cudaMemcpyDeviceToHost,
                           p->stream));
        if (p->q_mode) CK(cudaMemcpyAsync(p->h_err, p->dev_err, sizeof(int), cudaMemcpyDeviceToHost, p->stream));
        CK(cudaStreamSynchronize(p->stream));
        if (p->q_mode && *p->h_err)
            return fail(p, DTS_ERR_TIMEOUT, "k_moments_q: a bounded wait on a bulk copy or the tensor cores gave up");
        for (int gg = 0; gg < G; ++gg) {
            int trips = 0;   // the WHILE node's iterations: every one counts the members still active
            for (int b = 0; b < B; ++b) {
                const size_t bg = (size_t)b * G + gg;
                const int n_it = p->iters[bg];
                trips = std::max(trips, n_it);
                updates += (int64_t)n_it * u_per_sweep;
                sweeps += n_it;
                max_res = std::max(max_res, p->resid[bg]);
                if (p->d.tol > 0.0 && !(p->resid[bg] < p->d.tol)) all_conv = false;
            }
            launches += (int64_t)trips * (p->graph_launches + 1);   // + k_loop_control
            sweep_launches += (int64_t)trips * p->n_stages;
        }
        return DTS_OK;
    }

    dts_status finish(dts_solve_stats* st)
    {
        CK(cudaEventRecord(p->ev1, p->stream));
        CK(cudaEventSynchronize(p->ev1));
        if (p->host_out) {   // the last groups' copies to the host
            CK(cudaStreamSynchronize(p->copy_stream));
            p->copied_pending[0] = p->copied_pending[1] = false;
        }
        if (dev) TRY(collect_device_loop());
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, p->ev0, p->ev1));
        p->solved = true;
        if (st) {
            st->updates = updates;
            st->sweeps = sweeps;
            st->max_residual = max_res;
            st->solve_ms = ms;
            st->sweep_ms = sweep_ms;
            st->reduce_ms = reduce_ms;
            st->launches = launches;
            st->sweep_launches = sweep_launches;
            st->converged = all_conv ? 1 : 0;
            st->tile_x = p->TX;
            st->tile_y = p->TY;
            st->tile_z = p->TZ;
        }
        nvtxRangeEnd(r_solve);
        r_solve = 0;
        if (!all_conv) return fail(p, DTS_ERR_NOT_CONVERGED, "some (source, group) stopped above tol");
        return DTS_OK;
    }
};

dts_status run_solve(dts_problem* p, dts_solve_stats* st)
{
    SolveRun r(p);
    TRY(r.start());
    if (r.dev) {   // every group enqueued now: no host round trip per iteration
        while (!r.done) {
            TRY(r.launch_group_loop());
            TRY(r.end_group());
        }
        return r.finish(st);
    }
    while (!r.done) {
        while (r.group_iterating()) {
            TRY(r.launch_iteration());
            TRY(r.complete_iteration());
        }
        TRY(r.end_group());
    }
    return r.finish(st);
}

// the batched kernel addresses one warp's sources with 32-bit offsets
bool batch_offsets_fit(const dts_problem* p, int tx, int ty, int tz)
{
    const size_t padded = (size_t)((p->d.nx + tx - 1) / tx * tx) * ((p->d.ny + ty - 1) / ty * ty) *
                          ((p->d.nz + tz - 1) / tz * tz);
    return (size_t)(32 / p->ndo) * padded * p->K < (size_t)INT_MAX;
}

void choose_tile(dts_problem* p)
{
    if (p->d.tile_x > 0) {
        p->TX = p->d.tile_x;
        p->TY = p->d.tile_y;
        p->TZ = p->d.tile_z;
        p->TV = p->TX * p->TY * p->TZ;
        return;
    }
    // default: FP32 batches of at least a warp's worth of sources take the
    // batched kernel's 8 x 4 x 4 tile; otherwise 32 x-lines (4 in y, 8 in z)
    // per tile for the warp-synchronous kernel, 8 cells long in x (measured
    // fastest of 4..32 on the 96^3 S8 P3 batch)
    const bool batched = (p->q_mode || (p->d.precision == DTS_PREC_FP32 && p->d.batch >= 32 / p->ndo)) &&
                         batch_offsets_fit(p, 8, 4, 4);
    p->TX = 8;
    p->TY = 4;
    p->TZ = batched ? 4 : 8;
    p->TV = p->TX * p->TY * p->TZ;
}

dts_status setup_schedule(dts_problem* p)
{
    p->TV = p->TX * p->TY * p->TZ;
    p->NTx = (p->d.nx + p->TX - 1) / p->TX;
    p->NTy = (p->d.ny + p->TY - 1) / p->TY;
    p->NTz = (p->d.nz + p->TZ - 1) / p->TZ;
    if (batch_tile(p) && !batch_offsets_fit(p, p->TX, p->TY, p->TZ))
        return fail(p, DTS_ERR_INVALID_ARG, "grid too large for the batched 4 x 4 tiles; take an 8 x 4 x 8 tile");
    if (p->NTx > 1023 || p->NTy > 1023 || p->NTz > 1023)
        return fail(p, DTS_ERR_INVALID_ARG, "too many tiles along an axis (max 1023)");
    p->NT = p->NTx * p->NTy * p->NTz;
    p->NC = p->NT * p->TV;
    // tile stages: Eq. 9 applied to the NTx x NTy x NTz tile grid
    p->n_stages = p->NTx + p->NTy + p->NTz - 2;
    p->stage_off_h.assign(p->n_stages + 1, 0);
    for (int s = 0; s < p->n_stages; ++s)
        p->stage_off_h[s + 1] = p->stage_off_h[s] + (int)eq9(p->NTx, p->NTy, p->NTz, s);
    if (p->stage_off_h[p->n_stages] != p->NT) return fail(p, DTS_ERR_INTERNAL, "stage count mismatch");
    std::vector<unsigned> tiles(p->NT);
    std::vector<int> fill(p->stage_off_h.begin(), p->stage_off_h.end() - 1);
    for (int c = 0; c < p->NTz; ++c)
        for (int b = 0; b < p->NTy; ++b)
            for (int a = 0; a < p->NTx; ++a)
                if (fill[a + b + c] < p->stage_off_h[a + b + c + 1])
                    tiles[fill[a + b + c]++] = (unsigned)a | ((unsigned)b << 10) | ((unsigned)c << 20);
    for (int s = 0; s < p->n_stages; ++s)
        if (fill[s] != p->stage_off_h[s + 1]) return fail(p, DTS_ERR_INTERNAL, "Eq. 9 stage size mismatch");
    // intra-tile sub-sweeps (Table 1 ordering is irrelevant inside a sub-sweep)
    p->nsub = p->TX + p->TY + p->TZ - 2;
    std::vector<int> doff(p->nsub + 1, 0);
    for (int s = 0; s < p->nsub; ++s) doff[s + 1] = doff[s] + (int)eq9(p->TX, p->TY, p->TZ, s);
    std::vector<unsigned> cells(p->TV);
    std::vector<int> dfill(doff.begin(), doff.end() - 1);
    for (int z = 0; z < p->TZ; ++z)
        for (int y = 0; y < p->TY; ++y)
            for (int x = 0; x < p->TX; ++x)
                if (dfill[x + y + z] < doff[x + y + z + 1])
                    cells[dfill[x + y + z]++] = (unsigned)x | ((unsigned)y << 8) | ((unsigned)z << 16);
    for (int s = 0; s < p->nsub; ++s)
        if (dfill[s] != doff[s + 1]) return fail(p, DTS_ERR_INTERNAL, "Eq. 9 sub-sweep size mismatch");
    TRY(dalloc_t(p, &p->stage_tiles, tiles.size()));
    TRY(dalloc_t(p, &p->stage_off, p->stage_off_h.size()));
    TRY(dalloc_t(p, &p->diag_cells, cells.size()));
    TRY(dalloc_t(p, &p->diag_off, doff.size()));
    CK(cudaMemcpy(p->stage_tiles, tiles.data(), tiles.size() * sizeof(unsigned), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(p->stage_off, p->stage_off_h.data(), p->stage_off_h.size() * sizeof(int), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(p->diag_cells, cells.data(), cells.size() * sizeof(unsigned), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(p->diag_off, doff.data(), doff.size() * sizeof(int), cudaMemcpyHostToDevice));
    return DTS_OK;
}

template <typename R>
dts_status upload_tables(dts_problem* p, const std::vector<double>& Dkn, const std::vector<double>& Mnk)
{
    const int nd = p->nd, K = p->K;
    std::vector<R> M(nd * K), Dt(nd * K), A(nd * 3);
    std::vector<double> Lw(nd * 3);
    for (int n = 0; n < nd; ++n) {
        for (int k = 0; k < K; ++k) {
            M[n * K + k] = (R)Mnk[(size_t)n * K + k];
            Dt[n * K + k] = (R)Dkn[(size_t)k * nd + n];
        }
        const double om[3] = {std::fabs(p->mu[n]), std::fabs(p->eta[n]), std::fabs(p->xi[n])};
        const double h[3] = {p->d.dx, p->d.dy, p->d.dz};
        const double area[3] = {p->d.dy * p->d.dz, p->d.dx * p->d.dz, p->d.dx * p->d.dy};
        for (int a = 0; a < 3; ++a) {
            A[n * 3 + a] = (R)(2.0 * om[a] / h[a]);
            Lw[n * 3 + a] = p->w[n] * om[a] * area[a];
        }
    }
    TRY(dalloc(p, &p->Mt, M.size() * sizeof(R)));
    TRY(dalloc(p, &p->Dt, Dt.size() * sizeof(R)));
    TRY(dalloc(p, &p->At, A.size() * sizeof(R)));
    TRY(dalloc_t(p, &p->Lw, Lw.size()));
    CK(cudaMemcpy(p->Mt, M.data(), M.size() * sizeof(R), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(p->Dt, Dt.data(), Dt.size() * sizeof(R), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(p->At, A.data(), A.size() * sizeof(R), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(p->Lw, Lw.data(), Lw.size() * sizeof(double), cudaMemcpyHostToDevice));
    return DTS_OK;
}

// FP32 value of x rounded to nearest-even at `drop` low mantissa bits (16: bf16, 13: tf32)
float round_mantissa(double x, int drop)
{
    float f = (float)x;
    uint32_t u;
    std::memcpy(&u, &f, 4);
    const uint32_t half = (1u << (drop - 1)) - 1u + ((u >> drop) & 1u);
    u = (u + half) & ~((1u << drop) - 1u);
    std::memcpy(&f, &u, 4);
    return f;
}

// Operand parts of the tensor-core contractions, stored as (hi, lo) with
// hi = r(x), lo = r(x - hi): the source operator M' = 4 pi M padded to
// [NP][16] (N_d rounded up to a multiple of 16, K up to 16; r the rounding to
// bf16 for split BF16, to tf32 for split TF32), and, when N_d is a multiple of
// 16, the Eq. 3 operator D padded to [16][N_d] (r the rounding to bf16).
dts_status upload_qop(dts_problem* p, const std::vector<double>& Dkn, const std::vector<double>& Mnk)
{
    const int nd = p->nd, K = p->K, NP = (nd + 15) / 16 * 16;
    const int drop = p->q_kind == 0 ? 16 : 13;
    std::vector<float> op((size_t)2 * NP * 16, 0.f);
    for (int n = 0; n < nd; ++n)
        for (int k = 0; k < K; ++k) {
            const double m = 4.0 * kPi * Mnk[(size_t)n * K + k];
            const float hi = round_mantissa(m, drop);
            op[(size_t)n * 16 + k] = hi;
            op[(size_t)NP * 16 + (size_t)n * 16 + k] = round_mantissa(m - (double)hi, drop);
        }
    TRY(dalloc_t(p, &p->Mop, op.size()));
    CK(cudaMemcpy(p->Mop, op.data(), op.size() * sizeof(float), cudaMemcpyHostToDevice));
    if (nd % 16 == 0) {
        std::vector<float> dop((size_t)2 * 16 * nd, 0.f);
        for (int k = 0; k < K; ++k)
            for (int n = 0; n < nd; ++n) {
                const double v = Dkn[(size_t)k * nd + n];
                const float hi = round_mantissa(v, 16);
                dop[(size_t)k * nd + n] = hi;
                dop[(size_t)16 * nd + (size_t)k * nd + n] = round_mantissa(v - (double)hi, 16);
            }
        TRY(dalloc_t(p, &p->Dop, dop.size()));
        CK(cudaMemcpy(p->Dop, dop.data(), dop.size() * sizeof(float), cudaMemcpyHostToDevice));
    }
    return DTS_OK;
}

dts_status create(const dts_problem_desc* desc, dts_problem* p)
{
    p->d = *desc;
    const dts_problem_desc& d = p->d;
    if (d.nx < 1 || d.ny < 1 || d.nz < 1 || d.nx > 65536 || d.ny > 65536 || d.nz > 65536)
        return fail(p, DTS_ERR_INVALID_ARG, "grid extents must be in 1..65536");
    if (!(d.dx > 0 && d.dy > 0 && d.dz > 0) || !isfin(d.dx) || !isfin(d.dy) || !isfin(d.dz))
        return fail(p, DTS_ERR_INVALID_ARG, "voxel pitch must be finite and > 0");
    if (!isfin(d.x0) || !isfin(d.y0) || !isfin(d.z0))
        return fail(p, DTS_ERR_INVALID_ARG, "grid origin must be finite");
    if (d.n_groups < 1) return fail(p, DTS_ERR_INVALID_ARG, "n_groups must be >= 1");
    if (d.legendre_order < 0 || d.legendre_order > 3)
        return fail(p, DTS_ERR_INVALID_ARG, "legendre_order must be in 0..3");
    if (d.batch < 1) return fail(p, DTS_ERR_INVALID_ARG, "batch must be >= 1");
    if (d.precision != DTS_PREC_FP64 && d.precision != DTS_PREC_FP32 && d.precision != DTS_PREC_FP32_SPLITBF16 &&
        d.precision != DTS_PREC_FP32_TF32)
        return fail(p, DTS_ERR_INVALID_ARG, "unknown precision");
    if (!(d.tol >= 0.0) || !isfin(d.tol)) return fail(p, DTS_ERR_INVALID_ARG, "tol must be finite and >= 0");
    if (d.max_iters < 1) return fail(p, DTS_ERR_INVALID_ARG, "max_iters must be >= 1");
    const bool tile_given = d.tile_x || d.tile_y || d.tile_z;
    if (tile_given && (d.tile_x < 1 || d.tile_y < 1 || d.tile_z < 1 || d.tile_x > 64 ||
                       d.tile_y > 64 || d.tile_z > 64))
        return fail(p, DTS_ERR_INVALID_ARG, "tile extents must all be 0 or all in 1..64");
    if (!ls_set(d.sn_order, p->mu, p->eta, p->xi, p->w))
        return fail(p, DTS_ERR_INVALID_ARG, "sn_order must be 2, 4, 6 or 8");
    p->V = d.nx * d.ny * d.nz;
    p->G = d.n_groups;
    p->L = d.legendre_order;
    p->K = (p->L + 1) * (p->L + 1);
    p->nd = (int)p->w.size();
    p->ndo = p->nd / 8;
    p->B = d.batch;
    p->fp64 = d.precision == DTS_PREC_FP64;
    p->rsz = p->fp64 ? sizeof(double) : sizeof(float);
    p->q_mode = d.precision == DTS_PREC_FP32_SPLITBF16 || d.precision == DTS_PREC_FP32_TF32;
    p->q_kind = d.precision == DTS_PREC_FP32_TF32 ? 1 : 0;
    choose_tile(p);
    if (p->q_mode && !(p->TX == 8 && p->TY == 4 && p->TZ == 4))
        return fail(p, DTS_ERR_INVALID_ARG, "the tensor-core precisions need the 8 x 4 x 4 tile");
    p->psi_mode = p->q_mode || psi_form(p);

    int ndev = 0;
    CK(cudaGetDeviceCount(&ndev));
    if (d.device < 0 || d.device >= ndev) return fail(p, DTS_ERR_INVALID_ARG, "device ordinal out of range");
    DevGuard guard(d.device);
    cudaDeviceProp prop;
    CK(cudaGetDeviceProperties(&prop, d.device));
    p->n_sm = prop.multiProcessorCount;
    if (p->psi_mode && !p->q_mode) {
        RedPsiFn rf;
        PushPsiFn uf;
        psi_fns(p, rf, uf);
        if (!rf) p->psi_mode = false;   // octant partials instead
    }
    if (p->q_mode) {
        const int qs = dts_internal_q_smem(p->ndo, p->K, p->q_kind);
        if (qs < 0 || (size_t)qs > prop.sharedMemPerBlockOptin)
            return fail(p, DTS_ERR_INVALID_ARG, "no tensor-core moment kernel for this (S_N, P_L)");
        CK(dts_internal_q_prepare(p->ndo, p->K, p->q_kind));
        int per_sm = 0;
        CK(dts_internal_q_occupancy(p->ndo, p->K, p->q_kind, &per_sm));
        // every resident CTA holds kQTmemCols of the SM's 512 tensor-memory columns
        per_sm = std::max(1, std::min(per_sm, 512 / kQTmemCols));
        p->q_grid = per_sm * p->n_sm;
    }
    if (sweep_smem(p) > prop.sharedMemPerBlockOptin)
        return fail(p, DTS_ERR_INVALID_ARG, "wavefront tile needs more shared memory than a CTA has");
    if (d.cuda_stream) {
        p->stream = (cudaStream_t)d.cuda_stream;
    } else {
        CK(cudaStreamCreateWithFlags(&p->stream, cudaStreamNonBlocking));
        p->own_stream = true;
    }
    CK(cudaEventCreate(&p->ev0));
    CK(cudaEventCreate(&p->ev1));
    CK(cudaEventCreate(&p->eva));
    CK(cudaEventCreate(&p->evb));
    CK(cudaEventCreate(&p->evc));
    TRY(setup_schedule(p));
    std::vector<double> D, M;
    moment_tables(p->L, p->mu, p->eta, p->xi, p->w, D, M);
    TRY(p->fp64 ? upload_tables<double>(p, D, M) : upload_tables<float>(p, D, M));

    const size_t B = p->B, NC = p->NC, K = p->K, G = p->G, V = p->V;
    TRY(dalloc_t(p, &p->mat_t, NC));
    TRY(dalloc_t(p, &p->mat_nat, V));
    TRY(dalloc_t(p, &p->phi00, B * NC));
    TRY(dalloc(p, &p->T, p->q_mode ? 16 : B * NC * K * p->rsz));
    // octant partials [8][B][NT][K][TV], or in the direct-output form the
    // angular fluxes [B][8][NT][N_d/8][TV]
    TRY(dalloc(p, &p->part, 8 * B * NC * (p->psi_mode ? (size_t)p->ndo : (size_t)K) * p->rsz));
    if (p->q_mode) {
        TRY(dalloc(p, &p->Qbuf, 8 * B * NC * (size_t)p->ndo * sizeof(float)));
        TRY(upload_qop(p, D, M));
        TRY(dalloc_t(p, &p->dev_err, 1));
        CK(cudaMemset(p->dev_err, 0, sizeof(int)));
        TRY(dalloc_t(p, &p->dev_poison, 1));
        CK(cudaMemset(p->dev_poison, 0, sizeof(int)));
        CK(cudaMallocHost((void**)&p->h_err, sizeof(int)));
        *p->h_err = 0;
    }
    const size_t nf = (size_t)p->ndo;
    size_t fxs = 8 * B * (size_t)p->NTy * p->NTz * nf * p->TY * p->TZ * p->rsz;
    size_t fys = 8 * B * (size_t)p->NTx * p->NTz * nf * p->TX * p->TZ * p->rsz;
    size_t fzs = 8 * B * (size_t)p->NTx * p->NTy * nf * p->TX * p->TY * p->rsz;
    if (batch_tile(p)) {   // lane-major blocks per source group
        const int ngrp = (p->B + batch_sources_per_warp(p) - 1) / batch_sources_per_warp(p);
        fxs = std::max(fxs, sizeof(float) * batch_face_floats(ngrp, p->NTy * p->NTz, p->TY * p->TZ));
        fys = std::max(fys, sizeof(float) * batch_face_floats(ngrp, p->NTx * p->NTz, p->TX * p->TZ));
        fzs = std::max(fzs, sizeof(float) * batch_face_floats(ngrp, p->NTx * p->NTy, p->TX * p->TY));
    }
    TRY(dalloc(p, &p->xf, fxs));
    TRY(dalloc(p, &p->yf, fys));
    TRY(dalloc(p, &p->zf, fzs));
    TRY(dalloc(p, &p->sigt_r, NC * p->rsz));
    TRY(dalloc_t(p, &p->sigt64, NC));
    TRY(dalloc(p, &p->sigs, NC * (p->L + 1) * p->rsz));
    TRY(dalloc_t(p, &p->sigs0, NC));
    TRY(dalloc_t(p, &p->unc, B * G * V));
    TRY(dalloc_t(p, &p->col, B * G * V));
    TRY(dalloc_t(p, &p->tmp, G * V));
    if (d.keep_moments) TRY(dalloc_t(p, &p->mom, B * G * K * V));
    TRY(dalloc_t(p, &p->src, B * 8));
    TRY(dalloc_t(p, &p->spec, B * G));
    TRY(dalloc_t(p, &p->leak, B * 8 * p->NT));   // one slot per (source, octant, tile)
    p->nblk = (p->NC + kRedThreads - 1) / kRedThreads;
    TRY(dalloc_t(p, &p->blk, B * std::max(p->nblk, p->NT) * 4));   // k_moments_q: one partial per tile
    TRY(dalloc_t(p, &p->status, B * 4));
    TRY(dalloc_t(p, &p->active, B));
    TRY(dalloc_t(p, &p->ctl, 4));
    CK(cudaMemset(p->leak, 0, sizeof(double) * B * 8 * p->NT));
    CK(cudaMemset(p->col, 0, sizeof(double) * B * G * V));
    CK(cudaMallocHost((void**)&p->h_status, sizeof(double) * 4 * B));
    CK(cudaMallocHost((void**)&p->h_active, sizeof(int) * B));
    p->src_h.assign(B * 8, 0.0);
    for (size_t b = 0; b < B; ++b) p->src_h[b * 8] = -1.0;
    p->fan_h.assign(B * 8, 0.0);
    TRY(dalloc_t(p, &p->fan, B * 8));
    CK(cudaMemset(p->fan, 0, sizeof(double) * B * 8));
    p->cone_geo_h.assign(B, {});
    p->cone_spec_h.assign(B, {});
    p->cone_n_h.assign(B, 0);
    p->uslot_h.assign(B, -1);
    TRY(dalloc_t(p, &p->cone_n, B));
    TRY(dalloc_t(p, &p->uslot, B));
    CK(cudaMemset(p->cone_n, 0, sizeof(int) * B));
    CK(cudaMemset(p->uslot, 0, sizeof(int) * B));
    p->spec_h.assign(B * G, 0.0);
    p->src_set.assign(B, 0);
    p->iters.assign(B * G, 0);
    p->resid.assign(B * G, 0.0);
    p->balance.assign(B * G * 3, 0.0);
    return DTS_OK;
}

void destroy(dts_problem* p)
{
    DevGuard guard(p->d.device);
    if (p->stream) cudaStreamSynchronize(p->stream);
    if (p->graph) cudaGraphExecDestroy(p->graph);
    if (p->graph_red) cudaGraphExecDestroy(p->graph_red);
    if (p->graph_loop) cudaGraphExecDestroy(p->graph_loop);
    for (void* a : p->allocs) cudaFree(a);
    p->allocs.clear();
    if (p->h_status) cudaFreeHost(p->h_status);
    if (p->h_active) cudaFreeHost(p->h_active);
    if (p->h_err) cudaFreeHost(p->h_err);
    for (cudaEvent_t e : {p->ev0, p->ev1, p->eva, p->evb, p->evc, p->ev_staged[0], p->ev_staged[1],
                          p->ev_copied[0], p->ev_copied[1]})
        if (e) cudaEventDestroy(e);
    if (p->copy_stream) {
        cudaStreamSynchronize(p->copy_stream);
        cudaStreamDestroy(p->copy_stream);
    }
    if (p->own_stream && p->stream) cudaStreamDestroy(p->stream);
}

// natural [V] -> tiled [NC] (padding gets `pad`)
template <typename T>
std::vector<T> to_tiled(const dts_problem* p, const T* nat, T pad)
{
    std::vector<T> out(p->NC, pad);
    for (int tz = 0; tz < p->NTz; ++tz)
        for (int ty = 0; ty < p->NTy; ++ty)
            for (int tx = 0; tx < p->NTx; ++tx) {
                const size_t tile = ((size_t)tz * p->NTy + ty) * p->NTx + tx;
                for (int sz = 0; sz < p->TZ; ++sz)
                    for (int sy = 0; sy < p->TY; ++sy)
                        for (int sx = 0; sx < p->TX; ++sx) {
                            const int i = tx * p->TX + sx, j = ty * p->TY + sy, k = tz * p->TZ + sz;
                            if (i >= p->d.nx || j >= p->d.ny || k >= p->d.nz) continue;
                            out[tile * p->TV + (sz * p->TY + sy) * p->TX + sx] =
                                nat[((size_t)k * p->d.ny + j) * p->d.nx + i];
                        }
            }
    return out;
}

// ---------------------------------------------------------------------------
// discrete adjoint (FP64): see dts_adjoint.cuh
// ---------------------------------------------------------------------------
template <int NDO, int K>
void* adj_sweep_fn_k(int mode)
{
    return mode == 1 ? (void*)k_sweep_adj<NDO, K, 1> : (void*)k_sweep_adj<NDO, K, 2>;
}

template <int NDO>
void* adj_sweep_fn_n(int K, int mode)
{
    switch (K) {
    case 1: return adj_sweep_fn_k<NDO, 1>(mode);
    case 4: return adj_sweep_fn_k<NDO, 4>(mode);
    case 9: return adj_sweep_fn_k<NDO, 9>(mode);
    case 16: return adj_sweep_fn_k<NDO, 16>(mode);
    }
    return nullptr;
}

using AdjFn = void (*)(const AdjSweepParams, int);

AdjFn adj_sweep_fn(int ndo, int K, int mode)
{
    switch (ndo) {
    case 1: return (AdjFn)adj_sweep_fn_n<1>(K, mode);
    case 3: return (AdjFn)adj_sweep_fn_n<3>(K, mode);
    case 6: return (AdjFn)adj_sweep_fn_n<6>(K, mode);
    case 10: return (AdjFn)adj_sweep_fn_n<10>(K, mode);
    }
    return nullptr;
}

size_t adj_smem(const dts_problem* p)
{
    const size_t n = (size_t)p->ndo * p->TV +
                     (size_t)p->ndo * (p->TY * p->TZ + p->TX * p->TZ + p->TX * p->TY) + p->TV +
                     2 * p->ndo * p->K + 4 * p->ndo;
    return n * sizeof(double);
}

dts_status adj_alloc(dts_problem* p)
{
    if (p->adj_ready && p->adj_W != p->W) {   // band width changed: resize the source ring
        dfree(p, p->adj_S);
        p->adj_S = nullptr;
        TRY(dalloc_t(p, &p->adj_S, (size_t)(p->W + 1) * p->NC * p->K));
        p->adj_W = p->W;
    }
    if (p->adj_ready) return DTS_OK;
    p->adj_W = p->W;
    const size_t NC = p->NC, K = p->K, nd = p->nd, G = p->G, V = p->V, ndo = p->ndo;
    TRY(dalloc_t(p, &p->adj_T, NC * K));
    TRY(dalloc_t(p, &p->adj_part, 8 * NC * K));
    TRY(dalloc_t(p, &p->adj_xf, 8 * (size_t)p->NTy * p->NTz * ndo * p->TY * p->TZ));
    TRY(dalloc_t(p, &p->adj_yf, 8 * (size_t)p->NTx * p->NTz * ndo * p->TX * p->TZ));
    TRY(dalloc_t(p, &p->adj_zf, 8 * (size_t)p->NTx * p->NTy * ndo * p->TX * p->TY));
    TRY(dalloc_t(p, &p->adj_psi, nd * NC));
    TRY(dalloc_t(p, &p->adj_mask, nd * NC));
    TRY(dalloc_t(p, &p->adj_cpart, 8 * NC));
    TRY(dalloc_t(p, &p->adj_S, (size_t)(p->W + 1) * NC * K));
    TRY(dalloc_t(p, &p->adj_u00, NC));
    TRY(dalloc_t(p, &p->adj_a, G * V));
    TRY(dalloc_t(p, &p->adj_gt, V));
    TRY(dalloc_t(p, &p->adj_gs, V));
    TRY(dalloc_t(p, &p->adj_gsig, G * V));
    TRY(dalloc_t(p, &p->adj_dphiu, G * V));
    TRY(dalloc_t(p, &p->adj_blk, (size_t)p->nblk * 4));
    TRY(dalloc_t(p, &p->adj_status, 4));
    TRY(dalloc_t(p, &p->adj_leak, 1));
    TRY(dalloc_t(p, &p->adj_active, 1));
    TRY(dalloc_t(p, &p->adj_ctl, 4));
    const int one = 1;
    CK(cudaMemcpy(p->adj_active, &one, sizeof(int), cudaMemcpyHostToDevice));
    for (int mode = 1; mode <= 2; ++mode) {
        AdjFn f = adj_sweep_fn(p->ndo, p->K, mode);
        if (!f) return fail(p, DTS_ERR_INTERNAL, "no adjoint sweep kernel for this (S_N, P_L)");
        CK(cudaFuncSetAttribute((const void*)f, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)adj_smem(p)));
    }
    p->adj_ready = true;
    return DTS_OK;
}

dts_status run_adjoint(dts_problem* p, int b)
{
    const int G = p->G, W1 = p->W + 1;
    const size_t NC = p->NC, K = p->K, V = p->V;
    const dim3 cgrid((p->NC + 255) / 256);
    CK(cudaMemsetAsync(p->adj_gt, 0, sizeof(double) * V, p->stream));
    CK(cudaMemsetAsync(p->adj_gs, 0, sizeof(double) * V, p->stream));
    CK(cudaMemsetAsync(p->adj_dphiu, 0, sizeof(double) * G * V, p->stream));
    CK(cudaMemsetAsync(p->adj_leak, 0, sizeof(double), p->stream));

    AdjCellParams ac;
    ac.c = cell_params(p);
    ac.c.B = 1;
    ac.b = b; ac.V = p->V; ac.src = p->src; ac.unc = p->unc; ac.mom = p->mom; ac.q = p->q;
    ac.a = p->adj_a; ac.S = p->adj_S; ac.Sstride = NC * K; ac.W = p->W;
    AdjGradParams gp;
    gp.a = ac; gp.part = p->adj_part; gp.cpart = p->adj_cpart; gp.gt = p->adj_gt; gp.gs = p->adj_gs;
    gp.gsig = p->adj_gsig; gp.dphiu = p->adj_dphiu;

    AdjSweepParams sp;
    SweepParams<double>& q = sp.s;
    q.nx = p->d.nx; q.ny = p->d.ny; q.nz = p->d.nz;
    q.TX = p->TX; q.TY = p->TY; q.TZ = p->TZ; q.TV = p->TV;
    q.NTx = p->NTx; q.NTy = p->NTy; q.NTz = p->NTz; q.NT = p->NT;
    q.B = 1; q.nsub = p->nsub;
    q.stage_tiles = p->stage_tiles; q.stage_off = p->stage_off;
    q.diag_cells = p->diag_cells; q.diag_off = p->diag_off;
    q.A = (const double*)p->At; q.Lw = p->Lw;
    q.T = p->adj_T; q.sigt = (const double*)p->sigt_r; q.part = p->adj_part;
    q.xf = p->adj_xf; q.yf = p->adj_yf; q.zf = p->adj_zf;
    q.active = p->adj_active; q.leak = p->adj_leak;
    sp.rec_psi = p->adj_psi; sp.rec_mask = p->adj_mask; sp.cpart = p->adj_cpart; sp.NC = p->NC;
    const size_t smem = adj_smem(p);
    AdjFn rec = adj_sweep_fn(p->ndo, p->K, 1), adj = adj_sweep_fn(p->ndo, p->K, 2);

    RedParams<double> rp;
    rp.B = 1; rp.NT = p->NT; rp.TV = p->TV; rp.NC = p->NC;
    rp.part = p->adj_part; rp.phi00 = p->adj_u00; rp.T = p->adj_T; rp.F = p->adj_S;
    rp.Fstride = NC * K; rp.ctl = p->adj_ctl; rp.sigs = (const double*)p->sigs; rp.sigs0 = p->sigs0;
    rp.sigt64 = p->sigt64; rp.sigt = (const double*)p->sigt_r; rp.mat_t = p->mat_t; rp.active = p->adj_active;
    rp.vol = p->d.dx * p->d.dy * p->d.dz; rp.blk = p->adj_blk;
    RedFn<double> rf = reduce_fn<double>(p->K);

    p->adj_iters.assign(G, 0);
    for (int g = G - 1; g >= std::max(0, G - W1); --g)
        k_adj_source_init<<<cgrid, 256, 0, p->stream>>>(ac, g, g % W1);
    for (int g = G - 1; g >= 0; --g) {
        const int slot = g % W1;
        k_set_ctl<<<1, 1, 0, p->stream>>>(p->adj_ctl, g, slot);
        launch_group_xs<double>(p, g);
        k_adj_source_T<<<cgrid, 256, 0, p->stream>>>(ac, g, p->adj_T);
        // forward sweep of the converged source, recording psi and fixup sets
        q.M = (const double*)p->Mt;
        q.Dt = (const double*)p->Dt;
        for (int s = 0; s < p->n_stages; ++s) {
            const int cnt = p->stage_off_h[s + 1] - p->stage_off_h[s];
            rec<<<(unsigned)cnt * 8u, kSweepThreads, smem, p->stream>>>(sp, s);
        }
        // adjoint source iteration: the transposed sweep swaps the roles of D and M
        q.M = (const double*)p->Dt;
        q.Dt = (const double*)p->Mt;
        CK(cudaMemsetAsync(p->adj_u00, 0, sizeof(double) * NC, p->stream));
        k_group_init<double><<<(unsigned)((NC * K + 255) / 256), 256, 0, p->stream>>>(
            NC * K, p->adj_S + (size_t)slot * NC * K, p->adj_T);
        CK(cudaGetLastError());
        for (int it = 1; it <= p->d.max_iters; ++it) {
            for (int s = 0; s < p->n_stages; ++s) {
                const int cnt = p->stage_off_h[s + 1] - p->stage_off_h[s];
                adj<<<(unsigned)cnt * 8u, kSweepThreads, smem, p->stream>>>(sp, s);
            }
            rf<<<dim3(p->nblk, 1), kRedThreads, 0, p->stream>>>(rp);
            k_resid_final<<<1, 256, 0, p->stream>>>(p->adj_blk, p->nblk, p->adj_leak, 1, p->adj_status,
                                                    count_of<double>(p, p->adj_blk),
                                                    count_of<double>(p, p->adj_leak),
                                                    count_of<double>(p, p->adj_status));
            CK(cudaMemcpyAsync(p->h_status, p->adj_status, sizeof(double) * 4, cudaMemcpyDeviceToHost,
                               p->stream));
            CK(cudaStreamSynchronize(p->stream));
            p->adj_iters[g] = it;
            if (p->d.tol > 0.0 && p->h_status[0] < p->d.tol) break;
        }
        k_adj_grad<<<cgrid, 256, 0, p->stream>>>(gp, g);
        if (g - W1 >= 0) k_adj_source_init<<<cgrid, 256, 0, p->stream>>>(ac, g - W1, slot);
        CK(cudaGetLastError());
    }
    RayParams rp2;
    rp2.nx = p->d.nx; rp2.ny = p->d.ny; rp2.nz = p->d.nz; rp2.V = p->V; rp2.G = G;
    rp2.dx = p->d.dx; rp2.dy = p->d.dy; rp2.dz = p->d.dz;
    rp2.x0 = p->d.x0; rp2.y0 = p->d.y0; rp2.z0 = p->d.z0;
    rp2.mat = p->mat_nat; rp2.scale_t = p->scale_t_nat; rp2.sigma_t = p->sigma_t;
    rp2.src = p->src; rp2.spec = p->spec; rp2.unc = p->unc; rp2.n_mat = p->n_mat; rp2.fan = p->fan;
    k_adj_ray<<<(unsigned)((V + 127) / 128), 128, 0, p->stream>>>(rp2, p->adj_a, p->adj_dphiu, b, p->adj_gt);
    CK(cudaGetLastError());
    return DTS_OK;
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
// the beam of a kind-1 source: the cone half-angle, or a fan (aperture 1) with
// its plane normal and half angles; writes the 8-double aperture row
dts_status beam_row(dts_problem* p, const dts_source* s, double* row)
{
    for (int i = 0; i < 8; ++i) row[i] = 0.0;
    if (s->aperture == 0) return DTS_OK;
    if (s->aperture != 1) return fail(p, DTS_ERR_INVALID_ARG, "aperture must be 0 (cone) or 1 (fan)");
    const double an = std::sqrt(s->axis[0] * s->axis[0] + s->axis[1] * s->axis[1] + s->axis[2] * s->axis[2]);
    const double nn = std::sqrt(s->normal[0] * s->normal[0] + s->normal[1] * s->normal[1] +
                                s->normal[2] * s->normal[2]);
    if (!(nn > 0.0) || !isfin(nn)) return fail(p, DTS_ERR_INVALID_ARG, "fan normal must be non-zero and finite");
    const double c = (s->normal[0] * s->axis[0] + s->normal[1] * s->axis[1] + s->normal[2] * s->axis[2]) / (an * nn);
    if (!(std::fabs(c) < 1.0 - 1e-9)) return fail(p, DTS_ERR_INVALID_ARG, "fan normal parallel to the axis");
    if (!(s->half_azimuth > 0.0) || !(s->half_azimuth <= kPi + 1e-12))
        return fail(p, DTS_ERR_INVALID_ARG, "half_azimuth must be in (0, pi]");
    if (!(s->half_polar > 0.0) || !(s->half_polar <= 0.5 * kPi + 1e-12))
        return fail(p, DTS_ERR_INVALID_ARG, "half_polar must be in (0, pi/2]");
    row[0] = 1.0;
    for (int i = 0; i < 3; ++i) row[1 + i] = s->normal[i];
    row[4] = s->half_azimuth;
    row[5] = s->half_polar;
    return DTS_OK;
}

extern "C" {

dts_status dts_create_problem(const dts_problem_desc* desc, dts_problem** out)
{
    if (!out) return fail(nullptr, DTS_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!desc) return fail(nullptr, DTS_ERR_INVALID_ARG, "desc is NULL");
    dts_problem* p = new (std::nothrow) dts_problem();
    if (!p) return fail(nullptr, DTS_ERR_OOM, "host allocation failed");
    dts_status s = create(desc, p);
    if (s != DTS_OK) {
        g_thread_error = p->err;
        destroy(p);
        delete p;
        return s;
    }
    *out = p;
    return DTS_OK;
}

dts_status dts_set_materials(dts_problem* p, int n_mat, const double* sigma_t, const double* sigma_s,
                             const int32_t* mat_id, const double* scale_t, const double* scale_s)
{
    if (!p) return fail(nullptr, DTS_ERR_INVALID_ARG, "problem is NULL");
    if (n_mat < 1 || !sigma_t || !sigma_s || !mat_id)
        return fail(p, DTS_ERR_INVALID_ARG, "n_mat >= 1 and non-NULL sigma_t, sigma_s, mat_id required");
    const int G = p->G, L = p->L, V = p->V;
    for (size_t i = 0; i < (size_t)n_mat * G; ++i)
        if (!(sigma_t[i] > 0.0) || !isfin(sigma_t[i]))
            return fail(p, DTS_ERR_INVALID_ARG, "sigma_t must be finite and > 0");
    int W = 0;
    for (int m = 0; m < n_mat; ++m)
        for (int l = 0; l <= L; ++l)
            for (int gf = 0; gf < G; ++gf)
                for (int gt = 0; gt < G; ++gt) {
                    const double s = sigma_s[(((size_t)m * (L + 1) + l) * G + gf) * G + gt];
                    if (!isfin(s)) return fail(p, DTS_ERR_INVALID_ARG, "sigma_s must be finite");
                    if (l == 0 && s < 0.0) return fail(p, DTS_ERR_INVALID_ARG, "sigma_s0 must be >= 0");
                    if (s != 0.0 && gt < gf)
                        return fail(p, DTS_ERR_INVALID_ARG, "sigma_s must be downscatter only (g_to >= g_from)");
                    if (s != 0.0) W = std::max(W, gt - gf);
                }
    for (int v = 0; v < V; ++v)
        if (mat_id[v] < 0 || mat_id[v] >= n_mat) return fail(p, DTS_ERR_INVALID_ARG, "mat_id out of range");
    for (const double* sc : {scale_t, scale_s})
        if (sc)
            for (int v = 0; v < V; ++v)
                if (!(sc[v] > 0.0) || !isfin(sc[v]))
                    return fail(p, DTS_ERR_INVALID_ARG, "scale factors must be finite and > 0");
    DevGuard guard(p->d.device);
    CK(cudaStreamSynchronize(p->stream));
    if (n_mat != p->n_mat) {
        dfree(p, p->sigma_t);
        dfree(p, p->sigma_s);
        dfree(p, p->sigma_s_f);
        p->sigma_t = p->sigma_s = nullptr;
        p->sigma_s_f = nullptr;
        TRY(dalloc_t(p, &p->sigma_t, (size_t)n_mat * G));
        TRY(dalloc_t(p, &p->sigma_s, (size_t)n_mat * (L + 1) * G * G));
        TRY(dalloc_t(p, &p->sigma_s_f, (size_t)n_mat * (L + 1) * G * G));
        p->n_mat = n_mat;
    }
    CK(cudaMemcpy(p->sigma_t, sigma_t, sizeof(double) * n_mat * G, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(p->sigma_s, sigma_s, sizeof(double) * (size_t)n_mat * (L + 1) * G * G, cudaMemcpyHostToDevice));
    {
        std::vector<float> sf((size_t)n_mat * (L + 1) * G * G);
        for (size_t i = 0; i < sf.size(); ++i) sf[i] = (float)sigma_s[i];
        CK(cudaMemcpy(p->sigma_s_f, sf.data(), sizeof(float) * sf.size(), cudaMemcpyHostToDevice));
    }
    std::vector<int32_t> mt = to_tiled<int32_t>(p, mat_id, -1);
    CK(cudaMemcpy(p->mat_t, mt.data(), sizeof(int32_t) * p->NC, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(p->mat_nat, mat_id, sizeof(int32_t) * V, cudaMemcpyHostToDevice));
    struct { const double* h; double** t; double** n; } sc[2] = {
        {scale_t, &p->scale_t_t, &p->scale_t_nat}, {scale_s, &p->scale_s_t, nullptr}};
    for (auto& e : sc) {
        dfree(p, *e.t);
        *e.t = nullptr;
        if (e.n) {
            dfree(p, *e.n);
            *e.n = nullptr;
        }
        if (!e.h) continue;
        std::vector<double> tt = to_tiled<double>(p, e.h, 1.0);
        TRY(dalloc_t(p, e.t, p->NC));
        CK(cudaMemcpy(*e.t, tt.data(), sizeof(double) * p->NC, cudaMemcpyHostToDevice));
        if (e.n) {
            TRY(dalloc_t(p, e.n, V));
            CK(cudaMemcpy(*e.n, e.h, sizeof(double) * V, cudaMemcpyHostToDevice));
        }
    }
    p->W = std::min(W, G - 1);
    p->materials_set = true;
    p->solved = false;
    return DTS_OK;
}

dts_status dts_set_source(dts_problem* p, int batch_index, const dts_source* s)
{
    if (!p) return fail(nullptr, DTS_ERR_INVALID_ARG, "problem is NULL");
    if (!s) return fail(p, DTS_ERR_INVALID_ARG, "source is NULL");
    if (batch_index < 0 || batch_index >= p->B) return fail(p, DTS_ERR_INVALID_ARG, "batch_index out of range");
    const int G = p->G, V = p->V;
    DevGuard guard(p->d.device);
    double* row = &p->src_h[(size_t)batch_index * 8];
    if (p->cone_n_h[batch_index] != 0) {   // the member stops being a combined source
        p->cone_n_h[batch_index] = 0;
        CK(cudaMemcpy(p->cone_n + batch_index, &p->cone_n_h[batch_index], sizeof(int), cudaMemcpyHostToDevice));
    }
    if (s->kind == 0) {
        if (!s->q) return fail(p, DTS_ERR_INVALID_ARG, "kind 0 needs q");
        for (size_t i = 0; i < (size_t)G * V; ++i)
            if (!isfin(s->q[i])) return fail(p, DTS_ERR_INVALID_ARG, "q must be finite");
        if (!p->q) {
            TRY(dalloc_t(p, &p->q, (size_t)p->B * G * V));
            CK(cudaMemset(p->q, 0, sizeof(double) * (size_t)p->B * G * V));
        }
        CK(cudaMemcpy(p->q + (size_t)batch_index * G * V, s->q, sizeof(double) * G * V, cudaMemcpyHostToDevice));
        for (int i = 0; i < 8; ++i) row[i] = 0.0;
        for (int g = 0; g < G; ++g) p->spec_h[(size_t)batch_index * G + g] = 0.0;
    } else if (s->kind == 1) {
        if (!s->spectrum) return fail(p, DTS_ERR_INVALID_ARG, "kind 1 needs a spectrum");
        const double an = std::sqrt(s->axis[0] * s->axis[0] + s->axis[1] * s->axis[1] + s->axis[2] * s->axis[2]);
        if (!(an > 0.0) || !isfin(an)) return fail(p, DTS_ERR_INVALID_ARG, "cone axis must be non-zero");
        if (!(s->half_angle > 0.0) || !(s->half_angle <= kPi + 1e-12))
            return fail(p, DTS_ERR_INVALID_ARG, "half_angle must be in (0, pi]");
        for (int i = 0; i < 3; ++i)
            if (!isfin(s->pos[i])) return fail(p, DTS_ERR_INVALID_ARG, "source position must be finite");
        for (int g = 0; g < G; ++g) {
            if (!isfin(s->spectrum[g]) || s->spectrum[g] < 0.0)
                return fail(p, DTS_ERR_INVALID_ARG, "spectrum must be finite and >= 0");
            p->spec_h[(size_t)batch_index * G + g] = s->spectrum[g];
        }
        row[0] = 1.0;
        for (int i = 0; i < 3; ++i) {
            row[1 + i] = s->pos[i];
            row[4 + i] = s->axis[i];
        }
        row[7] = s->half_angle >= kPi ? kPi : s->half_angle;
    } else {
        return fail(p, DTS_ERR_INVALID_ARG, "source kind must be 0 or 1");
    }
    {
        double* frow = &p->fan_h[(size_t)batch_index * 8];
        if (s->kind == 1) TRY(beam_row(p, s, frow));
        else for (int i = 0; i < 8; ++i) frow[i] = 0.0;
        CK(cudaMemcpy(p->fan + (size_t)batch_index * 8, frow, sizeof(double) * 8, cudaMemcpyHostToDevice));
    }
    CK(cudaMemcpy(p->src + (size_t)batch_index * 8, row, sizeof(double) * 8, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(p->spec + (size_t)batch_index * G, &p->spec_h[(size_t)batch_index * G],
                  sizeof(double) * G, cudaMemcpyHostToDevice));
    p->src_set[batch_index] = 1;
    p->solved = false;
    return DTS_OK;
}

dts_status dts_set_source_cones(dts_problem* p, int batch_index, int n_cones, const dts_source* cones)
{
    if (!p) return fail(nullptr, DTS_ERR_INVALID_ARG, "problem is NULL");
    if (!cones) return fail(p, DTS_ERR_INVALID_ARG, "cones is NULL");
    if (batch_index < 0 || batch_index >= p->B) return fail(p, DTS_ERR_INVALID_ARG, "batch_index out of range");
    if (n_cones < 1 || n_cones > 4096) return fail(p, DTS_ERR_INVALID_ARG, "n_cones must be in 1..4096");
    const int G = p->G, B = p->B;
    std::vector<double> geo((size_t)n_cones * 16, 0.0), spec((size_t)n_cones * G);
    for (int c = 0; c < n_cones; ++c) {
        const dts_source* s = cones + c;
        if (s->kind != 1) return fail(p, DTS_ERR_INVALID_ARG, "every cone must be a kind-1 source");
        if (!s->spectrum) return fail(p, DTS_ERR_INVALID_ARG, "every cone needs a spectrum");
        const double an = std::sqrt(s->axis[0] * s->axis[0] + s->axis[1] * s->axis[1] + s->axis[2] * s->axis[2]);
        if (!(an > 0.0) || !isfin(an)) return fail(p, DTS_ERR_INVALID_ARG, "cone axis must be non-zero");
        if (!(s->half_angle > 0.0) || !(s->half_angle <= kPi + 1e-12))
            return fail(p, DTS_ERR_INVALID_ARG, "half_angle must be in (0, pi]");
        for (int i = 0; i < 3; ++i) {
            if (!isfin(s->pos[i])) return fail(p, DTS_ERR_INVALID_ARG, "source position must be finite");
            geo[(size_t)c * 16 + i] = s->pos[i];
            geo[(size_t)c * 16 + 3 + i] = s->axis[i];
        }
        geo[(size_t)c * 16 + 6] = s->half_angle >= kPi ? kPi : s->half_angle;
        TRY(beam_row(p, s, &geo[(size_t)c * 16 + 7]));   // aperture, normal, half azimuth, half polar
        for (int g = 0; g < G; ++g) {
            if (!isfin(s->spectrum[g]) || s->spectrum[g] < 0.0)
                return fail(p, DTS_ERR_INVALID_ARG, "spectrum must be finite and >= 0");
            spec[(size_t)c * G + g] = s->spectrum[g];
        }
    }
    DevGuard guard(p->d.device);
    CK(cudaStreamSynchronize(p->stream));
    p->cone_geo_h[batch_index] = geo;
    p->cone_spec_h[batch_index] = spec;
    p->cone_n_h[batch_index] = n_cones;
    if (n_cones > p->cone_cap) {   // wider tables: re-upload every member's cones
        dfree(p, p->cone_geo);
        dfree(p, p->cone_spec);
        p->cone_geo = p->cone_spec = nullptr;
        p->cone_cap = n_cones;
        TRY(dalloc_t(p, &p->cone_geo, (size_t)B * p->cone_cap * 16));
        TRY(dalloc_t(p, &p->cone_spec, (size_t)B * p->cone_cap * G));
        for (int b = 0; b < B; ++b) {
            const int n = (int)p->cone_geo_h[b].size() / 16;
            if (n == 0) continue;
            CK(cudaMemcpy(p->cone_geo + (size_t)b * p->cone_cap * 16, p->cone_geo_h[b].data(),
                          sizeof(double) * n * 16, cudaMemcpyHostToDevice));
            CK(cudaMemcpy(p->cone_spec + (size_t)b * p->cone_cap * G, p->cone_spec_h[b].data(),
                          sizeof(double) * (size_t)n * G, cudaMemcpyHostToDevice));
        }
    } else {
        CK(cudaMemcpy(p->cone_geo + (size_t)batch_index * p->cone_cap * 16, geo.data(), sizeof(double) * geo.size(),
                      cudaMemcpyHostToDevice));
        CK(cudaMemcpy(p->cone_spec + (size_t)batch_index * p->cone_cap * G, spec.data(),
                      sizeof(double) * spec.size(), cudaMemcpyHostToDevice));
    }
    if (p->uslot_h[batch_index] < 0) {   // a row of U for this member (recomputed by every solve)
        p->uslot_h[batch_index] = p->n_uslots++;
        dfree(p, p->U);
        p->U = nullptr;
        TRY(dalloc_t(p, &p->U, (size_t)p->n_uslots * G * p->K * p->V));
        CK(cudaMemcpy(p->uslot, p->uslot_h.data(), sizeof(int) * B, cudaMemcpyHostToDevice));
    }
    CK(cudaMemcpy(p->cone_n + batch_index, &p->cone_n_h[batch_index], sizeof(int), cudaMemcpyHostToDevice));
    double* row = &p->src_h[(size_t)batch_index * 8];
    for (int i = 0; i < 8; ++i) row[i] = 0.0;
    row[0] = 2.0;
    for (int g = 0; g < G; ++g) p->spec_h[(size_t)batch_index * G + g] = 0.0;
    CK(cudaMemcpy(p->src + (size_t)batch_index * 8, row, sizeof(double) * 8, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(p->spec + (size_t)batch_index * G, &p->spec_h[(size_t)batch_index * G], sizeof(double) * G,
                  cudaMemcpyHostToDevice));
    p->src_set[batch_index] = 1;
    p->solved = false;
    return DTS_OK;
}

dts_status dts_solve(dts_problem* p, dts_solve_stats* stats)
{
    if (!p) return fail(nullptr, DTS_ERR_INVALID_ARG, "problem is NULL");
    if (!p->materials_set) return fail(p, DTS_ERR_STATE, "dts_set_materials has not been called");
    for (int b = 0; b < p->B; ++b)
        if (!p->src_set[b]) return fail(p, DTS_ERR_STATE, "a batch member has no source");
    DevGuard guard(p->d.device);
    return run_solve(p, stats);
}

// Several problems (disjoint source sets, each on its own stream) solved together.
// Each problem's next source iteration is enqueued as soon as its last one is
// complete (the host polls the problems' events), so the problems' sweeps and
// moment graphs overlap on the GPU as they fall.
dts_status dts_solve_many(dts_problem* const* problems, int n, dts_solve_stats* stats)
{
    // every failure's message also goes to the thread's error (dts_last_error(NULL))
    auto bad = [](dts_problem* p, dts_status s, const char* msg) {
        fail(p, s, msg);
        g_thread_error = msg;
        return s;
    };
    if (!problems || n < 1) return bad(nullptr, DTS_ERR_INVALID_ARG, "problems is NULL or n < 1");
    for (int i = 0; i < n; ++i) {
        dts_problem* p = problems[i];
        if (!p) return bad(nullptr, DTS_ERR_INVALID_ARG, "a problem is NULL");
        for (int j = 0; j < i; ++j)
            if (problems[j] == p) return bad(p, DTS_ERR_INVALID_ARG, "a problem appears twice");
        if (p->d.device != problems[0]->d.device)
            return bad(p, DTS_ERR_INVALID_ARG, "the problems are on different devices");
        if (!p->materials_set) return bad(p, DTS_ERR_STATE, "dts_set_materials has not been called");
        for (int b = 0; b < p->B; ++b)
            if (!p->src_set[b]) return bad(p, DTS_ERR_STATE, "a batch member has no source");
    }
    DevGuard guard(problems[0]->d.device);
    std::vector<std::unique_ptr<SolveRun>> runs;
    for (int i = 0; i < n; ++i) runs.emplace_back(new SolveRun(problems[i]));
    std::vector<char> in_flight(n, 0), finished(n, 0);
    dts_status first_soft = DTS_OK;   // DTS_ERR_NOT_CONVERGED of some problem: the others still finish
    // a hard error of problem i: stop scheduling, let every stream drain, return the error
    auto abort_all = [&](int i, dts_status s) {
        for (int j = 0; j < n; ++j) cudaStreamSynchronize(problems[j]->stream);
        g_thread_error = problems[i]->err;
        return s;
    };
    for (int i = 0; i < n; ++i) {
        const dts_status s = runs[i]->start();
        if (s != DTS_OK) return abort_all(i, s);
    }
    // problems with the device-resident loop: every group enqueued on their streams now; they run
    // beside the others with no host step until they finish
    int remaining = n;
    for (int i = 0; i < n; ++i) {
        SolveRun& r = *runs[i];
        if (!r.dev) continue;
        dts_status s = DTS_OK;
        while (s == DTS_OK && !r.done) {
            s = r.launch_group_loop();
            if (s == DTS_OK) s = r.end_group();
        }
        if (s != DTS_OK) return abort_all(i, s);
        finished[i] = 1;
        --remaining;
    }
    while (remaining > 0) {
        bool progressed = false;
        for (int i = 0; i < n; ++i) {
            if (finished[i]) continue;
            SolveRun& r = *runs[i];
            dts_status s = DTS_OK;
            if (in_flight[i]) {
                const cudaError_t q = cudaEventQuery(r.p->evc);
                if (q == cudaErrorNotReady) continue;
                in_flight[i] = 0;
                s = r.complete_iteration();   // a failed query surfaces here
            }
            progressed = true;
            while (s == DTS_OK && !r.done && !r.group_iterating()) s = r.end_group();
            if (s == DTS_OK && r.done) {
                finished[i] = 1;
                --remaining;
                s = r.finish(stats ? &stats[i] : nullptr);
                if (s == DTS_ERR_NOT_CONVERGED) {
                    if (first_soft == DTS_OK) {
                        first_soft = s;
                        g_thread_error = r.p->err;
                    }
                    continue;
                }
            } else if (s == DTS_OK) {
                s = r.launch_iteration();
                in_flight[i] = 1;
            }
            if (s != DTS_OK) return abort_all(i, s);
        }
        if (!progressed) std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
    for (int i = 0; i < n; ++i) {
        if (!runs[i]->dev) continue;
        const dts_status s = runs[i]->finish(stats ? &stats[i] : nullptr);
        if (s == DTS_ERR_NOT_CONVERGED) {
            if (first_soft == DTS_OK) {
                first_soft = s;
                g_thread_error = problems[i]->err;
            }
        } else if (s != DTS_OK) {
            return abort_all(i, s);
        }
    }
    return first_soft;
}

dts_status dts_get_scalar_fluence(dts_problem* p, int batch_index, dts_component comp, double* out,
                                  size_t out_len, int out_is_device)
{
    if (!p) return fail(nullptr, DTS_ERR_INVALID_ARG, "problem is NULL");
    if (!p->solved) return fail(p, DTS_ERR_STATE, "no solve has completed");
    if (batch_index < 0 || batch_index >= p->B) return fail(p, DTS_ERR_INVALID_ARG, "batch_index out of range");
    if (!out) return fail(p, DTS_ERR_INVALID_ARG, "out is NULL");
    const size_t n = (size_t)p->G * p->V;
    if (out_len < n) return fail(p, DTS_ERR_INVALID_ARG, "out_len < G*V");
    DevGuard guard(p->d.device);
    const double* u = p->unc + (size_t)batch_index * n;
    const double* c = p->col + (size_t)batch_index * n;
    const double* srcp;
    if (comp == DTS_COMP_UNCOLLIDED) srcp = u;
    else if (comp == DTS_COMP_COLLIDED) srcp = c;
    else if (comp == DTS_COMP_TOTAL) {
        k_add<<<(unsigned)((n + 255) / 256), 256, 0, p->stream>>>(n, u, c, p->tmp);
        CK(cudaGetLastError());
        srcp = p->tmp;
    } else return fail(p, DTS_ERR_INVALID_ARG, "unknown component");
    if (out_is_device) {
        CK(cudaMemcpyAsync(out, srcp, sizeof(double) * n, cudaMemcpyDeviceToDevice, p->stream));
    } else {
        CK(cudaMemcpyAsync(out, srcp, sizeof(double) * n, cudaMemcpyDeviceToHost, p->stream));
        CK(cudaStreamSynchronize(p->stream));
    }
    return DTS_OK;
}

dts_status dts_get_dose(dts_problem* p, int batch_index, dts_component comp, const double* mu_en_rho,
                        const double* energy_mev, double* out, size_t out_len, int out_is_device)
{
    if (!p) return fail(nullptr, DTS_ERR_INVALID_ARG, "problem is NULL");
    if (!p->solved) return fail(p, DTS_ERR_STATE, "no solve has completed");
    if (batch_index < 0 || batch_index >= p->B) return fail(p, DTS_ERR_INVALID_ARG, "batch_index out of range");
    if (!mu_en_rho || !energy_mev || !out) return fail(p, DTS_ERR_INVALID_ARG, "NULL pointer");
    if (comp != DTS_COMP_UNCOLLIDED && comp != DTS_COMP_COLLIDED && comp != DTS_COMP_TOTAL)
        return fail(p, DTS_ERR_INVALID_ARG, "unknown component");
    if (out_len < (size_t)p->V) return fail(p, DTS_ERR_INVALID_ARG, "out_len < V");
    const int G = p->G, V = p->V;
    for (size_t i = 0; i < (size_t)p->n_mat * G; ++i)
        if (!isfin(mu_en_rho[i]) || mu_en_rho[i] < 0.0)
            return fail(p, DTS_ERR_INVALID_ARG, "mu_en_rho must be finite and >= 0");
    for (int g = 0; g < G; ++g)
        if (!isfin(energy_mev[g]) || energy_mev[g] < 0.0)
            return fail(p, DTS_ERR_INVALID_ARG, "energy_mev must be finite and >= 0");
    DevGuard guard(p->d.device);
    double* tab = nullptr;   // [n_mat][G] coefficients, then [G] energies
    CK(cudaMallocAsync((void**)&tab, sizeof(double) * ((size_t)p->n_mat * G + G + (out_is_device ? 0 : V)),
                       p->stream));
    double* dout = out_is_device ? out : tab + (size_t)p->n_mat * G + G;
    CK(cudaMemcpyAsync(tab, mu_en_rho, sizeof(double) * (size_t)p->n_mat * G, cudaMemcpyHostToDevice, p->stream));
    CK(cudaMemcpyAsync(tab + (size_t)p->n_mat * G, energy_mev, sizeof(double) * G, cudaMemcpyHostToDevice,
                       p->stream));
    const size_t n = (size_t)G * V;
    k_dose<<<(unsigned)((V + 255) / 256), 256, 0, p->stream>>>(
        V, G, p->unc + (size_t)batch_index * n, p->col + (size_t)batch_index * n,
        comp == DTS_COMP_UNCOLLIDED ? 0 : comp == DTS_COMP_COLLIDED ? 1 : 2, p->mat_nat, tab,
        tab + (size_t)p->n_mat * G, 1.602176634e-10, dout);
    CK(cudaGetLastError());
    if (!out_is_device)
        CK(cudaMemcpyAsync(out, dout, sizeof(double) * V, cudaMemcpyDeviceToHost, p->stream));
    CK(cudaFreeAsync(tab, p->stream));
    CK(cudaStreamSynchronize(p->stream));
    return DTS_OK;
}

dts_status dts_get_moments(dts_problem* p, int batch_index, int group, double* out, size_t out_len,
                           int out_is_device)
{
    if (!p) return fail(nullptr, DTS_ERR_INVALID_ARG, "problem is NULL");
    if (!p->d.keep_moments) return fail(p, DTS_ERR_STATE, "problem was created without keep_moments");
    if (!p->solved) return fail(p, DTS_ERR_STATE, "no solve has completed");
    if (batch_index < 0 || batch_index >= p->B || group < 0 || group >= p->G)
        return fail(p, DTS_ERR_INVALID_ARG, "batch_index or group out of range");
    const size_t n = (size_t)p->K * p->V;
    if (!out || out_len < n) return fail(p, DTS_ERR_INVALID_ARG, "out is NULL or out_len < K*V");
    DevGuard guard(p->d.device);
    const double* s = p->mom + ((size_t)batch_index * p->G + group) * n;
    CK(cudaMemcpyAsync(out, s, sizeof(double) * n,
                       out_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, p->stream));
    if (!out_is_device) CK(cudaStreamSynchronize(p->stream));
    return DTS_OK;
}

dts_status dts_get_iterations(dts_problem* p, int32_t* out, size_t out_len)
{
    if (!p) return fail(nullptr, DTS_ERR_INVALID_ARG, "problem is NULL");
    if (!out || out_len < p->iters.size()) return fail(p, DTS_ERR_INVALID_ARG, "out too small");
    std::copy(p->iters.begin(), p->iters.end(), out);
    return DTS_OK;
}

dts_status dts_get_residuals(dts_problem* p, double* out, size_t out_len)
{
    if (!p) return fail(nullptr, DTS_ERR_INVALID_ARG, "problem is NULL");
    if (!out || out_len < p->resid.size()) return fail(p, DTS_ERR_INVALID_ARG, "out too small");
    std::copy(p->resid.begin(), p->resid.end(), out);
    return DTS_OK;
}

dts_status dts_get_balance(dts_problem* p, double* out, size_t out_len)
{
    if (!p) return fail(nullptr, DTS_ERR_INVALID_ARG, "problem is NULL");
    if (!out || out_len < p->balance.size()) return fail(p, DTS_ERR_INVALID_ARG, "out too small");
    std::copy(p->balance.begin(), p->balance.end(), out);
    return DTS_OK;
}

dts_status dts_solve_adjoint(dts_problem* p, int batch_index, const double* dL_dphi, double* dL_dscale_t,
                             double* dL_dscale_s, double* dL_dsigma_t, int ptrs_are_device)
{
    if (!p) return fail(nullptr, DTS_ERR_INVALID_ARG, "problem is NULL");
    if (!p->fp64) return fail(p, DTS_ERR_STATE, "the adjoint needs a DTS_PREC_FP64 problem");
    if (!p->d.keep_moments) return fail(p, DTS_ERR_STATE, "the adjoint needs keep_moments = 1");
    if (!p->solved) return fail(p, DTS_ERR_STATE, "no forward solve has completed");
    if (batch_index < 0 || batch_index >= p->B) return fail(p, DTS_ERR_INVALID_ARG, "batch_index out of range");
    if (!dL_dphi || !dL_dscale_t || !dL_dscale_s) return fail(p, DTS_ERR_INVALID_ARG, "NULL pointer");
    if (p->cone_n_h[batch_index] > 0)
        return fail(p, DTS_ERR_STATE, "the adjoint covers volumetric and single-cone sources");
    DevGuard guard(p->d.device);
    TRY(adj_alloc(p));
    const size_t GV = (size_t)p->G * p->V, V = p->V;
    const cudaMemcpyKind in = ptrs_are_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    const cudaMemcpyKind out = ptrs_are_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    CK(cudaMemcpyAsync(p->adj_a, dL_dphi, sizeof(double) * GV, in, p->stream));
    TRY(run_adjoint(p, batch_index));
    CK(cudaMemcpyAsync(dL_dscale_t, p->adj_gt, sizeof(double) * V, out, p->stream));
    CK(cudaMemcpyAsync(dL_dscale_s, p->adj_gs, sizeof(double) * V, out, p->stream));
    if (dL_dsigma_t) CK(cudaMemcpyAsync(dL_dsigma_t, p->adj_gsig, sizeof(double) * GV, out, p->stream));
    CK(cudaStreamSynchronize(p->stream));
    return DTS_OK;
}

dts_status dts_get_adjoint_iterations(dts_problem* p, int32_t* out, size_t out_len)
{
    if (!p) return fail(nullptr, DTS_ERR_INVALID_ARG, "problem is NULL");
    if (!out || out_len < (size_t)p->G) return fail(p, DTS_ERR_INVALID_ARG, "out too small");
    if (p->adj_iters.size() != (size_t)p->G) return fail(p, DTS_ERR_STATE, "no adjoint solve has run");
    std::copy(p->adj_iters.begin(), p->adj_iters.end(), out);
    return DTS_OK;
}

const char* dts_last_error(const dts_problem* p) { return p ? p->err.c_str() : g_thread_error.c_str(); }

dts_status dts_debug_bounds_selftest(int plant, int* is_debug_build)
{
#ifdef DTS_DEBUG_BOUNDS
    if (is_debug_build) *is_debug_build = 1;
    take_bounds_word();
    k_bounds_selftest<<<1, 1>>>(plant, 1024);
    if (cudaDeviceSynchronize() != cudaSuccess) return fail(nullptr, DTS_ERR_CUDA, "selftest kernel failed");
    if (const unsigned long long w = take_bounds_word()) return fail(nullptr, DTS_ERR_INTERNAL, bounds_message(w));
    return DTS_OK;
#else
    (void)plant;
    if (is_debug_build) *is_debug_build = 0;
    return DTS_OK;
#endif
}

dts_status dts_set_initial_guess(dts_problem* p, int batch_index, const double* moments, size_t len,
                                 int is_device)
{
    if (!p) return fail(nullptr, DTS_ERR_INVALID_ARG, "problem is NULL");
    if (batch_index < 0 || batch_index >= p->B) return fail(p, DTS_ERR_INVALID_ARG, "batch_index out of range");
    const size_t n = (size_t)p->G * p->K * p->V;
    DevGuard guard(p->d.device);
    if (!moments) {   // clear: zeros are the default start exactly
        if (p->guess)
            CK(cudaMemsetAsync(p->guess + (size_t)batch_index * n, 0, n * sizeof(double), p->stream));
        CK(cudaStreamSynchronize(p->stream));
        return DTS_OK;
    }
    if (len < n) return fail(p, DTS_ERR_INVALID_ARG, "moments: need G*K*V doubles");
    if (!is_device)
        for (size_t i = 0; i < n; ++i)
            if (!isfin(moments[i])) return fail(p, DTS_ERR_INVALID_ARG, "moments: non-finite value");
    // the tensor-core forms' first-T buffer before the guess itself: a guess never exists without it
    if (p->q_mode && !p->guess_T) TRY(dalloc(p, &p->guess_T, (size_t)p->B * p->NC * p->K * sizeof(float)));
    if (!p->guess) {
        TRY(dalloc_t(p, &p->guess, (size_t)p->B * n));
        CK(cudaMemsetAsync(p->guess, 0, (size_t)p->B * n * sizeof(double), p->stream));
    }
    CK(cudaMemcpyAsync(p->guess + (size_t)batch_index * n, moments, n * sizeof(double),
                       is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, p->stream));
    CK(cudaStreamSynchronize(p->stream));
    p->solved = false;
    return DTS_OK;
}

dts_status dts_debug_poison_wait(dts_problem* p, int on)
{
    if (!p) return fail(nullptr, DTS_ERR_INVALID_ARG, "problem is NULL");
    if (on < 0 || on > 2) return fail(p, DTS_ERR_INVALID_ARG, "on must be 0, 1 or 2");
    if (!p->dev_poison) return fail(p, DTS_ERR_STATE, "only the tensor-core forms have device-side waits");
    DevGuard guard(p->d.device);
    const int v = on == 1 ? 1 : 0;
    CK(cudaStreamSynchronize(p->stream));
    CK(cudaMemcpy(p->dev_poison, &v, sizeof v, cudaMemcpyHostToDevice));
    const unsigned tx = on == 2 ? 16u : 0u;
    if (tx != p->poison_sweep_tx) {   // a sweep parameter: the captured graphs are made again
        p->poison_sweep_tx = tx;
        for (cudaGraphExec_t* g : {&p->graph, &p->graph_red, &p->graph_loop})
            if (*g) {
                cudaGraphExecDestroy(*g);
                *g = nullptr;
            }
    }
    return DTS_OK;
}

dts_status dts_set_host_output(dts_problem* p, dts_component comp, double* host, size_t len)
{
    if (!p) return fail(nullptr, DTS_ERR_INVALID_ARG, "problem is NULL");
    DevGuard guard(p->d.device);
    if (p->copy_stream) CK(cudaStreamSynchronize(p->copy_stream));
    if (!host) {
        p->host_out = nullptr;
        return DTS_OK;
    }
    if (comp != DTS_COMP_UNCOLLIDED && comp != DTS_COMP_COLLIDED && comp != DTS_COMP_TOTAL)
        return fail(p, DTS_ERR_INVALID_ARG, "comp must be UNCOLLIDED, COLLIDED or TOTAL");
    if (len < (size_t)p->B * p->G * p->V) return fail(p, DTS_ERR_INVALID_ARG, "host: need B*G*V doubles");
    // each resource on its own, so that a failed call leaves nothing half made for the next one
    for (int i = 0; i < 2; ++i)
        if (!p->out_stage[i]) TRY(dalloc_t(p, &p->out_stage[i], (size_t)p->B * p->V));
    for (int i = 0; i < 2; ++i) {
        if (!p->ev_staged[i]) CK(cudaEventCreateWithFlags(&p->ev_staged[i], cudaEventDisableTiming));
        if (!p->ev_copied[i]) CK(cudaEventCreateWithFlags(&p->ev_copied[i], cudaEventDisableTiming));
    }
    if (!p->copy_stream) CK(cudaStreamCreateWithFlags(&p->copy_stream, cudaStreamNonBlocking));
    p->host_out = host;
    p->host_comp = (int)comp;
    p->copied_pending[0] = p->copied_pending[1] = false;
    return DTS_OK;
}

dts_status dts_set_device_loop(dts_problem* p, int on)
{
    if (!p) return fail(nullptr, DTS_ERR_INVALID_ARG, "problem is NULL");
    if (on && !p->loop_mem) {
        // one allocation: it, last_improve [B], iters [B][G] (ints); best [B], resid [B][G],
        // balance [B][G][3] (doubles, 8-byte aligned)
        const size_t B = (size_t)p->B, BG = B * (size_t)p->G;
        const size_t ints = ((1 + B + BG) * sizeof(int) + 7) & ~size_t(7);
        DevGuard guard(p->d.device);
        TRY(dalloc(p, &p->loop_mem, ints + sizeof(double) * (B + 4 * BG)));
        char* m = static_cast<char*>(p->loop_mem);
        p->loop_it = reinterpret_cast<int*>(m);
        p->loop_last = p->loop_it + 1;
        p->loop_iters = p->loop_last + B;
        p->loop_best = reinterpret_cast<double*>(m + ints);
        p->loop_resid = p->loop_best + B;
        p->loop_bal = p->loop_resid + BG;
    }
    p->device_loop = on != 0;
    return DTS_OK;
}

dts_status dts_set_iteration_callback(dts_problem* p, dts_iteration_fn fn, void* user)
{
    if (!p) return fail(nullptr, DTS_ERR_INVALID_ARG, "problem is NULL");
    p->on_iter = fn;
    p->on_iter_user = user;
    return DTS_OK;
}

void dts_destroy_problem(dts_problem* p)
{
    if (!p) return;
    destroy(p);
    delete p;
}

const char* dts_status_string(dts_status s)
{
    switch (s) {
    case DTS_OK: return "DTS_OK";
    case DTS_ERR_INVALID_ARG: return "DTS_ERR_INVALID_ARG";
    case DTS_ERR_STATE: return "DTS_ERR_STATE";
    case DTS_ERR_OOM: return "DTS_ERR_OOM";
    case DTS_ERR_CUDA: return "DTS_ERR_CUDA";
    case DTS_ERR_NOT_CONVERGED: return "DTS_ERR_NOT_CONVERGED";
    case DTS_ERR_TIMEOUT: return "DTS_ERR_TIMEOUT";
    case DTS_ERR_INTERNAL: return "DTS_ERR_INTERNAL";
    }
    return "unknown status";
}

int dts_version(void) { return 1; }

void dts_debug_fail_allocation(int after) { g_fail_alloc_after.store(after < 0 ? -1 : (long long)after); }

dts_status dts_quadrature(int sn_order, double* mu, double* eta, double* xi, double* w, int* n_dirs)
{
    std::vector<double> a, b, c, d;
    if (!ls_set(sn_order, a, b, c, d)) return fail(nullptr, DTS_ERR_INVALID_ARG, "sn_order must be 2, 4, 6 or 8");
    if (!mu || !eta || !xi || !w) return fail(nullptr, DTS_ERR_INVALID_ARG, "NULL output");
    std::copy(a.begin(), a.end(), mu);
    std::copy(b.begin(), b.end(), eta);
    std::copy(c.begin(), c.end(), xi);
    std::copy(d.begin(), d.end(), w);
    if (n_dirs) *n_dirs = (int)d.size();
    return DTS_OK;
}

dts_status dts_moment_tables(int sn_order, int legendre_order, double* D, double* M)
{
    std::vector<double> a, b, c, w, Dv, Mv;
    if (!ls_set(sn_order, a, b, c, w)) return fail(nullptr, DTS_ERR_INVALID_ARG, "sn_order must be 2, 4, 6 or 8");
    if (legendre_order < 0 || legendre_order > 3)
        return fail(nullptr, DTS_ERR_INVALID_ARG, "legendre_order must be in 0..3");
    if (!D || !M) return fail(nullptr, DTS_ERR_INVALID_ARG, "NULL output");
    moment_tables(legendre_order, a, b, c, w, Dv, Mv);
    std::copy(Dv.begin(), Dv.end(), D);
    std::copy(Mv.begin(), Mv.end(), M);
    return DTS_OK;
}

// The tuner's results, per process and (when a cache file is named) on disk. A file line is
//   dts-tune-v1 <device name, blanks as '_'> <SMs> nx ny nz N L probe_batch precision tx ty tz rate
// keyed by everything but the tile and the rate; lines that do not parse are ignored, and a
// later line for the same key wins. New results are appended.
namespace {
std::mutex g_tune_mu;
std::map<std::vector<long long>, std::tuple<int, int, int, double>> g_tune_mem;
bool g_tune_path_set = false;   // dts_tune_cache_file was called (else DTS_TUNE_CACHE is read)
std::string g_tune_path;

std::string tune_path_locked()
{
    if (g_tune_path_set) return g_tune_path;
    const char* e = std::getenv("DTS_TUNE_CACHE");
    return e ? std::string(e) : std::string();
}

std::string tune_line_key(const std::string& dev, const std::vector<long long>& k)
{
    std::string out = "dts-tune-v1 " + dev;
    for (long long v : k) out += " " + std::to_string(v);
    return out;
}

// looks key up in the file at path; true and the entry when found
bool tune_file_lookup(const std::string& path, const std::string& keyline, std::tuple<int, int, int, double>* hit)
{
    FILE* f = std::fopen(path.c_str(), "r");
    if (!f) return false;
    bool found = false;
    char buf[512];
    while (std::fgets(buf, sizeof buf, f)) {
        std::string line(buf);
        while (!line.empty() && (line.back() == '\n' || line.back() == '\r')) line.pop_back();
        if (line.compare(0, keyline.size(), keyline) != 0 || line.size() <= keyline.size() ||
            line[keyline.size()] != ' ')
            continue;
        int tx = 0, ty = 0, tz = 0;
        double rate = 0.0;
        char extra = 0;
        if (std::sscanf(line.c_str() + keyline.size(), " %d %d %d %lf %c", &tx, &ty, &tz, &rate, &extra) == 4 &&
            tx >= 1 && tx <= 64 && ty >= 1 && ty <= 64 && tz >= 1 && tz <= 64) {
            *hit = std::make_tuple(tx, ty, tz, rate);
            found = true;   // keep reading: a later line for the key wins
        }
    }
    std::fclose(f);
    return found;
}
}  // namespace

dts_status dts_tune_cache_file(const char* path)
{
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_path_set = true;
    g_tune_path = path ? std::string(path) : std::string();
    return DTS_OK;
}

dts_status dts_tune_tile(dts_problem_desc* desc, double* best_updates_per_s)
{
    if (!desc) return fail(nullptr, DTS_ERR_INVALID_ARG, "desc is NULL");
    int nd = 0;
    {
        double a[80], b2[80], c[80], w[80];
        if (dts_quadrature(desc->sn_order, a, b2, c, w, &nd) != DTS_OK)
            return fail(nullptr, DTS_ERR_INVALID_ARG, "sn_order must be 2, 4, 6 or 8");
    }
    std::string dev;
    int n_sm = 0;
    {
        cudaDeviceProp prop;
        if (cudaGetDeviceProperties(&prop, desc->device) != cudaSuccess)
            return fail(nullptr, DTS_ERR_CUDA, "cannot query the device");
        for (const char* q = prop.name; *q; ++q) dev += (*q == ' ' || *q == '\t') ? '_' : *q;
        n_sm = prop.multiProcessorCount;
    }
    const int probe_b = std::min(desc->batch, 16);
    const std::vector<long long> key = {n_sm, desc->nx, desc->ny, desc->nz, desc->sn_order, desc->legendre_order,
                                        probe_b, (long long)desc->precision};
    const std::string keyline = tune_line_key(dev, key);
    std::vector<long long> mkey = key;
    mkey.push_back((long long)std::hash<std::string>()(dev));
    std::string path;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_mem.find(mkey);
        std::tuple<int, int, int, double> hit;
        path = tune_path_locked();
        bool found = it != g_tune_mem.end();
        if (found) hit = it->second;
        else if (!path.empty() && tune_file_lookup(path, keyline, &hit)) {
            g_tune_mem[mkey] = hit;
            found = true;
        }
        if (found) {
            desc->tile_x = std::get<0>(hit);
            desc->tile_y = std::get<1>(hit);
            desc->tile_z = std::get<2>(hit);
            if (best_updates_per_s) *best_updates_per_s = std::get<3>(hit);
            return DTS_OK;
        }
    }
    std::vector<std::array<int, 3>> cand;
    const bool tc = desc->precision == DTS_PREC_FP32_SPLITBF16 || desc->precision == DTS_PREC_FP32_TF32;
    if (desc->precision == DTS_PREC_FP32 || tc) cand.push_back({8, 4, 4});
    if (desc->precision == DTS_PREC_FP32) cand.push_back({4, 4, 4});
    if (!tc)
        for (auto t : std::vector<std::array<int, 3>>{{8, 4, 8}, {4, 4, 8}, {16, 4, 8}, {8, 8, 4}, {8, 8, 8}, {4, 4, 4}})
            cand.push_back(t);
    // probe: one group, homogeneous scatterer, unit volumetric source, two iterations
    const int L = desc->legendre_order, V = desc->nx * desc->ny * desc->nz;
    const double h = std::min(desc->dx, std::min(desc->dy, desc->dz));
    std::vector<double> st(1, 0.5 / h), ss(L + 1);
    for (int l = 0; l <= L; ++l) ss[l] = 0.25 / h * std::pow(0.3, l);
    std::vector<int32_t> mat(V, 0);
    std::vector<double> q(V, 1.0);
    dts_source src{};
    src.kind = 0;
    src.q = q.data();
    double best = -1.0;
    std::array<int, 3> best_t = {0, 0, 0};
    for (const auto& t : cand) {
        dts_problem_desc d = *desc;
        d.n_groups = 1;
        d.batch = probe_b;
        d.tol = 0.0;
        d.max_iters = 2;
        d.keep_moments = 0;
        d.tile_x = t[0];
        d.tile_y = t[1];
        d.tile_z = t[2];
        dts_problem* pr = nullptr;
        if (dts_create_problem(&d, &pr) != DTS_OK) continue;   // tile does not fit
        bool ok = dts_set_materials(pr, 1, st.data(), ss.data(), mat.data(), nullptr, nullptr) == DTS_OK;
        for (int b = 0; ok && b < probe_b; ++b) ok = dts_set_source(pr, b, &src) == DTS_OK;
        dts_solve_stats stats{};
        if (ok) ok = dts_solve(pr, &stats) == DTS_OK;
        if (ok && stats.sweep_ms > 0.0) {
            // sweep and reduction together: the direct-output form moves work between them
            const double ups = (double)stats.updates / ((stats.sweep_ms + stats.reduce_ms) * 1e-3);
            if (ups > best) {
                best = ups;
                best_t = t;
            }
        }
        dts_destroy_problem(pr);
    }
    if (best <= 0.0) return fail(nullptr, DTS_ERR_CUDA, "no candidate tile could be timed");
    desc->tile_x = best_t[0];
    desc->tile_y = best_t[1];
    desc->tile_z = best_t[2];
    if (best_updates_per_s) *best_updates_per_s = best;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_mem[mkey] = std::make_tuple(best_t[0], best_t[1], best_t[2], best);
    if (!path.empty()) {
        if (FILE* f = std::fopen(path.c_str(), "a")) {   // best effort: an unwritable file is skipped
            std::fprintf(f, "%s %d %d %d %.6e\n", keyline.c_str(), best_t[0], best_t[1], best_t[2], best);
            std::fclose(f);
        }
    }
    return DTS_OK;
}

long long dts_subsweep_size(int nx, int ny, int nz, int S)
{
    if (nx < 1 || ny < 1 || nz < 1 || S < 0 || S > nx + ny + nz - 3) return 0;
    return eq9(nx, ny, nz, S);
}

}  // extern "C"
