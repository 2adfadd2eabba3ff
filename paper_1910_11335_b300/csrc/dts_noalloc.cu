// dts_noalloc.cu -- one FP64 source-iteration sweep that allocates no memory.
//
// Some callers cannot allocate device memory at the point where they need a
// sweep: code running inside a caller-managed memory pool or arena that must
// not grow, or a host that has reserved the whole device for itself and
// forbids further cudaMalloc/cudaFree calls (which also synchronise the
// device). For them this file provides dts_sweep_once_noalloc: the caller
// passes device inputs and outputs, and every piece of scratch the wavefront
// sweep needs (tiled copies of the inputs, per-octant moment partials, face
// buffers, schedule and direction tables) lives in one file-scope device array
// of fixed size, reserved when the library is loaded on a device and held
// until the process exits.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/dts.h"
#define DTS_SWEEP_KERNEL_ONLY
#include "dts_kernels.cuh"

void dts_internal_set_thread_error(const char* msg);

namespace {

using namespace dts;

constexpr size_t kScratchBytes = (size_t)DTS_NOALLOC_SCRATCH_BYTES;
constexpr int kTile = 4;   // 4^3 tiles keep the FP64 S8/P3 shared memory near 12 KB

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mu;
void* g_scratch_ptr[256] = {};   // device address of g_scratch, per device ordinal

// the shape whose tables (schedule, direction operators) sit at the start of a
// device's scratch array; a call with the same shape reuses them
struct Shape {
    int nx = 0, ny = 0, nz = 0, sn = 0, L = -1;
    double dx = 0, dy = 0, dz = 0;
    bool operator==(const Shape& o) const
    {
        return nx == o.nx && ny == o.ny && nz == o.nz && sn == o.sn && L == o.L && dx == o.dx && dy == o.dy &&
               dz == o.dz;
    }
};
Shape g_tables[256];

dts_status err(dts_status s, const std::string& m)
{
    dts_internal_set_thread_error(m.c_str());
    return s;
}

// natural [K][V] (x fastest) -> tiled [NT][K][TV]; padding cells get zero
// source and unit sigma_t (they never feed a real cell); also arms the
// single batch member
__global__ void k_to_tiled(int nx, int ny, int nz, int NTx, int NTy, int K, int NC,
                           const double* src, const double* sig, double* T, double* st, int* active)
{
    const int ct = blockIdx.x * blockDim.x + threadIdx.x;
    if (ct == 0) *active = 1;
    if (ct >= NC) return;
    const int TV = kTile * kTile * kTile;
    const int tile = ct / TV, c = ct - tile * TV;
    const int tx = tile % NTx, ty = (tile / NTx) % NTy, tz = tile / (NTx * NTy);
    const int i = tx * kTile + c % kTile, j = ty * kTile + (c / kTile) % kTile,
              k = tz * kTile + c / (kTile * kTile);
    const bool valid = i < nx && j < ny && k < nz;
    const size_t V = (size_t)nx * ny * nz, v = ((size_t)k * ny + j) * nx + i;
    st[ct] = valid ? sig[v] : 1.0;
    for (int m = 0; m < K; ++m)
        T[((size_t)tile * K + m) * TV + c] = valid ? src[(size_t)m * V + v] : 0.0;
}

// Eq. 3 and its higher moments: octant partials summed in order 0..7 into the
// caller's natural-layout output
__global__ void k_octant_sum(int nx, int ny, int nz, int NTx, int NTy, int K, size_t ostride,
                             const double* part, double* phi)
{
    const size_t V = (size_t)nx * ny * nz;
    const size_t v = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= V) return;
    const int i = (int)(v % nx), j = (int)((v / nx) % ny), k = (int)(v / ((size_t)nx * ny));
    const int TV = kTile * kTile * kTile;
    const int tile = ((k / kTile) * NTy + j / kTile) * NTx + i / kTile;
    const int c = ((k % kTile) * kTile + j % kTile) * kTile + i % kTile;
    for (int m = 0; m < K; ++m) {
        const size_t ik = ((size_t)tile * K + m) * TV + c;
        double s = 0.0;
        for (int o = 0; o < 8; ++o) s += part[o * ostride + ik];
        phi[(size_t)m * V + v] = s;
    }
}

using SweepFnD = void (*)(const SweepParams<double>, int);

template <int NDO>
SweepFnD sweep_for(int K)
{
    switch (K) {
    case 1: return k_sweep_stage<double, NDO, 1>;
    case 4: return k_sweep_stage<double, NDO, 4>;
    case 9: return k_sweep_stage<double, NDO, 9>;
    case 16: return k_sweep_stage<double, NDO, 16>;
    }
    return nullptr;
}

SweepFnD sweep_fn(int ndo, int K)
{
    switch (ndo) {
    case 1: return sweep_for<1>(K);
    case 3: return sweep_for<3>(K);
    case 6: return sweep_for<6>(K);
    case 10: return sweep_for<10>(K);
    }
    return nullptr;
}

struct Carve {
    size_t off = 0;
    template <typename T>
    T* take(unsigned char* base, size_t count)
    {
        T* p = reinterpret_cast<T*>(base + off);
        off += (count * sizeof(T) + 255) & ~size_t(255);
        return p;
    }
};

}  // namespace

extern "C" dts_status dts_sweep_once_noalloc(int nx, int ny, int nz, double dx, double dy, double dz,
                                             int sn_order, int legendre_order, const double* src_moments,
                                             const double* sigma_t, double* phi, void* cuda_stream)
{
    if (nx < 1 || ny < 1 || nz < 1 || nx > 4096 || ny > 4096 || nz > 4096)
        return err(DTS_ERR_INVALID_ARG, "dts_sweep_once_noalloc: grid extents must be in 1..4096");
    if (!(dx > 0 && dy > 0 && dz > 0) || !std::isfinite(dx) || !std::isfinite(dy) || !std::isfinite(dz))
        return err(DTS_ERR_INVALID_ARG, "dts_sweep_once_noalloc: voxel pitch must be finite and > 0");
    if (legendre_order < 0 || legendre_order > 3)
        return err(DTS_ERR_INVALID_ARG, "dts_sweep_once_noalloc: legendre_order must be in 0..3");
    if (!src_moments || !sigma_t || !phi)
        return err(DTS_ERR_INVALID_ARG, "dts_sweep_once_noalloc: NULL input or output pointer");
    double mu[80], eta[80], xi[80], w[80];
    int nd = 0;
    if (dts_quadrature(sn_order, mu, eta, xi, w, &nd) != DTS_OK)
        return err(DTS_ERR_INVALID_ARG, "dts_sweep_once_noalloc: sn_order must be 2, 4, 6 or 8");
    const int K = (legendre_order + 1) * (legendre_order + 1), ndo = nd / 8;
    const int NTx = (nx + kTile - 1) / kTile, NTy = (ny + kTile - 1) / kTile, NTz = (nz + kTile - 1) / kTile;
    const int NT = NTx * NTy * NTz, TV = kTile * kTile * kTile, NC = NT * TV;
    const int n_stages = NTx + NTy + NTz - 2, nsub = 3 * kTile - 2;

    // scratch plan (offsets rounded up to 256 bytes)
    const size_t fx = (size_t)NTy * NTz * ndo * kTile * kTile, fy = (size_t)NTx * NTz * ndo * kTile * kTile,
                 fz = (size_t)NTx * NTy * ndo * kTile * kTile;
    Carve plan;
    unsigned char* const nul = nullptr;
    plan.take<unsigned>(nul, NT);
    plan.take<int>(nul, n_stages + 1);
    plan.take<unsigned>(nul, TV);
    plan.take<int>(nul, nsub + 1);
    plan.take<double>(nul, (size_t)nd * K);
    plan.take<double>(nul, (size_t)nd * K);
    plan.take<double>(nul, (size_t)nd * 3);
    plan.take<double>(nul, (size_t)nd * 3);
    plan.take<double>(nul, (size_t)NC * K);
    plan.take<double>(nul, (size_t)NC);
    plan.take<double>(nul, (size_t)8 * NC * K);
    plan.take<double>(nul, 8 * fx);
    plan.take<double>(nul, 8 * fy);
    plan.take<double>(nul, 8 * fz);
    plan.take<int>(nul, 1);
    if (plan.off > kScratchBytes) {
        char m[256];
        snprintf(m, sizeof m,
                 "dts_sweep_once_noalloc: this grid needs %zu bytes of scratch, more than the "
                 "fixed %zu-byte device array (reduce the grid or the Legendre order)",
                 plan.off, kScratchBytes);
        return err(DTS_ERR_INVALID_ARG, m);
    }

    // once per device: the device address of the scratch array; per device the shape of the tables
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return err(DTS_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= 256) return err(DTS_ERR_INVALID_ARG, "dts_sweep_once_noalloc: device ordinal >= 256");
    unsigned char* base;
    Shape shape;
    shape.nx = nx; shape.ny = ny; shape.nz = nz; shape.sn = sn_order; shape.L = legendre_order;
    shape.dx = dx; shape.dy = dy; shape.dz = dz;
    bool upload;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        upload = !(g_tables[dev] == shape);
        if (!g_scratch_ptr[dev]) {
            void* ptr = nullptr;
            e = cudaGetSymbolAddress(&ptr, g_scratch);
            if (e != cudaSuccess)
                return err(DTS_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            g_scratch_ptr[dev] = ptr;
        }
        base = static_cast<unsigned char*>(g_scratch_ptr[dev]);
    }

    // host-side tables: tile stages (Eq. 9 on the tile grid), intra-tile
    // sub-sweeps, and the direction operators of the quadrature
    std::vector<int> soff(n_stages + 1, 0), doff(nsub + 1, 0);
    for (int s = 0; s < n_stages; ++s) soff[s + 1] = soff[s] + (int)dts_subsweep_size(NTx, NTy, NTz, s);
    for (int s = 0; s < nsub; ++s) doff[s + 1] = doff[s] + (int)dts_subsweep_size(kTile, kTile, kTile, s);
    if (soff[n_stages] != NT || doff[nsub] != TV)
        return err(DTS_ERR_INTERNAL, "dts_sweep_once_noalloc: schedule size mismatch");
    std::vector<unsigned> tiles(NT), cells(TV);
    std::vector<int> sf(soff.begin(), soff.end() - 1), df(doff.begin(), doff.end() - 1);
    for (int c = 0; c < NTz; ++c)
        for (int b = 0; b < NTy; ++b)
            for (int a = 0; a < NTx; ++a)
                tiles[sf[a + b + c]++] = (unsigned)a | ((unsigned)b << 10) | ((unsigned)c << 20);
    for (int z = 0; z < kTile; ++z)
        for (int y = 0; y < kTile; ++y)
            for (int x = 0; x < kTile; ++x)
                cells[df[x + y + z]++] = (unsigned)x | ((unsigned)y << 8) | ((unsigned)z << 16);
    std::vector<double> D((size_t)K * nd), M((size_t)nd * K), Dt((size_t)nd * K), A((size_t)nd * 3),
        Lw((size_t)nd * 3);
    if (dts_moment_tables(sn_order, legendre_order, D.data(), M.data()) != DTS_OK)
        return err(DTS_ERR_INTERNAL, "dts_sweep_once_noalloc: moment tables");
    const double h[3] = {dx, dy, dz}, area[3] = {dy * dz, dx * dz, dx * dy};
    for (int n = 0; n < nd; ++n) {
        for (int k = 0; k < K; ++k) Dt[(size_t)n * K + k] = D[(size_t)k * nd + n];
        const double om[3] = {std::fabs(mu[n]), std::fabs(eta[n]), std::fabs(xi[n])};
        for (int a = 0; a < 3; ++a) {
            A[n * 3 + a] = 2.0 * om[a] / h[a];
            Lw[n * 3 + a] = w[n] * om[a] * area[a];
        }
    }

    Carve cv;
    SweepParams<double> sp;
    sp.nx = nx; sp.ny = ny; sp.nz = nz;
    sp.TX = sp.TY = sp.TZ = kTile; sp.TV = TV;
    sp.NTx = NTx; sp.NTy = NTy; sp.NTz = NTz; sp.NT = NT;
    sp.B = 1; sp.nsub = nsub;
    unsigned* d_tiles = cv.take<unsigned>(base, NT);
    int* d_soff = cv.take<int>(base, n_stages + 1);
    unsigned* d_cells = cv.take<unsigned>(base, TV);
    int* d_doff = cv.take<int>(base, nsub + 1);
    double* d_M = cv.take<double>(base, (size_t)nd * K);
    double* d_Dt = cv.take<double>(base, (size_t)nd * K);
    double* d_A = cv.take<double>(base, (size_t)nd * 3);
    double* d_Lw = cv.take<double>(base, (size_t)nd * 3);
    double* d_T = cv.take<double>(base, (size_t)NC * K);
    double* d_st = cv.take<double>(base, (size_t)NC);
    double* d_part = cv.take<double>(base, (size_t)8 * NC * K);
    double* d_xf = cv.take<double>(base, 8 * fx);
    double* d_yf = cv.take<double>(base, 8 * fy);
    double* d_zf = cv.take<double>(base, 8 * fz);
    int* d_active = cv.take<int>(base, 1);
    sp.stage_tiles = d_tiles; sp.stage_off = d_soff; sp.diag_cells = d_cells; sp.diag_off = d_doff;
    sp.M = d_M; sp.Dt = d_Dt; sp.A = d_A; sp.Lw = d_Lw;
    sp.T = d_T; sp.sigt = d_st; sp.part = d_part; sp.xf = d_xf; sp.yf = d_yf; sp.zf = d_zf;
    sp.active = d_active; sp.leak = nullptr;   // no leakage tally: the call returns moments only

    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
#define CKN(call)                                                                              \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            return err(DTS_ERR_CUDA, std::string("dts_sweep_once_noalloc: " #call ": ") +      \
                                         cudaGetErrorString(e_));                              \
    } while (0)
    if (upload) {
        // a new shape on this device: wait until no earlier call's work can still read the old
        // tables, then copy the new ones (blocking copies from host memory)
        CKN(cudaDeviceSynchronize());
        CKN(cudaMemcpy(d_tiles, tiles.data(), sizeof(unsigned) * NT, cudaMemcpyHostToDevice));
        CKN(cudaMemcpy(d_soff, soff.data(), sizeof(int) * (n_stages + 1), cudaMemcpyHostToDevice));
        CKN(cudaMemcpy(d_cells, cells.data(), sizeof(unsigned) * TV, cudaMemcpyHostToDevice));
        CKN(cudaMemcpy(d_doff, doff.data(), sizeof(int) * (nsub + 1), cudaMemcpyHostToDevice));
        CKN(cudaMemcpy(d_M, M.data(), sizeof(double) * nd * K, cudaMemcpyHostToDevice));
        CKN(cudaMemcpy(d_Dt, Dt.data(), sizeof(double) * nd * K, cudaMemcpyHostToDevice));
        CKN(cudaMemcpy(d_A, A.data(), sizeof(double) * nd * 3, cudaMemcpyHostToDevice));
        CKN(cudaMemcpy(d_Lw, Lw.data(), sizeof(double) * nd * 3, cudaMemcpyHostToDevice));
        std::lock_guard<std::mutex> lk(g_mu);
        g_tables[dev] = shape;
    }
    k_to_tiled<<<(NC + 255) / 256, 256, 0, st>>>(nx, ny, nz, NTx, NTy, K, NC, src_moments, sigma_t,
                                                 d_T, d_st, d_active);
    CKN(cudaGetLastError());
    SweepFnD fn = sweep_fn(ndo, K);
    if (!fn) return err(DTS_ERR_INTERNAL, "dts_sweep_once_noalloc: no sweep kernel for (S_N, P_L)");
    const size_t TVs = TV;
    const size_t smem = ((((size_t)ndo * TVs + (size_t)ndo * 3 * kTile * kTile + TVs + 2 * ndo * K + 4 * ndo) *
                          sizeof(double) + 15) & ~size_t(15)) + sizeof(double) * (3 * ndo + 32);
    for (int s = 0; s < n_stages; ++s) {
        const unsigned grid = (unsigned)(soff[s + 1] - soff[s]) * 8u;
        fn<<<grid, kSweepThreads, smem, st>>>(sp, s);
    }
    CKN(cudaGetLastError());
    const size_t V = (size_t)nx * ny * nz;
    k_octant_sum<<<(unsigned)((V + 255) / 256), 256, 0, st>>>(nx, ny, nz, NTx, NTy, K,
                                                               (size_t)NC * K, d_part, phi);
    CKN(cudaGetLastError());
#undef CKN
    return DTS_OK;
}
