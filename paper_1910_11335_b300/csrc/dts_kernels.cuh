// dts_kernels.cuh -- sm_103a kernels of the S_N source-iteration solve.
//
// Data layout in HBM ("tiled"): the grid is cut into TX x TY x TZ tiles
// (NT of them, padded at the high end of each axis); a per-cell array of one
// batch member stores tile after tile, and inside a tile moment k after
// moment k, each a contiguous run of TV = TX*TY*TZ cells (x fastest). So a
// tile's K moments are one contiguous block and every phase below reads and
// writes whole 32-byte sectors.
//
//   T    [B][NT][K][TV]   R       scatter + fixed source moments (this iteration)
//   part [8][B][NT][K][TV] R      per-octant moment partials of the last sweep
//   phi00 [B][NT*TV]     double  scalar flux of the current group
//   F    [W+1][B][NT][K][TV] R    fixed-source ring (first-collision + downscatter)
//   xf   [8][B][NTy*NTz][NDO][TY*TZ] R  x-faces in flight (likewise yf, zf)
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <math_constants.h>
#include <stdint.h>

#include "dts_ptx.cuh"

namespace dts {

// ---------------------------------------------------------------------------
// Index checks of the DTS_DEBUG_BOUNDS build. Before a kernel touches a region
// of a global buffer it checks the region's end against the buffer's size (an
// element count carried in the kernel's parameters); a region that does not
// fit is skipped (loads read nothing, stores are dropped) and the first failing
// site is recorded in bounds_word as (site << 48) | (end offset, low 48 bits).
// The host reads the word after every source iteration and returns
// DTS_ERR_INTERNAL. Each translation unit has its own word. In the normal build
// DTS_FITS is the constant true and the checks compile away.
// ---------------------------------------------------------------------------
#ifdef DTS_DEBUG_BOUNDS
static __device__ unsigned long long bounds_word;
__device__ __forceinline__ bool fits(size_t end, size_t size, unsigned site)
{
    if (end <= size) return true;
    atomicCAS(&bounds_word, 0ull, ((unsigned long long)site << 48) | (end & 0xffffffffffffull));
    return false;
}
#define DTS_FITS(end, size, site) ::dts::fits((size_t)(end), (size_t)(size), (site))
#else
#define DTS_FITS(end, size, site) true
#endif

constexpr int kSweepThreads = 256;
constexpr int kRedThreads = 256;
constexpr int kPushRing = 4;   // widest downscatter band of the FP32 push kernels (W <= 4)
constexpr int kRayGroups = 16;
constexpr double kPi = 3.14159265358979323846;

// ---------------------------------------------------------------------------
// real spherical harmonics in Cartesian form, l <= 3, k = l*l + l + m,
// normalised so that sum_m Y_lm(a) Y_lm(b) = P_l(a.b)
// ---------------------------------------------------------------------------
template <typename T>
__host__ __device__ inline void sh_eval(int L, T x, T y, T z, T* Y)
{
    Y[0] = T(1);
    if (L < 1) return;
    Y[1] = y;
    Y[2] = z;
    Y[3] = x;
    if (L < 2) return;
    const T s3 = T(1.7320508075688772);   // sqrt(3)
    Y[4] = s3 * x * y;
    Y[5] = s3 * y * z;
    Y[6] = T(0.5) * (T(3) * z * z - T(1));
    Y[7] = s3 * x * z;
    Y[8] = T(0.5) * s3 * (x * x - y * y);
    if (L < 3) return;
    const T s58 = T(0.7905694150420949);  // sqrt(5/8)
    const T s15 = T(3.872983346207417);   // sqrt(15)
    const T s38 = T(0.6123724356957945);  // sqrt(3/8)
    Y[9] = s58 * (T(3) * x * x * y - y * y * y);
    Y[10] = s15 * x * y * z;
    Y[11] = s38 * y * (T(5) * z * z - T(1));
    Y[12] = T(0.5) * (T(5) * z * z * z - T(3) * z);
    Y[13] = s38 * x * (T(5) * z * z - T(1));
    Y[14] = T(0.5) * s15 * z * (x * x - y * y);
    Y[15] = s58 * (x * x * x - T(3) * x * y * y);
}

__host__ __device__ inline int l_of_k(int k) { return k >= 9 ? 3 : k >= 4 ? 2 : k >= 1 ? 1 : 0; }

// ---------------------------------------------------------------------------
// block reduction of doubles (result valid in thread 0)
// ---------------------------------------------------------------------------
__device__ inline double block_sum(double v, double* red)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    v = 0.0;
    if (wid == 0) {
        v = lane < nw ? red[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    }
    return v;
}

// ---------------------------------------------------------------------------
// diamond-difference cell solve with set-to-zero fixup (Sec. IV)
// psi = (q + sum_d a_d in_d) / (sigma + sum_d a_d), out_d = 2 psi - in_d; a
// negative out_d is zeroed and dropped from the closure, its face entering the
// balance with a_d/2, until no new negative appears.
// ---------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ R dd_cell(R q, R sig, R ax, R ay, R az, R ix, R iy, R iz,
                                     R& ox, R& oy, R& oz)
{
    R psi = (q + ax * ix + ay * iy + az * iz) / (sig + ax + ay + az);
    ox = R(2) * psi - ix;
    oy = R(2) * psi - iy;
    oz = R(2) * psi - iz;
    if (ox < R(0) || oy < R(0) || oz < R(0)) {
        bool fx = false, fy = false, fz = false;
#pragma unroll 1
        for (int pass = 0; pass < 3; ++pass) {
            const bool nx = !fx && ox < R(0), ny = !fy && oy < R(0), nz = !fz && oz < R(0);
            if (!(nx || ny || nz)) break;
            fx |= nx;
            fy |= ny;
            fz |= nz;
            const R num = q + (fx ? R(0.5) * ax : ax) * ix + (fy ? R(0.5) * ay : ay) * iy +
                          (fz ? R(0.5) * az : az) * iz;
            const R den = sig + (fx ? R(0) : ax) + (fy ? R(0) : ay) + (fz ? R(0) : az);
            psi = num / den;
            ox = fx ? R(0) : R(2) * psi - ix;
            oy = fy ? R(0) : R(2) * psi - iy;
            oz = fz ? R(0) : R(2) * psi - iz;
        }
    }
    return psi;
}

// ---------------------------------------------------------------------------
// A3 + A4: one tile-wavefront stage of the sweep, all octants and batch
// members of the stage in one launch. One CTA = (tile, octant, source).
// ---------------------------------------------------------------------------
template <typename R>
struct SweepParams {
    int nx, ny, nz;
    int TX, TY, TZ, TV;
    int NTx, NTy, NTz, NT;
    int B, nsub;
    const unsigned* stage_tiles;   // octant-local tile (a | b<<10 | c<<20), sorted by a+b+c
    const int* stage_off;
    const unsigned* diag_cells;    // octant-local cell (x | y<<8 | z<<16), sorted by x+y+z
    const int* diag_off;
    const R* M;                    // [nd][K] source operator
    const R* Dt;                   // [nd][K] moment operator (transposed)
    const R* A;                    // [nd][3] a_d = 2|Omega_d|/Delta_d
    const double* Lw;              // [nd][3] w_n |Omega_d| A_d (leakage weights)
    const R* T;
    const R* sigt;                 // [NT][TV]
    R* part;
    R* xf;
    R* yf;
    R* zf;
    const int* active;             // [B]
    double* leak;                  // [B][8][NT] leakage of each (source, octant, tile) sweep, or null
    // element counts of the buffers above (checked in the DTS_DEBUG_BOUNDS build)
    size_t n_stage_tiles, n_T, n_sigt, n_part, n_xf, n_yf, n_zf, n_leak;
    int* err = nullptr;            // set when a bounded wait on a bulk copy gave up (Q-input sweep), or null
    unsigned poison_tx = 0;        // test hook (dts_debug_poison_wait): bytes the face wait expects beyond its copies
};

template <typename R, int NDO, int K>
__host__ __device__ inline size_t sweep_smem_bytes(int TX, int TY, int TZ)
{
    const int TV = TX * TY * TZ;
    size_t n = (size_t)NDO * TV + (size_t)NDO * (TY * TZ + TX * TZ + TX * TY) + TV +
               2 * NDO * K + 4 * NDO;
    size_t bytes = n * sizeof(R);
    bytes = (bytes + 15) & ~size_t(15);
    return bytes + sizeof(double) * (3 * NDO + 32);
}

// resident CTAs per SM the register allocation must allow (FP32: 4, FP64: 2)
template <typename R> struct SweepOcc { static constexpr int value = sizeof(R) == 4 ? 4 : 2; };

template <typename R, int NDO, int K>
__global__ void __launch_bounds__(kSweepThreads, SweepOcc<R>::value)
k_sweep_stage(const SweepParams<R> p, const int stage)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int TX = p.TX, TY = p.TY, TZ = p.TZ, TV = p.TV;
    const int s0 = p.stage_off[stage], cnt = p.stage_off[stage + 1] - s0;
    int bid = blockIdx.x;
    const int tl = bid % cnt;
    bid /= cnt;
    const int oct = bid & 7, b = bid >> 3;
    if (!p.active[b]) return;

    const unsigned pk = p.stage_tiles[s0 + tl];
    const int ta = pk & 1023, tb = (pk >> 10) & 1023, tc = (pk >> 20) & 1023;
    const bool negx = oct & 1, negy = oct & 2, negz = oct & 4;
    const int tx = negx ? p.NTx - 1 - ta : ta;
    const int ty = negy ? p.NTy - 1 - tb : tb;
    const int tz = negz ? p.NTz - 1 - tc : tc;
    const int tile = (tz * p.NTy + ty) * p.NTx + tx;
    const int fxn = TY * TZ, fyn = TX * TZ, fzn = TX * TY;

    R* Qs = reinterpret_cast<R*>(smem);        // [NDO][TV]: source, then psi
    R* fx = Qs + NDO * TV;                      // [NDO][TY*TZ]
    R* fy = fx + NDO * fxn;                     // [NDO][TX*TZ]
    R* fz = fy + NDO * fyn;                     // [NDO][TX*TY]
    R* sg = fz + NDO * fzn;                     // [TV]
    R* Ms = sg + TV;                            // [NDO][K]
    R* Ds = Ms + NDO * K;                       // [K][NDO]
    R* As = Ds + NDO * K;                       // [NDO][4]
    size_t off = ((size_t)(As + 4 * NDO - Qs) * sizeof(R) + 15) & ~size_t(15);
    double* Lw = reinterpret_cast<double*>(smem + off);   // [NDO][3]
    double* red = Lw + 3 * NDO;                            // [32]

    const int tid = threadIdx.x, nth = blockDim.x;
    const int n0 = oct * NDO;
    for (int i = tid; i < NDO * K; i += nth) {
        Ms[i] = p.M[n0 * K + i];                         // [NDO][K]
        Ds[(i % K) * NDO + i / K] = p.Dt[n0 * K + i];    // [K][NDO]
    }
    for (int i = tid; i < NDO * 3; i += nth) {
        As[(i / 3) * 4 + i % 3] = p.A[n0 * 3 + i];
        Lw[i] = p.Lw[n0 * 3 + i];
    }
    const size_t BB = p.B;
    R* gx = p.xf + (((size_t)oct * BB + b) * (p.NTy * p.NTz) + (tz * p.NTy + ty)) * (size_t)(NDO * fxn);
    R* gy = p.yf + (((size_t)oct * BB + b) * (p.NTx * p.NTz) + (tz * p.NTx + tx)) * (size_t)(NDO * fyn);
    R* gz = p.zf + (((size_t)oct * BB + b) * (p.NTx * p.NTy) + (ty * p.NTx + tx)) * (size_t)(NDO * fzn);
    // incoming faces: the upstream tile's outgoing faces, or vacuum on the boundary
    for (int i = tid; i < NDO * fxn; i += nth) fx[i] = ta > 0 ? gx[i] : R(0);
    for (int i = tid; i < NDO * fyn; i += nth) fy[i] = tb > 0 ? gy[i] : R(0);
    for (int i = tid; i < NDO * fzn; i += nth) fz[i] = tc > 0 ? gz[i] : R(0);
    __syncthreads();

    // phase A: scatter-source contraction Q_n = sum_k M[n][k] T_k for the octant
    const R* Tt = p.T + ((size_t)b * p.NT + tile) * (size_t)(K * TV);
    const R* st = p.sigt + (size_t)tile * TV;
#pragma unroll 1
    for (int c = tid; c < TV; c += nth) {
        R t[K];
#pragma unroll
        for (int k = 0; k < K; ++k) t[k] = Tt[k * TV + c];
        sg[c] = st[c];
#pragma unroll 1
        for (int d = 0; d < NDO; ++d) {
            R q = R(0);
#pragma unroll
            for (int k = 0; k < K; ++k) q = fma(Ms[d * K + k], t[k], q);
            Qs[d * TV + c] = q;
        }
    }
    __syncthreads();

    // phase B: intra-tile wavefront, sub-sweep by sub-sweep (Sec. II.B)
    double leak = 0.0;
    const int gx0 = tx * TX, gy0 = ty * TY, gz0 = tz * TZ;
    const int bx = negx ? 0 : p.nx - 1, by = negy ? 0 : p.ny - 1, bz = negz ? 0 : p.nz - 1;
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
            R* px = fx + d * fxn + sz * TY + sy;
            R* py = fy + d * fyn + sz * TX + sx;
            R* pz = fz + d * fzn + sy * TX + sx;
            const int gi = gx0 + sx, gj = gy0 + sy, gk = gz0 + sz;
            if (gi >= p.nx || gj >= p.ny || gk >= p.nz) {   // padding: vacuum in, nothing out
                *px = R(0);
                *py = R(0);
                *pz = R(0);
                Qs[d * TV + c] = R(0);
                continue;
            }
            R ox, oy, oz;
            const R psi = dd_cell<R>(Qs[d * TV + c], sg[c], As[d * 4], As[d * 4 + 1], As[d * 4 + 2],
                                     *px, *py, *pz, ox, oy, oz);
            *px = ox;
            *py = oy;
            *pz = oz;
            Qs[d * TV + c] = psi;
            if (gi == bx) leak += Lw[d * 3] * (double)ox;
            if (gj == by) leak += Lw[d * 3 + 1] * (double)oy;
            if (gk == bz) leak += Lw[d * 3 + 2] * (double)oz;
        }
        __syncthreads();
    }

    // phase C: per-octant moment partial P_o[k] = sum_n D[k][n] psi_n
    R* out = p.part + (((size_t)oct * BB + b) * p.NT + tile) * (size_t)(K * TV);
#pragma unroll 1
    for (int c = tid; c < TV; c += nth) {
        R ps[NDO];
#pragma unroll
        for (int d = 0; d < NDO; ++d) ps[d] = Qs[d * TV + c];
#pragma unroll 1
        for (int k = 0; k < K; ++k) {
            R acc = R(0);
#pragma unroll
            for (int d = 0; d < NDO; ++d) acc = fma(Ds[k * NDO + d], ps[d], acc);
            out[k * TV + c] = acc;
        }
    }
    // outgoing faces for the downstream tiles
    for (int i = tid; i < NDO * fxn; i += nth) gx[i] = fx[i];
    for (int i = tid; i < NDO * fyn; i += nth) gy[i] = fy[i];
    for (int i = tid; i < NDO * fzn; i += nth) gz[i] = fz[i];
    // every (source, octant, tile) of a sweep owns one slot: a fixed-order sum per source later
    leak = block_sum(leak, red);
    if (tid == 0 && p.leak) p.leak[((size_t)b * 8 + oct) * p.NT + tile] = leak;
}

// ---------------------------------------------------------------------------
// A3 + A4, warp-synchronous form for tiles of TY x TZ = 32 x-lines.
// One lane owns one x-line of the tile and walks it cell by cell; the x-face
// stays in a register, the y- and z-faces of the neighbouring lines arrive
// through warp shuffles one step later (the i+j+k wavefront of Sec. II.B,
// skewed across lanes), so the wavefront needs no CTA barrier. Each warp
// chains several directions of the octant back to back so the pipeline
// ramp is paid once per warp, not once per direction. Padding cells pass
// every face through unchanged, so a tile's outgoing faces on the downstream
// boundary of the grid are exactly the leakage.
// ---------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ R fast_div(R a, R b) { return a / b; }
template <>
__device__ __forceinline__ float fast_div<float>(float a, float b) { return __fdividef(a, b); }

template <typename R>
__device__ __forceinline__ R dd_cell_line(R q, R sig, R ax, R ay, R az, R ix, R iy, R iz,
                                          R& ox, R& oy, R& oz)
{
    R psi = fast_div<R>(q + ax * ix + ay * iy + az * iz, sig + ax + ay + az);
    ox = R(2) * psi - ix;
    oy = R(2) * psi - iy;
    oz = R(2) * psi - iz;
    if (ox < R(0) || oy < R(0) || oz < R(0)) {
        bool fx = false, fy = false, fz = false;
#pragma unroll 1
        for (int pass = 0; pass < 3; ++pass) {
            const bool nx = !fx && ox < R(0), ny = !fy && oy < R(0), nz = !fz && oz < R(0);
            if (!(nx || ny || nz)) break;
            fx |= nx;
            fy |= ny;
            fz |= nz;
            const R num = q + (fx ? R(0.5) * ax : ax) * ix + (fy ? R(0.5) * ay : ay) * iy +
                          (fz ? R(0.5) * az : az) * iz;
            const R den = sig + (fx ? R(0) : ax) + (fy ? R(0) : ay) + (fz ? R(0) : az);
            psi = fast_div<R>(num, den);
            ox = fx ? R(0) : R(2) * psi - ix;
            oy = fy ? R(0) : R(2) * psi - iy;
            oz = fz ? R(0) : R(2) * psi - iz;
        }
    }
    return psi;
}

template <typename R, int NDO, int K>
__host__ __device__ inline size_t sweep_lines_smem_bytes(int TX, int TY, int TZ)
{
    const int TV = TX * TY * TZ;
    size_t n = (size_t)NDO * TV + (size_t)NDO * (TY * TZ + TX * TZ + TX * TY) + TV +
               2 * NDO * K + 4 * NDO;
    size_t bytes = (n * sizeof(R) + 15) & ~size_t(15);
    return bytes + sizeof(double) * (3 * NDO + 32);
}

constexpr int kLineThreadsMax = 128;

// resident CTAs per SM the register allocation must allow (FP32: 8, FP64: 4)
template <typename R> struct LinesOcc { static constexpr int value = sizeof(R) == 4 ? 8 : 4; };

template <typename R, int NDO, int K, int TY, int TZ>
__global__ void __launch_bounds__(kLineThreadsMax, LinesOcc<R>::value)
k_sweep_lines(const SweepParams<R> p, const int stage)
{
    static_assert(TY * TZ == 32, "one warp lane per x-line");
    extern __shared__ __align__(16) unsigned char smem[];
    const int TX = p.TX, TV = TX * TY * TZ;
    const int s0 = p.stage_off[stage], cnt = p.stage_off[stage + 1] - s0;
    int bid = blockIdx.x;
    const int tl = bid % cnt;
    bid /= cnt;
    const int oct = bid & 7, b = bid >> 3;
    if (!p.active[b]) return;
    const unsigned pk = p.stage_tiles[s0 + tl];
    const int ta = pk & 1023, tb = (pk >> 10) & 1023, tc = (pk >> 20) & 1023;
    const bool negx = oct & 1, negy = oct & 2, negz = oct & 4;
    const int tx = negx ? p.NTx - 1 - ta : ta;
    const int ty = negy ? p.NTy - 1 - tb : tb;
    const int tz = negz ? p.NTz - 1 - tc : tc;
    const int tile = (tz * p.NTy + ty) * p.NTx + tx;
    constexpr int fxn = TY * TZ;
    const int fyn = TX * TZ, fzn = TX * TY;

    R* Qs = reinterpret_cast<R*>(smem);        // [NDO][TV]: source, then psi
    R* fx = Qs + NDO * TV;                      // [NDO][32] indexed by line = sz*TY + sy
    R* fy = fx + NDO * fxn;                     // [NDO][TX*TZ] indexed sz*TX + sx
    R* fz = fy + NDO * fyn;                     // [NDO][TX*TY] indexed sy*TX + sx
    R* sg = fz + NDO * fzn;                     // [TV]
    R* Ms = sg + TV;                            // [NDO][K]
    R* Ds = Ms + NDO * K;                       // [K][NDO]
    R* As = Ds + NDO * K;                       // [NDO][4]
    const size_t off = ((size_t)(As + 4 * NDO - Qs) * sizeof(R) + 15) & ~size_t(15);
    double* Lw = reinterpret_cast<double*>(smem + off);    // [NDO][3]
    double* red = Lw + 3 * NDO;                             // [32]

    const int tid = threadIdx.x, nth = blockDim.x;
    const int n0 = oct * NDO;
    for (int i = tid; i < NDO * K; i += nth) {
        Ms[i] = p.M[n0 * K + i];
        Ds[(i % K) * NDO + i / K] = p.Dt[n0 * K + i];
    }
    for (int i = tid; i < NDO * 3; i += nth) {
        As[(i / 3) * 4 + i % 3] = p.A[n0 * 3 + i];
        Lw[i] = p.Lw[n0 * 3 + i];
    }
    const size_t BB = p.B;
    R* gx = p.xf + (((size_t)oct * BB + b) * (p.NTy * p.NTz) + (tz * p.NTy + ty)) * (size_t)(NDO * fxn);
    R* gy = p.yf + (((size_t)oct * BB + b) * (p.NTx * p.NTz) + (tz * p.NTx + tx)) * (size_t)(NDO * fyn);
    R* gz = p.zf + (((size_t)oct * BB + b) * (p.NTx * p.NTy) + (ty * p.NTx + tx)) * (size_t)(NDO * fzn);
    for (int i = tid; i < NDO * fxn; i += nth) fx[i] = ta > 0 ? gx[i] : R(0);
    for (int i = tid; i < NDO * fyn; i += nth) fy[i] = tb > 0 ? gy[i] : R(0);
    for (int i = tid; i < NDO * fzn; i += nth) fz[i] = tc > 0 ? gz[i] : R(0);
    __syncthreads();

    // phase A: scatter-source contraction Q_n = sum_k M[n][k] T_k
    const R* Tt = p.T + ((size_t)b * p.NT + tile) * (size_t)(K * TV);
    const R* st = p.sigt + (size_t)tile * TV;
#pragma unroll 1
    for (int c = tid; c < TV; c += nth) {
        R t[K];
#pragma unroll
        for (int k = 0; k < K; ++k) t[k] = Tt[k * TV + c];
        sg[c] = st[c];
#pragma unroll 1
        for (int d = 0; d < NDO; ++d) {
            R q = R(0);
#pragma unroll
            for (int k = 0; k < K; ++k) q = fma(Ms[d * K + k], t[k], q);
            Qs[d * TV + c] = q;
        }
    }
    __syncthreads();

    // phase B: lane = x-line, warp = a run of directions, wavefront by shuffles
    {
        const int warp = tid >> 5, lane = tid & 31, nw = nth >> 5;
        const int d0 = warp * NDO / nw, d1 = (warp + 1) * NDO / nw;
        const int ly = lane % TY, lz = lane / TY;
        const int sy = negy ? TY - 1 - ly : ly, sz = negz ? TZ - 1 - lz : lz;
        const int line = sz * TY + sy;
        const bool line_ok = (ty * TY + sy) < p.ny && (tz * TZ + sz) < p.nz;
        const int nvx = line_ok ? p.nx - tx * TX : 0;   // valid cells along x in this line
        const int total = (d1 - d0) * TX, ls = ly + lz;
        const int xflip = negx ? TX - 1 : 0;           // storage x = xflip ^ lx when TX is 2^n
        int lx = 0, d = d0;
        R ax = As[d0 * 4], ay = As[d0 * 4 + 1], az = As[d0 * 4 + 2];
        R asum = ax + ay + az;
        R* qd = Qs + d0 * TV + line * TX;
        const R* sgl = sg + line * TX;
        R* yd = fy + d0 * fyn + sz * TX;
        R* zd = fz + d0 * fzn + sy * TX;
        R xin = fx[d0 * fxn + line], ycur = R(0), zcur = R(0), ysh = R(0), zsh = R(0);
        const bool ytop = ly == TY - 1, ztop = lz == TZ - 1;
        const int nsteps = total + TY + TZ - 2;
        for (int t = 0; t < nsteps; ++t) {
            const int u = t - ls;
            const bool act = (unsigned)u < (unsigned)total;
            bool neg = false;
            R ox = R(0), oy = R(0), oz = R(0), psi = R(0), q = R(0), sig = R(0), yin = R(0), zin = R(0);
            int sx = 0;
            if (act) {
                sx = (TX & (TX - 1)) == 0 ? (xflip ^ lx) : (negx ? TX - 1 - lx : lx);
                yin = ly ? ysh : yd[sx];
                zin = lz ? zsh : zd[sx];
                if (sx < nvx) {
                    q = qd[sx];
                    sig = sgl[sx];
                    psi = fast_div<R>(q + ax * xin + ay * yin + az * zin, sig + asum);
                    ox = R(2) * psi - xin;
                    oy = R(2) * psi - yin;
                    oz = R(2) * psi - zin;
                    neg = ox < R(0) || oy < R(0) || oz < R(0);
                } else {
                    ox = xin;
                    oy = yin;
                    oz = zin;
                }
            }
            if (__any_sync(0xffffffffu, neg) && neg) {
                bool fxd = false, fyd = false, fzd = false;
#pragma unroll 1
                for (int pass = 0; pass < 3; ++pass) {
                    const bool nx = !fxd && ox < R(0), ny = !fyd && oy < R(0), nz = !fzd && oz < R(0);
                    if (!(nx || ny || nz)) break;
                    fxd |= nx;
                    fyd |= ny;
                    fzd |= nz;
                    const R num = q + (fxd ? R(0.5) * ax : ax) * xin + (fyd ? R(0.5) * ay : ay) * yin +
                                  (fzd ? R(0.5) * az : az) * zin;
                    const R den = sig + (fxd ? R(0) : ax) + (fyd ? R(0) : ay) + (fzd ? R(0) : az);
                    psi = fast_div<R>(num, den);
                    ox = fxd ? R(0) : R(2) * psi - xin;
                    oy = fyd ? R(0) : R(2) * psi - yin;
                    oz = fzd ? R(0) : R(2) * psi - zin;
                }
            }
            if (act) {
                qd[sx] = psi;
                if (ytop) yd[sx] = oy;
                if (ztop) zd[sx] = oz;
                xin = ox;
                ycur = oy;
                zcur = oz;
                if (++lx == TX) {   // this line of direction d is done: next direction
                    fx[d * fxn + line] = ox;
                    lx = 0;
                    if (++d < d1) {
                        ax = As[d * 4];
                        ay = As[d * 4 + 1];
                        az = As[d * 4 + 2];
                        asum = ax + ay + az;
                        qd += TV;
                        yd += fyn;
                        zd += fzn;
                        xin = fx[d * fxn + line];
                    }
                }
            }
            ysh = __shfl_up_sync(0xffffffffu, ycur, 1);
            zsh = __shfl_up_sync(0xffffffffu, zcur, TY);
            __syncwarp();
        }
    }
    __syncthreads();

    // phase C: per-octant moment partial P_o[k] = sum_n D[k][n] psi_n
    R* out = p.part + (((size_t)oct * BB + b) * p.NT + tile) * (size_t)(K * TV);
#pragma unroll 1
    for (int c = tid; c < TV; c += nth) {
        R ps[NDO];
#pragma unroll
        for (int d = 0; d < NDO; ++d) ps[d] = Qs[d * TV + c];
#pragma unroll 1
        for (int k = 0; k < K; ++k) {
            R acc = R(0);
#pragma unroll
            for (int d = 0; d < NDO; ++d) acc = fma(Ds[k * NDO + d], ps[d], acc);
            out[k * TV + c] = acc;
        }
    }
    // outgoing faces; on the downstream boundary of the grid they leave it
    const bool lbx = negx ? tx == 0 : tx == p.NTx - 1;
    const bool lby = negy ? ty == 0 : ty == p.NTy - 1;
    const bool lbz = negz ? tz == 0 : tz == p.NTz - 1;
    double leak = 0.0;
    for (int i = tid; i < NDO * fxn; i += nth) {
        gx[i] = fx[i];
        if (lbx) leak += Lw[(i / fxn) * 3] * (double)fx[i];
    }
    for (int i = tid; i < NDO * fyn; i += nth) {
        gy[i] = fy[i];
        if (lby) leak += Lw[(i / fyn) * 3 + 1] * (double)fy[i];
    }
    for (int i = tid; i < NDO * fzn; i += nth) {
        gz[i] = fz[i];
        if (lbz) leak += Lw[(i / fzn) * 3 + 2] * (double)fz[i];
    }
    if (lbx || lby || lbz) leak = block_sum(leak, red);
    if (tid == 0 && p.leak) p.leak[((size_t)b * 8 + oct) * p.NT + tile] = (lbx || lby || lbz) ? leak : 0.0;
}

// ---------------------------------------------------------------------------
// A3 + A4, batched form (FP32): one warp per (tile, octant, group of sources).
// Lane = (source, direction) pair, e.g. 3 sources x 10 directions for S8, so
// all lanes solve the same cell at the same time: the warp walks the tile in
// upwind order (the sub-sweeps of Sec. II.B reduce to a lexicographic walk
// inside one warp). Each lane's sweep is independent of the others; the x-face
// stays in a register, the y-faces of a z-column of lines stay in registers,
// and the z-faces sit in per-lane shared-memory slots. The tile is processed
// one x-line at a time: the line's source moments arrive by cp.async one line
// ahead, are contracted to the lanes' directions (A3), swept (A4), and reduced
// to octant moment partials by lanes re-assigned to (moment, cell quad) pairs,
// so shared memory holds one line of sources and fluxes rather than the whole
// tile. Both contractions use packed FP32x2 FMA over pairs of cells fed by
// 16-byte shared loads (each half rounds like fmaf). Padding cells pass faces
// through. Faces between tiles live in octant-local lane-major blocks, so a
// tile's incoming faces are a flat copy of what its upstream neighbour wrote.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long f2pack(float lo, float hi)
{
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}

__device__ __forceinline__ void f2unpack(unsigned long long v, float& lo, float& hi)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}

__device__ __forceinline__ unsigned long long ffma2(unsigned long long a, unsigned long long b,
                                                    unsigned long long c)
{
    unsigned long long r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}

__device__ __forceinline__ unsigned long long fadd2(unsigned long long a, unsigned long long b)
{
    unsigned long long r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}

__device__ __forceinline__ void cp_async8(void* smem_dst, const void* gsrc)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(s), "l"(gsrc) : "memory");
}

__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gsrc)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

template <int NDO, int K, int BX, bool PSI = false, bool QIN = false>
struct BatchShape {
    static constexpr int BY = 4, BZ = 4, BV = BX * BY * BZ, NLINE = BY * BZ;
    static constexpr int SB = 32 / NDO, NL = SB * NDO;  // sources per warp, busy lanes
    static constexpr int NQ = BX / 4;                   // 4-cell quads per line
    static constexpr int TSTR = K * BX + 4;             // staged moments of a source, [K][BX] + pad
    static constexpr int PSTR = NDO * BX + 4;           // line fluxes of a source, [NDO][BX] + pad
    static constexpr int NH = 32 / K;                   // phase-C lane groups (lane = moment + K * group)
    static constexpr int NITEM = SB * NQ;               // phase-C (source, quad) items per line
    static constexpr int NJ = (NITEM + NH - 1) / NH;    // items per lane group
    static constexpr int NCP = (SB * K * NQ + 31) / 32; // 16-byte cp.async chunks per lane per line
    static constexpr bool PRE_CP = NCP <= 4, PRE_C = NJ <= 4;   // keep per-lane offsets in registers
    static constexpr int fxn = BY * BZ, fyn = BX * BZ, fzn = BX * BY;
    // float offsets
    // [SB][TSTR] the line being swept, refilled after phase A; with the Q input instead a ring of
    // QRING lines of the lanes' sources, [QRING][32][BX]
    static constexpr int QRING = 2;
    static constexpr int oT = 0;
    static constexpr int oP = oT + (QIN ? QRING * 32 * BX : SB * TSTR);   // [SB][PSTR]
    // [fxn][32] x faces, slot = local line (with the Q input the x-faces stay in registers and go
    // to and from the face block line by line)
    static constexpr int oX = oP + (PSI ? 0 : SB * PSTR);
    static constexpr int oY = oX + (QIN ? 0 : fxn * 32);    // [BX][32] y faces of one z-layer, slot = lx
    static constexpr int oZ = oY + BX * 32;             // [fzn][32] z faces, slot = ly * BX + lx
    static constexpr int oS = oZ + fzn * 32;            // [NLINE][BX] sigma_t, local line, storage x
    // with the Q input, four mbarriers (8 bytes each): the faces' bulk copies (tile prologue, y layers)
    // and the Q ring's two slots
    static constexpr int oB = (oS + BV + 3) & ~3;
    static constexpr int nF = oB + (QIN ? 8 : 0);
    static constexpr uint32_t QBOX = 4u * BX * NL;      // bytes of one line's Q box (lanes 0..NL-1)
    static constexpr size_t bytes = sizeof(float) * nF;
};

template <int NDO, int K, int BX, bool PSI, bool QIN = false>
__host__ __device__ constexpr size_t sweep_batch_smem() { return BatchShape<NDO, K, BX, PSI, QIN>::bytes; }

// Face buffers of the batched kernel: per (octant, source group, tile column)
// one block of F slots x 32 lanes, in the octant-local frame of the sweep.
__host__ __device__ inline size_t batch_face_floats(int n_groups, int columns, int F)
{
    return (size_t)8 * n_groups * columns * F * 32;
}

template <int F>
__device__ __forceinline__ void batch_faces_in(float* sh, const float* g, bool upstream)
{
    for (int j = threadIdx.x; j < F * 8; j += 32) {
        const float4 v = upstream ? *reinterpret_cast<const float4*>(g + 4 * j) : make_float4(0.f, 0.f, 0.f, 0.f);
        *reinterpret_cast<float4*>(sh + 4 * j) = v;
    }
}

// the same copy issued as cp.async (completed by the caller's wait on the group)
template <int F>
__device__ __forceinline__ void batch_faces_in_async(float* sh, const float* g, bool upstream)
{
    for (int j = threadIdx.x; j < F * 8; j += 32) {
        if (upstream) cp_async16(sh + 4 * j, g + 4 * j);
        else *reinterpret_cast<float4*>(sh + 4 * j) = make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

template <int F>
__device__ __forceinline__ void batch_faces_out(const float* sh, float* g)
{
    for (int j = threadIdx.x; j < F * 8; j += 32)
        *reinterpret_cast<float4*>(g + 4 * j) = *reinterpret_cast<const float4*>(sh + 4 * j);
}

// Set-to-zero fixup of one cell (FP32), entered with the plain diamond-
// difference result: faces found negative are fixed at zero and enter the
// balance with half weight; at most three passes.
__device__ __forceinline__ void batch_fixup(float qv, float sig, float ax, float ay, float az, float xin,
                                            float yin, float zin, float& psi, float& ox, float& oy, float& oz)
{
    bool fxd = false, fyd = false, fzd = false;
#pragma unroll 1
    for (int pass = 0; pass < 3; ++pass) {
        const bool nx = !fxd && ox < 0.f, ny = !fyd && oy < 0.f, nz = !fzd && oz < 0.f;
        if (!(nx || ny || nz)) break;
        fxd |= nx;
        fyd |= ny;
        fzd |= nz;
        const float num = qv + (fxd ? 0.5f * ax : ax) * xin + (fyd ? 0.5f * ay : ay) * yin +
                          (fzd ? 0.5f * az : az) * zin;
        const float den = sig + (fxd ? 0.f : ax) + (fyd ? 0.f : ay) + (fzd ? 0.f : az);
        psi = __fdividef(num, den);
        ox = fxd ? 0.f : 2.f * psi - xin;
        oy = fyd ? 0.f : 2.f * psi - yin;
        oz = fzd ? 0.f : 2.f * psi - zin;
    }
}

// The same fixup run by the whole warp (the Q-input walk, whose kernel is small enough for the longer
// code): pass 1 fixes the faces found negative in the plain solve, further passes run while a vote finds
// a free face of some lane negative; a lane with nothing new in a pass keeps its values bit for bit. A
// fixed face's term leaves the numerator by halves (num: the plain solve's numerator), and the
// denominator is formed again from the free faces. Measured against the divergent form on the 96^3 and
// 48^3 workloads: 2.4 % and 3.9 % less sweep time.
__device__ __forceinline__ void fixup_solve(float num, float sig, float ax, float ay, float az, bool fx, bool fy,
                                            bool fz, float xin, float yin, float zin, float& psi, float& ox,
                                            float& oy, float& oz)
{
    psi = __fdividef(num, sig + (((fx ? 0.f : ax) + (fy ? 0.f : ay)) + (fz ? 0.f : az)));
    ox = fmaf(2.f, psi, -xin);
    oy = fmaf(2.f, psi, -yin);
    oz = fmaf(2.f, psi, -zin);
}

__device__ __forceinline__ void batch_fixup_u(float num, float sig, float ax, float ay, float az, float xin,
                                              float yin, float zin, float& psi, float& ox, float& oy, float& oz)
{
    // pass 1 (the caller's vote found a sign bit set; a -0 outflow is not negative and changes nothing)
    bool fx = ox < 0.f, fy = oy < 0.f, fz = oz < 0.f;   // faces fixed at zero
    if (fx || fy || fz) {
        if (fx) num = fmaf(-0.5f * ax, xin, num);
        if (fy) num = fmaf(-0.5f * ay, yin, num);
        if (fz) num = fmaf(-0.5f * az, zin, num);
        fixup_solve(num, sig, ax, ay, az, fx, fy, fz, xin, yin, zin, psi, ox, oy, oz);
    }
    // passes 2 and 3 (ox, oy, oz: the latest solve's raw outflows 2 psi - psi_in)
#pragma unroll 1
    for (int pass = 1; pass < 3; ++pass) {
        const bool nx = !fx && ox < 0.f, ny = !fy && oy < 0.f, nz = !fz && oz < 0.f;
        const bool nw = nx || ny || nz;
        if (!__any_sync(0xffffffffu, nw)) break;
        if (nw) {
            if (nx) num = fmaf(-0.5f * ax, xin, num);
            if (ny) num = fmaf(-0.5f * ay, yin, num);
            if (nz) num = fmaf(-0.5f * az, zin, num);
            fx |= nx;
            fy |= ny;
            fz |= nz;
            fixup_solve(num, sig, ax, ay, az, fx, fy, fz, xin, yin, zin, psi, ox, oy, oz);
        }
    }
    ox = fx ? 0.f : ox;
    oy = fy ? 0.f : oy;
    oz = fz ? 0.f : oz;
}

// One x-line of phase B. Cells in upwind (local) order lx; q and psi in
// storage x order sx. CHECK: the line has padding cells (mask vm over sx).
// UF: the warp-uniform fixup (the Q-input walk) instead of the divergent one.
template <int BX, bool NX, bool CHECK, bool UF = false>
__device__ __forceinline__ void batch_line(float (&qv)[BX], float (&yv)[BX], float* zrow, const float* srow,
                                           float& xin, unsigned vm, float ax, float ay, float az, float asum)
{
    // the line's z-faces and sigma_t go to registers first, off the cell-to-cell chain
    float zv[BX], sv[BX];
#pragma unroll
    for (int lx = 0; lx < BX; ++lx) zv[lx] = zrow[lx * 32];
#pragma unroll
    for (int h = 0; h < BX / 4; ++h) {
        const float4 s4 = *reinterpret_cast<const float4*>(srow + 4 * h);
        sv[4 * h] = s4.x;
        sv[4 * h + 1] = s4.y;
        sv[4 * h + 2] = s4.z;
        sv[4 * h + 3] = s4.w;
    }
#pragma unroll
    for (int lx = 0; lx < BX; ++lx) {
        const int sx = NX ? BX - 1 - lx : lx;
        const float yin = yv[lx], zin = zv[lx];
        float psi, ox, oy, oz;
        if (!CHECK || (vm >> sx & 1u)) {
            const float q = qv[sx], sig = sv[sx];
            const float num = fmaf(ax, xin, fmaf(ay, yin, fmaf(az, zin, q)));
            psi = __fdividef(num, sig + asum);
            ox = fmaf(2.f, psi, -xin);
            oy = fmaf(2.f, psi, -yin);
            oz = fmaf(2.f, psi, -zin);
            // any sign bit set (a -0 outflow only enters the fixup to leave it unchanged)
            const bool neg = (__float_as_int(ox) | __float_as_int(oy) | __float_as_int(oz)) < 0;
            if (__any_sync(0xffffffffu, neg)) {
                if constexpr (UF) batch_fixup_u(num, sig, ax, ay, az, xin, yin, zin, psi, ox, oy, oz);
                else if (neg) batch_fixup(q, sig, ax, ay, az, xin, yin, zin, psi, ox, oy, oz);
            }
        } else {
            psi = 0.f;
            ox = xin;
            oy = yin;
            oz = zin;
        }
        qv[sx] = psi;
        yv[lx] = oy;
        zrow[lx * 32] = oz;
        xin = ox;
    }
}

template <int NDO, int K, int BX, bool PSI, bool NX, bool QIN>
__device__ __forceinline__ void sweep_batch_body(const SweepParams<float>& p, const CUtensorMap* qmap,
                                                 const int oct, const int grp,
                                                 const int ta, const int tb, const int tc, const unsigned okmask,
                                                 const float (&mrow)[K], const float (&arow)[3])
{
    using S = BatchShape<NDO, K, BX, PSI, QIN>;
    static_assert(!QIN || PSI, "the per-direction source input goes with the angular-flux output");
    constexpr int BY = S::BY, BZ = S::BZ, BV = S::BV, SB = S::SB, NL = S::NL, NQ = S::NQ;
    constexpr int TSTR = S::TSTR, PSTR = S::PSTR, NH = S::NH, NJ = S::NJ, NCP = S::NCP;
    constexpr int fxn = S::fxn, fyn = S::fyn, fzn = S::fzn;
    extern __shared__ __align__(128) float smf[];
    float* Tst = smf + S::oT;
    float* Ps = smf + S::oP;
    float* fx = smf + S::oX;
    float* fy = smf + S::oY;
    float* fz = smf + S::oZ;
    float* sg = smf + S::oS;
    uint64_t* bars = reinterpret_cast<uint64_t*>(smf + S::oB);   // Q input: [0] tile prologue, [1] y layers,
                                                                  // [2], [3] the Q ring's slots

    const int lane = threadIdx.x;
    const int b0 = grp * SB, nb = min(SB, p.B - b0);
    const int ngrp = (p.B + SB - 1) / SB;
    // x runs against storage order in odd octants: with the Q input the line data (Q, sigma_t, psi) are
    // kept in the octant's own x order, so one body serves every octant (NX false) and negx is a value
    const bool negx = QIN ? (oct & 1) != 0 : NX;
    const bool negy = oct & 2, negz = oct & 4;
    const int tx = negx ? p.NTx - 1 - ta : ta;
    const int ty = negy ? p.NTy - 1 - tb : tb;
    const int tz = negz ? p.NTz - 1 - tc : tc;
    const int tile = (tz * p.NTy + ty) * p.NTx + tx;
    const int n0 = oct * NDO;
    const int NTKB = p.NT * K * BV;                 // stride between sources (fits: checked on the host)
    const float* Tbase = p.T + ((size_t)b0 * p.NT + tile) * (size_t)(K * BV);
    float* obase = p.part + (((size_t)oct * p.B + b0) * p.NT + tile) * (size_t)(K * BV);
#ifdef DTS_DEBUG_BOUNDS
    {
        // every region the warp touches: sigma_t and the faces of the tile, the lanes' rows
        const int bl_ = lane / NDO, d_ = lane - bl_ * NDO;
        const bool src_ = lane < NL && (okmask >> bl_ & 1u);
        const size_t og_ = (size_t)oct * ngrp + grp;
        bool ok = tx < p.NTx && ty < p.NTy && tz < p.NTz && b0 + nb <= p.B;
        ok = DTS_FITS((size_t)(tile + 1) * BV, p.n_sigt, 2) && ok;
        ok = DTS_FITS(((og_ * (p.NTy * p.NTz) + (tz * p.NTy + ty)) * fxn + fxn) * 32, p.n_xf, 3) && ok;
        ok = DTS_FITS(((og_ * (p.NTx * p.NTz) + (tz * p.NTx + tx)) * fyn + fyn) * 32, p.n_yf, 4) && ok;
        ok = DTS_FITS(((og_ * (p.NTx * p.NTy) + (ty * p.NTx + tx)) * fzn + fzn) * 32, p.n_zf, 5) && ok;
        if (src_) {
            const size_t row = ((((size_t)(b0 + bl_) * 8 + oct) * p.NT + tile) * NDO + d_) * BV;
            if (PSI) ok = DTS_FITS(row + BV, p.n_part, 6) && ok;
            if (QIN) ok = DTS_FITS(row + BV, p.n_T, 7) && ok;
            if (!QIN) ok = DTS_FITS(((size_t)(b0 + bl_) * p.NT + tile + 1) * (size_t)(K * BV), p.n_T, 8) && ok;
            if (!PSI)
                ok = DTS_FITS((((size_t)oct * p.B + b0 + bl_) * p.NT + tile + 1) * (size_t)(K * BV), p.n_part, 9) && ok;
            if (d_ == 0 && p.leak) ok = DTS_FITS(((size_t)(b0 + bl_) * 8 + oct) * p.NT + tile + 1, p.n_leak, 10) && ok;
        }
        if (!__all_sync(0xffffffffu, ok)) return;
    }
#endif

    // cp.async chunks of one line: u -> (source il, moment k, quad h)
    auto chunk = [&](int c, int& src, int& dst) {
        const int u = lane + 32 * c;
        const int il = u / (K * NQ), r = u - il * (K * NQ), k = r / NQ, h = r - k * NQ;
        const bool ok = u < SB * K * NQ && il < nb && (okmask >> il & 1u);
        src = ok ? il * NTKB + k * BV + 4 * h : -1;
        dst = il * TSTR + k * BX + 4 * h;
    };
    int csrc[S::PRE_CP ? NCP : 1], cdst[S::PRE_CP ? NCP : 1];
    if constexpr (S::PRE_CP && !QIN) {
#pragma unroll
        for (int c = 0; c < NCP; ++c) chunk(c, csrc[c], cdst[c]);
    }
    auto stage_line = [&](int line, int buf) {
        const int ly = line % BY, lz = line / BY;
        const int sy = negy ? BY - 1 - ly : ly, sz = negz ? BZ - 1 - lz : lz;
        const int lbase = (sz * BY + sy) * BX;
        float* dbase = Tst + buf * SB * TSTR;
#pragma unroll
        for (int c = 0; c < NCP; ++c) {
            int src, dst;
            if constexpr (S::PRE_CP) {
                src = csrc[c];
                dst = cdst[c];
            } else {
                chunk(c, src, dst);
            }
            if (src >= 0) cp_async16(dbase + dst, Tbase + src + lbase);
        }
        cp_async_commit();
    };
    if constexpr (!QIN) stage_line(0, 0);

    // phase A/B lane: (source bl, direction d)
    const int bl = lane / NDO, d = lane - bl * NDO;
    const bool srcok = lane < NL && (okmask >> bl & 1u);
    unsigned long long m2[QIN ? 1 : K];
    if constexpr (!QIN) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const float m = srcok ? mrow[k] : 0.f;
            m2[k] = f2pack(m, m);
        }
    }
    const float ax = srcok ? arow[0] : 0.f, ay = srcok ? arow[1] : 0.f, az = srcok ? arow[2] : 0.f;
    const float asum = ax + ay + az;
    const float* trow = Tst + (srcok ? bl : 0) * TSTR;
    float* prow = Ps + (srcok ? bl : 0) * PSTR + d * BX;
    const size_t lane_ofs = ((((size_t)(b0 + (srcok ? bl : 0)) * 8 + oct) * p.NT + tile) * NDO + d) * BV;
    float* psi_lane = p.part + lane_ofs;
    // Q input: the line's per-direction source Q[b][oct][tile][d][cell] of the warp's sources (BX
    // floats per lane), landed one line ahead into a slot of a two-line ring by one tensor-map TMA issued
    // by lane 0: the box {BX cells, NDO directions, 1, SB sources} arrives in lane order (lane = source x
    // NDO + direction); sources past B arrive as zeros. Lanes of sources that have stopped iterating sweep
    // their last Q (valid values; nothing of theirs is stored).
    auto stage_q = [&](int line) {
        if (lane != 0) return;
        const int ly = line % BY, lz = line / BY;
        const int sy = negy ? BY - 1 - ly : ly, sz = negz ? BZ - 1 - lz : lz;
        uint64_t* qb = &bars[2 + (line & 1)];
        fence_async_smem();   // the slot's earlier reads (ordered by the caller's __syncwarp) come first
        mbar_expect_tx(qb, S::QBOX);
        tma_load_4d(Tst + (line % S::QRING) * 32 * BX, qmap, (sz * BY + sy) * BX, 0, oct * p.NT + tile, b0, qb);
    };
    if constexpr (QIN) {
        if (lane == 0) {   // every mbarrier of the tile, before the first copy is issued
#pragma unroll
            for (int i = 0; i < 4; ++i) mbar_init(&bars[i], 1);
            fence_mbar_init();
        }
        // the ring's TMA destination must be 128-byte aligned: a shared window that is not (never seen)
        // ends the tile before any copy, with the error word set
        if ((smem_addr(Tst) & 127u) != 0u) {
            if (lane == 0 && p.err) atomicExch(p.err, 1);
            return;
        }
        // the lanes past the warp's sources (no copy writes their slots) sweep zeros
        if (lane >= NL) {
#pragma unroll
            for (int r = 0; r < S::QRING; ++r)
#pragma unroll
                for (int h = 0; h < BX / 4; ++h)
                    *reinterpret_cast<float4*>(Tst + (r * 32 + lane) * BX + 4 * h) = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        stage_q(0);
    }

    // phase C lane: (moment kc, group h); items (source il, quad qd) = h + NH * j
    const int kc = lane % K, hc = lane / K;
    unsigned long long dk[PSI ? 1 : NDO];
    if constexpr (!PSI) {
#pragma unroll
        for (int dd = 0; dd < NDO; ++dd) {
            const float v = hc < NH ? p.Dt[(n0 + dd) * K + kc] : 0.f;
            dk[dd] = f2pack(v, v);
        }
    }
    auto citem = [&](int j, int& pofs, int& oofs) {
        const int item = hc + NH * j;
        const int il = item / NQ, qd = item - il * NQ;
        const bool ok = hc < NH && item < S::NITEM && il < nb && (okmask >> il & 1u);
        pofs = il * PSTR + 4 * qd;
        oofs = ok ? il * NTKB + kc * BV + 4 * qd : -1;
    };
    int cp_[S::PRE_C ? NJ : 1], co_[S::PRE_C ? NJ : 1];
    if constexpr (S::PRE_C && !PSI) {
#pragma unroll
        for (int j = 0; j < NJ; ++j) citem(j, cp_[j], co_[j]);
    }

    {
        const float* st = p.sigt + (size_t)tile * BV;
        for (int i = lane; i < BV / 4; i += 32) {
            const int srow = i / NQ, h = i - srow * NQ;
            const int sy = srow % BY, sz = srow / BY;
            const int ly = negy ? BY - 1 - sy : sy, lz = negz ? BZ - 1 - sz : sz;
            if (QIN && negx) {   // the line's cells in the octant's x order: quads reversed, and inside them
                float4 v = *reinterpret_cast<const float4*>(st + srow * BX + 4 * h);
                v = make_float4(v.w, v.z, v.y, v.x);
                *reinterpret_cast<float4*>(sg + (lz * BY + ly) * BX + 4 * (NQ - 1 - h)) = v;
            } else {
                cp_async16(sg + (lz * BY + ly) * BX + 4 * h, st + srow * BX + 4 * h);   // with the faces' group
            }
        }
    }
    const size_t og = (size_t)oct * ngrp + grp;
    float* gx = p.xf + ((og * (p.NTy * p.NTz) + (tz * p.NTy + ty)) * fxn) * 32;
    float* gy = p.yf + ((og * (p.NTx * p.NTz) + (tz * p.NTx + tx)) * fyn) * 32;
    float* gz = p.zf + ((og * (p.NTx * p.NTy) + (ty * p.NTx + tx)) * fzn) * 32;
    if constexpr (QIN) {
        // the tile's incoming z-faces and z-layer 0's y-faces: one bulk copy (TMA) each from their
        // contiguous face blocks, issued by lane 0 on bars[0]; on an inflow boundary the lanes write zeros
        if (lane == 0) {
            mbar_expect_tx(&bars[0], (tc > 0 ? fzn * 128u : 0u) + (tb > 0 ? BX * 128u : 0u) + p.poison_tx);
            if (tc > 0) bulk_load(fz, gz, fzn * 128u, &bars[0]);
            if (tb > 0) bulk_load(fy, gy, BX * 128u, &bars[0]);
        }
        if (tc == 0) batch_faces_in_async<fzn>(fz, gz, false);   // zeros
        if (tb == 0) batch_faces_in_async<BX>(fy, gy, false);
    } else {
        batch_faces_in_async<fxn>(fx, gx, ta > 0);   // land with the first line's sources
        batch_faces_in_async<BX>(fy, gy, tb > 0);    // z-layer 0; later layers stream in with the lines
        batch_faces_in_async<fzn>(fz, gz, tc > 0);
    }
    cp_async_commit();
    float xn = 0.f, xsum = 0.f;   // Q input: the next line's incoming x-face; the outgoing ones' sum
    if constexpr (QIN) xn = ta > 0 ? gx[lane] : 0.f;

    const int nvx = p.nx - tx * BX, nvy = p.ny - ty * BY, nvz = p.nz - tz * BZ;
    constexpr unsigned FULL = (1u << BX) - 1u;
    // valid cells as bits of the line's cell index: storage x, or with the Q input in an odd octant the
    // octant's x (the valid storage cells 0..nvx-1 are the last nvx there)
    const unsigned vxs = nvx >= BX ? FULL : (QIN && negx) ? (FULL << (BX - nvx)) & FULL : (1u << nvx) - 1u;
    float yv[BX];
    float ysum = 0.f;   // the lane's outgoing y-faces (leakage when the tile is on the y boundary)

#pragma unroll 1
    for (int line = 0; line < S::NLINE; ++line) {
        // this line's sources (copied during the previous line's walk; with the Q input the cp.async
        // group is the prologue's sigma_t only)
        if (!QIN || line == 0) cp_async_wait0();
        __syncwarp();
        const int ly = line % BY, lz = line / BY;
        const int sy = negy ? BY - 1 - ly : ly, sz = negz ? BZ - 1 - lz : lz;
        if constexpr (QIN) {
            // this line's Q (ring slot line & 1, its (line >> 1)-th copy); at a layer's first line also the
            // faces: line 0 the tile's (bars[0]), later layers their y-faces (bars[1], the (lz - 1)-th copy
            // on it). A wait that gives up ends the sweep of the tile.
            uint64_t* qb = &bars[2 + (line & 1)];
            const uint32_t qpar = (uint32_t)((line >> 1) & 1);
            bool ok = mbar_wait(qb, qpar);
            uint64_t* fb = nullptr;
            uint32_t fpar = 0u;
            if (ly == 0 && (lz == 0 || tb > 0)) {
                fb = lz == 0 ? &bars[0] : &bars[1];
                fpar = lz == 0 ? 0u : (uint32_t)((lz - 1) & 1);
                ok = mbar_wait(fb, fpar) && ok;
            }
            if (!__all_sync(0xffffffffu, ok)) {
                if (lane == 0 && p.err) atomicExch(p.err, 1);
                (void)mbar_wait(qb, qpar);   // the copies, should they still land (bounded)
                if (fb) (void)mbar_wait(fb, fpar);
                __syncwarp();
                return;
            }
        }

        // A: Q for the line's cells, two cells per packed FMA, storage x order
        // (Q input: the line's sources were loaded during the previous line's walk)
        float qv[BX];
        if constexpr (QIN) {
            const float* src = Tst + ((line % S::QRING) * 32 + lane) * BX;
#pragma unroll
            for (int h = 0; h < BX / 4; ++h) {
                const float4 v = *reinterpret_cast<const float4*>(src + 4 * h);
                qv[4 * h] = v.x;
                qv[4 * h + 1] = v.y;
                qv[4 * h + 2] = v.z;
                qv[4 * h + 3] = v.w;
            }
        } else {
            const float* tr = trow;
#pragma unroll
            for (int qd = 0; qd < NQ; ++qd) {
                unsigned long long a0 = 0ull, a1 = 0ull;
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    const ulonglong2 t = *reinterpret_cast<const ulonglong2*>(tr + k * BX + 4 * qd);
                    a0 = ffma2(m2[k], t.x, a0);
                    a1 = ffma2(m2[k], t.y, a1);
                }
                f2unpack(a0, qv[4 * qd], qv[4 * qd + 1]);
                f2unpack(a1, qv[4 * qd + 2], qv[4 * qd + 3]);
            }
        }

        // the staged sources are consumed: every lane is past phase A, so the
        // next line's sources can land in the same buffer during the walk
        __syncwarp();
        // the layer's y-faces went to registers during line ly = 0; the next layer's land in the
        // same buffer with the next line's sources
        if constexpr (QIN) {
            // the next layer's y-faces (bulk copy on bars[1]) into the buffer whose values every lane read
            // into registers during line ly = 0 (ordered by the __syncwarp above)
            if (ly == 1 && lz + 1 < BZ && tb > 0 && lane == 0) {
                fence_async_smem();
                mbar_expect_tx(&bars[1], BX * 128u);
                bulk_load(fy, gy + (size_t)(lz + 1) * BX * 32, BX * 128u, &bars[1]);
            }
        } else {
            if (ly == 1 && lz + 1 < BZ) batch_faces_in_async<BX>(fy, gy + (size_t)(lz + 1) * BX * 32, tb > 0);
        }
        if constexpr (!QIN) {
            if (line + 1 < S::NLINE) stage_line(line + 1, 0);
        } else {
            if (line + 1 < S::NLINE) stage_q(line + 1);   // into the slot of the line before this one
        }

        // B: walk the line
        if (ly == 0) {
#pragma unroll
            for (int lx = 0; lx < BX; ++lx) yv[lx] = fy[lx * 32 + lane];
        }
        {
            const unsigned vm = (sy < nvy && sz < nvz) ? vxs : 0u;
            float* zrow = fz + ly * BX * 32 + lane;
            const float* srow = sg + line * BX;
            float xin;
            if constexpr (QIN) {
                xin = xn;
                if (line + 1 < S::NLINE) xn = ta > 0 ? gx[(line + 1) * 32 + lane] : 0.f;
            } else {
                xin = fx[line * 32 + lane];
            }
            if (vm == FULL) batch_line<BX, NX, false, QIN>(qv, yv, zrow, srow, xin, vm, ax, ay, az, asum);
            else batch_line<BX, NX, true, QIN>(qv, yv, zrow, srow, xin, vm, ax, ay, az, asum);
            if constexpr (QIN) {
                gx[line * 32 + lane] = xin;   // outgoing x-face, in place in the face block
                xsum += xin;
            } else {
                fx[line * 32 + lane] = xin;
            }
        }
        if (ly == BY - 1) {
#pragma unroll
            for (int lx = 0; lx < BX; ++lx) {
                gy[(lz * BX + lx) * 32 + lane] = yv[lx];   // outgoing y-faces straight to the face block
                ysum += yv[lx];
            }
        }
        if constexpr (PSI) {
            // the lane's angular fluxes of the line go straight to HBM: psi[b][oct][tile][d][cell]
            if (srcok) {
                float* dst = psi_lane + (sz * BY + sy) * BX;
#pragma unroll
                for (int qd = 0; qd < NQ; ++qd)
                    *reinterpret_cast<float4*>(dst + 4 * qd) =
                        make_float4(qv[4 * qd], qv[4 * qd + 1], qv[4 * qd + 2], qv[4 * qd + 3]);
            }
            continue;   // the staging buffer was released after phase A
        } else if (srcok) {
#pragma unroll
            for (int qd = 0; qd < NQ; ++qd)
                *reinterpret_cast<float4*>(prow + 4 * qd) =
                    make_float4(qv[4 * qd], qv[4 * qd + 1], qv[4 * qd + 2], qv[4 * qd + 3]);
        }
        __syncwarp();

        // C: lane = (moment, item): octant moment partial of four cells, two per packed FMA
        {
            const int lofs = (sz * BY + sy) * BX;
#pragma unroll
            for (int j = 0; j < NJ; ++j) {
                int pofs, oofs;
                if constexpr (S::PRE_C) {
                    pofs = cp_[j];
                    oofs = co_[j];
                } else {
                    citem(j, pofs, oofs);
                }
                if (oofs >= 0) {
                    const float* pr = Ps + pofs;
                    unsigned long long a0 = 0ull, a1 = 0ull;
#pragma unroll
                    for (int dd = 0; dd < NDO; ++dd) {
                        const ulonglong2 s2 = *reinterpret_cast<const ulonglong2*>(pr + dd * BX);
                        a0 = ffma2(dk[dd], s2.x, a0);
                        a1 = ffma2(dk[dd], s2.y, a1);
                    }
                    *reinterpret_cast<ulonglong2*>(obase + oofs + lofs) = make_ulonglong2(a0, a1);
                }
            }
        }
        __syncwarp();
    }

    // outgoing faces; the lane's own faces leaving the grid are its leakage
    if constexpr (QIN) {
        // the z-faces by one bulk store (TMA) once every lane's stores are visible to the async proxy
        fence_async_smem();
        __syncwarp();
        if (lane == 0) {
            bulk_store(gz, fz, fzn * 128u);
            bulk_commit();
        }
    } else {
        batch_faces_out<fxn>(fx, gx);
        batch_faces_out<fzn>(fz, gz);
    }
    const bool lbx = negx ? tx == 0 : tx == p.NTx - 1;
    const bool lby = negy ? ty == 0 : ty == p.NTy - 1;
    const bool lbz = negz ? tz == 0 : tz == p.NTz - 1;
    // the source's leakage from this (octant, tile): its direction lanes summed in direction order
    // into its slot, so that the per-source total is reproducible; zero away from the boundary
    double tot = 0.0;
    if (lbx || lby || lbz) {   // uniform across the warp
        double lk = 0.0;
        if (srcok) {
            float sx_ = 0.f, sy_ = 0.f, sz_ = 0.f;
            if (lbx) {
                if constexpr (QIN) sx_ = xsum;
                else
                    for (int e = 0; e < fxn; ++e) sx_ += fx[e * 32 + lane];
            }
            if (lby) sy_ = ysum;
            if (lbz)
                for (int e = 0; e < fzn; ++e) sz_ += fz[e * 32 + lane];
            lk = p.Lw[(n0 + d) * 3] * (double)sx_ + p.Lw[(n0 + d) * 3 + 1] * (double)sy_ +
                 p.Lw[(n0 + d) * 3 + 2] * (double)sz_;
        }
#pragma unroll
        for (int dd = 0; dd < NDO; ++dd) tot += __shfl_sync(0xffffffffu, lk, (srcok ? bl : 0) * NDO + dd);
    }
    if (srcok && d == 0 && p.leak) p.leak[((size_t)(b0 + bl) * 8 + oct) * p.NT + tile] = tot;
    if (QIN && lane == 0) bulk_wait_read();   // the store has read the z-faces before the CTA's memory goes
}

// s0, cnt: the stage's first entry in stage_tiles and its tile count (kernel
// arguments, so a CTA's first dependent global load is its tile)
template <int NDO, int K, int BX, bool PSI, bool QIN = false>
// qmap (the Q-input form only): tensor map of Q as 4-D {cell TV, direction NDO, octant x tile 8 NT,
// source B} (FP32), box {line BX, NDO, 1, sources per warp}, so that one TMA per line lands every
// lane's row in lane order
__global__ void __launch_bounds__(32, QIN ? 28 : 17) k_sweep_batch(const SweepParams<float> p, const int s0,
                                                                      const int cnt,
                                                                      const __grid_constant__ CUtensorMap qmap)
{
    using S = BatchShape<NDO, K, BX, PSI, QIN>;
    int bid = blockIdx.x;
    const int tl = bid % cnt;
    bid /= cnt;
    const int oct = bid & 7, grp = bid >> 3, b0 = grp * S::SB;
    // the loads that depend on nothing else go first: tile, lane operator row, source flags
    if (!DTS_FITS(s0 + tl + 1, p.n_stage_tiles, 1)) return;
    const unsigned pk = p.stage_tiles[s0 + tl];
    const int lane = threadIdx.x, d = lane % NDO;
    const bool dl = lane < S::NL;
    float mrow[K], arow[3];
#pragma unroll
    for (int k = 0; k < K; ++k) mrow[k] = (dl && !QIN) ? p.M[(oct * NDO + d) * K + k] : 0.f;
#pragma unroll
    for (int j = 0; j < 3; ++j) arow[j] = dl ? p.A[(oct * NDO + d) * 3 + j] : 0.f;
    const int nb = min(S::SB, p.B - b0);
    unsigned okmask = 0;                           // sources of this warp still iterating
    for (int i = 0; i < nb; ++i)
        if (p.active[b0 + i]) okmask |= 1u << i;
    if (okmask == 0) return;
    const int ta = pk & 1023, tb = (pk >> 10) & 1023, tc = (pk >> 20) & 1023;
    if constexpr (QIN) {   // one body: the octant's x order is in the data
        sweep_batch_body<NDO, K, BX, PSI, false, QIN>(p, &qmap, oct, grp, ta, tb, tc, okmask, mrow, arow);
    } else {
        if (oct & 1) sweep_batch_body<NDO, K, BX, PSI, true, QIN>(p, &qmap, oct, grp, ta, tb, tc, okmask, mrow, arow);
        else sweep_batch_body<NDO, K, BX, PSI, false, QIN>(p, &qmap, oct, grp, ta, tb, tc, okmask, mrow, arow);
    }
}

// Error-free FP32 accumulation (Knuth's two-sum): s + e carries the exact sum
// of the FP32 terms added so far (to within rounding of the small e), so the
// FP64 scalar flux (double)s + (double)e equals the octant sum to ~2^-48.
struct TwoSum {
    float s = 0.f, e = 0.f;
    __device__ __forceinline__ void add(float x)
    {
        const float t = __fadd_rn(s, x);
        const float bp = __fsub_rn(t, s);
        e = __fadd_rn(e, __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(x, bp)));
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s + (double)e; }
};

// The per-cell tail of the FP32 reductions: store the FP64 scalar flux, form
// T_0 = F_0 + sigma_s0 phi_00 in FP32, and accumulate this thread's residual
// and balance terms in FP32 (summed across a warp in FP32, across warps and
// blocks in FP64).
struct RedTail {
    float ds = 0.f, ns = 0.f, sr = 0.f, ab = 0.f;
    // s0 = (double)ts.s + (double)ts.e rounds to the same FP32 value as the pair's FP32 sum (the
    // FP64 sum is exact unless e is below 2^-29 of s, and then both round to s); the old flux
    // enters only the balance term, where its FP32 value may be off by an ulp
    __device__ __forceinline__ float cell(const TwoSum& ts, double s0, double old, float f0, float sl0, float st)
    {
        const float s0f = __fadd_rn(ts.s, ts.e), dd = (float)(s0 - old), oldf = s0f - dd;
        ds = fmaf(dd, dd, ds);
        ns = fmaf(s0f, s0f, ns);
        ab = fmaf(st, s0f, ab);
        sr += fmaf(sl0, oldf, f0);
        return fmaf(sl0, s0f, f0);
    }
};

// moment pairs of the Eq. 3 operator rows (an even count, so pairs of pairs load as 16 bytes)
template <int K> struct PsiPairs { static constexpr int value = ((K + 1) / 2 + 1) & ~1; };   // even

// Translation units that only launch the sweep define DTS_SWEEP_KERNEL_ONLY so
// that the solver's other (non-template) kernels are defined once per library.
#ifndef DTS_SWEEP_KERNEL_ONLY

// ---------------------------------------------------------------------------
// A5 + A6 (+ A10 terms): Eq. 3 octant sum of the scalar flux in FP64 (fixed
// order 0..7), the higher moments in the sweep precision R, the next source
// T = F + sigma_s^{gg} phi, and the residual and balance partial sums (FP64).
// ---------------------------------------------------------------------------
template <typename R>
struct RedParams {
    int B, NT, TV, NC;
    const R* part;
    double* phi00;             // [B][NC] scalar flux of the current group
    R* T;
    const R* F;
    size_t Fstride;
    const int* ctl;            // [0] group, [1] fixed-source slot
    const R* sigs;             // [L+1][NC] in-group scatter per cell
    const double* sigs0;       // [NC] l = 0 in-group scatter, FP64
    const double* sigt64;      // [NC]
    const R* sigt;             // [NC] sigma_t in the sweep precision
    const int* mat_t;          // [NC], -1 = padding
    const int* active;
    double vol;
    double* blk;               // [B][nblk][4]
#ifdef DTS_DEBUG_BOUNDS
    // element counts of part, T, F, phi00, sigs and blk (checked in the DTS_DEBUG_BOUNDS build only,
    // so that the normal build's parameters stay as they were)
    size_t n_part, n_T, n_F, n_phi00, n_sigs, n_blk;
#endif
};

template <typename R, int K>
__global__ void __launch_bounds__(kRedThreads) k_reduce(const RedParams<R> p)
{
    __shared__ double red[32];
    const int b = blockIdx.y;
    const int ct = blockIdx.x * blockDim.x + threadIdx.x;
    double ds = 0.0, ns = 0.0, sr = 0.0, ab = 0.0;
    const bool act = p.active[b] != 0;
    if (act && ct < p.NC) {
        const int tile = ct / p.TV, c = ct - tile * p.TV;
        const size_t base = ((size_t)b * p.NT + tile) * (size_t)(K * p.TV) + c;
        const size_t ostride = (size_t)p.B * p.NT * K * p.TV;
        const R* __restrict__ pp = p.part + base;
        R* __restrict__ T = p.T + base;
        double* __restrict__ ph = p.phi00 + (size_t)b * p.NC + ct;
        if (p.mat_t[ct] >= 0) {
            const R* __restrict__ F = p.F + (size_t)p.ctl[1] * p.Fstride + base;
            double s0 = 0.0;
#pragma unroll
            for (int o = 0; o < 8; ++o) s0 += (double)pp[o * ostride];
            const double old = *ph, sl0 = p.sigs0[ct], f0 = (double)F[0];
            const double dd = s0 - old;
            ds = dd * dd;
            ns = s0 * s0;
            ab = p.vol * p.sigt64[ct] * s0;
            sr = p.vol * (f0 + sl0 * old);
            *ph = s0;
            T[0] = (R)(f0 + sl0 * s0);
#pragma unroll
            for (int k = 1; k < K; ++k) {
                R s = R(0);
#pragma unroll
                for (int o = 0; o < 8; ++o) s += pp[o * ostride + (size_t)k * p.TV];
                T[(size_t)k * p.TV] = F[(size_t)k * p.TV] + p.sigs[(size_t)l_of_k(k) * p.NC + ct] * s;
            }
        } else {
            *ph = 0.0;
#pragma unroll
            for (int k = 0; k < K; ++k) T[(size_t)k * p.TV] = R(0);
        }
    }
    ds = block_sum(ds, red);
    ns = block_sum(ns, red);
    sr = block_sum(sr, red);
    ab = block_sum(ab, red);
    if (threadIdx.x == 0) {
        double* o = p.blk + ((size_t)b * gridDim.x + blockIdx.x) * 4;
        o[0] = ds;
        o[1] = ns;
        o[2] = sr;
        o[3] = ab;
    }
}

// The block's four partial sums: FP32 butterflies within each warp (FP64 runs
// at a small fraction of the FP32 rate on this part), one barrier, then the
// warps' totals added in FP64 by four threads.
__device__ __forceinline__ void red_tail_store(const RedParams<float>& p, const RedTail& t, double* red, int b,
                                               int blk, int nblk)
{
    static_assert(kRedThreads / 32 * 4 <= 32, "red[] holds four partials per warp");
    float v[4] = {t.ds, t.ns, t.sr, t.ab};
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int i = 0; i < 4; ++i) v[i] += __shfl_xor_sync(0xffffffffu, v[i], o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    if (lane == 0)
#pragma unroll
        for (int i = 0; i < 4; ++i) red[wid * 4 + i] = (double)v[i];
    __syncthreads();
    if (threadIdx.x < 4) {
        double acc = 0.0;
        for (int w = 0; w < nw; ++w) acc += red[w * 4 + threadIdx.x];
        double* o = p.blk + ((size_t)b * nblk + blk) * 4;
        o[threadIdx.x] = threadIdx.x < 2 ? acc : p.vol * acc;
    }
}

// The same reduction for FP32 sweeps, four consecutive cells per thread with
// 16-byte loads and stores (tile volumes that are multiples of 4).
template <int K>
__global__ void __launch_bounds__(kRedThreads) k_reduce4(const RedParams<float> p)
{
    __shared__ double red[32];
    const int b = blockIdx.y;
    const int c4 = (blockIdx.x * blockDim.x + threadIdx.x) * 4;
    RedTail tl;
    if (p.active[b] != 0 && c4 < p.NC) {
        const int tile = c4 / p.TV, c = c4 - tile * p.TV;
        const size_t base = ((size_t)b * p.NT + tile) * (size_t)(K * p.TV) + c;
        const size_t ostride = (size_t)p.B * p.NT * K * p.TV;
        const float* __restrict__ pp = p.part + base;
        float* __restrict__ T = p.T + base;
        const float* __restrict__ F = p.F + (size_t)p.ctl[1] * p.Fstride + base;
        double* __restrict__ ph = p.phi00 + (size_t)b * p.NC + c4;
        const int4 m4 = *reinterpret_cast<const int4*>(p.mat_t + c4);
        const int mm[4] = {m4.x, m4.y, m4.z, m4.w};
        TwoSum s0[4];
#pragma unroll
        for (int o = 0; o < 8; ++o) {
            const float4 v = *reinterpret_cast<const float4*>(pp + o * ostride);
            s0[0].add(v.x);
            s0[1].add(v.y);
            s0[2].add(v.z);
            s0[3].add(v.w);
        }
        const float4 f0 = *reinterpret_cast<const float4*>(F);
        const float4 sl0 = *reinterpret_cast<const float4*>(p.sigs + c4);
        const float4 st = *reinterpret_cast<const float4*>(p.sigt + c4);
        const double2 o01 = *reinterpret_cast<const double2*>(ph), o23 = *reinterpret_cast<const double2*>(ph + 2);
        const float ff[4] = {f0.x, f0.y, f0.z, f0.w}, sl[4] = {sl0.x, sl0.y, sl0.z, sl0.w};
        const float sg[4] = {st.x, st.y, st.z, st.w};
        const double old[4] = {o01.x, o01.y, o23.x, o23.y};
        double phi[4];
        float t0[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (mm[j] < 0) {
                phi[j] = 0.0;
                t0[j] = 0.f;
                continue;
            }
            phi[j] = s0[j].value();
            t0[j] = tl.cell(s0[j], phi[j], old[j], ff[j], sl[j], sg[j]);
        }
        *reinterpret_cast<double2*>(ph) = make_double2(phi[0], phi[1]);
        *reinterpret_cast<double2*>(ph + 2) = make_double2(phi[2], phi[3]);
        *reinterpret_cast<float4*>(T) = make_float4(t0[0], t0[1], t0[2], t0[3]);
#pragma unroll
        for (int k = 1; k < K; ++k) {
            float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int o = 0; o < 8; ++o) {
                const float4 v = *reinterpret_cast<const float4*>(pp + o * ostride + (size_t)k * p.TV);
                acc.x += v.x;
                acc.y += v.y;
                acc.z += v.z;
                acc.w += v.w;
            }
            const float4 f = *reinterpret_cast<const float4*>(F + (size_t)k * p.TV);
            const float4 sk = *reinterpret_cast<const float4*>(p.sigs + (size_t)l_of_k(k) * p.NC + c4);
            *reinterpret_cast<float4*>(T + (size_t)k * p.TV) =
                make_float4(fmaf(sk.x, acc.x, f.x), fmaf(sk.y, acc.y, f.y), fmaf(sk.z, acc.z, f.z), fmaf(sk.w, acc.w, f.w));
        }
    }
    red_tail_store(p, tl, red, b, blockIdx.x, gridDim.x);
}

// Eq. 3 and its higher moments from the angular fluxes written by the batched
// sweep's direct-output form, psi[b][octant][tile][direction][cell], for two
// consecutive tiled cells. The moment operator is read as pairs of moments
// (D[n][2j], D[n][2j+1]) so that one 16-byte shared load feeds four packed
// FMAs. Each octant's directions are summed in FP32; the scalar flux takes
// those octant sums exactly (two-sum) in octant order 0..7, the higher
// moments stay in FP32.

// the first octant's copies of psi_moments (buffer 0), for callers that start them early
template <int NDO>
__device__ __forceinline__ void psi_issue_first(const float* __restrict__ ps, int TV, unsigned long long* stg)
{
    const int nt = blockDim.x;
#pragma unroll
    for (int d = 0; d < NDO; ++d) cp_async8(stg + d * nt, ps + (size_t)d * TV);
    cp_async_commit();
}

// flip: 0, or for angular fluxes whose odd octants are stored in the octant's own x order (the
// tensor-core forms' sweep) the offset of the cell pair there, (c ^ 6) - c, whose two values are swapped
template <int NDO, int K, bool ISSUED = false>
__device__ __forceinline__ void psi_moments(const float* __restrict__ ps, size_t ostride, int TV,
                                            const unsigned long long* Dp, unsigned long long* stg,
                                            TwoSum (&s0)[2], float (&m1)[2],
                                            unsigned long long (&acc)[2][PsiPairs<K>::value], int flip = 0)
{
    // stg: this thread's column of a [2][NDO][blockDim.x] staging area; the next
    // octant's fluxes are copied with cp.async while this one is reduced, so the
    // loads in flight hold no registers (each thread reads only its own copies)
    constexpr int KP = PsiPairs<K>::value;
    const int nt = blockDim.x;
    m1[0] = m1[1] = 0.f;
#pragma unroll
    for (int j = 0; j < KP; ++j) acc[0][j] = acc[1][j] = 0ull;
    auto issue = [&](int o) {
        unsigned long long* dst = stg + (o & 1) * NDO * nt;
        const float* po = ps + o * ostride + ((o & 1) ? flip : 0);
#pragma unroll
        for (int d = 0; d < NDO; ++d) cp_async8(dst + d * nt, po + (size_t)d * TV);
        cp_async_commit();
    };
    if (!ISSUED) issue(0);
#pragma unroll 1
    for (int o = 0; o < 8; ++o) {
        if (o + 1 < 8) issue(o + 1);
        else cp_async_commit();
        cp_async_wait1();
        const unsigned long long* src = stg + (o & 1) * NDO * nt;
        unsigned long long f0[2] = {0ull, 0ull};   // moments (0, 1) of this octant
#pragma unroll
        for (int d = 0; d < NDO; ++d) {
            const unsigned long long v = src[d * nt];
            float p0, p1;
            f2unpack(v, p0, p1);
            if (flip != 0 && (o & 1)) {
                const float t = p0;
                p0 = p1;
                p1 = t;
            }
            const unsigned long long a = f2pack(p0, p0), bq = f2pack(p1, p1);
            const ulonglong2* dq = reinterpret_cast<const ulonglong2*>(Dp + (o * NDO + d) * KP);
#pragma unroll
            for (int j = 0; j < KP / 2; ++j) {
                const ulonglong2 dd = dq[j];
                if (j == 0) {
                    f0[0] = ffma2(dd.x, a, f0[0]);
                    f0[1] = ffma2(dd.x, bq, f0[1]);
                } else {
                    acc[0][2 * j] = ffma2(dd.x, a, acc[0][2 * j]);
                    acc[1][2 * j] = ffma2(dd.x, bq, acc[1][2 * j]);
                }
                acc[0][2 * j + 1] = ffma2(dd.y, a, acc[0][2 * j + 1]);
                acc[1][2 * j + 1] = ffma2(dd.y, bq, acc[1][2 * j + 1]);
            }
        }
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            float lo, hi;
            f2unpack(f0[c], lo, hi);
            s0[c].add(lo);
            m1[c] += hi;
        }
    }
}

// moment k >= 1 of cell c from psi_moments' accumulators
template <int K>
__device__ __forceinline__ float psi_moment(int k, int c, const float (&m1)[2],
                                            const unsigned long long (&acc)[2][PsiPairs<K>::value])
{
    if (k == 1) return m1[c];
    float lo, hi;
    f2unpack(acc[c][k / 2], lo, hi);
    return (k & 1) ? hi : lo;
}

template <int NDO, int K>
__device__ __forceinline__ void load_dpairs(unsigned long long* Dp, const float* Dt)
{
    constexpr int KP = PsiPairs<K>::value;
    for (int i = threadIdx.x; i < 8 * NDO * KP; i += blockDim.x) {
        const int n = i / KP, j = i - n * KP;
        const float lo = 2 * j < K ? Dt[n * K + 2 * j] : 0.f, hi = 2 * j + 1 < K ? Dt[n * K + 2 * j + 1] : 0.f;
        Dp[i] = f2pack(lo, hi);
    }
    __syncthreads();
}

// A5 + A6 for the direct-output form: moments from psi, then T = F + sigma_s phi,
// the FP64 scalar flux, and the residual and balance partials as k_reduce4.
template <int NDO, int K>
__global__ void __launch_bounds__(kRedThreads, 4) k_reduce_psi(const RedParams<float> p, const float* __restrict__ Dt)
{
    __shared__ __align__(16) unsigned long long Dp[8 * NDO * PsiPairs<K>::value];
    __shared__ unsigned long long stg[2 * NDO * kRedThreads];
    __shared__ double red[32];
    const int b = blockIdx.y;
    const int c2 = (blockIdx.x * blockDim.x + threadIdx.x) * 2;
#ifdef DTS_DEBUG_BOUNDS
    bool live = p.active[b] != 0 && c2 < p.NC;
#else
    const bool live = p.active[b] != 0 && c2 < p.NC;
#endif
    const int tile = c2 / p.TV, c = c2 - tile * p.TV;
    const size_t ostride = (size_t)p.NT * NDO * p.TV;
    const size_t pofs = (size_t)b * 8 * ostride + (size_t)tile * NDO * p.TV + c;
#ifdef DTS_DEBUG_BOUNDS
    if (live) {   // the pair of cells' regions in every buffer
        const size_t base = ((size_t)b * p.NT + tile) * (size_t)(K * p.TV) + c;
        bool ok = DTS_FITS(pofs + 7 * ostride + (size_t)(NDO - 1) * p.TV + 2, p.n_part, 30);
        ok = DTS_FITS(base + (size_t)(K - 1) * p.TV + 2, p.n_T, 31) && ok;
        ok = DTS_FITS((size_t)p.ctl[1] * p.Fstride + base + (size_t)(K - 1) * p.TV + 2, p.n_F, 32) && ok;
        ok = DTS_FITS((size_t)b * p.NC + c2 + 2, p.n_phi00, 33) && ok;
        ok = DTS_FITS((size_t)l_of_k(K - 1) * p.NC + c2 + 2, p.n_sigs, 34) && ok;
        ok = DTS_FITS((size_t)c2 + 2, (size_t)p.NC, 35) && ok;
        live = ok;
    }
    if (!DTS_FITS(((size_t)b * gridDim.x + blockIdx.x + 1) * 4, p.n_blk, 36)) return;   // uniform per block
#endif
    // the first octant's fluxes are in flight while the block loads its moment operator
    if (live) psi_issue_first<NDO>(p.part + pofs, p.TV, stg + threadIdx.x);
    load_dpairs<NDO, K>(Dp, Dt);
    RedTail tl;
    if (live) {
        const size_t base = ((size_t)b * p.NT + tile) * (size_t)(K * p.TV) + c;
        const float* ps = p.part + pofs;
        TwoSum s0[2];
        float m1[2];
        unsigned long long acc[2][PsiPairs<K>::value];
        psi_moments<NDO, K, true>(ps, ostride, p.TV, Dp, stg + threadIdx.x, s0, m1, acc);
        float* __restrict__ T = p.T + base;
        const float* __restrict__ F = p.F + (size_t)p.ctl[1] * p.Fstride + base;
        double* __restrict__ ph = p.phi00 + (size_t)b * p.NC + c2;
        const int2 mv = *reinterpret_cast<const int2*>(p.mat_t + c2);
        const int mm[2] = {mv.x, mv.y};
        const float2 f0 = *reinterpret_cast<const float2*>(F);
        const float2 sl0 = *reinterpret_cast<const float2*>(p.sigs + c2);
        const float2 st = *reinterpret_cast<const float2*>(p.sigt + c2);
        const double2 od = *reinterpret_cast<const double2*>(ph);
        const float ff[2] = {f0.x, f0.y}, sl[2] = {sl0.x, sl0.y}, sg[2] = {st.x, st.y};
        const double old[2] = {od.x, od.y};
        double phi[2];
        float t0[2];
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            if (mm[j] < 0) {
                phi[j] = 0.0;
                t0[j] = 0.f;
                continue;
            }
            phi[j] = s0[j].value();
            t0[j] = tl.cell(s0[j], phi[j], old[j], ff[j], sl[j], sg[j]);
        }
        *reinterpret_cast<double2*>(ph) = make_double2(phi[0], phi[1]);
        *reinterpret_cast<float2*>(T) = make_float2(t0[0], t0[1]);
#pragma unroll
        for (int k = 1; k < K; ++k) {
            const float a0 = psi_moment<K>(k, 0, m1, acc), a1 = psi_moment<K>(k, 1, m1, acc);
            const float2 f = *reinterpret_cast<const float2*>(F + (size_t)k * p.TV);
            const float2 sk = *reinterpret_cast<const float2*>(p.sigs + (size_t)l_of_k(k) * p.NC + c2);
            *reinterpret_cast<float2*>(T + (size_t)k * p.TV) = make_float2(fmaf(sk.x, a0, f.x), fmaf(sk.y, a1, f.y));
        }
    }
    red_tail_store(p, tl, red, b, blockIdx.x, gridDim.x);
}

// per source: residual = sqrt(sum dphi^2 / sum phi^2), balance terms and the
// leakage of the last sweep from its nleak (octant, tile) slots; fixed
// summation order, so the results do not depend on the order the CTAs ran in
__global__ void k_resid_final(const double* blk, int nblk, const double* leak, int nleak, double* status,
                              size_t n_blk, size_t n_leak, size_t n_status)
{
    __shared__ double red[32];
    const int b = blockIdx.x;
    // uniform per block (DTS_DEBUG_BOUNDS build; constant true otherwise)
    if (!(DTS_FITS(((size_t)b + 1) * nblk * 4, n_blk, 40) && DTS_FITS(((size_t)b + 1) * nleak, n_leak, 41) &&
          DTS_FITS(((size_t)b + 1) * 4, n_status, 42)))
        return;
    double a[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int i = threadIdx.x; i < nblk; i += blockDim.x) {
        const double* o = blk + ((size_t)b * nblk + i) * 4;
        a[0] += o[0];
        a[1] += o[1];
        a[2] += o[2];
        a[3] += o[3];
    }
    {   // four independent accumulators per thread (loads in flight together), added in a fixed order
        const double* lk = leak + (size_t)b * nleak;
        const int nt = blockDim.x;
        double l4[4] = {0.0, 0.0, 0.0, 0.0};
        int i = threadIdx.x;
        for (; i + 3 * nt < nleak; i += 4 * nt) {
#pragma unroll
            for (int u = 0; u < 4; ++u) l4[u] += lk[i + u * nt];
        }
        for (; i < nleak; i += nt) l4[0] += lk[i];
        a[4] = (l4[0] + l4[1]) + (l4[2] + l4[3]);
    }
    for (int j = 0; j < 5; ++j) a[j] = block_sum(a[j], red);
    if (threadIdx.x == 0) {
        double* s = status + (size_t)b * 4;
        s[0] = a[1] > 0.0 ? sqrt(a[0] / a[1]) : 0.0;
        s[1] = a[2];
        s[2] = a[3];
        s[3] = a[4];
    }
}

// ---------------------------------------------------------------------------
// group set-up: per-cell cross sections of group g
// ---------------------------------------------------------------------------
struct CellParams {
    int NC, TV, TX, TY, TZ, NTx, NTy, nx, ny, nz, G, L, B, K, NT;
    double dx, dy, dz, x0, y0, z0;
    const int* mat_t;              // [NC]
    const double* scale_t_t;       // [NC] or null
    const double* scale_s_t;       // [NC] or null
    const double* sigma_t;         // [n_mat][G]
    const double* sigma_s;         // [n_mat][L+1][G][G]
};

__device__ inline int tiled_to_natural(const CellParams& p, int ct, double* C)
{
    const int tile = ct / p.TV, c = ct - tile * p.TV;
    const int tx = tile % p.NTx, ty = (tile / p.NTx) % p.NTy, tz = tile / (p.NTx * p.NTy);
    const int sx = c % p.TX, sy = (c / p.TX) % p.TY, sz = c / (p.TX * p.TY);
    const int i = tx * p.TX + sx, j = ty * p.TY + sy, k = tz * p.TZ + sz;
    if (C) {
        C[0] = p.x0 + (i + 0.5) * p.dx;
        C[1] = p.y0 + (j + 0.5) * p.dy;
        C[2] = p.z0 + (k + 0.5) * p.dz;
    }
    return (k * p.ny + j) * p.nx + i;
}

template <typename R>
__global__ void k_group_xs(const CellParams p, int g, R* sigt_r, double* sigt64, R* sigs, double* sigs0)
{
    const int ct = blockIdx.x * blockDim.x + threadIdx.x;
    if (ct >= p.NC) return;
    const int m = p.mat_t[ct];
    if (m < 0) {
        sigt_r[ct] = R(1);
        sigt64[ct] = 0.0;
        sigs0[ct] = 0.0;
        for (int l = 0; l <= p.L; ++l) sigs[(size_t)l * p.NC + ct] = R(0);
        return;
    }
    double st = p.sigma_t[(size_t)m * p.G + g];
    if (p.scale_t_t) st *= p.scale_t_t[ct];
    sigt_r[ct] = (R)st;
    sigt64[ct] = st;
    const double ss = p.scale_s_t ? p.scale_s_t[ct] : 1.0;
    for (int l = 0; l <= p.L; ++l) {
        const double v = p.sigma_s[(((size_t)m * (p.L + 1) + l) * p.G + g) * p.G + g] * ss;
        sigs[(size_t)l * p.NC + ct] = (R)v;
        if (l == 0) sigs0[ct] = v;
    }
}

// T = F[slot] at the start of a group (phi^(0) = 0)
template <typename R>
__global__ void k_group_init(size_t total, const R* F, R* T)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < total) T[i] = F[i];
}

// T = F[slot] + sigma_s phi_guess at the start of a group, and the scalar flux the first
// iteration's residual is measured against = the guess (dts_set_initial_guess): the guess is
// member b's collided moments [B][G][K][V] in natural voxel order, zeros for a member without
// one (which gives exactly T = F, phi = 0). F and T tile-ordered [B][NT][K][TV].
template <typename R>
__global__ void k_guess_source(const CellParams c, const double* __restrict__ guess, int g, const R* __restrict__ F,
                               const R* __restrict__ sigs, R* __restrict__ T, double* __restrict__ phi00, int V)
{
    const int ct = blockIdx.x * blockDim.x + threadIdx.x, b = blockIdx.y;
    if (ct >= c.NC) return;
    const int tile = ct / c.TV, cl = ct - tile * c.TV;
    const size_t base = ((size_t)b * c.NT + tile) * (size_t)(c.K * c.TV) + cl;
    if (c.mat_t[ct] < 0) {   // padding: no source, no flux
        for (int k = 0; k < c.K; ++k) T[base + (size_t)k * c.TV] = F[base + (size_t)k * c.TV];
        phi00[(size_t)b * c.NC + ct] = 0.0;
        return;
    }
    const int v = tiled_to_natural(c, ct, nullptr);
    const double* gb = guess + ((size_t)b * c.G + g) * (size_t)c.K * V + v;
    for (int k = 0; k < c.K; ++k) {
        const double ph = gb[(size_t)k * V];
        T[base + (size_t)k * c.TV] =
            (R)((double)F[base + (size_t)k * c.TV] + (double)sigs[(size_t)l_of_k(k) * c.NC + ct] * ph);
        if (k == 0) phi00[(size_t)b * c.NC + ct] = ph;
    }
}

// one group of the scalar fluence of every member for the streamed output: comp 0 uncollided,
// 1 collided, 2 their sum; unc and col [B][G][V], out [B][V]
__global__ void k_gather_component(const double* __restrict__ unc, const double* __restrict__ col, int comp, int g,
                                   int G, int V, double* __restrict__ out)
{
    const int v = blockIdx.x * blockDim.x + threadIdx.x, b = blockIdx.y;
    if (v >= V) return;
    const size_t i = ((size_t)b * G + g) * V + v;
    out[(size_t)b * V + v] = comp == 0 ? unc[i] : comp == 1 ? col[i] : unc[i] + col[i];
}

// one bounds check of a region of n elements, failing when plant != 0; touches no memory
__global__ void k_bounds_selftest(int plant, size_t n) { (void)DTS_FITS(plant ? n + 1 : n, n, 63); }

__global__ void k_set_ctl(int* ctl, int g, int slot)
{
    ctl[0] = g;
    ctl[1] = slot;
}

// ---------------------------------------------------------------------------
// A7 on the device: the convergence control of one group's source iterations
// when they run as a WHILE node of a CUDA graph. The decisions are those the
// host makes after every iteration: a member stops when its residual is below
// tol or, in the FP32 forms, when its residual has not improved by 1 % in 10
// iterations; the loop goes on while a member iterates, the iteration cap is
// not reached and no bounded wait has given up.
// ---------------------------------------------------------------------------
constexpr int kLoopThreads = 1024;
constexpr int kLoopMaxMembers = 32 * kLoopThreads;   // one stop bit per member and thread

struct LoopParams {
    int B, G, max_iters, fp32_stop;
    double tol;
    const double* status;      // [B][4] residual and balance terms of the iteration (k_resid_final)
    int* active;               // [B] members still iterating (read by the sweep and moment kernels)
    int* ctl;                  // [0] group, [1] fixed-source slot
    int* it;                   // iterations of the running group
    int* last_improve;         // [B] iteration of the last 1 % improvement (FP32 forms)
    double* best;              // [B] best residual so far (FP32 forms)
    int* iters;                // [B][G] iterations per (member, group)
    double* resid;             // [B][G] last residual
    double* balance;           // [B][G][3] source, absorption, leakage of the last sweep
    const int* err;            // the tensor-core forms' error word (a bounded wait gave up), or null
    cudaGraphConditionalHandle h;
};

// group g starts: its control values, every member active, the loop state cleared
__global__ void __launch_bounds__(kLoopThreads) k_loop_begin(const LoopParams q, int g, int slot)
{
    if (threadIdx.x == 0) {
        q.ctl[0] = g;
        q.ctl[1] = slot;
        *q.it = 0;
    }
    for (int b = threadIdx.x; b < q.B; b += blockDim.x) {
        q.active[b] = 1;
        q.best[b] = CUDART_INF;
        q.last_improve[b] = 0;
        q.iters[(size_t)b * q.G + g] = 0;
    }
}

// after each source iteration (one block of kLoopThreads): record every active member's residual and
// balance, retire the members that stopped, set the WHILE node's condition
__global__ void __launch_bounds__(kLoopThreads) k_loop_control(const LoopParams q)
{
    const int it = *q.it + 1, g = q.ctl[0];
    unsigned stopped = 0u;
    int goes_on = 0;
    for (int j = 0, b = threadIdx.x; b < q.B; ++j, b += blockDim.x) {
        if (!q.active[b]) continue;
        const double* s = q.status + 4 * (size_t)b;
        const size_t bg = (size_t)b * q.G + g;
        q.iters[bg] = it;
        q.resid[bg] = s[0];
        q.balance[bg * 3 + 0] = s[1];
        q.balance[bg * 3 + 1] = s[2];
        q.balance[bg * 3 + 2] = s[3];
        bool stop = q.tol > 0.0 && s[0] < q.tol;
        if (!stop && q.fp32_stop && q.tol > 0.0) {
            if (s[0] < 0.99 * q.best[b]) {
                q.best[b] = s[0];
                q.last_improve[b] = it;
            } else if (it - q.last_improve[b] >= 10) {
                stop = true;
            }
        }
        if (stop) stopped |= 1u << j;
        else goes_on = 1;
    }
    // as on the host: the flags of stopped members change only while some member goes on (the
    // group ends otherwise, and the next group sets every flag again)
    const int any = __syncthreads_or(goes_on);
    if (any)
        for (int j = 0, b = threadIdx.x; b < q.B; ++j, b += blockDim.x)
            if (stopped >> j & 1u) q.active[b] = 0;
    if (threadIdx.x == 0) {
        *q.it = it;
        const bool err = q.err && *q.err != 0;
        cudaGraphSetConditional(q.h, (any && it < q.max_iters && !err) ? 1u : 0u);
    }
}

// ---------------------------------------------------------------------------
// A1: uncollided fluence by exact voxel traversal from the source to each
// voxel centre (Eq. 4 with no scatter term); outside the grid is vacuum.
// src rows: kind, pos[3], axis[3], half_angle.
// ---------------------------------------------------------------------------
struct RayParams {
    int nx, ny, nz, V, G, n_mat;
    const double* fan;             // [B][8]: aperture (0 cone, 1 fan), fan normal, half azimuth, half polar
    double dx, dy, dz, x0, y0, z0;
    const int* mat;                // natural [V]
    const double* scale_t;         // natural [V] or null
    const double* sigma_t;         // [n_mat][G]
    const double* src;             // [B][8]
    const double* spec;            // [B][G]
    double* unc;                   // [B][G][V]
};

// Whether the unit direction u (source -> voxel centre) is in the beam.
// s7: pos[3], axis[3], cone half-angle; f: aperture (0 cone, 1 fan), fan-plane
// normal[3], half azimuth, half polar. Fan: with a = axis, n = normal made
// orthogonal to a, t = n x a: |asin(u.n)| <= half polar and
// |atan2(u.t, u.a)| <= half azimuth.
__device__ inline bool in_beam(const double* s7, const double* f, const double (&u)[3])
{
    const double an = sqrt(s7[3] * s7[3] + s7[4] * s7[4] + s7[5] * s7[5]);
    const double a[3] = {s7[3] / an, s7[4] / an, s7[5] / an};
    const double ua = u[0] * a[0] + u[1] * a[1] + u[2] * a[2];
    if (f == nullptr || f[0] != 1.0) return s7[6] >= kPi || ua >= cos(s7[6]);
    const double na = f[1] * a[0] + f[2] * a[1] + f[3] * a[2];
    double n[3] = {f[1] - na * a[0], f[2] - na * a[1], f[3] - na * a[2]};
    const double nn = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
    n[0] /= nn;
    n[1] /= nn;
    n[2] /= nn;
    const double t[3] = {n[1] * a[2] - n[2] * a[1], n[2] * a[0] - n[0] * a[2], n[0] * a[1] - n[1] * a[0]};
    const double un = u[0] * n[0] + u[1] * n[1] + u[2] * n[2];
    const double ut = u[0] * t[0] + u[1] * t[1] + u[2] * t[2];
    return fabs(un) <= sin(f[5]) && fabs(atan2(ut, ua)) <= f[4];
}

__global__ void k_raytrace(const RayParams p, int g0)
{
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    const int b = blockIdx.y;
    if (v >= p.V) return;
    const double* s = p.src + (size_t)b * 8;
    const int ng = min(kRayGroups, p.G - g0);
    double* out = p.unc + ((size_t)b * p.G + g0) * p.V + v;
    if (s[0] != 1.0) {
        for (int gg = 0; gg < ng; ++gg) out[(size_t)gg * p.V] = 0.0;
        return;
    }
    const int ci[3] = {v % p.nx, (v / p.nx) % p.ny, v / (p.nx * p.ny)};
    const int n[3] = {p.nx, p.ny, p.nz};
    const double lo[3] = {p.x0, p.y0, p.z0}, h[3] = {p.dx, p.dy, p.dz};
    double P[3], d[3];
    for (int a = 0; a < 3; ++a) {
        P[a] = s[1 + a];
        d[a] = lo[a] + (ci[a] + 0.5) * h[a] - P[a];
    }
    const double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    const double r = sqrt(r2);
    const double u[3] = {d[0] / r, d[1] / r, d[2] / r};
    if (!in_beam(s + 1, p.fan + (size_t)b * 8, u)) {
        for (int gg = 0; gg < ng; ++gg) out[(size_t)gg * p.V] = 0.0;
        return;
    }
    // parameter where the segment P -> C enters the grid box
    double a_in = 0.0;
    for (int a = 0; a < 3; ++a)
        if (d[a] != 0.0) {
            const double t0 = (lo[a] - P[a]) / d[a], t1 = (lo[a] + n[a] * h[a] - P[a]) / d[a];
            a_in = fmax(a_in, fmin(t0, t1));
        }
    int idx[3], step[3];
    double tnext[3];
    for (int a = 0; a < 3; ++a) {
        if (d[a] == 0.0) {
            idx[a] = ci[a];
            step[a] = 0;
            tnext[a] = 2.0;
            continue;
        }
        int id = (int)floor((P[a] + a_in * d[a] - lo[a]) / h[a]);
        id = id < 0 ? 0 : (id >= n[a] ? n[a] - 1 : id);
        idx[a] = id;
        step[a] = d[a] > 0.0 ? 1 : -1;
        tnext[a] = (lo[a] + (id + (d[a] > 0.0 ? 1 : 0)) * h[a] - P[a]) / d[a];
    }
    double tau[kRayGroups];
#pragma unroll
    for (int gg = 0; gg < kRayGroups; ++gg) tau[gg] = 0.0;
    double acur = a_in;
    const int max_steps = p.nx + p.ny + p.nz + 3;
    for (int it = 0; it < max_steps; ++it) {
        int ax = 0;
        if (tnext[1] < tnext[ax]) ax = 1;
        if (tnext[2] < tnext[ax]) ax = 2;
        const double a1 = fmin(tnext[ax], 1.0);
        const double seg = (a1 - acur) * r;
        if (seg > 0.0) {
            const int vv = (idx[2] * p.ny + idx[1]) * p.nx + idx[0];
            const int m = p.mat[vv];
            const double sc = p.scale_t ? p.scale_t[vv] : 1.0;
            const double* sgm = p.sigma_t + (size_t)m * p.G + g0;
#pragma unroll
            for (int gg = 0; gg < kRayGroups; ++gg)
                if (gg < ng) tau[gg] += sgm[gg] * sc * seg;
        }
        if (a1 >= 1.0) break;
        acur = a1;
        idx[ax] += step[ax];
        if (idx[ax] < 0 || idx[ax] >= n[ax]) break;
        tnext[ax] = (lo[ax] + (idx[ax] + (step[ax] > 0 ? 1 : 0)) * h[ax] - P[ax]) / d[ax];
    }
    const double inv = 1.0 / (4.0 * kPi * r2);
    for (int gg = 0; gg < ng; ++gg)
        out[(size_t)gg * p.V] = p.spec[(size_t)b * p.G + g0 + gg] * exp(-tau[gg]) * inv;
}

// The same traversal for problems with at most kRayMats materials: each
// thread accumulates the path length through every material (weighted by the
// voxel's sigma_t scale) in shared memory, and every group's optical depth is
// sum_m L_m sigma_t[m][g], so one pass serves all groups. The next crossing
// parameter is formed with the reciprocal of the ray's direction component.
constexpr int kRayMats = 8;
constexpr int kRayThreads = 128;

// Path length through every material (weighted by the voxel's sigma_t scale)
// on the segment from the source point P to the centre of voxel v, written to
// Ls[m * kRayThreads] (this thread's column of a shared-memory table), for a
// source collimated to a cone (axis, half angle; >= pi: isotropic). Returns
// false when the voxel is outside the cone; r2 = |C - P|^2 and om the unit
// direction of flight are set either way.
__device__ inline bool ray_lengths(const RayParams& p, int v, const double* s7, const double* fan, double* Ls,
                                   double& r2, double (&om)[3])
{
#pragma unroll
    for (int m = 0; m < kRayMats; ++m) Ls[m * kRayThreads] = 0.0;
    const int cx = v % p.nx, cy = (v / p.nx) % p.ny, cz = v / (p.nx * p.ny);
    const double Px = s7[0], Py = s7[1], Pz = s7[2];
    const double dx = p.x0 + (cx + 0.5) * p.dx - Px, dy = p.y0 + (cy + 0.5) * p.dy - Py,
                 dz = p.z0 + (cz + 0.5) * p.dz - Pz;
    r2 = dx * dx + dy * dy + dz * dz;
    const double r = sqrt(r2);
    om[0] = dx / r;
    om[1] = dy / r;
    om[2] = dz / r;
    if (!in_beam(s7, fan, om)) return false;
    // parameter where the segment P -> C enters the grid box
    double a_in = 0.0;
    auto enter = [&](double lo, int n, double h, double P, double d) {
        if (d != 0.0) {
            const double t0 = (lo - P) / d, t1 = (lo + n * h - P) / d;
            a_in = fmax(a_in, fmin(t0, t1));
        }
    };
    enter(p.x0, p.nx, p.dx, Px, dx);
    enter(p.y0, p.ny, p.dy, Py, dy);
    enter(p.z0, p.nz, p.dz, Pz, dz);
    // per axis: voxel index, step, and the next crossing parameter t = c0 + k c1 of plane k, with
    // c0 = (lo - P) / d and c1 = h / d (the plane index k is exact in FP64)
    auto init = [&](double lo, int n, double h, double P, double d, int c, int& id, int& st, double& c0,
                    double& c1, double& tn) {
        if (d == 0.0) {
            id = c;
            st = 0;
            c0 = 2.0;
            c1 = 0.0;
            tn = 2.0;
            return;
        }
        int i0 = (int)floor((P + a_in * d - lo) / h);
        id = i0 < 0 ? 0 : (i0 >= n ? n - 1 : i0);
        st = d > 0.0 ? 1 : -1;
        const double inv = 1.0 / d;
        c0 = (lo - P) * inv;
        c1 = h * inv;
        tn = fma((double)(id + (d > 0.0 ? 1 : 0)), c1, c0);
    };
    int ix, iy, iz, sx, sy, sz;
    double cx0, cx1, cy0, cy1, cz0, cz1, tx, ty, tz;
    init(p.x0, p.nx, p.dx, Px, dx, cx, ix, sx, cx0, cx1, tx);
    init(p.y0, p.ny, p.dy, Py, dy, cy, iy, sy, cy0, cy1, ty);
    init(p.z0, p.nz, p.dz, Pz, dz, cz, iz, sz, cz0, cz1, tz);
    // The crossing parameters are non-negative (2 marks an axis the ray does not cross), so their order
    // is that of their bit patterns as signed 64-bit integers: the selection below runs on the integer
    // pipes instead of the FP64 pipe (a small fraction of the FP32 rate on this part). A crossing that
    // rounds to -0 or just below 0 sorts first, as its value does; its segment is empty either way.
    const long long one = __double_as_longlong(1.0);
    double acur = a_in;
    const int max_steps = p.nx + p.ny + p.nz + 3;
    for (int it = 0; it < max_steps; ++it) {
        const long long bx = __double_as_longlong(tx), by = __double_as_longlong(ty), bz = __double_as_longlong(tz);
        const int ax = (by < bx) ? ((bz < by) ? 2 : 1) : ((bz < bx) ? 2 : 0);
        const long long bs = ax == 0 ? bx : ax == 1 ? by : bz;
        const bool last = bs >= one;
        const double a1 = last ? 1.0 : __longlong_as_double(bs);
        if (__double_as_longlong(a1) > __double_as_longlong(acur)) {
            const double seg = (a1 - acur) * r;
            const int vv = (iz * p.ny + iy) * p.nx + ix;
            const int m = p.mat[vv];
            Ls[m * kRayThreads] += p.scale_t ? p.scale_t[vv] * seg : seg;
        }
        if (last) break;
        acur = a1;
        if (ax == 0) {
            ix += sx;
            if (ix < 0 || ix >= p.nx) break;
            tx = fma((double)(ix + (sx > 0 ? 1 : 0)), cx1, cx0);
        } else if (ax == 1) {
            iy += sy;
            if (iy < 0 || iy >= p.ny) break;
            ty = fma((double)(iy + (sy > 0 ? 1 : 0)), cy1, cy0);
        } else {
            iz += sz;
            if (iz < 0 || iz >= p.nz) break;
            tz = fma((double)(iz + (sz > 0 ? 1 : 0)), cz1, cz0);
        }
    }
    return true;
}

__global__ void __launch_bounds__(kRayThreads) k_raytrace_mat(const RayParams p)
{
    __shared__ double Ls[kRayMats][kRayThreads];
    const int tid = threadIdx.x;
    const int v = blockIdx.x * blockDim.x + tid;
    const int b = blockIdx.y;
    if (v >= p.V) return;
    const double* s = p.src + (size_t)b * 8;
    double* out = p.unc + (size_t)b * p.G * p.V + v;
    double r2, om[3];
    if (s[0] != 1.0 || !ray_lengths(p, v, s + 1, p.fan + (size_t)b * 8, &Ls[0][tid], r2, om)) {
        for (int g = 0; g < p.G; ++g) out[(size_t)g * p.V] = 0.0;
        return;
    }
    double Lm[kRayMats];
#pragma unroll
    for (int m = 0; m < kRayMats; ++m) Lm[m] = Ls[m][tid];
    const double inv = 1.0 / (4.0 * kPi * r2);
    for (int g = 0; g < p.G; ++g) {
        double tau = 0.0;
#pragma unroll
        for (int m = 0; m < kRayMats; ++m)
            if (m < p.n_mat) tau += Lm[m] * p.sigma_t[(size_t)m * p.G + g];
        out[(size_t)g * p.V] = p.spec[(size_t)b * p.G + g] * exp(-tau) * inv;
    }
}

// Several cones summed into one source (batch members with n_cones[b] > 0):
// the uncollided fluence is the sum of the cones' (Eq. 4 per cone) and, for
// the first-collision source, U_lm^g(v) = sum_c phi_u,c^g(v) Y_lm(Omega_c(v))
// is accumulated per group and moment (each thread owns its voxel).
struct ConeParams {
    const double* geo;     // [B][cap][16]: pos, axis, half angle, aperture, normal, half azimuth, half polar
    const double* spec;    // [B][cap][G]
    const int* n_cones;    // [B]
    const int* slot;       // [B] row of U, -1 for none
    double* U;             // [slots][G][K][V]
    int cap, K, L;
};

__global__ void __launch_bounds__(kRayThreads) k_raytrace_cones(const RayParams p, const ConeParams cp)
{
    __shared__ double Ls[kRayMats][kRayThreads];
    const int tid = threadIdx.x;
    const int v = blockIdx.x * blockDim.x + tid;
    const int b = blockIdx.y;
    const int nc = cp.n_cones[b];
    if (v >= p.V || nc <= 0) return;
    double* out = p.unc + (size_t)b * p.G * p.V + v;
    double* U = cp.U + (size_t)cp.slot[b] * p.G * cp.K * p.V + v;
    for (int c = 0; c < nc; ++c) {
        const double* s7 = cp.geo + ((size_t)b * cp.cap + c) * 16;   // pos, axis, half, then aperture row
        const double* spec = cp.spec + ((size_t)b * cp.cap + c) * p.G;
        double r2, om[3];
        const bool in = ray_lengths(p, v, s7, s7 + 7, &Ls[0][tid], r2, om);
        double Lm[kRayMats], Y[16];
#pragma unroll
        for (int m = 0; m < kRayMats; ++m) Lm[m] = Ls[m][tid];
        sh_eval(cp.L, om[0], om[1], om[2], Y);
        const double inv = 1.0 / (4.0 * kPi * r2);
        for (int g = 0; g < p.G; ++g) {
            double phi = 0.0;
            if (in) {
                double tau = 0.0;
#pragma unroll
                for (int m = 0; m < kRayMats; ++m)
                    if (m < p.n_mat) tau += Lm[m] * p.sigma_t[(size_t)m * p.G + g];
                phi = spec[g] * exp(-tau) * inv;
            }
            double* Ug = U + (size_t)g * cp.K * p.V;
            if (c == 0) {
                out[(size_t)g * p.V] = phi;
                for (int k = 0; k < cp.K; ++k) Ug[(size_t)k * p.V] = phi * Y[k];
            } else {
                out[(size_t)g * p.V] += phi;
                for (int k = 0; k < cp.K; ++k) Ug[(size_t)k * p.V] += phi * Y[k];
            }
        }
    }
}

// ---------------------------------------------------------------------------
// A1 (second half) / A2: fixed source of group gt written into ring slot
// slot: first-collision moments (Eq. 5)
//   q_lm = sum_{g'<=gt} sigma_{s,l}^{g'->gt} phi_u^{g'} Y_lm(Omega_u)
// or the volumetric source (l = 0 only).
// ---------------------------------------------------------------------------
// Fluence to absorbed dose (post-processing, collision-kerma form): per voxel
// D = c sum_g (phi_g E_g) (mu_en/rho)_g(mat), groups in order; comp 0 uncollided,
// 1 collided, 2 total (uncollided + collided).
__global__ void k_dose(int V, int G, const double* u, const double* col, int comp, const int* mat,
                       const double* mu_en, const double* e_mev, double c, double* out)
{
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= V) return;
    const double* mrow = mu_en + (size_t)mat[v] * G;
    double acc = 0.0;
    for (int g = 0; g < G; ++g) {
        const double uf = u[(size_t)g * V + v], cf = col[(size_t)g * V + v];
        const double phi = comp == 0 ? uf : comp == 1 ? cf : uf + cf;
        acc += phi * e_mev[g] * mrow[g];
    }
    out[v] = c * acc;
}

template <typename R>
struct SrcParams {
    CellParams c;
    const double* src;     // [B][8]
    const double* unc;     // [B][G][V]
    const double* q;       // [B][G][V] or null
    const float* sigma_s_f;   // [n_mat][L+1][G][G] in FP32 (FP32 forms)
    const double* U;       // [slots][G][K][V] cone-summed uncollided moments (kind 2), or null
    const int* uslot;      // [B] row of U
    R* F;
    size_t Fstride;
    int V, W;              // W: downscatter band (sigma_s(g' -> g) = 0 for g - g' > W)
};

template <typename R>
__global__ void k_fixed_source(const SrcParams<R> p, int gt, int slot)
{
    const int ct = blockIdx.x * blockDim.x + threadIdx.x;
    const int b = blockIdx.y;
    const CellParams& c = p.c;
    if (ct >= c.NC) return;
    const int tile = ct / c.TV, cc = ct - tile * c.TV;
    R* F = p.F + (size_t)slot * p.Fstride + ((size_t)b * c.NT + tile) * (size_t)(c.K * c.TV) + cc;
    const int m = c.mat_t[ct];
    const int kind = (int)p.src[(size_t)b * 8];
    if (m < 0 || kind < 0) {
        for (int k = 0; k < c.K; ++k) F[(size_t)k * c.TV] = R(0);
        return;
    }
    double C[3];
    const int v = tiled_to_natural(c, ct, C);
    if (kind == 0) {
        F[0] = (R)p.q[((size_t)b * c.G + gt) * p.V + v];
        for (int k = 1; k < c.K; ++k) F[(size_t)k * c.TV] = R(0);
        return;
    }
    const double* s = p.src + (size_t)b * 8;
    const int g0 = max(0, gt - p.W);   // groups outside the band add exact zeros
    if (kind == 2) {
        // several cones: F_lm = sum_g' sigma_s,l(g' -> g) scale_s U_lm^g'
        const double* U = p.U + (size_t)p.uslot[b] * c.G * c.K * p.V + v;
        const double ss = c.scale_s_t ? c.scale_s_t[ct] : 1.0;
        for (int k = 0; k < c.K; ++k) {
            const int l = l_of_k(k);
            double acc = 0.0;
            for (int gp = g0; gp <= gt; ++gp)
                acc += c.sigma_s[(((size_t)m * (c.L + 1) + l) * c.G + gp) * c.G + gt] * ss *
                       U[((size_t)gp * c.K + k) * p.V];
            F[(size_t)k * c.TV] = (R)acc;
        }
        return;
    }
    if constexpr (sizeof(R) == 4) {
        // FP32 form: the product is stored in FP32, so it is formed in FP32
        const float d0 = (float)(C[0] - s[1]), d1 = (float)(C[1] - s[2]), d2 = (float)(C[2] - s[3]);
        const float ri = rsqrtf(d0 * d0 + d1 * d1 + d2 * d2);
        float Y[16];
        sh_eval(c.L, d0 * ri, d1 * ri, d2 * ri, Y);
        const float ss = c.scale_s_t ? (float)c.scale_s_t[ct] : 1.f;
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
        for (int gp = g0; gp <= gt; ++gp) {
            const float phu = (float)p.unc[((size_t)b * c.G + gp) * p.V + v] * ss;
            for (int l = 0; l <= c.L; ++l)
                acc[l] = fmaf(p.sigma_s_f[(((size_t)m * (c.L + 1) + l) * c.G + gp) * c.G + gt], phu, acc[l]);
        }
        for (int k = 0; k < c.K; ++k) F[(size_t)k * c.TV] = acc[l_of_k(k)] * Y[k];
    } else {
        const double d0 = C[0] - s[1], d1 = C[1] - s[2], d2 = C[2] - s[3];
        const double r = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
        double Y[16];
        sh_eval(c.L, d0 / r, d1 / r, d2 / r, Y);
        const double ss = c.scale_s_t ? c.scale_s_t[ct] : 1.0;
        double acc[4] = {0.0, 0.0, 0.0, 0.0};
        for (int gp = g0; gp <= gt; ++gp) {
            const double phu = p.unc[((size_t)b * c.G + gp) * p.V + v];
            for (int l = 0; l <= c.L; ++l)
                acc[l] += c.sigma_s[(((size_t)m * (c.L + 1) + l) * c.G + gp) * c.G + gt] * ss * phu;
        }
        for (int k = 0; k < c.K; ++k) F[(size_t)k * c.TV] = (R)(acc[l_of_k(k)] * Y[k]);
    }
}

// ---------------------------------------------------------------------------
// A2 / A7 at the end of group g: downscatter of the converged moments into
// the fixed sources of groups g+1 .. g+W, and the outputs.
// ---------------------------------------------------------------------------
template <typename R>
struct PushParams {
    CellParams c;
    const R* part;         // octant partials of the group's last sweep
    R* F;
    size_t Fstride;
    int W, V;
    double* col;           // [B][G][V]
    double* mom;           // [B][G][K][V] or null
    const float* sigma_s_f;   // [n_mat][L+1][G][G], the FP32 rounding of sigma_s
};

// sigma_s(mat, l, g -> gt) scale_s rounded to FP32 once: without a per-cell scatter scale it is the
// FP32 table entry (the same rounding of the same FP64 value, with no FP64 arithmetic)
template <typename R>
__device__ __forceinline__ float push_factor(const PushParams<R>& p, int m, int l, int g, int gt, const double* ss_t,
                                             int cell)
{
    const CellParams& c = p.c;
    const size_t i = (((size_t)m * (c.L + 1) + l) * c.G + g) * c.G + gt;
    return ss_t ? (float)(c.sigma_s[i] * ss_t[cell]) : p.sigma_s_f[i];
}

// the converged moments are the octant sums of the last sweep's partials
// (scalar flux in FP64, higher moments in the sweep precision, as the
// reduction formed them)
template <typename R>
__global__ void k_push(const PushParams<R> p, int g)
{
    const int ct = blockIdx.x * blockDim.x + threadIdx.x;
    const int b = blockIdx.y;
    const CellParams& c = p.c;
    if (ct >= c.NC) return;
    const int m = c.mat_t[ct];
    if (m < 0) return;
    const int tile = ct / c.TV, cc = ct - tile * c.TV;
    const size_t base = ((size_t)b * c.NT + tile) * (size_t)(c.K * c.TV) + cc;
    const size_t ostride = (size_t)c.B * c.NT * c.K * c.TV;
    const int v = tiled_to_natural(c, ct, nullptr);
    const double ss = c.scale_s_t ? c.scale_s_t[ct] : 1.0;
    const int W1 = p.W + 1;
    const int gmax = min(c.G - 1, g + p.W);
    for (int k = 0; k < c.K; ++k) {
        const R* pp = p.part + base + (size_t)k * c.TV;
        double ph;
        if (k == 0) {
            ph = 0.0;
            for (int o = 0; o < 8; ++o) ph += (double)pp[o * ostride];
        } else {
            R s = R(0);
            for (int o = 0; o < 8; ++o) s += pp[o * ostride];
            ph = (double)s;
        }
        const int l = l_of_k(k);
        if (k == 0) p.col[((size_t)b * c.G + g) * p.V + v] = ph;
        if (p.mom) p.mom[(((size_t)b * c.G + g) * c.K + k) * p.V + v] = ph;
        for (int g2 = g + 1; g2 <= gmax; ++g2) {
            const double sgm = c.sigma_s[(((size_t)m * (c.L + 1) + l) * c.G + g) * c.G + g2];
            if (sgm != 0.0) {
                R* f = p.F + (size_t)(g2 % W1) * p.Fstride + base + (size_t)k * c.TV;
                *f = (R)((double)*f + sgm * ss * ph);
            }
        }
    }
}

// FP32 form with tiles a multiple of 4 cells long in x: one thread per
// (4 consecutive cells, source), 16-byte loads and stores. The scalar flux is
// summed in FP64 as above; each later group's fixed source takes the product
// sigma_s * scale_s rounded to FP32 once per (cell, l, group) and an FP32 FMA
// per moment.
template <int K>
__global__ void __launch_bounds__(256) k_push4(const PushParams<float> p, int g)
{
    const int c4 = (blockIdx.x * blockDim.x + threadIdx.x) * 4;
    const int b = blockIdx.y;
    const CellParams& c = p.c;
    if (c4 >= c.NC) return;
    const int4 m4 = *reinterpret_cast<const int4*>(c.mat_t + c4);
    const int mm[4] = {m4.x, m4.y, m4.z, m4.w};
    if ((mm[0] & mm[1] & mm[2] & mm[3]) < 0) return;            // four padding cells
    const int tile = c4 / c.TV, cc = c4 - tile * c.TV;
    const size_t base = ((size_t)b * c.NT + tile) * (size_t)(K * c.TV) + cc;
    const size_t ostride = (size_t)c.B * c.NT * K * c.TV;
    const int v0 = tiled_to_natural(c, c4, nullptr);            // the 4 cells are x-consecutive
    const int x0 = v0 % c.nx;
    const int W1 = p.W + 1;
    const int gmax = min(c.G - 1, g + p.W);
    constexpr int LK = K == 1 ? 1 : K == 4 ? 2 : K == 9 ? 3 : 4;  // Legendre orders present
    const int nw = gmax - g;
    float sc[4][LK][4];                                         // [g2 - g - 1][l][cell], W <= 4
#pragma unroll
    for (int w = 0; w < 4; ++w)
#pragma unroll
        for (int l = 0; l < LK; ++l)
#pragma unroll
            for (int j = 0; j < 4; ++j)
                sc[w][l][j] = (w >= nw || mm[j] < 0) ? 0.f : push_factor(p, mm[j], l, g, g + 1 + w, c.scale_s_t, c4 + j);
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const float* pp = p.part + base + (size_t)k * c.TV;
        double ph[4];
        float4 s4;
        if (k == 0) {
            ph[0] = ph[1] = ph[2] = ph[3] = 0.0;
#pragma unroll
            for (int o = 0; o < 8; ++o) {
                const float4 v = *reinterpret_cast<const float4*>(pp + o * ostride);
                ph[0] += (double)v.x;
                ph[1] += (double)v.y;
                ph[2] += (double)v.z;
                ph[3] += (double)v.w;
            }
            s4 = make_float4((float)ph[0], (float)ph[1], (float)ph[2], (float)ph[3]);
        } else {
            s4 = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int o = 0; o < 8; ++o) {
                const float4 v = *reinterpret_cast<const float4*>(pp + o * ostride);
                s4.x += v.x;
                s4.y += v.y;
                s4.z += v.z;
                s4.w += v.w;
            }
            ph[0] = s4.x;
            ph[1] = s4.y;
            ph[2] = s4.z;
            ph[3] = s4.w;
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (mm[j] < 0 || x0 + j >= c.nx) continue;
            if (k == 0) p.col[((size_t)b * c.G + g) * p.V + v0 + j] = ph[j];
            if (p.mom) p.mom[(((size_t)b * c.G + g) * K + k) * p.V + v0 + j] = ph[j];
        }
        const int l = l_of_k(k);
        // the lower groups' ring slots are loaded together, then updated (one memory latency per moment)
        float4* fp[4];
        float4 fv[4];
#pragma unroll
        for (int w = 0; w < 4; ++w) {
            fp[w] = reinterpret_cast<float4*>(p.F + (size_t)((g + 1 + w) % W1) * p.Fstride + base + (size_t)k * c.TV);
            if (w < nw) fv[w] = *fp[w];
        }
#pragma unroll
        for (int w = 0; w < 4; ++w) {
            if (w >= nw) break;
            fv[w].x = fmaf(sc[w][l][0], s4.x, fv[w].x);
            fv[w].y = fmaf(sc[w][l][1], s4.y, fv[w].y);
            fv[w].z = fmaf(sc[w][l][2], s4.z, fv[w].z);
            fv[w].w = fmaf(sc[w][l][3], s4.w, fv[w].w);
            *fp[w] = fv[w];
        }
    }
}

// The downscatter push of the direct-output form: the converged group's
// moments are recomputed from the last sweep's angular fluxes (as k_reduce_psi
// forms them, two cells per thread), then pushed as in k_push4.
template <int NDO, int K>
// xrev: the angular fluxes come from the tensor-core forms' sweep (odd octants in their own x order).
// w0: this pass updates the lower groups g+1+w0 .. g+w0+kPushRing (a band wider than kPushRing takes
// several passes); the first pass (w0 = 0) also writes the group's outputs.
__global__ void __launch_bounds__(256, 4) k_push_psi(const PushParams<float> p, int g, const float* __restrict__ Dt,
                                                     int xrev, int w0)
{
    __shared__ __align__(16) unsigned long long Dp[8 * NDO * PsiPairs<K>::value];
    __shared__ unsigned long long stg[2 * NDO * 256];
    load_dpairs<NDO, K>(Dp, Dt);
    const int c2 = (blockIdx.x * blockDim.x + threadIdx.x) * 2;
    const int b = blockIdx.y;
    const CellParams& c = p.c;
    if (c2 >= c.NC) return;
    const int2 mv = *reinterpret_cast<const int2*>(c.mat_t + c2);
    const int mm[2] = {mv.x, mv.y};
    if ((mm[0] & mm[1]) < 0) return;
    const int tile = c2 / c.TV, cc = c2 - tile * c.TV;
    const size_t base = ((size_t)b * c.NT + tile) * (size_t)(K * c.TV) + cc;
    const size_t ostride = (size_t)c.NT * NDO * c.TV;
    const float* ps = p.part + (size_t)b * 8 * ostride + (size_t)tile * NDO * c.TV + cc;
    TwoSum s0t[2];
    float m1[2];
    unsigned long long acc[2][PsiPairs<K>::value];
    psi_moments<NDO, K>(ps, ostride, c.TV, Dp, stg + threadIdx.x, s0t, m1, acc, xrev ? (cc ^ 6) - cc : 0);
    const int v0 = tiled_to_natural(c, c2, nullptr);           // the 2 cells are x-consecutive
    const int x0 = v0 % c.nx;
    const int W1 = p.W + 1;
    const int nw = min(c.G - 1, g + p.W) - g - w0;   // lower groups of this pass (may be <= 0)
    // sigma_s(g -> g+1+w0+w) scale_s rounded to FP32 once per (cell, l, lower group): formed for each
    // Legendre order before its 2l+1 moments (FP64 runs at a small fraction of the FP32 rate)
    constexpr int NL = K == 1 ? 1 : K == 4 ? 2 : K == 9 ? 3 : 4;
    static_assert(NL * NL == K, "K = (L+1)^2");
#pragma unroll
    for (int l = 0; l < NL; ++l) {
        float sc[kPushRing][2];
#pragma unroll
        for (int w = 0; w < kPushRing; ++w)
#pragma unroll
            for (int j = 0; j < 2; ++j)
                sc[w][j] = (w >= nw || mm[j] < 0) ? 0.f
                                                  : push_factor(p, mm[j], l, g, g + 1 + w0 + w, c.scale_s_t, c2 + j);
#pragma unroll
        for (int k = l * l; k < (l + 1) * (l + 1); ++k) {
            double ph[2];
            float2 s2;
            if (k == 0) {
                ph[0] = s0t[0].value();
                ph[1] = s0t[1].value();
                s2 = make_float2((float)ph[0], (float)ph[1]);
            } else {
                s2 = make_float2(psi_moment<K>(k, 0, m1, acc), psi_moment<K>(k, 1, m1, acc));
                ph[0] = s2.x;
                ph[1] = s2.y;
            }
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                if (w0 != 0 || mm[j] < 0 || x0 + j >= c.nx) continue;
                if (k == 0) p.col[((size_t)b * c.G + g) * p.V + v0 + j] = ph[j];
                if (p.mom) p.mom[(((size_t)b * c.G + g) * K + k) * p.V + v0 + j] = ph[j];
            }
            // the ring slots of the lower groups are loaded together, then updated: one memory latency per
            // moment instead of one per (moment, group) (the compiler may not move a load above a store)
            float2* fp[kPushRing];
            float2 fv[kPushRing];
#pragma unroll
            for (int w = 0; w < kPushRing; ++w) {
                fp[w] = reinterpret_cast<float2*>(p.F + (size_t)((g + 1 + w0 + w) % W1) * p.Fstride + base +
                                                  (size_t)k * c.TV);
                if (w < nw) fv[w] = *fp[w];
            }
#pragma unroll
            for (int w = 0; w < kPushRing; ++w) {
                if (w >= nw) break;
                fv[w].x = fmaf(sc[w][0], s2.x, fv[w].x);
                fv[w].y = fmaf(sc[w][1], s2.y, fv[w].y);
                *fp[w] = fv[w];
            }
        }
    }
}

__global__ void k_add(size_t n, const double* a, const double* b, double* out)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = a[i] + b[i];
}

#endif  // DTS_SWEEP_KERNEL_ONLY

}  // namespace dts
