// dts_tc.cuh -- the Eq. 3 reduction fused with the scatter-source contraction
// on the fifth-generation tensor cores (tcgen05, sm_103a).
//
// One source iteration of the tensor-core forms is
//   sweep:   Q[b][o][tile][d][cell]  ->  psi[b][o][tile][d][cell]   (k_sweep_batch, Q input)
//   moments: psi -> phi_lm (Eq. 3, CUDA cores), T = F + sigma_s phi (Eq. 2),
//            Q = M T on the tensor cores                           (k_moments_q)
// so the sweep no longer contracts moments to directions itself: its
// per-update source arrives as one FP32 value per (cell, direction).
//
// The contraction of one (source, tile) item is the dense product
//   Q[128 cells x N_d] = T[128 cells x K] . M^T[K x N_d]
// with K = (L+1)^2 <= 16 moments, padded to 16, and N_d directions padded to a
// multiple of 16: one tcgen05.mma of M = 128 rows per (product, K step), the
// FP32 accumulator in tensor memory (one TMEM lane per cell), read back with
// tcgen05.ld and stored as coalesced 128-byte rows of Q.
//
// Operand precisions (dts_precision):
//   split BF16: T' = T_hi + T_lo and M' = M_hi + M_lo with bf16 parts, three
//               products hi.hi + hi.lo + lo.hi accumulated in FP32 (the
//               dropped lo.lo term and the rounding of the lo parts are
//               ~2^-17 of each term);
//   split TF32: the same three products with tf32 parts (10 explicit mantissa
//               bits each, round to nearest), ~2^-21 of each term; a single
//               TF32 product (T and M rounded once, ~2^-12 relative per
//               operand) measured 1.2e-4 relative L2 on the scalar fluence of
//               a small cone-beam case, above the 1e-4 gate of the
//               reduced-precision forms, so it is not offered.
// In both, the operator is scaled as M' = 4 pi M and the moments as
// T' = T / (4 pi), so that the isotropic column M'[n][0] = 1 is exact and the
// rounding of the operator adds no bias to the dominant l = 0 term.
#pragma once
#include <cuda_bf16.h>
#include <stdint.h>

#include <type_traits>

#include "dts_kernels.cuh"

namespace dts {

// --------------------------------------------------------------------------
// PTX wrappers: tcgen05 (mbarrier and bulk copy: dts_ptx.cuh)
// --------------------------------------------------------------------------
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// whole warp: allocate ncols (power of two >= 32) TMEM columns, address written to *slot
__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_free(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// Shared-memory matrix descriptor, K-major without swizzle: the operand is
// tiled into core matrices of 8 rows x 16 bytes (128 contiguous bytes); lbo
// is the byte distance between core matrices adjacent along K, sbo between
// core matrices adjacent along M (or N).
__device__ __forceinline__ uint64_t smem_desc(const void* p, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = (uint64_t)((smem_addr(p) & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;   // descriptor version of the fifth-generation tensor cores
    return d;                 // base offset 0, no swizzle
}

// Instruction descriptor of kind::f16 / kind::tf32: FP32 accumulator, A and B
// of format fmt (1 = BF16, 2 = TF32), both K-major, M x N.
__host__ __device__ constexpr uint32_t mma_idesc(uint32_t fmt, int M, int N)
{
    return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

template <int MODE>   // 0: kind::f16 (bf16 operands), 1: kind::tf32
__device__ __forceinline__ void mma_issue(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate)
{
    if constexpr (MODE == 0) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
            : "memory");
    } else {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
            : "memory");
    }
}

// arrive on *bar once every tcgen05.mma issued so far by this thread has completed
__device__ __forceinline__ void mma_commit(uint64_t* bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_addr(bar))
                 : "memory");
}

// 16 consecutive FP32 columns of this warp's 32 TMEM lanes (thread i: lane base + i)
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}

__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ uint32_t tf32_rn(float x)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ uint32_t bf16x2_bits(__nv_bfloat16 lo, __nv_bfloat16 hi)
{
    return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

// --------------------------------------------------------------------------
// k_moments_q
// --------------------------------------------------------------------------
constexpr int kQCells = 128;     // cells of an 8 x 4 x 4 tile = rows of the MMA = TMEM lanes
constexpr int kQThreads = 128;   // one thread per cell; 4 warps reach the 128 TMEM lanes
constexpr int kQTmemCols = 128;  // >= the padded direction count (<= 80) + 16 moment columns

struct QParams {
    int B, NT, TV, NC;
    int nitems;                  // B * NT
    int init;                    // 1: Q = M F (first iteration of a group; phi = 0, no psi read)
    const float* psi;            // [B][8][NT][NDO][TV]
    float* Q;                    // [B][8][NT][NDO][TV]
    double* phi00;               // [B][NC]
    const float* F;              // fixed-source ring, [slot][B][NT][K][TV]
    size_t Fstride;
    const int* ctl;              // [1] = ring slot of the group
    const float* sigs;           // [L+1][NC]
    const float* sigt;           // [NC]
    const int* mat_t;            // [NC]
    const int* active;           // [B]
    const float* Dt;             // [N_d][K] moment operator
    const float* Mop;            // [2][NP][16] operator parts M' = hi + lo (bf16 or tf32 values)
    const float* Dop;            // [2][16][N_d] Eq. 3 operator parts D = hi + lo (bf16 values), N_d % 16 == 0
    double vol;
    double* blk;                 // [B][NT][4] residual and balance partials per item
    int* err;                    // device error word (1: a bounded wait gave up)
    const int* poison;           // test hook (dts_debug_poison_wait): nonzero makes the flux-stage waits run out
    // element counts of the buffers above (checked in the DTS_DEBUG_BOUNDS build)
    size_t n_psi, n_Q, n_phi00, n_F, n_sigs, n_blk;
};

template <int NDO, int K, int MODE>
struct QShape {
    static constexpr int ND = 8 * NDO;
    static constexpr int NP = (ND + 15) / 16 * 16;            // N of the contraction to directions
    static constexpr int NCH = NP / 8;                        // 8-column TMEM chunks
    // the Eq. 3 moments on the tensor cores too when the directions fill whole bf16 K steps (S6, S8):
    // [128 cells x N_d] x [N_d x 16 moments], split-BF16 parts of the fluxes written in place of the
    // consumed flux stage (the two parts take exactly its bytes)
    static constexpr bool TC1 = ND % 16 == 0;
    static constexpr int KP = PsiPairs<K>::value;             // moment pairs of the CUDA-core Eq. 3 operator
    static constexpr int PSI_STAGE = ND * kQCells * 4;        // bytes of one item's angular fluxes
    static constexpr int ROWB = MODE == 0 ? 32 : 64;          // bytes of one 16-moment operand row
    static constexpr int SBO = 8 * ROWB;                      // bytes between 8-row groups
    static constexpr int A_BYTES = kQCells * ROWB;            // one operand part of T
    static constexpr int B_BYTES = NP * ROWB;                 // one operand part of M'
    static constexpr int SBO1 = ND / 8 * 128;                 // Eq. 3 operands: K = N_d bf16 per row
    static constexpr int A1_BYTES = kQCells * ND * 2;         // one part of the fluxes (hi or lo)
    static constexpr int B1_BYTES = 16 * ND * 2;              // one part of the Eq. 3 operator
    // byte offsets in dynamic shared memory
    static constexpr int oPsi = 0;                            // [ND][128] float: one item's fluxes
    static constexpr int oA = oPsi + PSI_STAGE;               // A parts (hi, lo) of T
    static constexpr int oB = oA + 2 * A_BYTES;               // B parts (hi, lo) of M'
    static constexpr int oB1 = oB + 2 * B_BYTES;              // TC1: B parts (hi, lo) of D
    static constexpr int oW = oB1 + (TC1 ? 2 * B1_BYTES : 0); // TC1: [ND] quadrature weights
    static constexpr int oD = oW + (TC1 ? ND * 4 : 0);        // !TC1: [ND][KP] moment pairs (8 B each)
    static constexpr int oRed = oD + (TC1 ? 0 : ND * KP * 8); // [4 warps][4] double
    static constexpr int oBar = oRed + 16 * 8;                // 3 mbarriers
    static constexpr int oSlot = oBar + 3 * 8;                // TMEM address
    static constexpr int bytes = oSlot + 16;
    static_assert(!TC1 || 2 * A1_BYTES == PSI_STAGE, "the flux parts replace their stage");
    static_assert(NP + 16 <= kQTmemCols, "the Eq. 3 accumulator sits after the direction columns");
};

template <int NDO, int K, int MODE>
__host__ __device__ constexpr int moments_q_smem() { return QShape<NDO, K, MODE>::bytes; }

// the byte offset of element (row, k) of a K-major operand part with 16-moment rows of ROWB bytes
template <int ROWB>
__device__ __forceinline__ int op_offset(int row, int kbyte)
{
    return (row >> 3) * (8 * ROWB) + (kbyte >> 4) * 128 + (row & 7) * 16 + (kbyte & 15);
}

// f(integral_constant<int, i>) for i = B .. E-1, unrolled at compile time
template <int B, int E, typename Fn>
__device__ __forceinline__ void static_for(Fn&& f)
{
    if constexpr (B < E) {
        f(std::integral_constant<int, B>{});
        static_for<B + 1, E>(f);
    }
}

// 8 consecutive FP32 columns of this warp's 32 TMEM lanes
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&r)[8])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
}

// (hi, lo) bf16 parts of the pair (a, b): hi = bf16(x), lo = bf16(x - hi)
__device__ __forceinline__ void bf16_split2(float a, float b, uint32_t& hi, uint32_t& lo)
{
    const __nv_bfloat16 ha = __float2bfloat16_rn(a), hb = __float2bfloat16_rn(b);
    hi = bf16x2_bits(ha, hb);
    lo = bf16x2_bits(__float2bfloat16_rn(a - __bfloat162float(ha)), __float2bfloat16_rn(b - __bfloat162float(hb)));
}

// Persistent: each CTA walks the (source, tile) items blockIdx.x, +gridDim.x,
// ... of active sources; thread t works on cell t of the item's tile. The
// item's angular fluxes arrive by bulk copies into one stage, whose next copy
// is issued as soon as the stage is consumed (after the Eq. 3 contraction), so
// it lands while the item's source is formed, contracted and stored; several
// CTAs per SM overlap their items.
template <int NDO, int K, int MODE>
__global__ void __launch_bounds__(kQThreads, 3) k_moments_q(const QParams p)
{
    using S = QShape<NDO, K, MODE>;
    constexpr int ND = S::ND, NP = S::NP, KP = S::KP, ROWB = S::ROWB;
    constexpr bool TC1 = S::TC1;
    extern __shared__ __align__(1024) unsigned char qsm[];
    float* spsi = reinterpret_cast<float*>(qsm + S::oPsi);
    unsigned char* sA = qsm + S::oA;
    unsigned char* sB = qsm + S::oB;
    unsigned char* sB1 = qsm + S::oB1;
    float* sw = reinterpret_cast<float*>(qsm + S::oW);
    unsigned long long* Dp = reinterpret_cast<unsigned long long*>(qsm + S::oD);
    double* red = reinterpret_cast<double*>(qsm + S::oRed);
    uint64_t* full = reinterpret_cast<uint64_t*>(qsm + S::oBar);   // the flux stage has landed
    uint64_t* mbar = full + 1;                                     // contraction to directions done
    uint64_t* mbar1 = full + 2;                                    // Eq. 3 contraction done
    uint32_t* slot = reinterpret_cast<uint32_t*>(qsm + S::oSlot);
    const int t = threadIdx.x, w = t >> 5, lane = t & 31, c = t;
    // the sweep keeps odd octants' (negative x cosine) Q and psi in the octant's own x order: cell c of
    // an 8 x 4 x 4 tile is c ^ 7 there
    static_assert(kQCells == 128, "8 x 4 x 4 tiles: x is the low 3 bits of the cell index");
    const int cr = c ^ 7;

    // bytes of a flux stage; the poison hook adds 16 that no copy delivers, so the stage's wait runs out
    __shared__ uint32_t stage_tx;
    if (t == 0) {
        stage_tx = (uint32_t)S::PSI_STAGE + ((!p.init && p.poison && *p.poison) ? 16u : 0u);
        mbar_init(full, 1);
        mbar_init(mbar, 1);
        mbar_init(mbar1, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (w == 0) tmem_alloc(slot, kQTmemCols);
    // B operand of the contraction to directions: the scaled operator parts, [n][k] K-major
    for (int i = t; i < 2 * NP * 16; i += kQThreads) {
        const int part = i / (NP * 16), r = i - part * NP * 16, n = r >> 4, k = r & 15;
        const float v = p.Mop[i];
        unsigned char* base = sB + part * S::B_BYTES;
        if constexpr (MODE == 0)
            *reinterpret_cast<__nv_bfloat16*>(base + op_offset<ROWB>(n, 2 * k)) = __float2bfloat16_rn(v);
        else
            *reinterpret_cast<float*>(base + op_offset<ROWB>(n, 4 * k)) = v;
    }
    if (!p.init) {
        if constexpr (TC1) {
            // B operand of the Eq. 3 contraction: D parts [k][n], K-major over the directions
            for (int i = t; i < 2 * 16 * ND; i += kQThreads) {
                const int part = i / (16 * ND), r = i - part * 16 * ND, k = r / ND, n = r - k * ND;
                *reinterpret_cast<__nv_bfloat16*>(sB1 + part * S::B1_BYTES + (k >> 3) * S::SBO1 + (n >> 3) * 128 +
                                                  (k & 7) * 16 + (n & 7) * 2) = __float2bfloat16_rn(p.Dop[i]);
            }
            for (int n = t; n < ND; n += kQThreads) sw[n] = p.Dt[n * K];   // D[0][n] = w_n
        } else {   // moment pairs (D[n][2j], D[n][2j+1]) of the Eq. 3 operator
            for (int i = t; i < ND * KP; i += kQThreads) {
                const int n = i / KP, j = i - n * KP;
                const float lo = 2 * j < K ? p.Dt[n * K + 2 * j] : 0.f, hi = 2 * j + 1 < K ? p.Dt[n * K + 2 * j + 1] : 0.f;
                Dp[i] = f2pack(lo, hi);
            }
        }
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *slot;
    const uint32_t lanes = tmem + ((uint32_t)(32 * w) << 16);   // this warp's TMEM lanes

    // the active items of this CTA, in order
    auto next_item = [&](int it) {
        for (; it < p.nitems; it += gridDim.x)
            if (p.active[it / p.NT]) return it;
        return p.nitems;
    };
    auto issue = [&](int it) {   // one item's psi: 8 octant blocks of ND/8 x 128 floats
        const int b = it / p.NT, tile = it - b * p.NT;
        constexpr uint32_t ob = NDO * kQCells * 4;
        if (!DTS_FITS((((size_t)b * 8 + 7) * p.NT + tile + 1) * (size_t)(NDO * kQCells), p.n_psi, 20)) {
            mbar_arrive(full);
            return;
        }
        mbar_expect_tx(full, stage_tx);   // set once per CTA, above
        for (int o = 0; o < 8; ++o)
            bulk_load(reinterpret_cast<unsigned char*>(spsi) + o * ob,
                      p.psi + (((size_t)b * 8 + o) * p.NT + tile) * (size_t)(NDO * kQCells), ob, full);
    };

    int it = next_item(blockIdx.x);
    if (!p.init && t == 0 && it < p.nitems) issue(it);
    uint32_t phase_full = 0u, phase_mma = 0u, phase_mma1 = 0u;
    bool failed = false;
    constexpr float kInv4Pi = 0.0795774715459476679f;
    constexpr uint32_t idesc = mma_idesc(MODE == 0 ? 1u : 2u, kQCells, NP);
    constexpr uint32_t idesc1 = mma_idesc(1u, kQCells, 16);
    constexpr int NLEG = K == 1 ? 1 : K == 4 ? 2 : K == 9 ? 3 : 4;

    while (it < p.nitems) {
        const int b = it / p.NT, tile = it - b * p.NT;
        const int nxt = next_item(it + gridDim.x);
        const int ct = tile * p.TV + c;
        float f[K], sl[NLEG], stc = 0.f;
        int mat = -1;
        double old = 0.0;
        double* ph = p.phi00 + (size_t)b * p.NC + ct;
        // the item's regions (DTS_DEBUG_BOUNDS build; constant true otherwise)
        const bool okF = DTS_FITS((size_t)p.ctl[1] * p.Fstride + ((size_t)b * p.NT + tile + 1) * (size_t)(K * p.TV),
                                  p.n_F, 21);
        const bool okS = DTS_FITS((size_t)(NLEG - 1) * p.NC + ct + 1, p.n_sigs, 22) &&
                         DTS_FITS((size_t)ct + 1, (size_t)p.NC, 26);
        const bool okP = DTS_FITS((size_t)b * p.NC + ct + 1, p.n_phi00, 23);
        const bool okQ = DTS_FITS((((size_t)b * 8 + 7) * p.NT + tile + 1) * (size_t)(NDO * p.TV), p.n_Q, 24);
        const bool okB = DTS_FITS(((size_t)b * p.NT + tile + 1) * 4, p.n_blk, 25);
        auto load_cell = [&]() {
            const float* __restrict__ F = p.F + (size_t)p.ctl[1] * p.Fstride +
                                          ((size_t)b * p.NT + tile) * (size_t)(K * p.TV) + c;
#pragma unroll
            for (int k = 0; k < K; ++k) f[k] = okF ? F[(size_t)k * p.TV] : 0.f;
#pragma unroll
            for (int l = 0; l < NLEG; ++l) sl[l] = okS ? p.sigs[(size_t)l * p.NC + ct] : 0.f;
            stc = okS ? p.sigt[ct] : 0.f;
            mat = okS ? p.mat_t[ct] : -1;
            if (!p.init && okP) old = *ph;
        };
        float T[K];
        RedTail tl;
        if (p.init) {
            load_cell();
#pragma unroll
            for (int k = 0; k < K; ++k) T[k] = f[k];
        } else {
            // the block agrees on the outcome, so that no thread leaves while others wait at a barrier
            if (__syncthreads_or(!mbar_wait(full, phase_full))) {
                failed = true;
                break;
            }
            phase_full ^= 1u;
            float os[8];   // moment 0 of each octant (FP32 sums of its directions)
            float mk[16];  // the cell's moments 1..K-1
            if constexpr (TC1) {
                uint32_t hw[ND / 2], lw[ND / 2];
#pragma unroll
                for (int o = 0; o < 8; ++o) {
                    float v[NDO];
#pragma unroll
                    for (int d = 0; d < NDO; ++d) v[d] = spsi[(o * NDO + d) * kQCells + ((o & 1) ? cr : c)];
                    float s = 0.f;
#pragma unroll
                    for (int d = 0; d < NDO; ++d) s = fmaf(sw[o * NDO + d], v[d], s);
                    os[o] = s;
#pragma unroll
                    for (int j = 0; j < NDO / 2; ++j)
                        bf16_split2(v[2 * j], v[2 * j + 1], hw[o * (NDO / 2) + j], lw[o * (NDO / 2) + j]);
                }
                __syncthreads();   // the stage is read: its bytes become the fluxes' operand parts
                unsigned char* a1 = reinterpret_cast<unsigned char*>(spsi);
#pragma unroll
                for (int q = 0; q < ND / 8; ++q) {
                    const int ofs = (c >> 3) * S::SBO1 + q * 128 + (c & 7) * 16;
                    *reinterpret_cast<uint4*>(a1 + ofs) = make_uint4(hw[4 * q], hw[4 * q + 1], hw[4 * q + 2], hw[4 * q + 3]);
                    *reinterpret_cast<uint4*>(a1 + S::A1_BYTES + ofs) =
                        make_uint4(lw[4 * q], lw[4 * q + 1], lw[4 * q + 2], lw[4 * q + 3]);
                }
                fence_async_smem();
                tc_fence_before();
                __syncthreads();
                if (t == 0) {
                    tc_fence_after();
                    const unsigned char* As[3] = {a1, a1, a1 + S::A1_BYTES};
                    const unsigned char* Bs[3] = {sB1, sB1 + S::B1_BYTES, sB1};
#pragma unroll
                    for (int pr = 0; pr < 3; ++pr)
#pragma unroll
                        for (int ks = 0; ks < ND / 16; ++ks)
                            mma_issue<0>(tmem + NP, smem_desc(As[pr] + ks * 256, 128, S::SBO1),
                                         smem_desc(Bs[pr] + ks * 256, 128, S::SBO1), idesc1,
                                         (pr | ks) ? 1u : 0u);
                    mma_commit(mbar1);
                }
                load_cell();
                if (__syncthreads_or(!mbar_wait(mbar1, phase_mma1))) {
                    failed = true;
                    break;
                }
                phase_mma1 ^= 1u;
                tc_fence_after();
                if (t == 0 && nxt < p.nitems) issue(nxt);   // the stage's operand parts are consumed
                uint32_t r[16];
                tmem_ld16(lanes + (uint32_t)NP, r);
                tmem_ld_wait();
#pragma unroll
                for (int k = 0; k < 16; ++k) mk[k] = __uint_as_float(r[k]);
            } else {
                float m1 = 0.f;
                unsigned long long acc[KP];
#pragma unroll
                for (int j = 0; j < KP; ++j) acc[j] = 0ull;
#pragma unroll 1
                for (int o = 0; o < 8; ++o) {
                    unsigned long long f0 = 0ull;   // moments (0, 1) of this octant
#pragma unroll
                    for (int d = 0; d < NDO; ++d) {
                        const float v = spsi[(o * NDO + d) * kQCells + ((o & 1) ? cr : c)];
                        const unsigned long long a = f2pack(v, v);
                        const ulonglong2* dq = reinterpret_cast<const ulonglong2*>(Dp + (o * NDO + d) * KP);
#pragma unroll
                        for (int j = 0; j < KP / 2; ++j) {
                            const ulonglong2 dd = dq[j];
                            if (j == 0) f0 = ffma2(dd.x, a, f0);
                            else acc[2 * j] = ffma2(dd.x, a, acc[2 * j]);
                            acc[2 * j + 1] = ffma2(dd.y, a, acc[2 * j + 1]);
                        }
                    }
                    float hi;
                    f2unpack(f0, os[o], hi);
                    m1 += hi;
                }
                __syncthreads();   // the stage is read
                if (t == 0 && nxt < p.nitems) issue(nxt);
                load_cell();
                mk[1] = m1;
#pragma unroll
                for (int k = 2; k < 16; ++k) {
                    if (k >= K) break;
                    float lo, hi;
                    f2unpack(acc[k / 2], lo, hi);
                    mk[k] = (k & 1) ? hi : lo;
                }
            }
            TwoSum s0;   // the scalar flux: the eight FP32 octant sums added exactly, in octant order
#pragma unroll
            for (int o = 0; o < 8; ++o) s0.add(os[o]);
            if (mat < 0) {
                if (okP) *ph = 0.0;
#pragma unroll
                for (int k = 0; k < K; ++k) T[k] = 0.f;
            } else {
                const double phi = s0.value();
                T[0] = tl.cell(s0, phi, old, f[0], sl[0], stc);
                if (okP) *ph = phi;
#pragma unroll
                for (int k = 1; k < K; ++k) T[k] = fmaf(sl[l_of_k(k)], mk[k], f[k]);
            }
        }
        // A operand row c: T' = T / (4 pi), padded to 16 moments, as (hi, lo) parts
        if constexpr (MODE == 0) {
            uint32_t hw[8], lw[8];
#pragma unroll
            for (int j = 0; j < 8; ++j)
                bf16_split2(2 * j < K ? T[2 * j] * kInv4Pi : 0.f, 2 * j + 1 < K ? T[2 * j + 1] * kInv4Pi : 0.f,
                            hw[j], lw[j]);
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                *reinterpret_cast<uint4*>(sA + op_offset<ROWB>(c, 16 * q)) =
                    make_uint4(hw[4 * q], hw[4 * q + 1], hw[4 * q + 2], hw[4 * q + 3]);
                *reinterpret_cast<uint4*>(sA + S::A_BYTES + op_offset<ROWB>(c, 16 * q)) =
                    make_uint4(lw[4 * q], lw[4 * q + 1], lw[4 * q + 2], lw[4 * q + 3]);
            }
        } else {
            uint32_t hv[16], lv[16];
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                const float a = k < K ? T[k] * kInv4Pi : 0.f;
                hv[k] = tf32_rn(a);
                lv[k] = tf32_rn(a - __uint_as_float(hv[k]));
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                *reinterpret_cast<uint4*>(sA + op_offset<ROWB>(c, 16 * q)) =
                    make_uint4(hv[4 * q], hv[4 * q + 1], hv[4 * q + 2], hv[4 * q + 3]);
                *reinterpret_cast<uint4*>(sA + S::A_BYTES + op_offset<ROWB>(c, 16 * q)) =
                    make_uint4(lv[4 * q], lv[4 * q + 1], lv[4 * q + 2], lv[4 * q + 3]);
            }
        }
        fence_async_smem();
        tc_fence_before();
        __syncthreads();   // A complete; this item's and the last item's TMEM reads are done
        if (t == 0) {
            tc_fence_after();
            // products hi.hi, hi.lo, lo.hi; bf16 takes K = 16 per instruction, tf32 K = 8 (two
            // core matrices along K, so the second K step starts 256 bytes further)
            constexpr int KSTEPS = MODE == 0 ? 1 : 2;
            const unsigned char* As[3] = {sA, sA, sA + S::A_BYTES};
            const unsigned char* Bs[3] = {sB, sB + S::B_BYTES, sB};
#pragma unroll
            for (int pr = 0; pr < 3; ++pr)
#pragma unroll
                for (int ks = 0; ks < KSTEPS; ++ks)
                    mma_issue<MODE>(tmem, smem_desc(As[pr] + ks * 256, 128, S::SBO),
                                    smem_desc(Bs[pr] + ks * 256, 128, S::SBO), idesc,
                                    (pr | ks) ? 1u : 0u);
            mma_commit(mbar);
        }
        // residual and balance partials of the item while the MMA runs
        if (!p.init) {
            float v[4] = {tl.ds, tl.ns, tl.sr, tl.ab};
#pragma unroll
            for (int o = 16; o > 0; o >>= 1)
#pragma unroll
                for (int i = 0; i < 4; ++i) v[i] += __shfl_xor_sync(0xffffffffu, v[i], o);
            if (lane == 0)
#pragma unroll
                for (int i = 0; i < 4; ++i) red[w * 4 + i] = (double)v[i];
        }
        // one barrier: the MMA wait's outcome is shared, and red[] is visible to the threads below
        if (__syncthreads_or(!mbar_wait(mbar, phase_mma))) {
            failed = true;
            break;
        }
        phase_mma ^= 1u;
        tc_fence_after();
        {
            // column n = o NDO + d of cell c goes to Q[b][o][tile][d][c], odd octants at c ^ 7
            float* qb = p.Q + ((size_t)b * 8 * p.NT + tile) * (size_t)(NDO * p.TV) + c;
            float* qbr = qb + (cr - c);
            const size_t ostr = (size_t)p.NT * (NDO * p.TV);
            static_for<0, S::NCH>([&](auto chv) {
                constexpr int ch = decltype(chv)::value;
                uint32_t r[8];
                tmem_ld8(lanes + (uint32_t)(8 * ch), r);
                tmem_ld_wait();
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    constexpr int nb = 8 * ch;
                    const int n = nb + i;
                    if (n < ND && okQ)
                        (((n / NDO) & 1) ? qbr : qb)[(size_t)(n / NDO) * ostr + (n % NDO) * p.TV] = __uint_as_float(r[i]);
                }
            });
        }
        if (!p.init && t < 4 && okB) {
            double a = 0.0;
#pragma unroll
            for (int i = 0; i < kQThreads / 32; ++i) a += red[i * 4 + t];
            p.blk[((size_t)b * p.NT + tile) * 4 + t] = t < 2 ? a : p.vol * a;
        }
        it = nxt;
    }
    if (failed && t == 0) atomicExch(p.err, 1);
    tc_fence_before();
    __syncthreads();
    if (w == 0) tmem_free(tmem, kQTmemCols);
}

}  // namespace dts
