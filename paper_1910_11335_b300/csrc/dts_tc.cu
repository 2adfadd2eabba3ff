// dts_tc.cu -- instantiations and launchers of the tensor-core forms: the
// fused Eq. 3 reduction + scatter-source contraction (k_moments_q) and the
// batched sweep that reads its per-direction source. Compiled as its own
// translation unit; dts_runtime.cu calls the launchers below.
#include <cuda_runtime.h>

#define DTS_SWEEP_KERNEL_ONLY
#include "dts_kernels.cuh"
#include "dts_tc.cuh"
#include "dts_tc_launch.h"

namespace dts {
namespace {

using QFn = void (*)(const QParams);

template <int NDO, int MODE>
QFn q_fn_k(int K)
{
    switch (K) {
    case 1: return k_moments_q<NDO, 1, MODE>;
    case 4: return k_moments_q<NDO, 4, MODE>;
    case 9: return k_moments_q<NDO, 9, MODE>;
    case 16: return k_moments_q<NDO, 16, MODE>;
    }
    return nullptr;
}

template <int NDO, int MODE>
int q_smem_k(int K)
{
    switch (K) {
    case 1: return moments_q_smem<NDO, 1, MODE>();
    case 4: return moments_q_smem<NDO, 4, MODE>();
    case 9: return moments_q_smem<NDO, 9, MODE>();
    case 16: return moments_q_smem<NDO, 16, MODE>();
    }
    return -1;
}

template <int MODE>
QFn q_fn_m(int ndo, int K)
{
    switch (ndo) {
    case 1: return q_fn_k<1, MODE>(K);
    case 3: return q_fn_k<3, MODE>(K);
    case 6: return q_fn_k<6, MODE>(K);
    case 10: return q_fn_k<10, MODE>(K);
    }
    return nullptr;
}

template <int MODE>
int q_smem_m(int ndo, int K)
{
    switch (ndo) {
    case 1: return q_smem_k<1, MODE>(K);
    case 3: return q_smem_k<3, MODE>(K);
    case 6: return q_smem_k<6, MODE>(K);
    case 10: return q_smem_k<10, MODE>(K);
    }
    return -1;
}

QFn q_fn(int ndo, int K, int mode) { return mode == 0 ? q_fn_m<0>(ndo, K) : q_fn_m<1>(ndo, K); }
int q_smem(int ndo, int K, int mode) { return mode == 0 ? q_smem_m<0>(ndo, K) : q_smem_m<1>(ndo, K); }

}  // namespace
}  // namespace dts

int dts_internal_q_smem(int ndo, int K, int mode) { return dts::q_smem(ndo, K, mode); }

cudaError_t dts_internal_q_prepare(int ndo, int K, int mode)
{
    const dts::QFn f = dts::q_fn(ndo, K, mode);
    if (!f) return cudaErrorInvalidValue;
    const cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, dts::q_smem(ndo, K, mode));
    if (e != cudaSuccess) return e;
    // all of the unified L1/shared array as shared memory, so that more than one CTA fits per SM
    return cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
}

// resident CTAs per SM from the kernel's registers and shared memory (all of the L1/shared array
// as shared memory, as dts_internal_q_prepare requests)
cudaError_t dts_internal_q_occupancy(int ndo, int K, int mode, int* per_sm)
{
    const dts::QFn f = dts::q_fn(ndo, K, mode);
    if (!f) return cudaErrorInvalidValue;
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, f);
    if (e != cudaSuccess) return e;
    int dev = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    int smem_sm = 0, smem_rsv = 0, regs_sm = 0;
    if ((e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&smem_rsv, cudaDevAttrReservedSharedMemoryPerBlock, dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev)) != cudaSuccess) return e;
    const int by_smem = smem_sm / (dts::q_smem(ndo, K, mode) + smem_rsv);
    const int by_regs = regs_sm / (dts::kQThreads * (fa.numRegs > 0 ? fa.numRegs : 1));
    *per_sm = by_smem < by_regs ? by_smem : by_regs;
    return cudaSuccess;
}

cudaError_t dts_internal_q_launch(int ndo, int K, int mode, const dts::QParams& p, int grid, cudaStream_t s)
{
    const dts::QFn f = dts::q_fn(ndo, K, mode);
    if (!f) return cudaErrorInvalidValue;
    f<<<grid, dts::kQThreads, (size_t)dts::q_smem(ndo, K, mode), s>>>(p);
    return cudaGetLastError();
}

dts_internal_batch_fn dts_internal_qsweep_fn(int ndo)
{
    switch (ndo) {
    case 1: return dts::k_sweep_batch<1, 1, 8, true, true>;
    case 3: return dts::k_sweep_batch<3, 1, 8, true, true>;
    case 6: return dts::k_sweep_batch<6, 1, 8, true, true>;
    case 10: return dts::k_sweep_batch<10, 1, 8, true, true>;
    }
    return nullptr;
}

size_t dts_internal_qsweep_smem(int ndo)
{
    switch (ndo) {
    case 1: return dts::sweep_batch_smem<1, 1, 8, true, true>();
    case 3: return dts::sweep_batch_smem<3, 1, 8, true, true>();
    case 6: return dts::sweep_batch_smem<6, 1, 8, true, true>();
    case 10: return dts::sweep_batch_smem<10, 1, 8, true, true>();
    }
    return 0;
}

unsigned long long dts_internal_tc_bounds_take()
{
#ifdef DTS_DEBUG_BOUNDS
    unsigned long long w = 0, z = 0;
    cudaMemcpyFromSymbol(&w, dts::bounds_word, sizeof w);
    cudaMemcpyToSymbol(dts::bounds_word, &z, sizeof z);
    return w;
#else
    return 0;
#endif
}
