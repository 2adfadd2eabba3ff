// dts_tc_launch.h -- launchers of the tensor-core forms (defined in dts_tc.cu,
// called by dts_runtime.cu; not part of the public ABI).
#pragma once
#include <cuda_runtime.h>

#include "dts_kernels.cuh"

namespace dts {
struct QParams;
}

using dts_internal_batch_fn = void (*)(const dts::SweepParams<float>, int, int, const CUtensorMap);

// dynamic shared memory of k_moments_q<ndo, K, mode> (mode 0 split BF16, 1 TF32); -1 if unsupported
int dts_internal_q_smem(int ndo, int K, int mode);
// opt the kernel into its shared-memory size (once per process and device is enough)
cudaError_t dts_internal_q_prepare(int ndo, int K, int mode);
// resident CTAs of k_moments_q per SM at its shared-memory size
cudaError_t dts_internal_q_occupancy(int ndo, int K, int mode, int* per_sm);
// one launch of k_moments_q on stream s
cudaError_t dts_internal_q_launch(int ndo, int K, int mode, const dts::QParams& p, int grid, cudaStream_t s);
// the batched sweep that reads the per-direction source Q (8 x 4 x 4 tiles) and its shared memory
dts_internal_batch_fn dts_internal_qsweep_fn(int ndo);
size_t dts_internal_qsweep_smem(int ndo);
// the first failed bounds check of this unit's kernels (DTS_DEBUG_BOUNDS build), read and cleared;
// always 0 in the normal build
unsigned long long dts_internal_tc_bounds_take();
