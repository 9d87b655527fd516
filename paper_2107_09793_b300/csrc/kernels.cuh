// Host-visible launchers of the device kernels (one per kernel family).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "kernel_args.h"
#include "tc_args.h"

#define JET_COMMA ,

namespace jet {

struct LaunchCfg {
    int gx, gy, gz, block, smem, variant;
};

cudaError_t launch_direct(const DirectArgs &a, const LaunchCfg &c, cudaStream_t s);
cudaError_t set_direct_smem_limits();
cudaError_t launch_splitk_reduce(const SplitKReduceArgs &a, const LaunchCfg &c, cudaStream_t s);
cudaError_t launch_slice_reduce(const ReduceArgs &a, const LaunchCfg &c, cudaStream_t s);
cudaError_t launch_small_batch(const SmallBatchArgs &a, const LaunchCfg &c, cudaStream_t s);
cudaError_t launch_accum(const AccumArgs &a, const LaunchCfg &c, cudaStream_t s);
cudaError_t launch_accum_batch(const AccumBatchArgs &a, const LaunchCfg &c, cudaStream_t s);
cudaError_t launch_apply(const ApplyArgs &a, const LaunchCfg &c, cudaStream_t s);
cudaError_t set_apply_tc_smem_limits();
cudaError_t launch_permute(const PermuteArgs &a, const LaunchCfg &c, cudaStream_t s);
cudaError_t launch_gemm_simt(const GemmArgs &a, const LaunchCfg &c, cudaStream_t s);
cudaError_t launch_tc_split(const TcSplitArgs &a, const LaunchCfg &c, cudaStream_t s);
cudaError_t launch_tc_gemm(const TcGemmArgs &a, const LaunchCfg &c, cudaStream_t s);
cudaError_t set_tc_smem_limits();
int encode_tc_maps(TcGemmArgs &a);
cudaError_t launch_c64_to_c128(const void *src, void *dst, int64_t n, cudaStream_t s);

}  // namespace jet
