// Transpose half and GEMM half of a pairwise contraction (Section 3.1: each
// contraction = two partial transposes + one matrix multiply), on CUDA cores.
//
//  * permute_kernel: dst (dense, destination label order) <- src (any strides).
//  * gemm_simt_kernel: C[m][n] = sum_k A[m][k] B[k][n], complex, FP32 FMA
//    (FP64 for the FP64 mode).  This is the plain CUDA-core path the
//    tensor-core split-precision GEMM is measured against.
#include <cuda_runtime.h>
#include <stdint.h>

#include "kernel_args.h"
#include "kernels.cuh"

namespace jet {

template <typename V>
__global__ void __launch_bounds__(256) permute_kernel(const __grid_constant__ PermuteArgs a)
{
    const uint64_t *pS = (const uint64_t *)a.ptrSrc, *pD = (const uint64_t *)a.ptrDst;
    for (int64_t inst = blockIdx.y; inst < a.n_inst; inst += gridDim.y) {
        const V *__restrict__ S = (const V *)pS[inst];
        V *__restrict__ D = (V *)pD[inst];
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += (int64_t)gridDim.x * blockDim.x) {
            int64_t r = i, off = 0;
            for (int j = 0; j < a.rank; ++j) {
                int64_t d = a.dim[j];
                int64_t q = r / d;
                off += (r - q * d) * a.sstride[j];
                r = q;
            }
            D[i] = __ldg(S + off);
        }
    }
}

constexpr int SB_M = 64, SB_N = 64, SB_K = 16;

template <typename V>
__device__ __forceinline__ V czero()
{
    V z;
    z.x = 0;
    z.y = 0;
    return z;
}

template <typename V, bool AK, bool BK>
__global__ void __launch_bounds__(256) gemm_simt_kernel(const __grid_constant__ GemmArgs a)
{
    __shared__ V As[SB_K][SB_M + 1];
    __shared__ V Bs[SB_K][SB_N + 1];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int64_t M = a.M, N = a.N, K = a.K;
    const int64_t n0 = (int64_t)blockIdx.x * SB_N, tiles_m = (M + SB_M - 1) / SB_M;
    // row tiles and instances beyond the grid's y/z extent are walked by stride
    for (int64_t inst = blockIdx.z; inst < a.n_inst; inst += gridDim.z)
    for (int64_t mt = blockIdx.y; mt < tiles_m; mt += gridDim.y) {
    const int64_t m0 = mt * SB_M;
    const V *__restrict__ A = (const V *)((const uint64_t *)a.ptrA)[inst];
    const V *__restrict__ B = (const V *)((const uint64_t *)a.ptrB)[inst];
    V *__restrict__ C = (V *)((const uint64_t *)a.ptrC)[inst];
    V acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = czero<V>();
    for (int64_t k0 = 0; k0 < K; k0 += SB_K) {
#pragma unroll
        for (int l = 0; l < 4; ++l) {
            int idx = tid + 256 * l;
            int mm, kk;
            if (AK) { mm = idx >> 4; kk = idx & 15; }
            else { kk = idx >> 6; mm = idx & 63; }
            int64_t gm = m0 + mm, gk = k0 + kk;
            V v = czero<V>();
            if (gm < M && gk < K) v = AK ? __ldg(A + gm * K + gk) : __ldg(A + gk * M + gm);
            As[kk][mm] = v;
            int nn;
            if (BK) { nn = idx >> 4; kk = idx & 15; }
            else { kk = idx >> 6; nn = idx & 63; }
            int64_t gn = n0 + nn;
            gk = k0 + kk;
            V w = czero<V>();
            if (gn < N && gk < K) w = BK ? __ldg(B + gn * K + gk) : __ldg(B + gk * N + gn);
            Bs[kk][nn] = w;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < SB_K; ++kk) {
            V x[4], y[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) x[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) y[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    acc[i][j].x = fma(x[i].x, y[j].x, acc[i][j].x);
                    acc[i][j].x = fma(-x[i].y, y[j].y, acc[i][j].x);
                    acc[i][j].y = fma(x[i].x, y[j].y, acc[i][j].y);
                    acc[i][j].y = fma(x[i].y, y[j].x, acc[i][j].y);
                }
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        int64_t gm = m0 + ty + 16 * i;
        if (gm >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            int64_t gn = n0 + tx + 16 * j;
            if (gn < N) C[gm * N + gn] = acc[i][j];
        }
    }
    }
}

cudaError_t launch_permute(const PermuteArgs &a, const LaunchCfg &c, cudaStream_t s)
{
    dim3 grid(c.gx, c.gy, 1);
    if (c.variant & 1) permute_kernel<double2><<<grid, 256, 0, s>>>(a);
    else permute_kernel<float2><<<grid, 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_gemm_simt(const GemmArgs &a, const LaunchCfg &c, cudaStream_t s)
{
    dim3 grid(c.gx, c.gy, c.gz);
    const bool fp64 = c.variant & 1;
#define JET_G(V)                                                                                \
    do {                                                                                        \
        if (a.a_kmajor && a.b_kmajor) gemm_simt_kernel<V, true, true><<<grid, 256, 0, s>>>(a);   \
        else if (a.a_kmajor) gemm_simt_kernel<V, true, false><<<grid, 256, 0, s>>>(a);           \
        else if (a.b_kmajor) gemm_simt_kernel<V, false, true><<<grid, 256, 0, s>>>(a);           \
        else gemm_simt_kernel<V, false, false><<<grid, 256, 0, s>>>(a);                          \
    } while (0)
    if (fp64) JET_G(double2);
    else JET_G(float2);
#undef JET_G
    return cudaGetLastError();
}

}  // namespace jet
