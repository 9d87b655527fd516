// Small-operand application (Section 2.3, one step of Eq. sequence, in the
// shape a circuit's gate takes when it is absorbed into a large state-like
// tensor):
//     C[r, f] = sum_q B[f, q] * A[r, q]
// A is the large operand, B a small one (at most JET_APPLY_MAXK summed and
// JET_APPLY_MAXF free entries, JET_APPLY_MAXB in all: a gate, a bra
// projection, an outer factor);
// r runs over A's free labels ("fibers"), q over the summed labels and f over
// B's free labels.  Each thread takes two fibers: it reads their nk values of
// A once into registers, multiplies them by B (staged in shared memory, read
// as warp-wide broadcasts) and writes the nf results, so every element of A is
// loaded by one thread only (the generic strided direct kernel loads it once
// per output it feeds) and A and C cross HBM once.  Fibers are numbered along
// A's smallest free stride first, so a warp's loads of one summed entry are
// coalesced whenever the summed labels are not the fastest ones.  The
// contraction is HBM-bound (8 * nk * nf FLOP per 8 * (nk + nf) bytes).
#include <cuda_runtime.h>
#include <stdint.h>

#include "kernel_args.h"
#include "kernels.cuh"

namespace jet {

template <typename V>
__device__ __forceinline__ void cfma(V &acc, V b, V x)
{
    acc.x = fma(b.x, x.x, acc.x);
    acc.x = fma(-b.y, x.y, acc.x);
    acc.y = fma(b.x, x.y, acc.y);
    acc.y = fma(b.y, x.x, acc.y);
}

// Packed FP32 pair FMA of sm_100+ (fma.rn.f32x2): d = a * b + c lane-wise,
// each lane rounded once like a scalar fma.  One instruction does the two FMAs
// a complex multiply-add needs per operand entry (see cmac2 below), halving
// the issue slots of the FP32 contraction.
__device__ __forceinline__ unsigned long long ffma2(unsigned long long a, unsigned long long b, unsigned long long c)
{
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

__device__ __forceinline__ unsigned long long pack2(float lo, float hi)
{
    return (unsigned long long)__float_as_uint(lo) | ((unsigned long long)__float_as_uint(hi) << 32);
}

__device__ __forceinline__ float2 unpack2(unsigned long long v)
{
    return make_float2(__uint_as_float((unsigned)(v & 0xffffffffu)), __uint_as_float((unsigned)(v >> 32)));
}

// Complex multiply-add split over two packed accumulators: with b = br + i bi,
//   p += (br, br) * (xr, xi),   m += (bi, bi) * (xr, xi),
// and the product sum is (p.x - m.y) + i (p.y + m.x) (cfinish).  sb holds the
// pairs (br, br, bi, bi) of one entry of B.
__device__ __forceinline__ void cmac2(unsigned long long &p, unsigned long long &m, const ulonglong2 &sb,
                                      unsigned long long x)
{
    p = ffma2(sb.x, x, p);
    m = ffma2(sb.y, x, m);
}

__device__ __forceinline__ float2 cfinish(unsigned long long p, unsigned long long m)
{
    const float2 a = unpack2(p), b = unpack2(m);
    return make_float2(a.x - b.y, a.y + b.x);
}

template <bool POW2>
__device__ __forceinline__ void fiber_offsets(int64_t r, const ApplyArgs &a, int64_t &oa, int64_t &oc)
{
    oa = 0;
    oc = 0;
    for (int j = 0; j < a.rank; ++j) {
        const int64_t d = a.dim[j];
        int64_t q, dg;
        if (POW2) {
            const int sh = __ffsll((unsigned long long)d) - 1;
            q = r >> sh;
            dg = r & (d - 1);
        } else {
            q = r / d;
            dg = r - q * d;
        }
        oa += dg * a.sA[j];
        oc += dg * a.sC[j];
        r = q;
    }
}

// complex64: B staged as packed pairs (br, br, bi, bi); FIB fibers per thread
// (two up to 16 summed entries, one for 32), every B entry read from shared
// memory once feeds the packed FMAs of all of them.
template <int NK, int FIB, bool POW2>
__global__ void __launch_bounds__(256) apply_kernel_c64(const __grid_constant__ ApplyArgs a)
{
    // B as plain complex values, read two summed entries per 16-byte load; the
    // packed pairs (br, br), (bi, bi) are formed in registers
    __shared__ __align__(16) float2 sB[JET_APPLY_MAXB];
    const uint64_t *pA = (const uint64_t *)a.ptrA, *pB = (const uint64_t *)a.ptrB, *pC = (const uint64_t *)a.ptrC;
    const int nf = a.nf;
    const int64_t step = (int64_t)gridDim.x * blockDim.x * FIB;
    for (int64_t inst = blockIdx.y; inst < a.n_inst; inst += gridDim.y) {
        const unsigned long long *__restrict__ A = (const unsigned long long *)pA[inst];
        const float2 *__restrict__ B = (const float2 *)pB[inst];
        unsigned long long *__restrict__ C = (unsigned long long *)pC[inst];
        __syncthreads();   // the previous instance's readers of sB are done
        for (int i = threadIdx.x; i < nf * NK; i += blockDim.x) {
            const int f = i / NK, q = i - f * NK;
            sB[i] = q < a.nk ? B[a.bF[f] + a.bK[q]] : make_float2(0.f, 0.f);   // padding is zero
        }
        __syncthreads();
        for (int64_t r0 = (int64_t)blockIdx.x * blockDim.x * FIB + threadIdx.x; r0 < a.n_fib; r0 += step) {
            int64_t oa[FIB], oc[FIB];
            bool ok[FIB];
            unsigned long long x[FIB][NK];
#pragma unroll
            for (int u = 0; u < FIB; ++u) {
                const int64_t r = r0 + (int64_t)u * blockDim.x;
                ok[u] = r < a.n_fib;
                fiber_offsets<POW2>(ok[u] ? r : 0, a, oa[u], oc[u]);
#pragma unroll
                for (int q = 0; q < NK; ++q) x[u][q] = ok[u] ? __ldg(A + oa[u] + a.kA[q]) : 0ull;
            }
            for (int f = 0; f < nf; ++f) {
                unsigned long long p[FIB], m[FIB];
#pragma unroll
                for (int u = 0; u < FIB; ++u) p[u] = m[u] = 0ull;
                if (NK == 1) {
                    const float2 v = sB[f];
                    const ulonglong2 b = make_ulonglong2(pack2(v.x, v.x), pack2(v.y, v.y));
#pragma unroll
                    for (int u = 0; u < FIB; ++u) cmac2(p[u], m[u], b, x[u][0]);
                } else {
                    const float4 *row = (const float4 *)(sB + f * NK);
#pragma unroll
                    for (int q = 0; q < NK; q += 2) {
                        const float4 v = row[q / 2];
                        const ulonglong2 b0 = make_ulonglong2(pack2(v.x, v.x), pack2(v.y, v.y));
                        const ulonglong2 b1 = make_ulonglong2(pack2(v.z, v.z), pack2(v.w, v.w));
#pragma unroll
                        for (int u = 0; u < FIB; ++u) {
                            cmac2(p[u], m[u], b0, x[u][q]);
                            cmac2(p[u], m[u], b1, x[u][q + 1]);
                        }
                    }
                }
                const int64_t cf = a.cF[f];
#pragma unroll
                for (int u = 0; u < FIB; ++u)
                    if (ok[u]) {
                        const float2 c = cfinish(p[u], m[u]);
                        __stcs(C + oc[u] + cf, pack2(c.x, c.y));
                    }
            }
        }
    }
}

// Streamed form, for a small operand with more summed entries (up to
// JET_APPLY_MAXK) and few free ones (up to JET_APPLY_STREAMF): the thread keeps
// NF outputs of its fibers in registers at a time (free entries in chunks of
// NF) and walks the summed index, one entry of A at a time, instead of holding
// the whole fiber.
template <int NF, int FIB, bool POW2>
__global__ void __launch_bounds__(256) apply_stream_c64(const __grid_constant__ ApplyArgs a)
{
    __shared__ ulonglong2 sB[JET_APPLY_MAXK * 4];   // [q][f], rows of nfp <= 4 entries
    const uint64_t *pA = (const uint64_t *)a.ptrA, *pB = (const uint64_t *)a.ptrB, *pC = (const uint64_t *)a.ptrC;
    const int nk = a.nk, nf = a.nf;
    const int nfp = (nf + NF - 1) / NF * NF;   // row length: free entries padded to whole chunks
    const int64_t step = (int64_t)gridDim.x * blockDim.x * FIB;
    for (int64_t inst = blockIdx.y; inst < a.n_inst; inst += gridDim.y) {
        const unsigned long long *__restrict__ A = (const unsigned long long *)pA[inst];
        const float2 *__restrict__ B = (const float2 *)pB[inst];
        unsigned long long *__restrict__ C = (unsigned long long *)pC[inst];
        __syncthreads();
        for (int i = threadIdx.x; i < nk * nfp; i += blockDim.x) {
            const int q = i / nfp, f = i - q * nfp;
            const float2 b = f < nf ? B[a.bF[f] + a.bK[q]] : make_float2(0.f, 0.f);
            sB[i] = make_ulonglong2(pack2(b.x, b.x), pack2(b.y, b.y));
        }
        __syncthreads();
        for (int64_t r0 = (int64_t)blockIdx.x * blockDim.x * FIB + threadIdx.x; r0 < a.n_fib; r0 += step) {
            int64_t oa[FIB], oc[FIB];
            bool ok[FIB];
#pragma unroll
            for (int u = 0; u < FIB; ++u) {
                const int64_t r = r0 + (int64_t)u * blockDim.x;
                ok[u] = r < a.n_fib;
                fiber_offsets<POW2>(ok[u] ? r : 0, a, oa[u], oc[u]);
            }
            for (int f0 = 0; f0 < nf; f0 += NF) {
                unsigned long long p[FIB][NF], m[FIB][NF];
#pragma unroll
                for (int u = 0; u < FIB; ++u)
#pragma unroll
                    for (int f = 0; f < NF; ++f) p[u][f] = m[u][f] = 0ull;
#pragma unroll 2
                for (int q = 0; q < nk; ++q) {
                    unsigned long long x[FIB];
#pragma unroll
                    for (int u = 0; u < FIB; ++u) x[u] = ok[u] ? __ldg(A + oa[u] + a.kA[q]) : 0ull;
#pragma unroll
                    for (int f = 0; f < NF; ++f) {
                        const ulonglong2 b = sB[q * nfp + f0 + f];
#pragma unroll
                        for (int u = 0; u < FIB; ++u) cmac2(p[u][f], m[u][f], b, x[u]);
                    }
                }
#pragma unroll
                for (int f = 0; f < NF; ++f)
                    if (f0 + f < nf) {
                        const int64_t cf = a.cF[f0 + f];
#pragma unroll
                        for (int u = 0; u < FIB; ++u)
                            if (ok[u]) {
                                const float2 c = cfinish(p[u][f], m[u][f]);
                                __stcs(C + oc[u] + cf, pack2(c.x, c.y));
                            }
                    }
            }
        }
    }
}

// Streamed form for 4 < nf <= JET_APPLY_STREAMF: a group of four lanes shares
// four fibers and splits the free entries, each lane keeping 4 fibers x 4
// outputs in registers (16 free entries per pass).  Every entry of B read from
// shared memory feeds 8 packed FMAs, and the four lanes of a group load the
// same A addresses (one request).  Fibers of a warp: w0 + 8 i + group.
template <bool POW2>
__global__ void __launch_bounds__(256, 2) apply_quad_c64(const __grid_constant__ ApplyArgs a)
{
    __shared__ __align__(16) float2 sB[JET_APPLY_STREAMB];   // [q][f], rows of nfp entries
    const uint64_t *pA = (const uint64_t *)a.ptrA, *pB = (const uint64_t *)a.ptrB, *pC = (const uint64_t *)a.ptrC;
    const int nk = a.nk, nf = a.nf;
    const int nfp = (nf + 15) / 16 * 16;
    const int lane = threadIdx.x & 31, grp = lane >> 2, t = lane & 3, warp = threadIdx.x >> 5;
    const int64_t step = (int64_t)gridDim.x * (blockDim.x / 32) * 32;
    constexpr int QC = 4;   // summed entries loaded ahead per round
    for (int64_t inst = blockIdx.y; inst < a.n_inst; inst += gridDim.y) {
        const unsigned long long *__restrict__ A = (const unsigned long long *)pA[inst];
        const float2 *__restrict__ B = (const float2 *)pB[inst];
        unsigned long long *__restrict__ C = (unsigned long long *)pC[inst];
        __syncthreads();
        for (int i = threadIdx.x; i < nk * nfp; i += blockDim.x) {
            const int q = i / nfp, f = i - q * nfp;
            sB[i] = f < nf ? B[a.bF[f] + a.bK[q]] : make_float2(0.f, 0.f);
        }
        __syncthreads();
        for (int64_t w0 = ((int64_t)blockIdx.x * (blockDim.x / 32) + warp) * 32; w0 < a.n_fib; w0 += step) {
            int64_t oa[4], oc[4];
            bool ok[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int64_t r = w0 + 8 * i + grp;
                ok[i] = r < a.n_fib;
                fiber_offsets<POW2>(ok[i] ? r : 0, a, oa[i], oc[i]);
            }
            for (int f0 = 0; f0 < nf; f0 += 16) {
                unsigned long long p[4][4], m[4][4];
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int ff = 0; ff < 4; ++ff) p[i][ff] = m[i][ff] = 0ull;
                const float4 *brow = (const float4 *)(sB + f0 + 4 * t);   // 4 free entries = 2 float4
                for (int q0 = 0; q0 < nk; q0 += QC) {
                    unsigned long long x[QC][4];
#pragma unroll
                    for (int qq = 0; qq < QC; ++qq)
#pragma unroll
                        for (int i = 0; i < 4; ++i)
                            x[qq][i] = (ok[i] && q0 + qq < nk) ? __ldg(A + oa[i] + a.kA[q0 + qq]) : 0ull;
#pragma unroll
                    for (int qq = 0; qq < QC; ++qq) {
                        if (q0 + qq >= nk) break;
                        const float4 v01 = brow[(size_t)(q0 + qq) * nfp / 2], v23 = brow[(size_t)(q0 + qq) * nfp / 2 + 1];
                        const ulonglong2 b[4] = {make_ulonglong2(pack2(v01.x, v01.x), pack2(v01.y, v01.y)),
                                                 make_ulonglong2(pack2(v01.z, v01.z), pack2(v01.w, v01.w)),
                                                 make_ulonglong2(pack2(v23.x, v23.x), pack2(v23.y, v23.y)),
                                                 make_ulonglong2(pack2(v23.z, v23.z), pack2(v23.w, v23.w))};
#pragma unroll
                        for (int ff = 0; ff < 4; ++ff)
#pragma unroll
                            for (int i = 0; i < 4; ++i) cmac2(p[i][ff], m[i][ff], b[ff], x[qq][i]);
                    }
                }
#pragma unroll
                for (int ff = 0; ff < 4; ++ff) {
                    const int f = f0 + 4 * t + ff;
                    if (f < nf) {
                        const int64_t cf = a.cF[f];
#pragma unroll
                        for (int i = 0; i < 4; ++i)
                            if (ok[i]) {
                                const float2 c = cfinish(p[i][ff], m[i][ff]);
                                __stcs(C + oc[i] + cf, pack2(c.x, c.y));
                            }
                    }
                }
            }
        }
    }
}

// NK: summed entries (compile time, so the fiber stays in registers); FIB:
// fibers per thread (complex128: 1).
template <typename V, int NK, int FIB, bool POW2>
__global__ void __launch_bounds__(256) apply_kernel(const __grid_constant__ ApplyArgs a)
{
    __shared__ V sB[JET_APPLY_MAXB];
    const uint64_t *pA = (const uint64_t *)a.ptrA, *pB = (const uint64_t *)a.ptrB, *pC = (const uint64_t *)a.ptrC;
    const int nf = a.nf;
    const int64_t step = (int64_t)gridDim.x * blockDim.x * FIB;
    for (int64_t inst = blockIdx.y; inst < a.n_inst; inst += gridDim.y) {
        const V *__restrict__ A = (const V *)pA[inst];
        const V *__restrict__ B = (const V *)pB[inst];
        V *__restrict__ C = (V *)pC[inst];
        __syncthreads();   // the previous instance's readers of sB are done
        for (int i = threadIdx.x; i < nf * NK; i += blockDim.x) {
            const int f = i / NK, q = i - f * NK;
            sB[i] = q < a.nk ? B[a.bF[f] + a.bK[q]] : V{0, 0};   // padded entries are zero
        }
        __syncthreads();
        for (int64_t r0 = (int64_t)blockIdx.x * blockDim.x * FIB + threadIdx.x; r0 < a.n_fib; r0 += step) {
            int64_t oa[FIB], oc[FIB];
            bool ok[FIB];
            V x[FIB][NK];
#pragma unroll
            for (int u = 0; u < FIB; ++u) {
                const int64_t r = r0 + (int64_t)u * blockDim.x;
                ok[u] = r < a.n_fib;
                fiber_offsets<POW2>(ok[u] ? r : 0, a, oa[u], oc[u]);
#pragma unroll
                for (int q = 0; q < NK; ++q) x[u][q] = ok[u] ? __ldg(A + oa[u] + a.kA[q]) : V{0, 0};
            }
            for (int f = 0; f < nf; ++f) {
                V acc[FIB];
#pragma unroll
                for (int u = 0; u < FIB; ++u) acc[u] = V{0, 0};
#pragma unroll
                for (int q = 0; q < NK; ++q) {
                    const V b = sB[f * NK + q];
#pragma unroll
                    for (int u = 0; u < FIB; ++u) cfma(acc[u], b, x[u][q]);
                }
                const int64_t cf = a.cF[f];
#pragma unroll
                for (int u = 0; u < FIB; ++u)
                    if (ok[u]) __stcs(C + oc[u] + cf, acc[u]);
            }
        }
    }
}

template <typename V, int FIB>
static void launch_nk(const ApplyArgs &a, dim3 grid, bool pow2, cudaStream_t s)
{
#define JET_APPLY(NK)                                                                       \
    do {                                                                                    \
        if (pow2) apply_kernel<V, NK, FIB, true><<<grid, 256, 0, s>>>(a);                    \
        else apply_kernel<V, NK, FIB, false><<<grid, 256, 0, s>>>(a);                        \
    } while (0)
    switch (a.nk_tmpl) {
    case 1: JET_APPLY(1); break;
    case 2: JET_APPLY(2); break;
    case 4: JET_APPLY(4); break;
    case 8: JET_APPLY(8); break;
    default: JET_APPLY(16); break;
    }
#undef JET_APPLY
}

cudaError_t launch_apply(const ApplyArgs &a, const LaunchCfg &c, cudaStream_t s)
{
    if (a.nf_tmpl > 0) {   // streamed form (complex64)
        // nf_tmpl: free entries per register chunk (1, 2, 4); 16: lane groups of four
        const int nfp = a.nf_tmpl == 16 ? (a.nf + 15) / 16 * 16 : (a.nf + a.nf_tmpl - 1) / a.nf_tmpl * a.nf_tmpl;
        const bool ok = (a.nf_tmpl == 1 || a.nf_tmpl == 2 || a.nf_tmpl == 4 || a.nf_tmpl == 16) &&
                        a.nf >= 1 && a.nf <= JET_APPLY_STREAMF && a.nk >= 1 && a.nk <= JET_APPLY_MAXK &&
                        (a.nf_tmpl == 16 ? a.nk * nfp <= JET_APPLY_STREAMB : nfp <= 4) && a.rank <= JET_MAXR &&
                        !(c.variant & 1);
        if (!ok) return cudaErrorInvalidValue;
        dim3 grid(c.gx, c.gy, 1);
        const bool pow2 = c.variant & 4;
        if (a.nf_tmpl == 16) {
            if (pow2) apply_quad_c64<true><<<grid, 256, 0, s>>>(a);
            else apply_quad_c64<false><<<grid, 256, 0, s>>>(a);
            return cudaGetLastError();
        }
#define JET_ST(NF, FIB)                                                                     \
    do {                                                                                    \
        if (pow2) apply_stream_c64<NF, FIB, true><<<grid, 256, 0, s>>>(a);                   \
        else apply_stream_c64<NF, FIB, false><<<grid, 256, 0, s>>>(a);                       \
    } while (0)
        switch (a.nf_tmpl) {
        case 1: JET_ST(1, 2); break;
        case 2: JET_ST(2, 2); break;
        default: JET_ST(4, 2); break;
        }
#undef JET_ST
        return cudaGetLastError();
    }
    const bool tmpl_ok = a.nk_tmpl == 1 || a.nk_tmpl == 2 || a.nk_tmpl == 4 || a.nk_tmpl == 8 || a.nk_tmpl == 16 ||
                         (a.nk_tmpl == 32 && !(c.variant & 1));
    if (!tmpl_ok || a.nk < 1 || a.nk > a.nk_tmpl || a.nk_tmpl > JET_APPLY_HOLDK || a.nf < 1 || a.nf > JET_APPLY_MAXF ||
        a.nf * a.nk_tmpl > JET_APPLY_MAXB || a.rank > JET_MAXR)
        return cudaErrorInvalidValue;
    dim3 grid(c.gx, c.gy, 1);
    const bool pow2 = c.variant & 4;
    if (c.variant & 1) {
        launch_nk<double2, 1>(a, grid, pow2, s);
        return cudaGetLastError();
    }
#define JET_C64(NK, FIB)                                                                   \
    do {                                                                                   \
        if (pow2) apply_kernel_c64<NK, FIB, true><<<grid, 256, 0, s>>>(a);                  \
        else apply_kernel_c64<NK, FIB, false><<<grid, 256, 0, s>>>(a);                      \
    } while (0)
    switch (a.nk_tmpl) {
    case 1: JET_C64(1, 2); break;
    case 2: JET_C64(2, 2); break;
    case 4: JET_C64(4, 2); break;
    case 8: JET_C64(8, 2); break;
    case 16: JET_C64(16, 2); break;
    default: JET_C64(32, 1); break;
    }
#undef JET_C64
    return cudaGetLastError();
}

}  // namespace jet
