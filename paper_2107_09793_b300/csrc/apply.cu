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
#include <type_traits>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "kernel_args.h"
#include "kernels.cuh"
#include "tc_ptx.cuh"

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

// Offsets in A and C of fiber r (mixed radix over A's free labels, fastest
// first).  Power-of-two dims: digit j is the bit field of r at shift[j], so the
// digits decode independently of one another.
template <bool POW2>
__device__ __forceinline__ void fiber_offsets(int64_t r, const ApplyArgs &a, int64_t &oa, int64_t &oc)
{
    oa = 0;
    oc = 0;
    if (POW2) {
#pragma unroll 4
        for (int j = 0; j < a.rank; ++j) {
            const int64_t dg = (r >> a.shift[j]) & (a.dim[j] - 1);
            oa += dg * a.sA[j];
            oc += dg * a.sC[j];
        }
        return;
    }
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

// Offsets of the fiber indices b0 + k * stride (k = 0, 1, ...), the same for a
// whole warp, when every digit is a power of two (a fiber's offsets are then
// linear in the bits of its index, so a thread adds its own low part): lane l
// decodes index k0 + l, 32 values of k at a time, read by shuffle.  Calls are
// warp-uniform.
struct TileWindow {
    int64_t k0 = -64, oa = 0, oc = 0;
    __device__ __forceinline__ void get(const ApplyArgs &a, int64_t b0, int64_t stride, int64_t k, int64_t &ra,
                                        int64_t &rc)
    {
        if (k < k0 || k - k0 >= 32) {
            k0 = k;
            fiber_offsets<true>(b0 + (k0 + (int64_t)(threadIdx.x & 31)) * stride, a, oa, oc);
        }
        const int src = (int)(k - k0);
        ra = (int64_t)__shfl_sync(0xffffffffu, (long long)oa, src);
        rc = (int64_t)__shfl_sync(0xffffffffu, (long long)oc, src);
    }
};

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
    const int64_t step = (int64_t)gridDim.x * blockDim.x * FIB, b0 = (int64_t)blockIdx.x * blockDim.x * FIB;
    int64_t t_oa[FIB], t_oc[FIB];   // power-of-two digits: this thread's part of its fibers' offsets
#pragma unroll
    for (int u = 0; u < FIB; ++u) {
        t_oa[u] = t_oc[u] = 0;
        if (POW2) fiber_offsets<true>(threadIdx.x + (int64_t)u * blockDim.x, a, t_oa[u], t_oc[u]);
    }
    TileWindow win;
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
        int64_t k = 0;
        for (int64_t rb = b0; rb < a.n_fib; rb += step, ++k) {   // block-uniform fiber bases
            int64_t oa[FIB], oc[FIB], wa = 0, wc = 0;
            bool ok[FIB];
            unsigned long long x[FIB][NK];
            if (POW2) win.get(a, b0, step, k, wa, wc);
#pragma unroll
            for (int u = 0; u < FIB; ++u) {
                const int64_t r = rb + threadIdx.x + (int64_t)u * blockDim.x;
                ok[u] = r < a.n_fib;
                if (POW2) {
                    oa[u] = wa + t_oa[u];
                    oc[u] = wc + t_oc[u];
                } else {
                    fiber_offsets<false>(ok[u] ? r : 0, a, oa[u], oc[u]);
                }
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
    const int64_t step = (int64_t)gridDim.x * blockDim.x * FIB, b0 = (int64_t)blockIdx.x * blockDim.x * FIB;
    int64_t t_oa[FIB], t_oc[FIB];   // power-of-two digits: this thread's part of its fibers' offsets
#pragma unroll
    for (int u = 0; u < FIB; ++u) {
        t_oa[u] = t_oc[u] = 0;
        if (POW2) fiber_offsets<true>(threadIdx.x + (int64_t)u * blockDim.x, a, t_oa[u], t_oc[u]);
    }
    TileWindow win;
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
        int64_t k = 0;
        for (int64_t rb = b0; rb < a.n_fib; rb += step, ++k) {   // block-uniform fiber bases
            int64_t oa[FIB], oc[FIB], wa = 0, wc = 0;
            bool ok[FIB];
            if (POW2) win.get(a, b0, step, k, wa, wc);
#pragma unroll
            for (int u = 0; u < FIB; ++u) {
                const int64_t r = rb + threadIdx.x + (int64_t)u * blockDim.x;
                ok[u] = r < a.n_fib;
                if (POW2) {
                    oa[u] = wa + t_oa[u];
                    oc[u] = wc + t_oc[u];
                } else {
                    fiber_offsets<false>(ok[u] ? r : 0, a, oa[u], oc[u]);
                }
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

// ------------------------------------------------------------ tensor-core form
// The same contraction on the 5th-generation tensor cores, for a small operand
// with many summed entries (where the CUDA-core forms above are bound by their
// FMA issue rate rather than by HBM).  Written as one real matrix product per
// tile of 128 fibers:
//     D[m, 2f + c'] = sum_{q, c} A2[m, 2q + c] * B2[2f + c', 2q + c]
// with A2 the interleaved (re, im) values of A's fiber m and B2 the 2 x 2 real
// block [[Br, -Bi], [Bi, Br]] of each entry B[f, q], so row m of D holds the
// fiber's nf complex outputs as (re, im) pairs.  Both operands are split into
// TF32 hi + lo parts and the products hi.hi + hi.lo + lo.hi (one term in plain
// TF32 mode) accumulate in FP32 in tensor memory, restarting every 32 summed
// entries; chunk results are added up in FP32 registers.
//
// A CTA holds G groups of 128 threads (one fiber per thread; warp w of a group
// owns TMEM lanes 32 (w % 4) ..).  The CTA walks a contiguous range of units
// (instance, G consecutive tiles), group g taking tile g of each unit; the
// small operand's planes are rebuilt in shared memory when the instance
// changes.  Per chunk of 32 summed entries a thread: splits its gathered values
// into the group's K-major SWIZZLE_64B planes, issues the gathers of its next
// chunk (before the group barrier with one chunk per tile, after the MMA issue
// with several; they stay in flight through the wait and the epilogue), the
// group synchronises, one thread issues the MMAs and commits them to the
// group's mbarrier, every thread waits for the MMAs (bounded: ~2 s, then the
// group stops and the kernel records status bit 2) and reads its row of D.
constexpr int ATC_M = 128;     // fibers per tile: MMA M, TMEM lanes
constexpr int ATC_KC = 32;     // summed entries per chunk (64 real K = 4 blocks of 16 TF32)
constexpr int ATC_KBB = ATC_M * 64;   // bytes of one 64-byte-wide K block of an A plane

__device__ __forceinline__ uint32_t sw64(int row, int chunk16)
{
    // SWIZZLE_64B: 16-byte chunk index XOR row bits 1..2 (rows of 64 bytes, 512-byte atoms)
    return (uint32_t)(row * 64 + ((chunk16 ^ ((row >> 1) & 3)) << 4));
}

__device__ __forceinline__ void st_shared_v4(uint32_t addr, float x, float y, float z, float w)
{
    asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "f"(x), "f"(y), "f"(z), "f"(w) : "memory");
}

__device__ __forceinline__ void group_sync(int id)
{
    asm volatile("bar.sync %0, 128;" ::"r"(id) : "memory");
}

__device__ __forceinline__ bool group_any(bool v, int id)
{
    uint32_t r;
    asm volatile("{\n .reg .pred p, q;\n setp.ne.u32 q, %1, 0;\n bar.red.or.pred p, %2, 128, q;\n selp.u32 %0, 1, 0, p;\n}"
                 : "=r"(r)
                 : "r"((uint32_t)v), "r"(id)
                 : "memory");
    return r != 0;
}

// TF32 hi / lo planes of the small operand for one instance: row 2f + c' of
// K block kb holds, for the 8 summed entries q of the block, the pairs that
// multiply (re, im) of A[., q] into the real (c' = 0) or imaginary (c' = 1)
// part of output f.
__device__ __forceinline__ void atc_fill_b(const ApplyArgs &a, const float2 *__restrict__ B, uint32_t sB, int nkb,
                                           int nrl, uint32_t bplane, int tid, int nthr)
{
    const int per_blk = nrl * 4;   // 16-byte chunks per K block
    for (int i = tid; i < nkb * per_blk; i += nthr) {
        const int kb = i / per_blk, rem = i - kb * per_blk, row = rem >> 2, j = rem & 3;
        const int f = row >> 1, q0 = kb * 8 + 2 * j;
        float v[4];
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const int q = q0 + e;
            float2 b = make_float2(0.f, 0.f);
            if (f < a.nf && q < a.nk) b = B[a.bF[f] + a.bK[q]];
            if (row & 1) {   // imaginary output: Bi * Ar + Br * Ai
                v[2 * e] = b.y;
                v[2 * e + 1] = b.x;
            } else {         // real output: Br * Ar - Bi * Ai
                v[2 * e] = b.x;
                v[2 * e + 1] = -b.y;
            }
        }
        float h[4], l[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            h[e] = tf32_rna(v[e]);
            l[e] = tf32_rna(v[e] - h[e]);
        }
        const uint32_t off = (uint32_t)kb * (uint32_t)(nrl * 64) + sw64(row, j);
        st_shared_v4(sB + off, h[0], h[1], h[2], h[3]);
        st_shared_v4(sB + bplane + off, l[0], l[1], l[2], l[3]);
    }
}

// FP16 form: the power-of-two exponent that brings a chunk's largest magnitude
// m into [2^14, 2^15) (m = f 2^e, f in [0.5, 1), e = biased exponent - 126 for
// normal m; clamped to [-100, 100], 0 for m = 0), and 2^x as a float.
__device__ __forceinline__ int atc_exp16(float m)
{
    return m > 0.f ? max(-100, min(100, 141 - (int)((__float_as_uint(m) >> 23) & 0xffu))) : 0;
}
__device__ __forceinline__ float atc_pow2(int x) { return __uint_as_float((uint32_t)(127 + x) << 23); }
__device__ __forceinline__ uint32_t h2u(__half2 h) { return *(const uint32_t *)&h; }
// x = hi + lo up to rounding, both FP16 (x already scaled into FP16's range)
__device__ __forceinline__ void split_h2(float x0, float x1, uint32_t &hi, uint32_t &lo)
{
    const __half2 h = __floats2half2_rn(x0, x1);
    const float2 hf = __half22float2(h);
    hi = h2u(h);
    lo = h2u(__floats2half2_rn(x0 - hf.x, x1 - hf.y));
}

// FP16 form of atc_fill_b: K block kb holds 16 summed entries (32 halves, 64
// bytes) of each row; row r (= 2f + c') is scaled by 2^bex[sc nrl + r] in
// chunk sc of 32 entries (bex: the exponents, binv: their inverses, kept for
// the epilogue).
__device__ __forceinline__ void atc_fill_b16(const ApplyArgs &a, const float2 *__restrict__ B, uint32_t sB, int nkb16,
                                             int nrl, uint32_t bplane, int tid, int nthr, int *bex, float *binv)
{
    const int nsc = (a.nk + 31) >> 5;
    for (int i = tid; i < nsc * nrl; i += nthr) {   // one (chunk, row) per step: its largest magnitude
        const int sc = i / nrl, row = i - sc * nrl, f = row >> 1;
        float mx = 0.f;
        if (f < a.nf)
            for (int q = 32 * sc; q < min(a.nk, 32 * sc + 32); ++q) {
                const float2 b = B[a.bF[f] + a.bK[q]];
                mx = fmaxf(mx, fmaxf(fabsf(b.x), fabsf(b.y)));
            }
        const int ex = atc_exp16(mx);
        bex[i] = ex;
        binv[i] = atc_pow2(-ex);
    }
    __syncthreads();
    const int per_blk = nrl * 4;   // 16-byte chunks per K block
    for (int i = tid; i < nkb16 * per_blk; i += nthr) {
        const int kb = i / per_blk, rem = i - kb * per_blk, row = rem >> 2, j = rem & 3;
        const int f = row >> 1, q0 = kb * 16 + 4 * j;
        const float sf = atc_pow2(bex[(q0 >> 5) * nrl + row]);
        uint32_t hi[4], lo[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int q = q0 + e;
            float2 b = make_float2(0.f, 0.f);
            if (f < a.nf && q < a.nk) b = B[a.bF[f] + a.bK[q]];
            // imaginary output row: Bi * Ar + Br * Ai; real: Br * Ar - Bi * Ai
            const float v0 = (row & 1) ? b.y : b.x, v1 = (row & 1) ? b.x : -b.y;
            split_h2(v0 * sf, v1 * sf, hi[e], lo[e]);
        }
        const uint32_t off = (uint32_t)kb * (uint32_t)(nrl * 64) + sw64(row, j);
        asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(sB + off), "r"(hi[0]), "r"(hi[1]), "r"(hi[2]),
                     "r"(hi[3])
                     : "memory");
        asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(sB + bplane + off), "r"(lo[0]), "r"(lo[1]),
                     "r"(lo[2]), "r"(lo[3])
                     : "memory");
    }
}

// Bounded mbarrier wait, inlined so that the gathers a thread has in flight
// stay in flight across it (~2 s, or until another group has given up).
__device__ __forceinline__ bool mbar_wait_inline(uint32_t bar, uint32_t parity, volatile int *abort_flag)
{
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer();
    for (uint32_t it = 1; it < (1u << 30); ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 255) == 0) {
            if (*abort_flag) return false;
            if (globaltimer() - t0 > 2000000000ull) return false;
        }
    }
    return false;
}

// MULTI: more than one chunk per tile (summed entries above 32), partial sums
// promoted into FP32 registers; without it a tile is one chunk.  HALF (more
// than 64 free entries, or operand planes too large for whole chunks; two
// groups): each gathered chunk of 32 is staged in two halves of 16 summed
// entries accumulated in the same TMEM columns (as many accumulations per
// promotion as a whole chunk).
// F16: FP16 hi + lo parts (kind::f16, 16 summed reals per MMA) with a
// power-of-two scale per row and 32-entry chunk of each operand, undone when
// the chunk is promoted, instead of TF32 hi + lo (8 per MMA): half the MMAs and
// half the plane bytes for the same three products.
template <int G, bool MULTI, bool POW2, bool HALF, bool F16>
__global__ void __launch_bounds__(128 * G, 1) apply_tc_c64(const __grid_constant__ ApplyArgs a)
{
    constexpr int KC = HALF ? ATC_KC / 2 : ATC_KC;   // summed entries per staged chunk
    constexpr int EK = F16 ? 16 : 8;                 // summed entries per 64-byte K block of a plane row
    constexpr uint32_t ABY = (HALF ? JET_APPLY_TC_ABYTES / 2 : JET_APPLY_TC_ABYTES) / (F16 ? 2 : 1);   // a group's A planes
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t bars[G];
    __shared__ uint32_t tmem_holder;
    __shared__ int fail_any;
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int tid = threadIdx.x, g = tid >> 7, m = tid & 127, warp = tid >> 5;
    const int nk = a.nk, nf = a.nf, nkb = (nk + 7) >> 3, nch = (MULTI || HALF) ? (nk + KC - 1) / KC : 1;
    const int nkbx = (nk + EK - 1) / EK;    // K blocks of the small operand's planes
    const int nr = (nf + 7) >> 3;           // 16-column groups of D (8 complex outputs each)
    const int nrl = 16 * nr;                // real columns: the MMA's N
    const uint32_t bplane = (uint32_t)(nkb * nrl * 64);
    const int64_t T = (a.n_fib + ATC_M - 1) / ATC_M, U = (T + G - 1) / G, total = U * a.n_inst;
    const int64_t u0 = total * blockIdx.x / gridDim.x, u1 = total * (blockIdx.x + 1) / gridDim.x;
    const uint32_t sA = smem_u32(smem + g * ABY), sB = smem_u32(smem + G * ABY);
    // F16: the small operand's exponents and inverse scales per (32-entry chunk, row)
    int *bex = (int *)(smem + G * ABY + 2 * (size_t)nkb * (16 * ((nf + 7) >> 3)) * 64);
    float *binv = (float *)(bex + 512);
    const uint32_t bar = smem_u32(&bars[g]);
    const uint64_t *pA = (const uint64_t *)a.ptrA, *pB = (const uint64_t *)a.ptrB, *pC = (const uint64_t *)a.ptrC;
    // TMEM columns per group (the MMA's N: up to 64, 128 or 256), allocated as a power of two
    const uint32_t span = nrl <= 64 ? 64u : nrl <= 128 ? 128u : 256u, COLS = (G <= 2 ? 2u : 4u) * span;

    if (tid == 0) {
        for (int i = 0; i < G; ++i) mbar_init(smem_u32(&bars[i]), 1);
        fail_any = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_holder)),
                     "r"(COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_holder + span * g;
    const uint32_t trow = tmem + ((uint32_t)((warp & 3) * 32) << 16);
    // kind::tf32 (operand format 2) or kind::f16 with F16 operands (0), FP32 D,
    // K-major A and B, M = 128, N = nrl
    constexpr uint32_t FMT = F16 ? 0u : 2u;
    const uint32_t idesc = (1u << 4) | (FMT << 7) | (FMT << 10) | ((uint32_t)(nrl >> 3) << 17) | ((uint32_t)(ATC_M >> 4) << 24);
    const int terms = a.tc_terms;

    // Unit u is tile group u % U of instance u / U; positions advance by counters.
    // The prefetch position (the next unit whose chunk is gathered):
    int64_t p_u = u0, p_inst = u0 / U, p_tt = u0 - (u0 / U) * U;
    auto p_valid = [&]() { return p_tt * G + g < T; };
    auto p_advance = [&]() {
        ++p_u;
        if (++p_tt == U) {
            p_tt = 0;
            ++p_inst;
        }
    };
    // Power-of-two dims: a fiber's offsets are linear in the bits of its index, so
    // they are the sum of this thread's part (bits 0..6, the row m of the tile) and
    // the tile's (the higher bits, the same for the whole group).  Each warp decodes
    // the tile parts of 32 consecutive units at a time, lane l holding unit w_u + l.
    int64_t m_oa = 0, m_oc = 0, w_u = -1, w_oa = 0, w_oc = 0;
    if (POW2) fiber_offsets<true>(m, a, m_oa, m_oc);
    const int lane = tid & 31;
    auto tile_offsets = [&](int64_t &oa, int64_t &oc) {   // of the prefetch unit (warp-uniform)
        if (w_u < 0 || p_u - w_u >= 32) {
            w_u = p_u;
            const int64_t tt = (p_tt + lane) % U;
            fiber_offsets<true>((tt * G + g) * ATC_M, a, w_oa, w_oc);
        }
        const int src = (int)(p_u - w_u);
        oa = (int64_t)__shfl_sync(0xffffffffu, (long long)w_oa, src);
        oc = (int64_t)__shfl_sync(0xffffffffu, (long long)w_oc, src);
    };
    // gather one chunk of one fiber (zeros outside the operand)
    uint64_t X[ATC_KC];
    int64_t oc_next = 0, a_inst = -1;
    const unsigned long long *a_base = nullptr;
    auto gather = [&](int c) {
        const int64_t r = (p_tt * G + g) * ATC_M + m;
        const bool ok = r < a.n_fib;
        int64_t oa, oc;
        if (POW2) {
            tile_offsets(oa, oc);
            oa += m_oa;
            oc += m_oc;
        } else {
            fiber_offsets<false>(ok ? r : 0, a, oa, oc);
        }
        oc_next = oc;
        if (p_inst != a_inst) {   // the instance's base address, loaded once per instance
            a_inst = p_inst;
            a_base = (const unsigned long long *)pA[p_inst];
        }
        const unsigned long long *A = a_base + oa;
        const int kv = min(ATC_KC, nk - c * ATC_KC);
#pragma unroll
        for (int q = 0; q < ATC_KC; ++q)   // one chunk: compile-time table offsets
            X[q] = (ok && q < kv) ? __ldg(A + a.kA[(MULTI ? c * ATC_KC : 0) + q]) : 0ull;
    };

    while (p_u < u1 && !p_valid()) p_advance();
    int pc = 0;
    if (p_u < u1) gather(0);
    int64_t cur_inst = -1;
    unsigned long long *C = nullptr;
    uint32_t phase = 0;
    bool failed = false;
    float acc[MULTI ? 64 : 1];

    int64_t n_inst_u = u0 / U, n_tt = u0 - (u0 / U) * U;   // position of the loop's next unit
    for (int64_t u = u0; u < u1; ++u) {
        const int64_t inst = n_inst_u, tt = n_tt;
        if (++n_tt == U) {
            n_tt = 0;
            ++n_inst_u;
        }
        if (inst != cur_inst) {   // CTA-uniform: every group's MMAs on the old planes have completed
            __syncthreads();
            if (F16) atc_fill_b16(a, (const float2 *)pB[inst], sB, nkbx, nrl, bplane, tid, 128 * G, bex, binv);
            else atc_fill_b(a, (const float2 *)pB[inst], sB, nkb, nrl, bplane, tid, 128 * G);
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncthreads();
            cur_inst = inst;
            C = (unsigned long long *)pC[inst];
        }
        if (failed || tt * G + g >= T) continue;   // group-uniform
        const int64_t r = (tt * G + g) * ATC_M + m;
        const bool rok = r < a.n_fib;
        const int64_t oc = oc_next;
        float a_inv = 1.f;   // F16: the inverse of this fiber's scale in the current chunk of 32
        for (int c = 0; c < nch; ++c) {
            const int kv = min(KC, nk - c * KC), kbc = (kv + EK - 1) / EK;
            const int sc = HALF ? c >> 1 : c;   // the chunk of 32 entries (scale chunk)
            float a_f = 1.f;
            if (F16) {   // the chunk's scale, from all 32 gathered entries (zeros past the end)
                if (!HALF || !(c & 1)) {
                    float mx = 0.f;
#pragma unroll
                    for (int q = 0; q < ATC_KC; ++q) {
                        const float2 v = unpack2(X[q]);
                        mx = fmaxf(mx, fmaxf(fabsf(v.x), fabsf(v.y)));
                    }
                    const int ex = atc_exp16(mx);
                    a_inv = atc_pow2(-ex);
                }
                a_f = 1.f / a_inv;   // exact: a power of two in range
            }
            // split the staged entries X[OFF ..] into the hi / lo planes of row m
            // (OFF a compile-time offset: the second half of a chunk)
            auto stage = [&](auto off_tag) {
                constexpr int OFF = decltype(off_tag)::value;
                if (F16) {   // 4 entries (8 halves) per 16-byte chunk, 4 chunks per K block
#pragma unroll
                    for (int p = 0; p < KC / 4; ++p) {
                        if ((p >> 2) < kbc) {
                            uint32_t hi[4], lo[4];
#pragma unroll
                            for (int e = 0; e < 4; ++e) {
                                const float2 v = unpack2(X[OFF + 4 * p + e]);
                                split_h2(v.x * a_f, v.y * a_f, hi[e], lo[e]);
                            }
                            const uint32_t off = (uint32_t)(p >> 2) * ATC_KBB + sw64(m, p & 3);
                            asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(sA + off), "r"(hi[0]),
                                         "r"(hi[1]), "r"(hi[2]), "r"(hi[3])
                                         : "memory");
                            asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(sA + ABY / 2 + off),
                                         "r"(lo[0]), "r"(lo[1]), "r"(lo[2]), "r"(lo[3])
                                         : "memory");
                        }
                    }
                    return;
                }
#pragma unroll
                for (int p = 0; p < KC / 2; ++p) {
                    if ((p >> 2) < kbc) {
                        const float2 v0 = unpack2(X[OFF + 2 * p]), v1 = unpack2(X[OFF + 2 * p + 1]);
                        const float h0 = tf32_rna(v0.x), h1 = tf32_rna(v0.y), h2 = tf32_rna(v1.x), h3 = tf32_rna(v1.y);
                        const uint32_t off = (uint32_t)(p >> 2) * ATC_KBB + sw64(m, p & 3);
                        st_shared_v4(sA + off, h0, h1, h2, h3);
                        st_shared_v4(sA + ABY / 2 + off, tf32_rna(v0.x - h0), tf32_rna(v0.y - h1),
                                     tf32_rna(v1.x - h2), tf32_rna(v1.y - h3));
                    }
                }
            };
            if (HALF && (c & 1)) stage(std::integral_constant<int, KC>{});
            else stage(std::integral_constant<int, 0>{});
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            // The gathers of this group's next chunk (the staged registers are free;
            // a chunk's second half is already in registers) stay in flight through
            // the MMA wait and the epilogue.  With one chunk per tile they go out
            // here, ahead of the barrier and of the MMA issue, whose thread would
            // otherwise hold back the rest of its warp: the next tile's loads are
            // the tile's critical path.  With several chunks the MMAs are (the next
            // chunk is staged only once they have read the planes), so they go out
            // after the issue.
            auto gather_next = [&]() {
                bool next = true;
                if (c + 1 < nch) {
                    pc = HALF ? (c + 1) >> 1 : c + 1;   // the next chunk of 32
                    next = MULTI && (!HALF || (c & 1));
                } else {
                    p_advance();
                    while (p_u < u1 && !p_valid()) p_advance();
                    pc = 0;
                }
                if (next && p_u < u1) gather(pc);
            };
            if (!MULTI) gather_next();
            group_sync(1 + g);
            // Several chunks: a plain issue loop (the unrolled form below measured a few
            // per cent slower on those tiles, faster on one-chunk tiles).
            if (MULTI && m == 0) {
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                for (int kb = 0; kb < kbc; ++kb)
                    for (int sub = 0; sub < 2; ++sub)
                        for (int t = 0; t < terms; ++t) {
                            const int pa = t == 2, pb = t == 1;   // hi.hi, hi.lo, lo.hi
                            const uint64_t ad = sdesc(sA + pa * (ABY / 2) + kb * ATC_KBB + sub * 32);
                            const uint64_t bd =
                                sdesc(sB + pb * bplane + (uint32_t)(c * (KC / EK) + kb) * (uint32_t)(nrl * 64) + sub * 32);
                            umma<F16 ? 0 : 1>(tmem, ad, bd, idesc, ((HALF ? (c & 1) : 0) | kb | sub | t) ? 1u : 0u);
                        }
                umma_commit(bar);
            }
            if (!MULTI && m == 0) {
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                // The issue loop is unrolled with the descriptors of the chunk's first
                // K block formed once: every other operand position is an added
                // constant (descriptor start addresses count 16-byte units and all
                // planes lie below 256 KB, so an add never carries out of that field).
                // Products per (K block, 32-byte half): hi.hi, hi.lo, lo.hi.
                const uint64_t ad0 = sdesc(sA);
                const uint64_t bd0 = sdesc(sB + (uint32_t)(c * (KC / EK)) * (uint32_t)(nrl * 64));
                const uint64_t b_kb = (uint64_t)(nrl * 4), b_lo = (uint64_t)(bplane >> 4);
                constexpr uint64_t a_lo = (ABY / 2) >> 4;
                const uint32_t acc0 = HALF ? (uint32_t)(c & 1) : 0u;   // a second half adds to the first in TMEM
#pragma unroll
                for (int kb = 0; kb < KC / EK; ++kb) {
                    if (kb < kbc) {
#pragma unroll
                        for (int sub = 0; sub < 2; ++sub) {
                            const uint64_t ad = ad0 + (uint64_t)((kb * ATC_KBB + sub * 32) >> 4);
                            const uint64_t bd = bd0 + (uint64_t)kb * b_kb + (uint64_t)(sub * 2);
                            umma<F16 ? 0 : 1>(tmem, ad, bd, idesc, (acc0 | (uint32_t)kb | (uint32_t)sub) ? 1u : 0u);
                            if (terms > 1) {
                                umma<F16 ? 0 : 1>(tmem, ad, bd + b_lo, idesc, 1u);
                                umma<F16 ? 0 : 1>(tmem, ad + a_lo, bd, idesc, 1u);
                            }
                        }
                    }
                }
                umma_commit(bar);
            }
            if (MULTI) gather_next();
            const bool ok = mbar_wait_inline(bar, phase, (volatile int *)&fail_any);
            phase ^= 1u;
            if (group_any(!ok, 1 + g)) {
                failed = true;
                if (m == 0) fail_any = 1;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const bool last = c + 1 == nch;
            // D is read after every chunk of 32 (promotion) or once at the end
            const bool read_d = MULTI ? (!HALF || (c & 1) || last) : last;
            const bool first = (HALF ? c >> 1 : c) == 0;   // the tile's first chunk of 32
            // 16-column groups of D
            constexpr int HMAX = MULTI ? JET_APPLY_TC_MAXF_MULTI / 8 : HALF ? JET_APPLY_TC_MAXF / 8 : JET_APPLY_TC_WIDEF / 8;
            auto emit = [&](const int h, const uint32_t (&R)[16]) {
                // F16: undo the fiber's and the column's scales of this chunk
                float sbv[16];
#pragma unroll
                for (int j = 0; j < 16; ++j) sbv[j] = F16 ? a_inv * binv[sc * nrl + 16 * h + j] : 1.f;
                if (MULTI) {
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const float v = F16 ? __uint_as_float(R[j]) * sbv[j] : __uint_as_float(R[j]);
                        acc[(16 * h + j) % (MULTI ? 64 : 1)] = first ? v : acc[(16 * h + j) % (MULTI ? 64 : 1)] + v;
                    }
                }
                if (last && rok) {
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const int f = 8 * h + j;
                        if (f < nf) {
                            const float re = MULTI ? acc[(16 * h + 2 * j) % (MULTI ? 64 : 1)]
                                                   : __uint_as_float(R[2 * j]) * sbv[2 * j];
                            const float im = MULTI ? acc[(16 * h + 2 * j + 1) % (MULTI ? 64 : 1)]
                                                   : __uint_as_float(R[2 * j + 1]) * sbv[2 * j + 1];
                            __stcs(C + oc + a.cF[f], pack2(re, im));
                        }
                    }
                }
            };
            // 16-column groups read two at a time, one wait per pair
#pragma unroll
            for (int h = 0; h < HMAX; h += 2) {
                if (h < nr && read_d) {
                    uint32_t R0[16], R1[16];
                    JET_TMEM_LD16(trow + 16 * h, R0);
                    if (h + 1 < nr) JET_TMEM_LD16(trow + 16 * (h + 1), R1);
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                    emit(h, R0);
                    if (h + 1 < nr) emit(h + 1, R1);
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_holder), "r"(COLS));
    if (tid == 0 && fail_any) atomicOr((unsigned int *)a.status, 2u);
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

constexpr int ATC_SMEM_MAX = JET_APPLY_TC_SMEM_MAX;

cudaError_t set_apply_tc_smem_limits()
{
    cudaError_t e = cudaSuccess;
#define JET_ATCSM(G, MU, P2, W)                                                                                   \
    if (e == cudaSuccess)                                                                                         \
        e = cudaFuncSetAttribute(apply_tc_c64<G JET_COMMA MU JET_COMMA P2 JET_COMMA W JET_COMMA false>,            \
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, ATC_SMEM_MAX);                      \
    if (e == cudaSuccess)                                                                                         \
        e = cudaFuncSetAttribute(apply_tc_c64<G JET_COMMA MU JET_COMMA P2 JET_COMMA W JET_COMMA true>,             \
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, ATC_SMEM_MAX)
    JET_ATCSM(2, true, true, false);
    JET_ATCSM(2, true, false, false);
    JET_ATCSM(2, false, true, false);
    JET_ATCSM(2, false, false, false);
    JET_ATCSM(3, false, true, false);
    JET_ATCSM(3, false, false, false);
    JET_ATCSM(2, false, true, true);
    JET_ATCSM(2, false, false, true);
    JET_ATCSM(2, true, true, true);
    JET_ATCSM(2, true, false, true);
#undef JET_ATCSM
    return e;
}

template <bool F16>
static void launch_apply_tc_form(const ApplyArgs &a, const LaunchCfg &c, cudaStream_t s, int G, bool pow2, bool multi,
                                 bool half, int smem)
{
    if (multi && half) {
        if (pow2) apply_tc_c64<2, true, true, true, F16><<<c.gx, 256, smem, s>>>(a);
        else apply_tc_c64<2, true, false, true, F16><<<c.gx, 256, smem, s>>>(a);
    } else if (multi) {
        if (pow2) apply_tc_c64<2, true, true, false, F16><<<c.gx, 256, smem, s>>>(a);
        else apply_tc_c64<2, true, false, false, F16><<<c.gx, 256, smem, s>>>(a);
    } else if (half) {
        if (pow2) apply_tc_c64<2, false, true, true, F16><<<c.gx, 256, smem, s>>>(a);
        else apply_tc_c64<2, false, false, true, F16><<<c.gx, 256, smem, s>>>(a);
    } else if (G == 2) {
        if (pow2) apply_tc_c64<2, false, true, false, F16><<<c.gx, 256, smem, s>>>(a);
        else apply_tc_c64<2, false, false, false, F16><<<c.gx, 256, smem, s>>>(a);
    } else {
        if (pow2) apply_tc_c64<3, false, true, false, F16><<<c.gx, 384, smem, s>>>(a);
        else apply_tc_c64<3, false, false, false, F16><<<c.gx, 384, smem, s>>>(a);
    }
}

static cudaError_t launch_apply_tc(const ApplyArgs &a, const LaunchCfg &c, cudaStream_t s)
{
    const int G = c.block / 128;
    if ((G != 2 && G != 3) || c.block != 128 * G || a.nk < 1 || a.nk > JET_APPLY_MAXK || a.nf < 1 ||
        a.nf > JET_APPLY_TC_MAXF || (a.tc_terms != 1 && a.tc_terms != 3) || (a.tc_f16 && a.tc_terms != 3) ||
        a.rank > JET_MAXR || a.n_inst < 1 || a.n_fib < 1 || !a.status || (c.variant & 1) || c.gx < 1 || c.gy != 1)
        return cudaErrorInvalidValue;
    const int smem = jet_apply_tc_smem(G, a.nk, a.nf, a.tc_f16);
    if (smem > ATC_SMEM_MAX) return cudaErrorInvalidValue;
    const bool pow2 = c.variant & 4, multi = a.nk > ATC_KC, half = jet_apply_tc_half(a.nk, a.nf);
    // promotion registers: two groups and at most 32 free entries only; halves:
    // two groups (up to 256 TMEM columns each)
    if (multi && (G != 2 || a.nf > JET_APPLY_TC_MAXF_MULTI)) return cudaErrorInvalidValue;
    if (half && G != 2) return cudaErrorInvalidValue;
    if (a.tc_f16) launch_apply_tc_form<true>(a, c, s, G, pow2, multi, half, smem);
    else launch_apply_tc_form<false>(a, c, s, G, pow2, multi, half, smem);
    return cudaGetLastError();
}

cudaError_t launch_apply(const ApplyArgs &a, const LaunchCfg &c, cudaStream_t s)
{
    if (c.variant & 8) return launch_apply_tc(a, c, s);   // tensor-core form
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
