// Direct strided pairwise contraction (Section 2.3, one step of Eq. sequence):
//   C[out] = sum_k A[offA(out) + offA(k)] * B[offB(out) + offB(k)]
// evaluated from label strides, with no operand transpose.  This is the route
// for the many small contractions of a circuit network (gate absorption,
// gate-gate fusion, leaf/bra attachment, Section 2.2.1) and for
// contractions with few outputs and a long summed index (split-K).
//
// Also: the deterministic split-K partial sum, and the FP64 slice/amplitude
// reduction of Eq. sliced_sum.
#include <cuda_runtime.h>
#include <stdint.h>

#include "kernel_args.h"
#include "kernels.cuh"
#include "tc_ptx.cuh"

namespace jet {

template <typename V>
__device__ __forceinline__ V cmul_add(V acc, V x, V y)
{
    acc.x = fma(x.x, y.x, acc.x);
    acc.x = fma(-x.y, y.y, acc.x);
    acc.y = fma(x.x, y.y, acc.y);
    acc.y = fma(x.y, y.x, acc.y);
    return acc;
}

template <typename V>
__device__ __forceinline__ V vzero()
{
    V z;
    z.x = 0;
    z.y = 0;
    return z;
}

// Row decode: POW2 uses shifts (every dim a power of two), else div/mod.
template <bool POW2>
__device__ __forceinline__ void decode(int64_t r, int rank, const int64_t *dim, const int64_t *sA,
                                       const int64_t *sB, int64_t &oa, int64_t &ob)
{
    for (int j = 0; j < rank; ++j) {
        int64_t d = dim[j];
        int64_t q, dg;
        if (POW2) {
            int sh = __ffsll((unsigned long long)d) - 1;
            q = r >> sh;
            dg = r & (d - 1);
        } else {
            q = r / d;
            dg = r - q * d;
        }
        oa += dg * sA[j];
        ob += dg * sB[j];
        r = q;
    }
}

template <typename V, bool POW2>
__global__ void __launch_bounds__(256) direct_kernel(const __grid_constant__ DirectArgs a)
{
    extern __shared__ int32_t sm[];
    int32_t *sColA = sm, *sColB = sm + a.n_cols;
    int32_t *sKA = sColB + a.n_cols, *sKB = sKA + a.n_klo;
    const int32_t *gColA = (const int32_t *)a.colA, *gColB = (const int32_t *)a.colB;
    const int32_t *gKA = (const int32_t *)a.kA, *gKB = (const int32_t *)a.kB;
    for (int i = threadIdx.x; i < a.n_cols; i += blockDim.x) {
        sColA[i] = gColA[i];
        sColB[i] = gColB[i];
    }
    for (int i = threadIdx.x; i < a.n_klo; i += blockDim.x) {
        sKA[i] = gKA[i];
        sKB[i] = gKB[i];
    }
    __syncthreads();
    const uint64_t *pA = (const uint64_t *)a.ptrA, *pB = (const uint64_t *)a.ptrB, *pC = (const uint64_t *)a.ptrC;
    for (int64_t inst = blockIdx.y; inst < a.n_inst; inst += gridDim.y) {
        const V *__restrict__ A = (const V *)pA[inst];
        const V *__restrict__ B = (const V *)pB[inst];
        V *__restrict__ C = (V *)pC[inst];
        for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < a.n_out;
             e += (int64_t)gridDim.x * blockDim.x) {
            int64_t r = e / a.n_cols;
            int c = (int)(e - r * a.n_cols);
            int64_t oa = sColA[c], ob = sColB[c];
            decode<POW2>(r, a.row_rank, a.row_dim, a.row_sA, a.row_sB, oa, ob);
            V acc = vzero<V>();
            for (int64_t h = 0; h < a.n_khi; ++h) {
                int64_t ha = oa, hb = ob;
                decode<POW2>(h, a.khi_rank, a.khi_dim, a.khi_sA, a.khi_sB, ha, hb);
                for (int q = 0; q < a.n_klo; ++q) acc = cmul_add(acc, __ldg(A + ha + sKA[q]), __ldg(B + hb + sKB[q]));
            }
            C[e] = acc;
        }
    }
}

// Few outputs, long summed index: block (part, output group, instance) sums
// its slice of khi values over all klo entries, block-reduces, writes a partial.
// P > 0: the group's 8 outputs are the outer product of values of A and B, each
// loaded once per summed entry (NA + NB loads, not 16): P = NA in {1, 2, 4, 8}
// with A's NA values fastest (output j = ib * NA + ia), or P = 16 + NB with B's
// NB values fastest (j = ia * NB + ib); P = 32: one output (a dot product).
// A thread loads U table entries ahead (their loads overlap) and adds them in
// increasing entry order; with power-of-two digits the outer summed values are
// decoded 32 at a time, one per lane, and read by shuffle.
template <typename V, bool POW2, int P>
__global__ void __launch_bounds__(256) direct_splitk_kernel(const __grid_constant__ DirectArgs a)
{
    extern __shared__ __align__(16) int32_t sm[];
    int32_t *sKA = sm, *sKB = sm + a.n_klo, *sQB = sm + 2 * a.n_klo;
    __shared__ V red[JET_SPLITK_G][8];
    const int32_t *gKA = (const int32_t *)a.kA, *gKB = (const int32_t *)a.kB;
    const int32_t *gColA = (const int32_t *)a.colA, *gColB = (const int32_t *)a.colB;
    for (int i = threadIdx.x; i < a.n_klo; i += blockDim.x) {
        sKA[i] = gKA[i];
        sKB[i] = gKB[i];
        if (P == 66) sQB[i] = ((const int32_t *)a.qB)[i];
    }
    __syncthreads();
    const int64_t inst = blockIdx.z;   // P = 64: an instance block
    if (inst >= a.n_inst) return;
    const int32_t *itab = (const int32_t *)a.itab;
    const int nbk = P >= 64 ? a.blk_na * a.blk_nb : 1;
    const V *__restrict__ A = (const V *)((const uint64_t *)a.ptrA)[P >= 64 ? itab[inst * nbk] : inst];
    const V *__restrict__ B = (const V *)((const uint64_t *)a.ptrB)[P >= 64 ? itab[inst * nbk] : inst];
    const int64_t out0 = (int64_t)blockIdx.y * JET_SPLITK_G;
    const int nout = P >= 64 ? nbk : (int)((a.n_out - out0) < JET_SPLITK_G ? (a.n_out - out0) : JET_SPLITK_G);
    int64_t oa[JET_SPLITK_G], ob[JET_SPLITK_G];
    V acc[JET_SPLITK_G];
#pragma unroll
    for (int j = 0; j < JET_SPLITK_G; ++j) {
        oa[j] = ob[j] = 0;
        acc[j] = vzero<V>();
        if (j < (P >= 64 ? 1 : nout)) {   // (an instance block has one output per instance)
            int64_t e = out0 + j;
            int64_t r = e / a.n_cols;
            int c = (int)(e - r * a.n_cols);
            oa[j] = gColA[c];
            ob[j] = gColB[c];
            decode<POW2>(r, a.row_rank, a.row_dim, a.row_sA, a.row_sB, oa[j], ob[j]);
        }
    }
    const int64_t h0 = (int64_t)blockIdx.x * a.khi_per_part;
    const int64_t h1 = (h0 + a.khi_per_part) < a.n_khi ? (h0 + a.khi_per_part) : a.n_khi;
    int64_t w_h = -1, w_a = 0, w_b = 0;
    auto h_offsets = [&](int64_t h, int64_t &ha, int64_t &hb) {   // block-uniform h
        ha = hb = 0;
        if (POW2) {
            if (w_h < 0 || h - w_h >= 32) {
                w_h = h;
                w_a = w_b = 0;
                decode<true>(h + (threadIdx.x & 31), a.khi_rank, a.khi_dim, a.khi_sA, a.khi_sB, w_a, w_b);
            }
            ha = (int64_t)__shfl_sync(0xffffffffu, (long long)w_a, (int)(h - w_h));
            hb = (int64_t)__shfl_sync(0xffffffffu, (long long)w_b, (int)(h - w_h));
        } else {
            decode<false>(h, a.khi_rank, a.khi_dim, a.khi_sA, a.khi_sB, ha, hb);
        }
    };
    const int nklo = a.n_klo, bd = blockDim.x;
    constexpr bool BLK = P >= 64;          // dot products of instance blocks
    constexpr int MB = P == 64 ? 4 : 2;    // at most MB A and MB B vectors per block
    V accB[BLK ? MB : 1][BLK ? MB : 1];
    if (BLK && P == 66) {
        // B's entries of each outer value h pass through shared memory (two
        // buffers): read in B's own order (kB: B offsets ascending, so a warp's
        // loads are adjacent), stored at their inner index (qB) with one padding
        // entry per 32, and read back at the inner index q of A's loads; the
        // next h's B loads are in flight while this h is summed.  Each product
        // adds the same terms in the same order as the direct block form.
        constexpr int U = 4;
        const int na = a.blk_na, nb = a.blk_nb;
        const int PAD = nklo + (nklo >> 5);
        V *Bs = (V *)((uint8_t *)sm + (((size_t)3 * nklo * 4 + 15) & ~(size_t)15));   // [2][MB][PAD]
#pragma unroll
        for (int j = 0; j < MB; ++j)
#pragma unroll
            for (int l = 0; l < MB; ++l) accB[j][l] = vzero<V>();
        const V *__restrict__ Aj[MB];
        const V *__restrict__ Bl[MB];
#pragma unroll
        for (int j = 0; j < MB; ++j) {
            Aj[j] = j < na ? (const V *)((const uint64_t *)a.ptrA)[itab[inst * nbk + j * nb]] + oa[0] : A;
            Bl[j] = j < nb ? (const V *)((const uint64_t *)a.ptrB)[itab[inst * nbk + j]] + ob[0] : B;
        }
        V xb[U][MB];
        int64_t ha = 0, hb = 0;
        auto load_b = [&]() {
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int jq = threadIdx.x + u * bd;
                const bool ok = jq < nklo;
                const int64_t kb = hb + (ok ? sKB[jq] : 0);
#pragma unroll
                for (int l = 0; l < MB; ++l) xb[u][l] = ok && l < nb ? __ldg(Bl[l] + kb) : vzero<V>();
            }
        };
        if (h0 < h1) {
            h_offsets(h0, ha, hb);
            load_b();
        }
        int buf = 0;
        for (int64_t h = h0; h < h1; ++h) {
            V *Bb = Bs + (size_t)buf * MB * PAD;
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int jq = threadIdx.x + u * bd;
                if (jq < nklo) {
                    const int q = sQB[jq], qq = q + (q >> 5);
#pragma unroll
                    for (int l = 0; l < MB; ++l) Bb[l * PAD + qq] = xb[u][l];
                }
            }
            const int64_t ha_c = ha;
            if (h + 1 < h1) {   // block-uniform
                h_offsets(h + 1, ha, hb);
                load_b();
            }
            __syncthreads();   // this h's B entries are in place; the other buffer's readers are done
            V xa[U][MB];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int q = threadIdx.x + u * bd;
                const bool ok = q < nklo;
                const int64_t ka = ha_c + (ok ? sKA[q] : 0);
#pragma unroll
                for (int j = 0; j < MB; ++j) xa[u][j] = ok && j < na ? __ldg(Aj[j] + ka) : vzero<V>();
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int q = threadIdx.x + u * bd;
                if (q < nklo) {
                    const int qq = q + (q >> 5);
#pragma unroll
                    for (int l = 0; l < MB; ++l) {
                        if (l >= nb) continue;
                        const V vb = Bb[l * PAD + qq];
#pragma unroll
                        for (int j = 0; j < MB; ++j)
                            if (j < na) accB[j][l] = cmul_add(accB[j][l], xa[u][j], vb);
                    }
                }
            }
            buf ^= 1;
        }
    } else if (BLK) {   // dot products of an instance block: blk_na A vectors x blk_nb B vectors
        constexpr int U = 4;
        const int na = a.blk_na, nb = a.blk_nb;
#pragma unroll
        for (int j = 0; j < (BLK ? MB : 1); ++j)
#pragma unroll
            for (int l = 0; l < (BLK ? MB : 1); ++l) accB[j][l] = vzero<V>();
        const V *__restrict__ Aj[MB];
        const V *__restrict__ Bl[MB];
#pragma unroll
        for (int j = 0; j < MB; ++j) {
            Aj[j] = j < na ? (const V *)((const uint64_t *)a.ptrA)[itab[inst * nbk + j * nb]] + oa[0] : A;
            Bl[j] = j < nb ? (const V *)((const uint64_t *)a.ptrB)[itab[inst * nbk + j]] + ob[0] : B;
        }
        for (int64_t h = h0; h < h1; ++h) {
            int64_t ha, hb;
            h_offsets(h, ha, hb);
            for (int q0 = threadIdx.x; q0 < nklo; q0 += U * bd) {
                V xa[U][MB], xb[U][MB];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int q = q0 + u * bd;
                    const bool ok = q < nklo;
                    const int64_t ka = ha + (ok ? sKA[q] : 0), kb = hb + (ok ? sKB[q] : 0);
#pragma unroll
                    for (int j = 0; j < MB; ++j) {
                        xa[u][j] = ok && j < na ? __ldg(Aj[j] + ka) : vzero<V>();
                        xb[u][j] = ok && j < nb ? __ldg(Bl[j] + kb) : vzero<V>();
                    }
                }
#pragma unroll
                for (int u = 0; u < U; ++u)
                    if (q0 + u * bd < nklo) {
#pragma unroll
                        for (int j = 0; j < (BLK ? MB : 1); ++j)
#pragma unroll
                            for (int l = 0; l < (BLK ? MB : 1); ++l)
                                if (j < na && l < nb) accB[j][l] = cmul_add(accB[j][l], xa[u][j], xb[u][l]);
                    }
            }
        }
    } else if (P == 32) {   // one output
        constexpr int U = 8;
        const V *__restrict__ A0 = A + oa[0];
        const V *__restrict__ B0 = B + ob[0];
        for (int64_t h = h0; h < h1; ++h) {
            int64_t ha, hb;
            h_offsets(h, ha, hb);
            for (int q0 = threadIdx.x; q0 < nklo; q0 += U * bd) {
                V xa[U], xb[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int q = q0 + u * bd;
                    xa[u] = q < nklo ? __ldg(A0 + ha + sKA[q]) : vzero<V>();
                    xb[u] = q < nklo ? __ldg(B0 + hb + sKB[q]) : vzero<V>();
                }
#pragma unroll
                for (int u = 0; u < U; ++u)
                    if (q0 + u * bd < nklo) acc[0] = cmul_add(acc[0], xa[u], xb[u]);
            }
        }
    } else if (P > 0) {
        constexpr bool BF = P & 16;   // B's values fastest
        constexpr int NF = (P & 15) ? (P & 15) : 1, NS = JET_SPLITK_G / NF;   // fastest side's values, slowest side's
        constexpr int NA = BF ? NS : NF, NB = BF ? NF : NS, U = 4;
        for (int64_t h = h0; h < h1; ++h) {
            int64_t ha, hb;
            h_offsets(h, ha, hb);
            for (int q0 = threadIdx.x; q0 < nklo; q0 += U * bd) {
                V xa[U][NA], xb[U][NB];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int q = q0 + u * bd;
                    const bool ok = q < nklo;
                    const int64_t ka = ha + (ok ? sKA[q] : 0), kb = hb + (ok ? sKB[q] : 0);
#pragma unroll
                    for (int i = 0; i < NA; ++i) xa[u][i] = ok ? __ldg(A + oa[BF ? i * NB : i] + ka) : vzero<V>();
#pragma unroll
                    for (int i = 0; i < NB; ++i) xb[u][i] = ok ? __ldg(B + ob[BF ? i : i * NA] + kb) : vzero<V>();
                }
#pragma unroll
                for (int u = 0; u < U; ++u)
                    if (q0 + u * bd < nklo) {
#pragma unroll
                        for (int j = 0; j < JET_SPLITK_G; ++j)
                            acc[j] = cmul_add(acc[j], xa[u][BF ? j / NB : j % NA], xb[u][BF ? j % NB : j / NA]);
                    }
            }
        }
    } else {
        constexpr int U = 2;
        for (int64_t h = h0; h < h1; ++h) {
            int64_t ha, hb;
            h_offsets(h, ha, hb);
            for (int q0 = threadIdx.x; q0 < nklo; q0 += U * bd) {
                V xa[U][JET_SPLITK_G], xb[U][JET_SPLITK_G];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int q = q0 + u * bd;
                    const bool ok = q < nklo;
                    const int64_t ka = ha + (ok ? sKA[q] : 0), kb = hb + (ok ? sKB[q] : 0);
#pragma unroll
                    for (int j = 0; j < JET_SPLITK_G; ++j) {
                        xa[u][j] = ok && j < nout ? __ldg(A + oa[j] + ka) : vzero<V>();
                        xb[u][j] = ok && j < nout ? __ldg(B + ob[j] + kb) : vzero<V>();
                    }
                }
#pragma unroll
                for (int u = 0; u < U; ++u)
                    if (q0 + u * bd < nklo) {
#pragma unroll
                        for (int j = 0; j < JET_SPLITK_G; ++j)
                            if (j < nout) acc[j] = cmul_add(acc[j], xa[u][j], xb[u][j]);
                    }
            }
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (BLK) {   // product (j, l) of the block goes to slot j nb + l
#pragma unroll
        for (int j = 0; j < (BLK ? MB : 1); ++j)
#pragma unroll
            for (int l = 0; l < (BLK ? MB : 1); ++l)
                if (j < a.blk_na && l < a.blk_nb) {
                    V s = accB[j][l];
                    for (int o = 16; o > 0; o >>= 1) {
                        s.x += __shfl_xor_sync(0xffffffffu, s.x, o);
                        s.y += __shfl_xor_sync(0xffffffffu, s.y, o);
                    }
                    if (lane == 0) red[j * a.blk_nb + l][warp] = s;
                }
    } else {
#pragma unroll
        for (int j = 0; j < JET_SPLITK_G; ++j) {
            V s = acc[j];
            for (int o = 16; o > 0; o >>= 1) {
                s.x += __shfl_xor_sync(0xffffffffu, s.x, o);
                s.y += __shfl_xor_sync(0xffffffffu, s.y, o);
            }
            if (lane == 0) red[j][warp] = s;
        }
    }
    __syncthreads();
    if (threadIdx.x < nout) {
        V s = vzero<V>();
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            s.x += red[threadIdx.x][w].x;
            s.y += red[threadIdx.x][w].y;
        }
        V *part = (V *)a.partials;
        if (P >= 64) part[(int64_t)itab[inst * nbk + threadIdx.x] * a.ksplit + blockIdx.x] = s;   // one output each
        else part[(inst * a.ksplit + blockIdx.x) * a.n_out + out0 + threadIdx.x] = s;
    }
}

// Single outputs with many parts (a GEMM's dot epilogue, FP64 parts; a split-K
// dot product): a warp per output, lane l adding parts l, l + 32, ... in order
// (in the parts' precision, or FP64 for FP64 parts), then the 32 lane sums in a
// fixed butterfly (deterministic), rounded once to V.
template <typename V, typename P>
__global__ void splitk_reduce_warp_kernel(const __grid_constant__ SplitKReduceArgs a)
{
    using R = decltype(P().x);
    const int64_t inst = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (inst >= a.n_inst) return;   // warp-uniform
    const P *part = (const P *)a.partials + inst * a.ksplit;
    R sx = 0, sy = 0;
    for (int p = lane; p < a.ksplit; p += 32) {
        const P v = part[p];
        sx += v.x;
        sy += v.y;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        sx += __shfl_xor_sync(0xffffffffu, sx, o);
        sy += __shfl_xor_sync(0xffffffffu, sy, o);
    }
    if (lane == 0) {
        V r;
        r.x = sx;
        r.y = sy;
        *(V *)((const uint64_t *)a.ptrC)[inst] = r;
    }
}

// (P: the partials' type, V: the output's; FP64 partials are added in FP64 and
// rounded once)
template <typename V, typename P = V>
__global__ void splitk_reduce_kernel(const __grid_constant__ SplitKReduceArgs a)
{
    const P *part = (const P *)a.partials;
    const uint64_t *pC = (const uint64_t *)a.ptrC;
    const int64_t total = a.n_out * a.n_inst;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        int64_t inst = e / a.n_out, o = e - inst * a.n_out;
        P s = vzero<P>();
        // 8 partials loaded at a time, added in increasing part order
        for (int p0 = 0; p0 < a.ksplit; p0 += 8) {
            P x[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) x[u] = p0 + u < a.ksplit ? part[(inst * a.ksplit + p0 + u) * a.n_out + o] : vzero<P>();
#pragma unroll
            for (int u = 0; u < 8; ++u)
                if (p0 + u < a.ksplit) {
                    s.x += x[u].x;
                    s.y += x[u].y;
                }
        }
        V r;
        r.x = s.x;
        r.y = s.y;
        ((V *)pC[inst])[o] = r;
    }
}

// Many small contractions of one tree level in one launch.  Task t owns blocks
// [block0_t, block0_{t+1}); a block finds its task by binary search and walks
// the task's (instance, output) items with full offset tables.
template <typename V>
__global__ void __launch_bounds__(256) small_batch_kernel(const __grid_constant__ SmallBatchArgs a)
{
    const SmallTask *T = (const SmallTask *)a.tasks;
    int lo = 0, hi = a.n_tasks - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (T[mid].block0 <= (int)blockIdx.x) lo = mid;
        else hi = mid - 1;
    }
    const SmallTask t = T[lo];
    const int nb = (lo + 1 < a.n_tasks ? T[lo + 1].block0 : a.n_blocks) - t.block0;
    const int32_t *__restrict__ oA = (const int32_t *)t.offA, *__restrict__ oB = (const int32_t *)t.offB;
    const int32_t *__restrict__ kA = (const int32_t *)t.kA, *__restrict__ kB = (const int32_t *)t.kB;
    const int64_t total = (int64_t)t.n_inst * t.n_out;
    for (int64_t i = (int64_t)(blockIdx.x - t.block0) * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)nb * blockDim.x) {
        const int inst = (int)(i / t.n_out), o = (int)(i - (int64_t)inst * t.n_out);
        const V *__restrict__ A = (const V *)((const uint64_t *)t.ptrA)[inst];
        const V *__restrict__ B = (const V *)((const uint64_t *)t.ptrB)[inst];
        V *__restrict__ C = (V *)((const uint64_t *)t.ptrC)[inst];
        const int32_t xa = oA[o], xb = oB[o];
        V acc = vzero<V>();
        for (int q = 0; q < t.n_k; ++q) acc = cmul_add(acc, A[xa + kA[q]], B[xb + kB[q]]);
        C[o] = acc;
    }
}

// A chain of small levels in one cooperative launch (its blocks co-resident):
// a level's items are spread over every thread of the grid (task by binary
// search on its first item), and a grid barrier separates the levels.  One
// launch instead of one per level, where each would be mostly launch latency.
// The barrier is an arrival counter that block leaders wait on with a bounded
// spin (1 s, then status bit 8 and the kernel stops); the last block out sets
// both counters back to zero for the next launch.
template <typename V>
__global__ void __launch_bounds__(256) small_chain_kernel(const __grid_constant__ SmallBatchArgs a)
{
    const SmallTask *T = (const SmallTask *)a.tasks;
    __shared__ int32_t item0[JET_CHAIN_TASKS];   // the level's first items, searched here
    __shared__ int stop;
    uint32_t *arrive = (uint32_t *)a.barrier, *depart = arrive + 1;
    if (threadIdx.x == 0) stop = 0;
    const int64_t nthr = (int64_t)gridDim.x * blockDim.x;
    int t0 = 0;
    for (int l = 0; l < a.n_levels; ++l) {
        const int t1 = a.lv_end[l];
        __syncthreads();   // the previous level's readers of item0 are done
        for (int k = threadIdx.x; k < t1 - t0; k += blockDim.x) item0[k] = T[t0 + k].block0;
        __syncthreads();
        const SmallTask &tl = T[t1 - 1];
        const int64_t total = (int64_t)tl.block0 + (int64_t)tl.n_inst * tl.n_out;
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += nthr) {
            int lo = 0, hi = t1 - t0 - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if ((int64_t)item0[mid] <= i) lo = mid;
                else hi = mid - 1;
            }
            const SmallTask &t = T[t0 + lo];
            const int64_t j = i - t.block0;
            const int inst = (int)(j / t.n_out), o = (int)(j - (int64_t)inst * t.n_out);
            const int32_t *__restrict__ kA = (const int32_t *)t.kA, *__restrict__ kB = (const int32_t *)t.kB;
            const V *__restrict__ A = (const V *)((const uint64_t *)t.ptrA)[inst];
            const V *__restrict__ B = (const V *)((const uint64_t *)t.ptrB)[inst];
            V *__restrict__ C = (V *)((const uint64_t *)t.ptrC)[inst];
            const int32_t xa = ((const int32_t *)t.offA)[o], xb = ((const int32_t *)t.offB)[o];
            V acc = vzero<V>();
            for (int q = 0; q < t.n_k; ++q) acc = cmul_add(acc, A[xa + kA[q]], B[xb + kB[q]]);
            C[o] = acc;
        }
        t0 = t1;
        if (l + 1 < a.n_levels) {   // every block's outputs of this level before any block reads them
            __syncthreads();
            if (threadIdx.x == 0 && !grid_arrive_wait(arrive, (uint32_t)(l + 1) * gridDim.x, 1000000000ull)) {
                stop = 1;
                atomicOr((unsigned int *)a.status, 8u);
            }
            __syncthreads();
            if (stop) break;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {   // the last block out resets the counters
        __threadfence();
        if (atomicAdd(depart, 1u) == gridDim.x - 1) {
            atomicExch(arrive, 0u);
            atomicExch(depart, 0u);
        }
    }
}

cudaError_t launch_small_batch(const SmallBatchArgs &a, const LaunchCfg &c, cudaStream_t s)
{
    if (c.variant & 2) {   // chain of small levels: one cooperative launch, at most one block per SM
        if (a.n_levels < 1 || a.n_levels > JET_CHAIN_LEVELS || a.lv_end[a.n_levels - 1] != a.n_tasks || c.gx < 1 ||
            c.gx > 148 || c.gx != a.n_blocks || !a.barrier || !a.status)
            return cudaErrorInvalidValue;
        for (int l = 0; l < a.n_levels; ++l)
            if (a.lv_end[l] <= (l ? a.lv_end[l - 1] : 0) || a.lv_end[l] - (l ? a.lv_end[l - 1] : 0) > JET_CHAIN_TASKS)
                return cudaErrorInvalidValue;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeCooperative;
        at[0].val.cooperative = 1;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)c.gx);
        cfg.blockDim = dim3(256);
        cfg.dynamicSmemBytes = 0;
        cfg.stream = s;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        if (c.variant & 1) return cudaLaunchKernelEx(&cfg, small_chain_kernel<double2>, a);
        return cudaLaunchKernelEx(&cfg, small_chain_kernel<float2>, a);
    }
    if (c.variant & 1) small_batch_kernel<double2><<<c.gx, 256, 0, s>>>(a);
    else small_batch_kernel<float2><<<c.gx, 256, 0, s>>>(a);
    return cudaGetLastError();
}

template <typename VS, typename VT>
__global__ void __launch_bounds__(256) accum_kernel(const __grid_constant__ AccumArgs a)
{
    const int32_t *ptr = (const int32_t *)a.csr_ptr, *src = (const int32_t *)a.csr_src;
    const uint64_t *tgt = (const uint64_t *)a.tgt;
    const VS *S = (const VS *)a.src;
    const int64_t total = (int64_t)a.n_tgt * a.n;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = idx / a.n, e = idx - t * a.n;
        int64_t r = e, off = 0;
        for (int j = 0; j < a.rank; ++j) {
            const int64_t q = r / a.dim[j];
            off += (r - q * a.dim[j]) * a.tstride[j];
            r = q;
        }
        VT acc = vzero<VT>();
        for (int p = ptr[t]; p < ptr[t + 1]; ++p) {
            const VS v = S[(int64_t)src[p] * a.n + e];
            acc.x += v.x;
            acc.y += v.y;
        }
        VT *d = (VT *)tgt[t] + off;
        VT cur = *d;
        cur.x += acc.x;
        cur.y += acc.y;
        *d = cur;
    }
}

// One element of an accumulation: target t, source element e (dense source layout).
template <typename VS, typename VT>
__device__ __forceinline__ void accum_one(const AccumArgs &a, int64_t idx)
{
    const int32_t *ptr = (const int32_t *)a.csr_ptr, *src = (const int32_t *)a.csr_src;
    const uint64_t *tgt = (const uint64_t *)a.tgt;
    const VS *S = (const VS *)a.src;
    const int64_t t = idx / a.n, e = idx - t * a.n;
    int64_t r = e, off = 0;
    for (int j = 0; j < a.rank; ++j) {
        const int64_t q = r / a.dim[j];
        off += (r - q * a.dim[j]) * a.tstride[j];
        r = q;
    }
    VT acc = vzero<VT>();
    for (int p = ptr[t]; p < ptr[t + 1]; ++p) {
        const VS v = S[(int64_t)src[p] * a.n + e];
        acc.x += v.x;
        acc.y += v.y;
    }
    VT *d = (VT *)tgt[t] + off;
    VT cur = *d;
    cur.x += acc.x;
    cur.y += acc.y;
    *d = cur;
}

__global__ void __launch_bounds__(256) accum_batch_kernel(const __grid_constant__ AccumBatchArgs b)
{
    const AccumTask *T = (const AccumTask *)b.tasks;
    int lo = 0, hi = b.n_tasks - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (T[mid].block0 <= (int)blockIdx.x) lo = mid;
        else hi = mid - 1;
    }
    const AccumArgs &a = T[lo].a;
    const int nb = (lo + 1 < b.n_tasks ? T[lo + 1].block0 : b.n_blocks) - T[lo].block0;
    const int64_t total = (int64_t)a.n_tgt * a.n;
    for (int64_t i = (int64_t)(blockIdx.x - T[lo].block0) * blockDim.x + threadIdx.x; i < total;
         i += (int64_t)nb * blockDim.x) {
        if (a.src_fp64 && a.tgt_fp64) accum_one<double2, double2>(a, i);
        else if (a.tgt_fp64) accum_one<float2, double2>(a, i);
        else accum_one<float2, float2>(a, i);
    }
}

cudaError_t launch_accum_batch(const AccumBatchArgs &a, const LaunchCfg &c, cudaStream_t s)
{
    accum_batch_kernel<<<c.gx, 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_accum(const AccumArgs &a, const LaunchCfg &c, cudaStream_t s)
{
    if (a.src_fp64 && a.tgt_fp64) accum_kernel<double2, double2><<<c.gx, 256, 0, s>>>(a);
    else if (a.tgt_fp64) accum_kernel<float2, double2><<<c.gx, 256, 0, s>>>(a);
    else accum_kernel<float2, float2><<<c.gx, 256, 0, s>>>(a);
    return cudaGetLastError();
}

// amp[b][e] = sum_{s = 0 .. n_sl-1} root(b, s)[e], in FP64, one thread per
// value (e runs over the free open legs, one value when there are none).
__global__ void slice_reduce_kernel(const __grid_constant__ ReduceArgs a)
{
    const uint64_t *roots = (const uint64_t *)a.roots;
    const int64_t *eoff = (const int64_t *)a.eoff;
    const int64_t es = a.fp64_in ? 16 : 8, ne = a.n_elem;
    auto load = [&](uint64_t p, int64_t e) {
        if (ne > 1) p += (uint64_t)(eoff[e] * es);
        if (a.fp64_in) return *(const double2 *)p;
        const float2 f = *(const float2 *)p;
        return make_double2(f.x, f.y);
    };
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (a.partials) {   // per-slice partials, no summation
        if (i >= (int64_t)a.n_amps * a.n_slices * ne) return;
        ((double2 *)a.amps)[i] = load(roots[i / ne], i % ne);
        return;
    }
    if (i >= (int64_t)a.n_amps * ne) return;
    const int64_t b = i / ne, e = i % ne;
    double re = 0, im = 0;
    // 16 partials loaded at a time (their loads overlap), added in increasing slice id
    constexpr int U = 16;
    for (int s0 = 0; s0 < a.n_slices; s0 += U) {
        double2 v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) v[u] = s0 + u < a.n_slices ? load(roots[b * a.n_slices + s0 + u], e) : double2{0, 0};
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (s0 + u < a.n_slices) {
                re += v[u].x;
                im += v[u].y;
            }
    }
    ((double2 *)a.amps)[i] = make_double2(re, im);
}

__global__ void c64_to_c128_kernel(const float2 *src, double2 *dst, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        float2 v = src[i];
        dst[i] = make_double2(v.x, v.y);
    }
}

// ------------------------------------------------------------ launchers
cudaError_t launch_direct(const DirectArgs &a, const LaunchCfg &c, cudaStream_t s)
{
    dim3 grid(c.gx, c.gy, c.gz);
    bool fp64 = c.variant & 1, splitk = c.variant & 2, pow2 = c.variant & 4;
    size_t smem = c.smem;
    const int na = a.splitk_na;
    if (na != 0 && (!splitk || (na != 1 && na != 2 && na != 4 && na != 8 && na != 18 && na != 20 && na != 32 && na != 64 &&
                                na != 65 && na != 66) ||
                    (na >= 32 ? a.n_out != 1 : a.n_out % JET_SPLITK_G != 0)))
        return cudaErrorInvalidValue;
    if (na >= 64 && (!a.itab || a.blk_na < 1 || a.blk_nb < 1 || a.blk_na > (na == 64 ? 4 : 2) ||
                     a.blk_nb > (na == 64 ? 4 : 2) || a.blk_na * a.blk_nb > JET_SPLITK_G || c.gy != 1))
        return cudaErrorInvalidValue;
    // staged form: complex64 only, its tables and two buffers of 2 B vectors within the default
    // 48 KB of shared memory, every inner entry one of a thread's U = 4 loads
    if (na == 66 && (fp64 || !a.qB || a.n_klo > 4 * (int)c.block ||
                     smem < (((size_t)3 * a.n_klo * 4 + 15) & ~(size_t)15) + (size_t)2 * 2 * (a.n_klo + (a.n_klo >> 5)) * 8 ||
                     smem > 48 * 1024 - sizeof(float2) * JET_SPLITK_G * 8))
        return cudaErrorInvalidValue;
#define JET_DIRECT_LAUNCH(V, P)                                                                 \
    do {                                                                                        \
        if (splitk) {                                                                           \
            switch (na) {                                                                       \
            case 1: direct_splitk_kernel<V, P, 1><<<grid, c.block, smem, s>>>(a); break;        \
            case 2: direct_splitk_kernel<V, P, 2><<<grid, c.block, smem, s>>>(a); break;        \
            case 4: direct_splitk_kernel<V, P, 4><<<grid, c.block, smem, s>>>(a); break;        \
            case 8: direct_splitk_kernel<V, P, 8><<<grid, c.block, smem, s>>>(a); break;        \
            case 18: direct_splitk_kernel<V, P, 18><<<grid, c.block, smem, s>>>(a); break;      \
            case 20: direct_splitk_kernel<V, P, 20><<<grid, c.block, smem, s>>>(a); break;      \
            case 32: direct_splitk_kernel<V, P, 32><<<grid, c.block, smem, s>>>(a); break;      \
            case 64: direct_splitk_kernel<V, P, 64><<<grid, c.block, smem, s>>>(a); break;      \
            case 65: direct_splitk_kernel<V, P, 65><<<grid, c.block, smem, s>>>(a); break;      \
            case 66: direct_splitk_kernel<V, P, 66><<<grid, c.block, smem, s>>>(a); break;      \
            default: direct_splitk_kernel<V, P, 0><<<grid, c.block, smem, s>>>(a); break;       \
            }                                                                                   \
        } else direct_kernel<V, P><<<grid, c.block, smem, s>>>(a);                              \
    } while (0)
    if (fp64) {
        if (pow2) JET_DIRECT_LAUNCH(double2, true);
        else JET_DIRECT_LAUNCH(double2, false);
    } else {
        if (pow2) JET_DIRECT_LAUNCH(float2, true);
        else JET_DIRECT_LAUNCH(float2, false);
    }
#undef JET_DIRECT_LAUNCH
    return cudaGetLastError();
}

cudaError_t set_direct_smem_limits()
{
    const int bytes = 8 * (JET_COLMAX + JET_KLOMAX);
    cudaError_t e = cudaSuccess;
#define JET_SMEM(K)                                                                             \
    if (e == cudaSuccess) e = cudaFuncSetAttribute(K, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes)
    JET_SMEM(direct_kernel<float2 JET_COMMA true>);
    JET_SMEM(direct_kernel<float2 JET_COMMA false>);
    JET_SMEM(direct_kernel<double2 JET_COMMA true>);
    JET_SMEM(direct_kernel<double2 JET_COMMA false>);
#undef JET_SMEM
    return e;
}

cudaError_t launch_splitk_reduce(const SplitKReduceArgs &a, const LaunchCfg &c, cudaStream_t s)
{
    if (a.n_out == 1 && (a.parts64 || a.ksplit >= 64)) {   // a warp per output (grid from the outputs)
        const unsigned g = (unsigned)(((int64_t)a.n_inst * 32 + 255) / 256);
        if (a.parts64 || (c.variant & 1)) {
            if (c.variant & 1) splitk_reduce_warp_kernel<double2, double2><<<g, 256, 0, s>>>(a);
            else splitk_reduce_warp_kernel<float2, double2><<<g, 256, 0, s>>>(a);
        } else {
            splitk_reduce_warp_kernel<float2, float2><<<g, 256, 0, s>>>(a);
        }
    } else if (a.parts64) {
        if (c.variant & 1) splitk_reduce_kernel<double2, double2><<<c.gx, 256, 0, s>>>(a);
        else splitk_reduce_kernel<float2, double2><<<c.gx, 256, 0, s>>>(a);
    } else if (c.variant & 1) splitk_reduce_kernel<double2><<<c.gx, 256, 0, s>>>(a);
    else splitk_reduce_kernel<float2><<<c.gx, 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_slice_reduce(const ReduceArgs &a, const LaunchCfg &c, cudaStream_t s)
{
    if (a.n_elem < 1 || (a.n_elem > 1 && !a.eoff)) return cudaErrorInvalidValue;
    slice_reduce_kernel<<<c.gx, c.block, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_c64_to_c128(const void *src, void *dst, int64_t n, cudaStream_t s)
{
    int64_t blocks = std::min<int64_t>((n + 255) / 256, 148 * 8);
    if (blocks < 1) blocks = 1;
    c64_to_c128_kernel<<<(unsigned)blocks, 256, 0, s>>>((const float2 *)src, (double2 *)dst, n);
    return cudaGetLastError();
}

}  // namespace jet
