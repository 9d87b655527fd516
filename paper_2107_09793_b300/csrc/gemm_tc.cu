// Tensor-core route of a pairwise contraction (Section 3.1's matrix multiply),
// written for the 5th-generation tensor cores of sm_103a.
//
// Complex product in the 4M real form with split precision:
//   x = x_hi + x_lo (+ x_mid) in BF16 or TF32;  a*b ~ sum of the split terms
//   whose magnitude is above the working precision (3 terms for a 2-way split,
//   6 for BF16 3-way), accumulated in FP32.
//   Re C = sum Ar.Br + (-Ai).Bi,  Im C = sum Ar.Bi + Ai.Br, each in one FP32
//   accumulator, term by term (the negated product uses the instruction
//   descriptor's negate-A bit).
//
// tc_split_kernel gathers a complex64 operand from any strides into K-major
// padded planes (the transpose of Section 3.1 fused with the split).
// tc_gemm_kernel: persistent over 128x128 output tiles; warp 0 issues TMA
// loads of all planes of a K-block into a SWIZZLE_64B stage ring, warp 1
// allocates TMEM and one thread issues tcgen05.mma into 32-wide K chunks of
// double-buffered TMEM accumulators, warps 2-9 add each chunk into FP32
// registers and write complex64 C.  Every mbarrier wait is bounded: on
// time-out the CTA records a status bit, frees its TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "kernels.cuh"
#include "tc_args.h"
#include "tc_ptx.cuh"

namespace jet {

constexpr int TC_BM = 128;          // tile rows (M) and tile columns (N)
constexpr int TC_BN = 128;
constexpr int TC_ROWB = 64;         // bytes of K per stage row (SWIZZLE_64B span)
constexpr int TC_PLANE_TILE = TC_BM * TC_ROWB;   // 8 KiB per plane tile
constexpr uint32_t TC_TMEM_COLS = 512;   // two chunk buffers x (Re 128 + Im 128 columns)

template <int MODE>
struct TcCfg;
// FMT: operand format code of the instruction descriptor (F16 0, BF16 1, TF32 2).
// SCALED: operand rows carry a power-of-two scale per 32-wide K chunk.
template <>
struct TcCfg<JET_PREC_TF32> {
    static constexpr int NP = 2, NT = 1, EB = 4, KIND = 1, STAGES = 4, FMT = 2, CHUNK_K = 64;
    static constexpr bool SCALED = false;
    __device__ static void term(int t, int &p, int &q) { p = 0; q = 0; }
};
template <>
struct TcCfg<JET_PREC_TF32X3> {
    static constexpr int NP = 4, NT = 3, EB = 4, KIND = 1, STAGES = 2, FMT = 2, CHUNK_K = 32;
    static constexpr bool SCALED = false;
    __device__ static void term(int t, int &p, int &q) { p = (t == 2); q = (t == 1); }   // lo.lo dropped
};
template <>
struct TcCfg<JET_PREC_BF16X3> {
    static constexpr int NP = 4, NT = 3, EB = 2, KIND = 0, STAGES = 2, FMT = 1, CHUNK_K = 64;
    static constexpr bool SCALED = false;
    __device__ static void term(int t, int &p, int &q) { p = (t == 2); q = (t == 1); }
};
template <>
struct TcCfg<JET_PREC_FP16X3> {
    static constexpr int NP = 4, NT = 3, EB = 2, KIND = 0, STAGES = 2, FMT = 0, CHUNK_K = 64;
    static constexpr bool SCALED = true;
    __device__ static void term(int t, int &p, int &q) { p = (t == 2); q = (t == 1); }
};
template <>
struct TcCfg<JET_PREC_BF16X6> {
    static constexpr int NP = 6, NT = 6, EB = 2, KIND = 0, STAGES = 2, FMT = 1, CHUNK_K = 32;
    static constexpr bool SCALED = false;
    // hi=0, mid=1, lo=2: hh, hm, mh, hl, lh, mm
    __device__ static void term(int t, int &p, int &q)
    {
        const int P[6] = {0, 0, 1, 0, 2, 1}, Q[6] = {0, 1, 0, 2, 0, 1};
        p = P[t];
        q = Q[t];
    }
};

// ------------------------------------------------------------------ split kernel

// The mode's parts of one value, largest first (x = p0 + p1 + p2 up to rounding).
template <int MODE>
__device__ __forceinline__ void split_parts(float x, float (&p)[3])
{
    if (MODE == JET_PREC_TF32) {
        p[0] = tf32_rna(x);
    } else if (MODE == JET_PREC_TF32X3) {
        p[0] = tf32_rna(x);
        p[1] = tf32_rna(x - p[0]);
    } else if (MODE == JET_PREC_BF16X3) {
        p[0] = __bfloat162float(__float2bfloat16_rn(x));
        p[1] = __bfloat162float(__float2bfloat16_rn(x - p[0]));
    } else if (MODE == JET_PREC_FP16X3) {   // x already scaled into FP16 range
        p[0] = __half2float(__float2half_rn(x));
        p[1] = __half2float(__float2half_rn(x - p[0]));
    } else {
        p[0] = __bfloat162float(__float2bfloat16_rn(x));
        const float r = x - p[0];
        p[1] = __bfloat162float(__float2bfloat16_rn(r));
        p[2] = __bfloat162float(__float2bfloat16_rn(r - p[1]));
    }
}

// Four adjacent values of one component (re or im) split into the mode's
// planes, each plane's four parts packed as they are stored: 16-bit formats two
// per word (w[p][0..1]), TF32 one per word (w[p][0..3]).  Every part is the
// same rounding of the same remainder as split_parts.
__device__ __forceinline__ uint32_t h2_bits(__half2 h) { return *(const uint32_t *)&h; }
__device__ __forceinline__ uint32_t b2_bits(__nv_bfloat162 h) { return *(const uint32_t *)&h; }
template <int MODE>
__device__ __forceinline__ void split4(const float (&x)[4], uint32_t (&w)[TcCfg<MODE>::NP / 2][TcCfg<MODE>::EB])
{
    if constexpr (MODE == JET_PREC_FP16X3) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const __half2 hi = __floats2half2_rn(x[2 * h], x[2 * h + 1]);
            const float2 hf = __half22float2(hi);
            w[0][h] = h2_bits(hi);
            w[1][h] = h2_bits(__floats2half2_rn(x[2 * h] - hf.x, x[2 * h + 1] - hf.y));
        }
    } else if constexpr (MODE == JET_PREC_BF16X3) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const __nv_bfloat162 hi = __floats2bfloat162_rn(x[2 * h], x[2 * h + 1]);
            const float2 hf = __bfloat1622float2(hi);
            w[0][h] = b2_bits(hi);
            w[1][h] = b2_bits(__floats2bfloat162_rn(x[2 * h] - hf.x, x[2 * h + 1] - hf.y));
        }
    } else if constexpr (MODE == JET_PREC_BF16X6) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const __nv_bfloat162 hi = __floats2bfloat162_rn(x[2 * h], x[2 * h + 1]);
            const float2 hf = __bfloat1622float2(hi);
            const float r0 = x[2 * h] - hf.x, r1 = x[2 * h + 1] - hf.y;
            const __nv_bfloat162 mid = __floats2bfloat162_rn(r0, r1);
            const float2 mf = __bfloat1622float2(mid);
            w[0][h] = b2_bits(hi);
            w[1][h] = b2_bits(mid);
            w[2][h] = b2_bits(__floats2bfloat162_rn(r0 - mf.x, r1 - mf.y));
        }
    } else {   // TF32, TF32x3: FP32 words
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            float p[3];
            split_parts<MODE>(x[c], p);
#pragma unroll
            for (int q = 0; q < TcCfg<MODE>::NP / 2; ++q) w[q][c] = __float_as_uint(p[q]);
        }
    }
}

constexpr int SPLIT_TR = 64, SPLIT_TK = 64;
constexpr int SPLIT_ROW = SPLIT_TK + 2;   // padded tile row (float2; even: 16-byte pairs stay aligned)
constexpr int SPLIT_SMEM = 2 * SPLIT_TR * SPLIT_ROW * 8               // two tiles
                           + 2 * (SPLIT_TR + SPLIT_TK) * 8            // their row / column offsets
                           + 3 * SPLIT_TR * 8;                        // plane rows (three tiles: one is
                                                                      // read while the next-but-one's are decoded)

// (no memory clobber: the copies' shared-memory writes are ordered by the
// wait_group and barrier that follow, which carry it; the offsets they read
// stay in registers across a tile's copies)
__device__ __forceinline__ void cp_async8_zfill(uint32_t dst, const void *src, uint32_t src_bytes)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(dst), "l"(src), "r"(src_bytes));
}
__device__ __forceinline__ void cp_async16_zfill(uint32_t dst, const void *src, uint32_t src_bytes)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(src_bytes));
}

// Tiled gather + split: a block walks 64-row x 64-column tiles of the planes.
// Two tiles are in flight: while one is split and written, the next one's
// source elements are already being copied into shared memory by cp.async
// (8-byte copies, zero-filled outside the operand), so the loads of a block
// never wait behind its own conversion work.  The source offsets of a tile's
// rows and columns are decoded once into shared memory; elements are read with
// threads running along the source's fastest label (rows or K, fast_k) and
// written along K, two values per thread.
template <int MODE, bool POW2>
__global__ void __launch_bounds__(256, 3) tc_split_kernel(const __grid_constant__ TcSplitArgs a)
{
    constexpr int NP = TcCfg<MODE>::NP, EB = TcCfg<MODE>::EB, NPH = NP / 2;
    extern __shared__ __align__(16) uint8_t split_smem[];
    float2 *tiles_s = (float2 *)split_smem;                                        // [2][64][65]
    int64_t *offs = (int64_t *)(split_smem + 2 * SPLIT_TR * SPLIT_ROW * 8);       // [2][64 + 64]
    int64_t *prows = offs + 2 * (SPLIT_TR + SPLIT_TK);                              // [3][64]
    const int tid = threadIdx.x;
    const int64_t k_tiles = (a.k_pad + SPLIT_TK - 1) / SPLIT_TK;
    const int64_t plane_elems = a.rows_group * a.k_pad;

    auto decode = [&](int64_t t, int buf, int pbuf) {   // threads 0..127: one row or column offset each
        static_assert(SPLIT_TR + SPLIT_TK <= 256, "one decoding thread per tile row and column");
        if (tid < SPLIT_TR + SPLIT_TK) {
            const int64_t rt = t / k_tiles, kt = t - rt * k_tiles;
            const bool is_row = tid < SPLIT_TR;
            int64_t x = is_row ? rt * SPLIT_TR + tid : kt * SPLIT_TK + (tid - SPLIT_TR), off = -1;
            int64_t prow = x;   // (rows: plane row; padding rows and the identity order: x)
            if (x < (is_row ? a.rows : a.k)) {
                off = 0;
                const bool perm = is_row && a.row_perm;
                if (perm) prow = 0;
                const int rank = is_row ? a.rank_r : a.rank_k;
                const int64_t *dim = is_row ? a.r_dim : a.k_dim, *str = is_row ? a.r_s : a.k_s;
                for (int jj = 0; jj < rank; ++jj) {
                    const int64_t d = dim[jj];
                    int64_t q, r;
                    if (POW2) {
                        const int sh = __ffsll((unsigned long long)d) - 1;
                        q = x >> sh;
                        r = x & (d - 1);
                    } else {
                        q = x / d;
                        r = x - q * d;
                    }
                    off += r * str[jj];
                    if (perm) prow += r * a.p_s[jj];
                    x = q;
                }
            }
            offs[buf * (SPLIT_TR + SPLIT_TK) + tid] = off;
            if (is_row) prows[pbuf * SPLIT_TR + tid] = prow;
        }
    };
    auto issue = [&](const float2 *S, int buf) {   // 16 zero-filling 8-byte copies per thread
        const int64_t *rowOff = offs + buf * (SPLIT_TR + SPLIT_TK), *kOff = rowOff + SPLIT_TR;
        float2 *tile = tiles_s + (size_t)buf * SPLIT_TR * SPLIT_ROW;
        if (a.pair16) {
            // the fastest summed label has stride 1 (and K is even): entries 2c and
            // 2c + 1 of a row are adjacent in the source and in the tile, one
            // 16-byte copy each (8 per thread)
#pragma unroll
            for (int i = 0; i < (SPLIT_TR * SPLIT_TK) / 512; ++i) {
                const int kk = 2 * (tid & (SPLIT_TK / 2 - 1)), r = (tid >> 5) + (256 / (SPLIT_TK / 2)) * i;
                const int64_t ro = rowOff[r], ko = kOff[kk];
                const bool in = ro >= 0 && ko >= 0;
                cp_async16_zfill(smem_u32(tile + r * SPLIT_ROW + kk), in ? (const void *)(S + ro + ko) : (const void *)S,
                                 in ? 16u : 0u);
            }
            return;
        }
        if (a.fast_k) {
#pragma unroll
            for (int i = 0; i < (SPLIT_TR * SPLIT_TK) / 256; ++i) {
                const int kk = tid & (SPLIT_TK - 1), r = (tid >> 6) + (256 / SPLIT_TK) * i;
                const int64_t ro = rowOff[r], ko = kOff[kk];
                const bool in = ro >= 0 && ko >= 0;
                cp_async8_zfill(smem_u32(tile + r * SPLIT_ROW + kk), in ? (const void *)(S + ro + ko) : (const void *)S,
                                in ? 8u : 0u);
            }
            return;
        }
        // rows along the source's fastest label: a warp takes 16 rows x 2 columns
        // (two 128-byte runs of a row-contiguous source; with 66-entry tile rows
        // the 32 lanes' 8-byte writes fall on all 32 banks, two wavefronts)
        static_assert(SPLIT_TR == 64 && SPLIT_TK == 64 && SPLIT_ROW == 66, "warp: 16 rows x 2 columns");
        const int lane = tid & 31, w = tid >> 5;
        const int r = 16 * (w & 3) + (lane & 15), kk0 = 2 * (w >> 2) + (lane >> 4);
        const int64_t ro = rowOff[r];
        const float2 *Sr = S + (ro >= 0 ? ro : 0);
        const uint32_t dst0 = smem_u32(tile + r * SPLIT_ROW + kk0);
#pragma unroll
        for (int i = 0; i < (SPLIT_TR * SPLIT_TK) / 256; ++i) {
            const int64_t ko = kOff[kk0 + 4 * i];
            const bool in = ro >= 0 && ko >= 0;
            cp_async8_zfill(dst0 + 4 * i * 8, in ? (const void *)(Sr + ko) : (const void *)S, in ? 8u : 0u);
        }
    };

    for (int64_t inst = blockIdx.y; inst < a.n_inst; inst += gridDim.y) {
        const float2 *__restrict__ S = (const float2 *)((const uint64_t *)a.ptrSrc)[inst];
        // instance j of group g: rows j * rows.. of the group's planes; the last
        // instance of a group also writes the group's padding rows (zeros)
        const int64_t g = inst / a.per_group, j = inst - g * a.per_group;
        const int64_t row_base = j * a.rows;
        const int64_t rows_w = j == a.per_group - 1 ? a.rows_group - row_base : a.rows;
        const int64_t n_tiles = ((rows_w + SPLIT_TR - 1) / SPLIT_TR) * k_tiles;
        uint8_t *base = (uint8_t *)a.planes + (g * NP * plane_elems + row_base * a.k_pad) * EB;
        __syncthreads();   // the previous instance's readers of the buffers are done
        if (blockIdx.x < n_tiles) decode(blockIdx.x, 0, 0);
        __syncthreads();
        if (blockIdx.x < n_tiles) issue(S, 0);
        asm volatile("cp.async.commit_group;" ::: "memory");
        int k = 0;
        for (int64_t t = blockIdx.x; t < n_tiles; t += gridDim.x, ++k) {
            const int cur = k & 1, nxt = cur ^ 1;
            const int64_t t1 = t + gridDim.x;
            if (t1 < n_tiles) decode(t1, nxt, (k + 1) % 3);
            __syncthreads();   // next offsets visible; the buffer of tile k-1 is free
            if (t1 < n_tiles) issue(S, nxt);
            asm volatile("cp.async.commit_group;" ::: "memory");
            asm volatile("cp.async.wait_group 1;" ::: "memory");   // this thread's copies of tile t
            __syncthreads();                                        // everyone's
            const float2 *tile = tiles_s + (size_t)cur * SPLIT_TR * SPLIT_ROW;
            const int64_t rt = t / k_tiles, kt = t - rt * k_tiles;
            const int64_t row0 = rt * SPLIT_TR, k0 = kt * SPLIT_TK;
            // a half-warp takes one row of the tile per step, its lanes four adjacent
            // columns each (written as one 8- or 16-byte vector per plane), so the
            // row's power-of-two scale comes from a reduction over 16 lanes (FP16x3:
            // one scale per row and 64-wide K chunk, this tile's columns; the chunk's
            // largest |re| or |im| lands in [2^14, 2^15), inside FP16's range;
            // padding columns and rows hold zeros)
            static_assert(SPLIT_TK == 64 && SPLIT_ROW % 2 == 0, "16 lanes x 4 columns cover one 16-byte aligned row");
            const int q16 = tid & 15, rsub = tid >> 4;
            // a lane reads its two 16-byte halves in the order that puts the 8 lanes
            // of a quarter-warp on 8 different 16-byte bank groups
            const int sw = (q16 >> 2) & 1;
            const int kq = 4 * q16;
            const bool col_in = k0 + kq < a.k_pad;   // k_pad is a multiple of 16
            const int64_t pstep = plane_elems * EB;
            const int64_t *prow = prows + (k % 3) * SPLIT_TR;   // the tile rows' plane rows (relative to row_base)
            float *sc = nullptr;
            if (TcCfg<MODE>::SCALED) sc = (float *)a.scales + (g * k_tiles + kt) * a.rows_group + row_base;
#pragma unroll
            for (int i = 0; i < SPLIT_TR / 16; ++i) {
                const int r = rsub + 16 * i;
                const bool valid = row0 + r < rows_w;
                const float4 *row4 = (const float4 *)(tile + r * SPLIT_ROW) + 2 * q16;
                const float4 x0 = row4[sw], x1 = row4[1 - sw];
                const float4 lo = sw ? x1 : x0, hi = sw ? x0 : x1;
                float re[4] = {lo.x, lo.z, hi.x, hi.z}, im[4] = {lo.y, lo.w, hi.y, hi.w};
                if (TcCfg<MODE>::SCALED) {
                    float m = fmaxf(fmaxf(fmaxf(fabsf(re[0]), fabsf(re[1])), fmaxf(fabsf(re[2]), fabsf(re[3]))),
                                    fmaxf(fmaxf(fabsf(im[0]), fabsf(im[1])), fmaxf(fabsf(im[2]), fabsf(im[3]))));
#pragma unroll
                    for (int o = 8; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
                    // m = f 2^e with f in [0.5, 1) and e = (biased exponent) - 126 for
                    // normal m; scale 2^(15 - e), clamped to [-100, 100] (subnormal m: 100)
                    int ex = 0;
                    if (m > 0.f) ex = max(-100, min(100, 141 - (int)((__float_as_uint(m) >> 23) & 0xffu)));
                    const float f = __uint_as_float((uint32_t)(127 + ex) << 23);
                    if (q16 == 0 && valid) sc[prow[r]] = __uint_as_float((uint32_t)(127 - ex) << 23);
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        re[c] *= f;
                        im[c] *= f;
                    }
                }
                if (!valid || !col_in) continue;
                uint32_t wr[NPH][EB], wi[NPH][EB];
                split4<MODE>(re, wr);
                split4<MODE>(im, wi);
                uint8_t *q = base + (prow[r] * a.k_pad + k0 + kq) * EB;
#pragma unroll
                for (int p = 0; p < NPH; ++p) {
                    if (EB == 2) {
                        *(uint2 *)(q + p * pstep) = make_uint2(wr[p][0], wr[p][1]);
                        *(uint2 *)(q + (NPH + p) * pstep) = make_uint2(wi[p][0], wi[p][1]);
                    } else {
                        *(uint4 *)(q + p * pstep) = make_uint4(wr[p][0], wr[p][1], wr[p][2 % EB], wr[p][3 % EB]);
                        *(uint4 *)(q + (NPH + p) * pstep) = make_uint4(wi[p][0], wi[p][1], wi[p][2 % EB], wi[p][3 % EB]);
                    }
                }
            }
        }
        asm volatile("cp.async.wait_group 0;" ::: "memory");
    }
}

// ------------------------------------------------------------------ fused split
// FP16X3 epilogue that writes a row's 16-column group straight into the parent
// GEMM's operand planes (see TcGemmArgs::fz_*): NK consecutive columns are the
// NK fastest summed entries of one parent row, and the 2^lgsz lanes of a lane
// group (consecutive m_k) hold the rest of a 64-entry chunk, so the chunk's
// scale is a max over the group's lanes; each lane then stores NK halves per
// plane (contiguous across the group).
__device__ __forceinline__ uint32_t fz_h2(float x0, float x1, uint32_t &lo)
{
    const __half2 h = __floats2half2_rn(x0, x1);
    const float2 hf = __half22float2(h);
    const __half2 l = __floats2half2_rn(x0 - hf.x, x1 - hf.y);
    lo = *(const uint32_t *)&l;
    return *(const uint32_t *)&h;
}
// (it, ibase, sbase: the group's node instance and its plane and scale bases;
// rn: the parent-row contributions of the group's 16 / NK n_f values, all
// looked up at the start of the tile)
template <int NK>
__device__ __forceinline__ void fz_store_group(const TcGemmArgs &a, const float *re, const float *im, int64_t it,
                                               int64_t ibase, int64_t sbase, const int32_t *rn, int32_t rm, int64_t mk,
                                               int lane)
{
    constexpr int LNK = NK == 4 ? 2 : 3;
    constexpr int GSZ = 64 / NK;   // lanes of one chunk
    const int64_t k0 = mk << LNK, ch = k0 >> 6;
    __half *gp = (__half *)a.fz_planes + ibase + k0;                       // plane 0, row 0 of the group's rows
    float *gs = (float *)a.fz_scales + sbase + ch * a.fz_rows_pad;         // the chunk's scales
    const uint32_t kpad = (uint32_t)a.fz_kpad;
    const int64_t pe = a.fz_plane_elems;
#pragma unroll
    for (int t = 0; t < 16 / NK; ++t) {
        const uint32_t r = (uint32_t)(rm + rn[t]);
        float m = 0.f;
#pragma unroll
        for (int c = 0; c < NK; ++c) m = fmaxf(m, fmaxf(fabsf(re[t * NK + c]), fabsf(im[t * NK + c])));
#pragma unroll
        for (int o = GSZ / 2; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        const int ex = m > 0.f ? max(-100, min(100, 141 - (int)((__float_as_uint(m) >> 23) & 0xffu))) : 0;
        const float f = __uint_as_float((uint32_t)(127 + ex) << 23);
        if (it < 0) continue;
        if ((lane & (GSZ - 1)) == 0) gs[r] = __uint_as_float((uint32_t)(127 - ex) << 23);
        uint32_t rh[NK / 2], rl[NK / 2], ih[NK / 2], il[NK / 2];
#pragma unroll
        for (int c = 0; c < NK / 2; ++c) {
            rh[c] = fz_h2(re[t * NK + 2 * c] * f, re[t * NK + 2 * c + 1] * f, rl[c]);
            ih[c] = fz_h2(im[t * NK + 2 * c] * f, im[t * NK + 2 * c + 1] * f, il[c]);
        }
        __half *e = gp + (uint64_t)r * kpad;
        if (NK == 4) {
            *(uint2 *)e = make_uint2(rh[0], rh[1 % (NK / 2)]);
            *(uint2 *)(e + pe) = make_uint2(rl[0], rl[1 % (NK / 2)]);
            *(uint2 *)(e + 2 * pe) = make_uint2(ih[0], ih[1 % (NK / 2)]);
            *(uint2 *)(e + 3 * pe) = make_uint2(il[0], il[1 % (NK / 2)]);
        } else {
            *(uint4 *)e = make_uint4(rh[0], rh[1], rh[2 % (NK / 2)], rh[3 % (NK / 2)]);
            *(uint4 *)(e + pe) = make_uint4(rl[0], rl[1], rl[2 % (NK / 2)], rl[3 % (NK / 2)]);
            *(uint4 *)(e + 2 * pe) = make_uint4(ih[0], ih[1], ih[2 % (NK / 2)], ih[3 % (NK / 2)]);
            *(uint4 *)(e + 3 * pe) = make_uint4(il[0], il[1], il[2 % (NK / 2)], il[3 % (NK / 2)]);
        }
    }
}

// ------------------------------------------------------------------ GEMM kernel
// Persistent: CTA c handles tiles c, c + gridDim.x, ...  Roles (10 warps):
//   warp 0     TMA producer (one thread): all planes of each K-block into the stage ring
//   warp 1     TMEM owner; one thread issues the MMAs
//   warps 2-9  promotion/epilogue: warp w owns TMEM lanes 32*(w%4).. and half the columns
// The K range of a tile is cut into chunks of 32; each chunk accumulates into a
// fresh TMEM buffer (two buffers alternate, 256 columns each: Re 128 + Im 128).
// The epilogue warps add every finished chunk into FP32 registers (round to
// nearest) and release the buffer; after the tile's last chunk they write C.
// Restarting the tensor-core accumulator every 32 of K keeps the long sums as
// accurate as an FP32 FMA chain.
constexpr int TC_EPI_WARPS = 8;
// C staging: each epilogue warp writes its 32 rows x 16 columns through shared
// memory (rows padded by one complex value) so that global stores cover whole
// 128-byte lines, four rows per instruction.
constexpr int TC_CST_ROW = 17;
// with bulk stores (c_tma) each epilogue warp alternates two dense 32 x 16
// complex boxes (4 KB each, 128-byte swizzle) instead
constexpr int TC_CST_BYTES = TC_EPI_WARPS * 32 * TC_CST_ROW * 8 > TC_EPI_WARPS * 2 * 4096
                                 ? TC_EPI_WARPS * 32 * TC_CST_ROW * 8
                                 : TC_EPI_WARPS * 2 * 4096;
// dot epilogue: each epilogue warp stages A in TC_DOT_BUFS units of 32 rows x 8
// complex values
constexpr int TC_DOT_BUFS = 5;
constexpr int TC_DOT_WARP_BYTES = TC_DOT_BUFS * 2048;
constexpr int TC_SMEM_LIMIT = 232448;   // opt-in dynamic shared memory per block
constexpr int TC_STATIC_SMEM = 6144;    // barriers, scale staging and flags (upper bound)
// K blocks (pipeline stages) per accumulator chunk
template <int MODE>
__host__ __device__ constexpr int tc_chunk_kb()
{
    return TcCfg<MODE>::CHUNK_K / (TC_ROWB / TcCfg<MODE>::EB) > 0 ? TcCfg<MODE>::CHUNK_K / (TC_ROWB / TcCfg<MODE>::EB)
                                                                  : 1;
}
template <int MODE>
__host__ __device__ constexpr bool tc_dot_fits()
{
    return TcCfg<MODE>::STAGES * 2 * TcCfg<MODE>::NP * TC_PLANE_TILE + 1024 + TC_EPI_WARPS * TC_DOT_WARP_BYTES +
               TC_STATIC_SMEM <=
           TC_SMEM_LIMIT;
}
template <int MODE>
__host__ __device__ constexpr bool tc_cstage()
{
    return TcCfg<MODE>::STAGES * 2 * TcCfg<MODE>::NP * TC_PLANE_TILE + 1024 + TC_CST_BYTES + TC_STATIC_SMEM <=
           TC_SMEM_LIMIT;
}
constexpr int TC_THREADS = 64 + 32 * TC_EPI_WARPS;
constexpr int TC_GROUP_M = 8;   // tile rasterisation: groups of 8 M-tiles walk the N-tiles together

__device__ __forceinline__ void tile_coords(int64_t t, int tiles_m, int tiles_n, int &inst, int &tm, int &tn)
{
    const int64_t per = (int64_t)tiles_m * tiles_n;
    inst = (int)(t / per);
    const int r = (int)(t - (int64_t)inst * per);
    const int group = r / (TC_GROUP_M * tiles_n);
    const int first_m = group * TC_GROUP_M;
    const int gm = min(TC_GROUP_M, tiles_m - first_m);
    const int idx = r - group * TC_GROUP_M * tiles_n;
    tm = first_m + idx % gm;
    tn = idx / gm;
}

// Dot epilogue: copy A's values of the warp's 32 rows (row offsets xm, one per
// lane) x the 8 columns of unit q of its 64 (column offsets xn0, xn1: columns
// lane and 32 + lane) into buf as one group of 16-byte asynchronous copies
// (through L2 only), each of two values adjacent in A:
//   dot_lcol 1: columns 2p, 2p + 1 of a row, at r 8 + 2 (p ^ (r / 2 % 4))
//   dot_lcol 0: rows 2p, 2p + 1 of a column, at c 32 + r
// (a quarter warp's copies and a row's reads then meet every bank once).
__device__ __forceinline__ void dot_stage(const TcGemmArgs &a, const float2 *A, int64_t xm, int32_t xn0, int32_t xn1,
                                          int q, float2 *buf, int lane)
{
    const uint32_t b0 = smem_u32(buf);
    const int32_t xq = q < 4 ? xn0 : xn1;
    if (a.dot_lcol) {   // a quarter warp covers two rows, a lane a column pair
        const int p = lane & 3;
        const int64_t xc = __shfl_sync(0xffffffffu, xq, (q & 3) * 8 + 2 * p);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int r = 8 * i + (lane >> 2);
            const int64_t xr = __shfl_sync(0xffffffffu, xm, r);
            cp_async16_zfill(b0 + (uint32_t)(r * 8 + 2 * (p ^ ((r >> 1) & 3))) * 8u, A + xr + xc, 16);
        }
    } else {            // half a warp covers a column's 32 rows, a lane a row pair
        const int p = lane & 15;
        const int64_t xr = __shfl_sync(0xffffffffu, xm, 2 * p);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int c = 2 * i + (lane >> 4);
            const int64_t xc = __shfl_sync(0xffffffffu, xq, (q & 3) * 8 + c);
            cp_async16_zfill(b0 + (uint32_t)(c * 32 + 2 * p) * 8u, A + xr + xc, 16);
        }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}

// Dot epilogue: the lane's row of a staged unit (layouts above)
__device__ __forceinline__ void dot_read(const TcGemmArgs &a, const float2 *buf, int lane, float2 (&av)[8])
{
    if (a.dot_lcol) {
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            const float4 v = *(const float4 *)(buf + lane * 8 + 2 * (p ^ ((lane >> 1) & 3)));
            av[2 * p] = make_float2(v.x, v.y);
            av[2 * p + 1] = make_float2(v.z, v.w);
        }
    } else {
#pragma unroll
        for (int c = 0; c < 8; ++c) av[c] = buf[c * 32 + lane];
    }
}

// wait until at most n (0 .. 4) of this thread's copy groups are pending
__device__ __forceinline__ void cp_async_wait_upto(int n)
{
    if (n >= 4) asm volatile("cp.async.wait_group 4;" ::: "memory");
    else if (n == 3) asm volatile("cp.async.wait_group 3;" ::: "memory");
    else if (n == 2) asm volatile("cp.async.wait_group 2;" ::: "memory");
    else if (n == 1) asm volatile("cp.async.wait_group 1;" ::: "memory");
    else asm volatile("cp.async.wait_group 0;" ::: "memory");
}

// Dot form: step st is tile position (tmi, tni) of dot block d = st % dot_nblk
// (blocks fastest, so that blocks sharing sibling instances read them at about
// the same time, the later ones from L2); its tile k (0, 1) is that of the
// block's instance c_k (c_0 again when the block has one), entry (j, l) of GEMM
// block b: rows j Mi + 128 tmi, columns l Ni + 128 tni.
__device__ __forceinline__ void tile_coords_pair(int64_t st, int k, const TcGemmArgs &a, int &inst, int &tm, int &tn)
{
    const int64_t tmi_n = a.Mi >> 7, tni_n = a.Ni >> 7, nb = a.dot_nblk;
    const int64_t d = st % nb, r = st / nb, tni = r % tni_n, tmi = r / tni_n;
    const int32_t *blk = (const int32_t *)a.dot_pair + 8 * d;
    int32_t c = __ldg(blk + k);
    if (c < 0) c = __ldg(blk);
    const int32_t *cp = (const int32_t *)a.dot_cpos + 3 * (int64_t)c;
    inst = __ldg(cp);
    tm = (int)(__ldg(cp + 1) * tmi_n + tmi);
    tn = (int)(__ldg(cp + 2) * tni_n + tni);
}

// (DOT: the dot-epilogue form, launched when a.dot_parts is set; a form of its
// own so that its registers do not weigh on the others)
template <int MODE, bool DOT>
__global__ void __launch_bounds__(TC_THREADS, 1) tc_gemm_kernel(const __grid_constant__ TcGemmArgs a)
{
    using Cfg = TcCfg<MODE>;
    constexpr int NP = Cfg::NP, NPH = NP / 2, S = Cfg::STAGES;
    constexpr int STAGE_BYTES = 2 * NP * TC_PLANE_TILE;
    constexpr int KE = TC_ROWB / Cfg::EB;               // K elements per stage
    constexpr int KSUB = TC_ROWB / 32;                   // MMAs of 32 bytes of K per stage
    constexpr int CHUNK_KB = tc_chunk_kb<MODE>();   // stages per K chunk
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t bars[2 * S + 4];
    __shared__ uint32_t tmem_holder;
    __shared__ int abort_flag;
    __shared__ int dot_cnt[4];   // dot epilogue: warps done with the step (a ring of four steps)

    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t full0 = smem_u32(&bars[0]), empty0 = smem_u32(&bars[S]);
    const uint32_t tfull0 = smem_u32(&bars[2 * S]), tempty0 = smem_u32(&bars[2 * S + 2]);
    const int tiles_m = (int)(a.m_pad / TC_BM), tiles_n = (int)(a.n_pad / TC_BN);
    const int64_t total_tiles = (int64_t)a.n_inst * tiles_m * tiles_n;
    const int n_kb = a.n_kb;
    const int n_chunks = (n_kb + CHUNK_KB - 1) / CHUNK_KB;
    // steps of the launch: tiles, or (dot form) tile positions of a dot block,
    // PER tiles each
    constexpr int PER = DOT ? 2 : 1;
    const int64_t n_steps = DOT ? (int64_t)a.dot_nblk * (a.Mi >> 7) * (a.Ni >> 7) : total_tiles;

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(full0 + 8 * s, 1);
            mbar_init(empty0 + 8 * s, 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(tfull0 + 8 * b, 1);
            mbar_init(tempty0 + 8 * b, TC_EPI_WARPS);
        }
        abort_flag = 0;
        dot_cnt[0] = dot_cnt[1] = dot_cnt[2] = dot_cnt[3] = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_holder)),
                     "r"(TC_TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_holder;

    if (warp == 0) {
        if (lane == 0) {
            int64_t kg = 0, issued = 0;
            for (int64_t st = blockIdx.x; st < n_steps && !abort_flag; st += gridDim.x)
                for (int k = 0; k < PER && !abort_flag; ++k) {
                int inst, tm, tn;
                if (DOT) tile_coords_pair(st, k, a, inst, tm, tn);
                else tile_coords(st, tiles_m, tiles_n, inst, tm, tn);
                const int zA = ((const int32_t *)a.zA)[inst], zB = ((const int32_t *)a.zB)[inst];
                for (int kb = 0; kb < n_kb; ++kb, ++kg) {
                    const int s = (int)(kg % S);
                    if (kg >= S && !mbar_wait_bounded(empty0 + 8 * s, (uint32_t)(((kg / S) - 1) & 1), &abort_flag)) {
                        abort_flag = 1;
                        break;
                    }
                    const uint32_t st = smem_u32(smem + (size_t)s * STAGE_BYTES);
                    mbar_expect_tx(full0 + 8 * s, STAGE_BYTES);
                    for (int p = 0; p < NP; ++p)
                        tma_load_3d(st + p * TC_PLANE_TILE, &a.tmA, full0 + 8 * s, kb * KE, tm * TC_BM, zA + p);
                    for (int p = 0; p < NP; ++p)
                        tma_load_3d(st + (NP + p) * TC_PLANE_TILE, &a.tmB, full0 + 8 * s, kb * KE, tn * TC_BN, zB + p);
                    issued = kg + 1;
                }
            }
            if (abort_flag) {   // let copies already in flight land before the CTA exits
                for (int64_t k = issued - S > 0 ? issued - S : 0; k < issued; ++k)
                    mbar_wait_bounded(full0 + 8 * (int)(k % S), (uint32_t)((k / S) & 1), &abort_flag);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // kind::f16 / kind::tf32 instruction descriptor: FP32 D, K-major A and B, M=128, N=128;
            // the negate-A variant accumulates (-Ai).Bi into the real part
            const uint32_t fmt = (uint32_t)Cfg::FMT;
            const uint32_t idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(TC_BN >> 3) << 17) |
                                   ((uint32_t)(TC_BM >> 4) << 24);
            const uint32_t idesc_neg = idesc | (1u << 13);
            int64_t kg = 0, cg = 0;
            for (int64_t st = blockIdx.x; st < n_steps && !abort_flag; st += gridDim.x)
                for (int k = 0; k < PER && !abort_flag; ++k) {
                for (int c = 0; c < n_chunks && !abort_flag; ++c, ++cg) {
                    const int buf = (int)(cg & 1);
                    if (cg >= 2 && !mbar_wait_bounded(tempty0 + 8 * buf, (uint32_t)(((cg >> 1) - 1) & 1), &abort_flag)) {
                        abort_flag = 1;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t dR = tmem + buf * 2 * TC_BN, dI = dR + TC_BN;
                    const int kb_end = min(n_kb, (c + 1) * CHUNK_KB);
                    for (int kb = c * CHUNK_KB; kb < kb_end; ++kb, ++kg) {
                        const int s = (int)(kg % S);
                        if (!mbar_wait_bounded(full0 + 8 * s, (uint32_t)((kg / S) & 1), &abort_flag)) {
                            abort_flag = 1;
                            break;
                        }
                        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                        const uint32_t st = smem_u32(smem + (size_t)s * STAGE_BYTES);
                        const bool first_kb = kb == c * CHUNK_KB;
#pragma unroll
                        for (int sub = 0; sub < KSUB; ++sub) {
#pragma unroll
                            for (int tt = 0; tt < Cfg::NT; ++tt) {
                                int p, q;
                                Cfg::term(tt, p, q);
                                const uint64_t aRe = sdesc(st + p * TC_PLANE_TILE + sub * 32);
                                const uint64_t aIm = sdesc(st + (NPH + p) * TC_PLANE_TILE + sub * 32);
                                const uint64_t bRe = sdesc(st + (NP + q) * TC_PLANE_TILE + sub * 32);
                                const uint64_t bIm = sdesc(st + (NP + NPH + q) * TC_PLANE_TILE + sub * 32);
                                const uint32_t acc = (!first_kb || sub || tt) ? 1u : 0u;
                                umma<Cfg::KIND>(dR, aRe, bRe, idesc, acc);
                                umma<Cfg::KIND>(dR, aIm, bIm, idesc_neg, 1u);
                                umma<Cfg::KIND>(dI, aRe, bIm, idesc, acc);
                                umma<Cfg::KIND>(dI, aIm, bRe, idesc, 1u);
                            }
                        }
                        umma_commit(empty0 + 8 * s);
                    }
                    umma_commit(tfull0 + 8 * buf);
                }
            }
        }
    } else {
        // promotion + epilogue: rows 32*(warp%4) + lane, columns half*64 .. +63 of the tile
        const int quarter = warp & 3, half = (warp - 2) >> 2;
        __shared__ float sfn[TC_EPI_WARPS][64];   // SCALED: this warp's 64 column scales of the chunk
        int64_t cg = 0;
        // fused split: this warp's per-tile lookups (instances, plane and scale
        // bases of its four 16-column groups, parent-row parts of its n_f values),
        // staged in its slice of the C staging area while the chunks accumulate
        int64_t *fz_t64 = (int64_t *)(smem + (size_t)S * STAGE_BYTES + (size_t)(warp - 2) * 8192);
        // dot epilogue: TC_DOT_BUFS staged 32 x 8 units of A per warp, in place
        // of the C staging
        float2 *dstage = (float2 *)(smem + (size_t)S * STAGE_BYTES + (size_t)(warp - 2) * TC_DOT_WARP_BYTES);
        int32_t *fz_rn = (int32_t *)(fz_t64 + 12);
        if (DOT) {
            // dot epilogue (the whole summed extent in one accumulator chunk): per
            // step, the parts of up to four products (the block's two tiles times
            // its two sibling instances), read straight from the two accumulators,
            // which the warp holds until the step is done.  A's values are staged
            // 8 columns at a time (TC_DOT_BUFS 2 KB buffers: the copies of the units
            // after this one run while it is read, the first ones while the
            // accumulators fill), each unit dotted with both tiles.  The block's
            // lookups are loaded one step ahead.  The epilogue warps may be up to
            // two steps apart, so the parts and counters live in a ring of four
            __shared__ float2 dred[4][TC_EPI_WARPS][4];
            __shared__ float sfn1[TC_EPI_WARPS][64];   // the second tile's column scales
            const int64_t tmi_n = a.Mi >> 7, tni_n = a.Ni >> 7, nb = a.dot_nblk;
            int32_t n_c[2] = {-1, -1}, n_p[4] = {-1, -1, -1, -1};
            const float2 *n_A[2] = {nullptr, nullptr};
            auto lookup = [&](int64_t st) {
                if (st >= n_steps) return;
                const int64_t d = st % nb;
                const int4 v0 = __ldg((const int4 *)a.dot_pair + 2 * d), v1 = __ldg((const int4 *)a.dot_pair + 2 * d + 1);
                n_c[0] = v0.x;
                n_c[1] = v0.y;
                n_p[0] = v0.z;
                n_p[1] = v0.w;
                n_p[2] = v1.x;
                n_p[3] = v1.y;
                n_A[0] = (const float2 *)__ldg((const unsigned long long *)a.dot_ptrA + 2 * d);
                n_A[1] = (const float2 *)__ldg((const unsigned long long *)a.dot_ptrA + 2 * d + 1);
            };
            lookup(blockIdx.x);
            int64_t i = 0;
            for (int64_t st = blockIdx.x; st < n_steps; st += gridDim.x, ++i) {
                const int64_t r = st / nb, tni = r % tni_n, tmi = r / tni_n;
                const int32_t c0 = n_c[0], c1 = n_c[1] >= 0 ? n_c[1] : n_c[0];
                const int32_t p00 = n_p[0], p01 = n_p[1], p10 = n_p[2], p11 = n_p[3];
                const float2 *A0 = n_A[0], *A1 = n_A[1];
                lookup(st + gridDim.x);
                // units: sibling m = u / 8, columns 8 (u % 8) ..; sibling 1 only when
                // a product uses it
                const int U = (p01 >= 0 || p11 >= 0) ? 16 : 8;
                const int32_t *xn = (const int32_t *)a.dot_xn + (tni << 7) + half * 64;
                const int32_t xn0 = __ldg(xn + lane), xn1 = __ldg(xn + 32 + lane);
                const int64_t mm = (tmi << 7) + quarter * 32 + lane;
                int64_t xm = 0;
                for (int b = 0; b < a.dot_mbits; ++b)
                    if ((mm >> b) & 1) xm += a.dot_sm[b];
#pragma unroll
                for (int u = 0; u < TC_DOT_BUFS - 1; ++u) dot_stage(a, A0, xm, xn0, xn1, u, dstage + u * 256, lane);
                // SCALED: the two tiles' row and column scales
                float fm0 = 1.f, fm1 = 1.f;
                if (Cfg::SCALED) {
                    __syncwarp();
#pragma unroll
                    for (int k = 0; k < 2; ++k) {
                        const int32_t *cp = (const int32_t *)a.dot_cpos + 3 * (int64_t)(k ? c1 : c0);
                        const int b = __ldg(cp);
                        const int64_t tm = __ldg(cp + 1) * tmi_n + tmi, tn = __ldg(cp + 2) * tni_n + tni;
                        const int64_t instA = ((const int32_t *)a.zA)[b] / NP, instB = ((const int32_t *)a.zB)[b] / NP;
                        const float f = __ldg((const float *)a.scaleA + instA * a.m_pad + tm * TC_BM + quarter * 32 + lane);
                        const float *g = (const float *)a.scaleB + instB * a.n_pad + tn * TC_BN + half * 64;
                        float *fnk = k ? sfn1[warp - 2] : sfn[warp - 2];
                        fnk[lane] = __ldg(g + lane);
                        fnk[lane + 32] = __ldg(g + lane + 32);
                        if (k) fm1 = f;
                        else fm0 = f;
                    }
                    __syncwarp();
                }
                // the step's two tiles: buffers 0 and 1 (cg is even here)
                if (!mbar_wait_bounded(tfull0, (uint32_t)((cg >> 1) & 1), &abort_flag) ||
                    !mbar_wait_bounded(tfull0 + 8, (uint32_t)((cg >> 1) & 1), &abort_flag)) {
                    abort_flag = 1;
                    asm volatile("cp.async.wait_all;" ::: "memory");   // no staged copy outlives the block
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t base0 = tmem + ((uint32_t)(quarter * 32) << 16) + half * 64, base1 = base0 + 2 * TC_BN;
                float s[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};   // (re, im) of (k, m) = (0,0) (0,1) (1,0) (1,1)
#pragma unroll
                for (int u = 0; u < 16; ++u) {
                    if (u < U) {   // warp-uniform
                        constexpr int AH = TC_DOT_BUFS - 1;   // units in flight ahead of this one
                        if (u + AH < U)
                            dot_stage(a, u + AH < 8 ? A0 : A1, xm, xn0, xn1, (u + AH) & 7,
                                      dstage + ((u + AH) % TC_DOT_BUFS) * 256, lane);
                        uint32_t R0[8], I0[8], R1[8], I1[8];
                        JET_TMEM_LD8(base0 + (u & 7) * 8, R0);
                        JET_TMEM_LD8(base0 + TC_BN + (u & 7) * 8, I0);
                        JET_TMEM_LD8(base1 + (u & 7) * 8, R1);
                        JET_TMEM_LD8(base1 + TC_BN + (u & 7) * 8, I1);
                        cp_async_wait_upto(min(AH, U - 1 - u));   // unit u has landed
                        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                        __syncwarp();
                        float2 avs[8];
                        dot_read(a, dstage + (u % TC_DOT_BUFS) * 256, lane, avs);
                        float x0 = 0.f, y0 = 0.f, x1 = 0.f, y1 = 0.f;
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            const int cj = (u & 7) * 8 + j;
                            const float f0 = Cfg::SCALED ? fm0 * sfn[warp - 2][cj] : 1.f;
                            const float f1 = Cfg::SCALED ? fm1 * sfn1[warp - 2][cj] : 1.f;
                            const float ar = __uint_as_float(R0[j]) * f0, ai = __uint_as_float(I0[j]) * f0;
                            const float br = __uint_as_float(R1[j]) * f1, bi = __uint_as_float(I1[j]) * f1;
                            const float2 av = avs[j];
                            x0 = fmaf(ar, av.x, fmaf(-ai, av.y, x0));
                            y0 = fmaf(ar, av.y, fmaf(ai, av.x, y0));
                            x1 = fmaf(br, av.x, fmaf(-bi, av.y, x1));
                            y1 = fmaf(br, av.y, fmaf(bi, av.x, y1));
                        }
                        const int m = u < 8 ? 0 : 1;
                        s[2 * m] += x0;
                        s[2 * m + 1] += y0;
                        s[4 + 2 * m] += x1;
                        s[4 + 2 * m + 1] += y1;
                        __syncwarp();   // the buffer is refilled TC_DOT_BUFS - 1 units on
                    }
                }
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                __syncwarp();
                if (lane == 0) {   // both accumulators are free
                    mbar_arrive(tempty0);
                    mbar_arrive(tempty0 + 8);
                }
                cg += 2;
#pragma unroll
                for (int q = 0; q < 8; ++q)
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) s[q] += __shfl_xor_sync(0xffffffffu, s[q], o);
                const int par = (int)(i & 3);   // this CTA's step count, mod 4
                if (lane == 0) {
#pragma unroll
                    for (int q = 0; q < 4; ++q) dred[par][warp - 2][q] = make_float2(s[2 * q], s[2 * q + 1]);
                }
                // the last of the eight epilogue warps to finish the step adds their
                // parts in warp order (no barrier: a warp that gave up on a wait
                // never holds the others)
                int last = 0;
                if (lane == 0) {
                    __threadfence_block();
                    last = atomicAdd(&dot_cnt[par], 1) == TC_EPI_WARPS - 1;
                }
                last = __shfl_sync(0xffffffffu, last, 0);
                if (last) {
                    __threadfence_block();
                    const int32_t pr = lane == 0 ? p00 : lane == 1 ? p01 : lane == 2 ? p10 : p11;
                    if (lane < 4 && pr >= 0) {   // the eight parts added in FP64, the tile's part kept in FP64
                        const volatile float2 *dr = dred[par][0] + lane;
                        double ax = dr[0].x, ay = dr[0].y;
                        for (int w = 1; w < TC_EPI_WARPS; ++w) {
                            ax += dr[4 * w].x;
                            ay += dr[4 * w].y;
                        }
                        ((double2 *)a.dot_parts)[(int64_t)pr * a.dot_tiles + tmi * tni_n + tni] = make_double2(ax, ay);
                    }
                    __syncwarp();
                    if (lane == 0) dot_cnt[par] = 0;
                }
            }
        } else
        for (int64_t t = blockIdx.x; t < total_tiles; t += gridDim.x) {
            int inst, tm, tn;
            tile_coords(t, tiles_m, tiles_n, inst, tm, tn);
            if (Cfg::SCALED && a.fz_planes) {
                const int64_t c0 = (int64_t)tn * TC_BN + half * 64;
                __syncwarp();   // the previous tile's readers of the lookups are done
                if (c0 < a.N) {
                    const bool grp = a.itab != 0;
                    int64_t jj = 0;
                    if (grp) {
                        const int64_t R0 = (int64_t)tm * TC_BM + quarter * 32;
                        jj = a.mi_shift >= 0 ? R0 >> a.mi_shift : R0 / a.Mi;
                    }
                    auto col_split = [&](int64_t c, int64_t &ll, int64_t &nn) {
                        if (!grp) {
                            ll = 0;
                            nn = c;
                        } else if (a.ni_shift >= 0) {
                            ll = c >> a.ni_shift;
                            nn = c & (a.Ni - 1);
                        } else {
                            ll = c / a.Ni;
                            nn = c - ll * a.Ni;
                        }
                    };
                    if (lane < 4) {
                        int64_t ll, nn;
                        col_split(c0 + 16 * lane, ll, nn);
                        const int64_t it =
                            grp ? (int64_t)__ldg((const int32_t *)a.itab + ((int64_t)inst * a.nA + jj) * a.nB + ll) : inst;
                        fz_t64[lane] = it;
                        fz_t64[4 + lane] = it >= 0 ? __ldg((const long long *)a.fz_ibase + 2 * it) : 0;
                        fz_t64[8 + lane] = it >= 0 ? __ldg((const long long *)a.fz_ibase + 2 * it + 1) : 0;
                    }
                    const int nv = 64 >> a.fz_lnk;   // n_f values of the warp's 64 columns
                    if (lane < nv) {
                        int64_t ll, nn;
                        col_split(c0 + ((int64_t)lane << a.fz_lnk), ll, nn);
                        fz_rn[lane] = __ldg((const int *)a.fz_pn + (nn >> a.fz_lnk));
                    }
                }
                __syncwarp();
            }
            float racc[64], iacc[64];
#pragma unroll
            for (int j = 0; j < 64; ++j) racc[j] = iacc[j] = 0.f;
            bool ok = !abort_flag;
            // SCALED: the operands' power-of-two chunk scales (undone exactly), each
            // chunk's loaded while the chunk before it accumulates: this row's, and
            // the warp's 64 column scales (two per lane, read back as broadcasts)
            float *fn = sfn[warp - 2];
            const float *sc_a = nullptr, *sc_b = nullptr;
            float fm_nx = 1.f, fn_nx0 = 1.f, fn_nx1 = 1.f;
            if (Cfg::SCALED && n_chunks > 0) {
                const int64_t instA = ((const int32_t *)a.zA)[inst] / NP, instB = ((const int32_t *)a.zB)[inst] / NP;
                sc_a = (const float *)a.scaleA + instA * n_chunks * a.m_pad + (int64_t)tm * TC_BM + quarter * 32 + lane;
                sc_b = (const float *)a.scaleB + instB * n_chunks * a.n_pad + (int64_t)tn * TC_BN + half * 64 + lane;
                fm_nx = __ldg(sc_a);
                fn_nx0 = __ldg(sc_b);
                fn_nx1 = __ldg(sc_b + 32);
            }
            for (int c = 0; c < n_chunks && ok; ++c, ++cg) {
                const int buf = (int)(cg & 1);
                float fm = 1.f;
                if (Cfg::SCALED) {
                    fm = fm_nx;
                    __syncwarp();
                    fn[lane] = fn_nx0;
                    fn[lane + 32] = fn_nx1;
                    __syncwarp();
                    if (c + 1 < n_chunks) {
                        fm_nx = __ldg(sc_a + (int64_t)(c + 1) * a.m_pad);
                        fn_nx0 = __ldg(sc_b + (int64_t)(c + 1) * a.n_pad);
                        fn_nx1 = __ldg(sc_b + (int64_t)(c + 1) * a.n_pad + 32);
                    }
                }
                if (!mbar_wait_bounded(tfull0 + 8 * buf, (uint32_t)((cg >> 1) & 1), &abort_flag)) {
                    abort_flag = 1;
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t base = tmem + buf * 2 * TC_BN + ((uint32_t)(quarter * 32) << 16) + half * 64;
                // 16 columns per TMEM load (8 in the scaled mode, whose scales need registers too)
                constexpr int LW = Cfg::SCALED ? 8 : 16;
#pragma unroll
                for (int h = 0; h < 64 / LW; ++h) {
                    uint32_t R[LW], I[LW];
                    if (LW == 8) {
                        JET_TMEM_LD8(base + h * LW, R);
                        JET_TMEM_LD8(base + TC_BN + h * LW, I);
                    } else {
                        JET_TMEM_LD16(base + h * LW, R);
                        JET_TMEM_LD16(base + TC_BN + h * LW, I);
                    }
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                    for (int j = 0; j < LW; ++j) {
                        if (Cfg::SCALED) {
                            const float f = fm * fn[h * LW + j];
                            racc[h * LW + j] = fmaf(__uint_as_float(R[j]), f, racc[h * LW + j]);
                            iacc[h * LW + j] = fmaf(__uint_as_float(I[j]), f, iacc[h * LW + j]);
                        } else {
                            racc[h * LW + j] += __uint_as_float(R[j]);
                            iacc[h * LW + j] += __uint_as_float(I[j]);
                        }
                    }
                }
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                __syncwarp();
                if (lane == 0) mbar_arrive(tempty0 + 8 * buf);
            }
            if (!ok) break;
            const int64_t row = (int64_t)tm * TC_BM + quarter * 32 + lane;
            const uint64_t *ptrC = (const uint64_t *)a.ptrC;
            const bool grouped = a.itab != 0;
            const int64_t col0 = (int64_t)tn * TC_BN + half * 64;
            const int32_t *itab = (const int32_t *)a.itab;
            // a block entry (R, c) is entry (m, n) of instance itab[(inst nA + j) nB + l]
            // with R = j Mi + m and c = l Ni + n (shifts for power-of-two Mi, Ni)
            auto split_row = [&](int64_t R, int64_t &jj, int64_t &mm) {
                if (a.mi_shift >= 0) {
                    jj = R >> a.mi_shift;
                    mm = R & (a.Mi - 1);
                } else {
                    jj = R / a.Mi;
                    mm = R - jj * a.Mi;
                }
            };
            auto split_col = [&](int64_t c, int64_t &ll, int64_t &nn) {
                if (a.ni_shift >= 0) {
                    ll = c >> a.ni_shift;
                    nn = c & (a.Ni - 1);
                } else {
                    ll = c / a.Ni;
                    nn = c - ll * a.Ni;
                }
            };
            // the output base of (j, l), looked up again only when (j, l) changes
            // (rows and columns of a tile mostly share one instance)
            int64_t cj = -1, cl = -1;
            float2 *cptr = grouped ? nullptr : (float2 *)ptrC[inst];
            auto inst_ptr = [&](int64_t jj, int64_t ll) -> float2 * {
                if (!grouped) return cptr;
                if (jj != cj || ll != cl) {
                    cj = jj;
                    cl = ll;
                    const int32_t it = __ldg(itab + ((int64_t)inst * a.nA + jj) * a.nB + ll);
                    cptr = it < 0 ? nullptr : (float2 *)__ldg((const unsigned long long *)ptrC + it);
                }
                return cptr;
            };
            if (Cfg::SCALED && a.fz_planes) {
                // fused split: the parent's planes (whole tiles of rows, columns in 64s:
                // a warp's half tile is all in or all out; a warp's 32 rows lie in one
                // instance, each 16-column group too)
                if (col0 >= a.N) continue;
                const int64_t R = (int64_t)tm * TC_BM + quarter * 32 + lane;
                int64_t jj = 0, mm = R;
                if (grouped) split_row(R, jj, mm);
                const int64_t mk = mm & (((int64_t)1 << a.fz_lmk) - 1), mf = mm >> a.fz_lmk;
                const int32_t rm = __ldg((const int *)a.fz_pm + mf);
                if (a.fz_lnk == 2) {   // 4 or 8 summed entries from the N side (the planner's two forms)
#pragma unroll
                    for (int p = 0; p < 4; ++p)
                        fz_store_group<4>(a, racc + p * 16, iacc + p * 16, fz_t64[p], fz_t64[4 + p], fz_t64[8 + p],
                                          fz_rn + 4 * p, rm, mk, lane);
                } else {
#pragma unroll
                    for (int p = 0; p < 4; ++p)
                        fz_store_group<8>(a, racc + p * 16, iacc + p * 16, fz_t64[p], fz_t64[4 + p], fz_t64[8 + p],
                                          fz_rn + 2 * p, rm, mk, lane);
                }
            } else if (tc_cstage<MODE>() && a.c_tma && (a.Ni & 15) == 0 && col0 + 64 <= a.N) {
                // bulk tensor stores: the warp's 32 rows x 16 columns staged as one
                // dense box (16-byte chunk c of row r at chunk c ^ (r % 8): 128-byte
                // swizzle), stored by lane 0; two boxes alternate, a box rewritten
                // only once the store that read it two steps before has
                const uint32_t stb = smem_u32(smem + (size_t)S * STAGE_BYTES) + (uint32_t)(warp - 2) * 8192u;
                // the warp's 32 rows lie in one instance (grouped blocks: Mi a multiple
                // of 32), each 16-column group too (Ni a multiple of 16)
                const int64_t R0 = (int64_t)tm * TC_BM + quarter * 32;
                int64_t jj = 0, m0 = R0;
                if (grouped) split_row(R0, jj, m0);
#pragma unroll
                for (int p = 0; p < 4; ++p) {
                    const uint32_t box = stb + (uint32_t)(p & 1) * 4096u;
                    int64_t ll = 0, n0 = col0 + p * 16;
                    if (grouped) split_col(col0 + p * 16, ll, n0);
                    const int64_t it = grouped ? (int64_t)__ldg(itab + ((int64_t)inst * a.nA + jj) * a.nB + ll) : inst;
                    if (lane == 0) bulk_wait_read1();
                    __syncwarp();
#pragma unroll
                    for (int c = 0; c < 8; ++c)
                        sts_v4(box + (uint32_t)lane * 128u + ((uint32_t)(c ^ (lane & 7)) << 4), racc[p * 16 + 2 * c],
                               iacc[p * 16 + 2 * c], racc[p * 16 + 2 * c + 1], iacc[p * 16 + 2 * c + 1]);
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    __syncwarp();
                    if (lane == 0 && R0 < a.M && it >= 0) tma_store_3d(&a.tmC, box, (int)(n0 * 2), (int)m0, (int)it);
                }
            } else if (tc_cstage<MODE>() && (a.Ni & 15) == 0 && col0 + 64 <= a.N) {
                // whole 64-column half tile in range: stage 16 columns at a time (a
                // 16-column group lies in one instance); each lane stores 8 rows
                float2 *st = (float2 *)(smem + (size_t)S * STAGE_BYTES) + (size_t)(warp - 2) * 32 * TC_CST_ROW;
                const int64_t row0 = (int64_t)tm * TC_BM + quarter * 32;
                const int cc = (lane & 7) * 2;
#pragma unroll
                for (int p = 0; p < 4; ++p) {
#pragma unroll
                    for (int j = 0; j < 16; ++j) st[lane * TC_CST_ROW + j] = make_float2(racc[p * 16 + j], iacc[p * 16 + j]);
                    __syncwarp();
                    int64_t lq = 0, nq = col0 + p * 16 + cc;
                    if (grouped) split_col(col0 + p * 16 + cc, lq, nq);
#pragma unroll
                    for (int it = 0; it < 8; ++it) {
                        const int r = it * 4 + (lane >> 3);
                        if (row0 + r < a.M) {
                            int64_t jj = 0, mm = row0 + r;
                            if (grouped) split_row(row0 + r, jj, mm);
                            float2 *C = inst_ptr(jj, lq);
                            const float2 v0 = st[r * TC_CST_ROW + cc], v1 = st[r * TC_CST_ROW + cc + 1];
                            if (C) *(float4 *)(C + mm * a.Ni + nq) = make_float4(v0.x, v0.y, v1.x, v1.y);
                        }
                    }
                    __syncwarp();
                }
            } else if (row < a.M) {
                int64_t jj = 0, mm = row, ll = 0, nn = col0;
                if (grouped) {
                    split_row(row, jj, mm);
                    split_col(col0, ll, nn);
                }
                if ((a.Ni & 1) == 0 && col0 + 64 <= a.N) {
#pragma unroll
                    for (int j = 0; j < 64; j += 2) {
                        float2 *C = inst_ptr(jj, ll);
                        if (C) *(float4 *)(C + mm * a.Ni + nn) = make_float4(racc[j], iacc[j], racc[j + 1], iacc[j + 1]);
                        nn += 2;
                        if (nn >= a.Ni) {
                            nn -= a.Ni;
                            ++ll;
                        }
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < 64; ++j) {
                        if (col0 + j < a.N) {
                            float2 *C = inst_ptr(jj, ll);
                            if (C) C[mm * a.Ni + nn] = make_float2(racc[j], iacc[j]);
                        }
                        if (++nn >= a.Ni) {
                            nn -= a.Ni;
                            ++ll;
                        }
                    }
                }
            }
        }
    }
    if (warp >= 2 && lane == 0 && a.c_tma) bulk_wait_all();   // this lane's bulk stores have completed
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 1) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS));
    }
    if (threadIdx.x == 0 && abort_flag) atomicOr((unsigned int *)a.status, 1u);
}

// ------------------------------------------------------------------ host side
template <int MODE>
static int tc_smem_bytes(bool dot = false)
{
    return TcCfg<MODE>::STAGES * 2 * TcCfg<MODE>::NP * TC_PLANE_TILE + 1024 +
           (dot ? TC_EPI_WARPS * TC_DOT_WARP_BYTES : tc_cstage<MODE>() ? TC_CST_BYTES : 0);
}

int tc_planes(int mode)
{
    switch (mode) {
    case JET_PREC_TF32: return TcCfg<JET_PREC_TF32>::NP;
    case JET_PREC_TF32X3: return TcCfg<JET_PREC_TF32X3>::NP;
    case JET_PREC_BF16X3: return TcCfg<JET_PREC_BF16X3>::NP;
    case JET_PREC_BF16X6: return TcCfg<JET_PREC_BF16X6>::NP;
    case JET_PREC_FP16X3: return TcCfg<JET_PREC_FP16X3>::NP;
    default: return 0;
    }
}

int tc_elem_bytes(int mode) { return (mode == JET_PREC_TF32 || mode == JET_PREC_TF32X3) ? 4 : 2; }
int tc_k_block(int mode) { return TC_ROWB / tc_elem_bytes(mode); }
int tc_tile() { return TC_BM; }
// The dot epilogue stages its sibling values after the pipeline stages (modes
// whose stages leave room for it) and reads one accumulator chunk: the
// largest summed extent it takes (0: none)
template <int MODE>
static int tc_dot_max_k_of()
{
    return tc_dot_fits<MODE>() ? tc_chunk_kb<MODE>() * (TC_ROWB / TcCfg<MODE>::EB) : 0;
}
int tc_dot_max_k(int mode)
{
    switch (mode) {
    case JET_PREC_TF32: return tc_dot_max_k_of<JET_PREC_TF32>();
    case JET_PREC_TF32X3: return tc_dot_max_k_of<JET_PREC_TF32X3>();
    case JET_PREC_BF16X3: return tc_dot_max_k_of<JET_PREC_BF16X3>();
    case JET_PREC_BF16X6: return tc_dot_max_k_of<JET_PREC_BF16X6>();
    case JET_PREC_FP16X3: return tc_dot_max_k_of<JET_PREC_FP16X3>();
    default: return 0;
    }
}

cudaError_t set_tc_smem_limits()
{
    cudaError_t e = cudaSuccess;
#define JET_TCSM(M)                                                                                        \
    if (e == cudaSuccess)                                                                                  \
        e = cudaFuncSetAttribute(tc_gemm_kernel<M JET_COMMA false>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                 tc_smem_bytes<M>());                                                       \
    if (e == cudaSuccess)                                                                                  \
        e = cudaFuncSetAttribute(tc_gemm_kernel<M JET_COMMA true>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                 tc_dot_fits<M>() ? tc_smem_bytes<M>(true) : tc_smem_bytes<M>())
    JET_TCSM(JET_PREC_TF32);
    JET_TCSM(JET_PREC_TF32X3);
    JET_TCSM(JET_PREC_BF16X3);
    JET_TCSM(JET_PREC_BF16X6);
    JET_TCSM(JET_PREC_FP16X3);
#undef JET_TCSM
#define JET_SPSM(M)                                                                                          \
    if (e == cudaSuccess)                                                                                    \
        e = cudaFuncSetAttribute(tc_split_kernel<M JET_COMMA true>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                 SPLIT_SMEM);                                                                \
    if (e == cudaSuccess)                                                                                    \
        e = cudaFuncSetAttribute(tc_split_kernel<M JET_COMMA false>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                 SPLIT_SMEM);
    JET_SPSM(JET_PREC_TF32)
    JET_SPSM(JET_PREC_TF32X3)
    JET_SPSM(JET_PREC_BF16X3)
    JET_SPSM(JET_PREC_BF16X6)
    JET_SPSM(JET_PREC_FP16X3)
#undef JET_SPSM
    return e;
}

cudaError_t launch_tc_split(const TcSplitArgs &a, const LaunchCfg &c, cudaStream_t s)
{
    dim3 grid(c.gx, c.gy, 1);
    const bool pow2 = c.variant & 2;
#define JET_SPLIT(M)                                                                         \
    do {                                                                                     \
        if (pow2) tc_split_kernel<M, true><<<grid, 256, SPLIT_SMEM, s>>>(a);                 \
        else tc_split_kernel<M, false><<<grid, 256, SPLIT_SMEM, s>>>(a);                     \
    } while (0)
    switch (a.mode) {
    case JET_PREC_TF32: JET_SPLIT(JET_PREC_TF32); break;
    case JET_PREC_TF32X3: JET_SPLIT(JET_PREC_TF32X3); break;
    case JET_PREC_BF16X3: JET_SPLIT(JET_PREC_BF16X3); break;
    case JET_PREC_BF16X6: JET_SPLIT(JET_PREC_BF16X6); break;
    case JET_PREC_FP16X3: JET_SPLIT(JET_PREC_FP16X3); break;
    default: return cudaErrorInvalidValue;
    }
#undef JET_SPLIT
    return cudaGetLastError();
}

static int sm_count()
{
    static int n = 0;
    if (!n) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1)
            n = 148;
    }
    return n;
}

cudaError_t launch_tc_gemm(const TcGemmArgs &a, const LaunchCfg &c, cudaStream_t s)
{
    const int64_t tiles = (int64_t)c.gx * c.gy * c.gz;   // persistent: one CTA per SM at most
    dim3 grid((unsigned)std::min<int64_t>(tiles, sm_count()), 1, 1);
#define JET_GEMM(M)                                                                                      \
    do {                                                                                                 \
        if (a.dot_parts && (!tc_dot_fits<M>() || a.n_kb > tc_chunk_kb<M>()))                             \
            return cudaErrorInvalidValue; /* no staging area, or more than one accumulator chunk */      \
        if (a.dot_parts) tc_gemm_kernel<M, true><<<grid, TC_THREADS, tc_smem_bytes<M>(true), s>>>(a);    \
        else tc_gemm_kernel<M, false><<<grid, TC_THREADS, tc_smem_bytes<M>(), s>>>(a);                   \
    } while (0)
    switch (a.mode) {
    case JET_PREC_TF32: JET_GEMM(JET_PREC_TF32); break;
    case JET_PREC_TF32X3: JET_GEMM(JET_PREC_TF32X3); break;
    case JET_PREC_BF16X3: JET_GEMM(JET_PREC_BF16X3); break;
    case JET_PREC_BF16X6: JET_GEMM(JET_PREC_BF16X6); break;
    case JET_PREC_FP16X3: JET_GEMM(JET_PREC_FP16X3); break;
    default: return cudaErrorInvalidValue;
    }
#undef JET_GEMM
    return cudaGetLastError();
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no -lcuda).
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn()
{
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        cudaDriverEntryPointQueryResult q;
        void *p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
    }
    return fn;
}

int encode_tc_maps(TcGemmArgs &a)
{
    EncodeTiledFn fn = encode_fn();
    if (!fn) return -1;
    const int eb = tc_elem_bytes(a.mode);
    const CUtensorMapDataType dt = eb == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                   : a.mode == JET_PREC_FP16X3 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                                               : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    cuuint32_t box[3] = {(cuuint32_t)(TC_ROWB / eb), (cuuint32_t)TC_BM, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    {
        cuuint64_t dims[3] = {(cuuint64_t)a.k_pad, (cuuint64_t)a.m_pad, (cuuint64_t)a.planesA_total};
        cuuint64_t strides[2] = {(cuuint64_t)(a.k_pad * eb), (cuuint64_t)(a.m_pad * a.k_pad * eb)};
        if (fn(&a.tmA, dt, 3, (void *)a.planesA, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return -2;
    }
    {
        cuuint64_t dims[3] = {(cuuint64_t)a.k_pad, (cuuint64_t)a.n_pad, (cuuint64_t)a.planesB_total};
        cuuint64_t strides[2] = {(cuuint64_t)(a.k_pad * eb), (cuuint64_t)(a.n_pad * a.k_pad * eb)};
        if (fn(&a.tmB, dt, 3, (void *)a.planesB, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return -3;
    }
    if (a.c_tma) {   // node outputs as floats: (2 Ni, Mi, instances), boxes of 32 floats x 32 rows
        if ((a.Ni & 1) || (a.baseC & 15) || a.c_inst < 1) return -4;
        cuuint64_t dims[3] = {(cuuint64_t)(2 * a.Ni), (cuuint64_t)a.Mi, (cuuint64_t)a.c_inst};
        cuuint64_t strides[2] = {(cuuint64_t)(2 * a.Ni * 4), (cuuint64_t)(a.Mi * 2 * a.Ni * 4)};
        cuuint32_t cbox[3] = {32, 32, 1};
        if (fn(&a.tmC, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, (void *)a.baseC, dims, strides, cbox, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_NONE,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return -5;
    }
    return 0;
}

}  // namespace jet
