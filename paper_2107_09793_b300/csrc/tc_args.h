// Argument blocks of the tensor-core route (split planes + tcgen05 GEMM).
#pragma once
#include <cuda.h>
#include <stdint.h>

#include "kernel_args.h"
#include "../../include/jet.h"

// Operand split: a complex64 operand, gathered from any strides into
// K-contiguous planes.  Instances come in groups of per_group; group g owns
// planes z = g * n_planes + p of rows_group rows x k_pad, and its j-th
// instance fills rows [j * rows, (j + 1) * rows) of each (the last one also
// zeroes the group's padding rows up to rows_group).  Plane order per group:
//   bf16x3 / tf32x3 : re_hi, re_lo, im_hi, im_lo
//   bf16x6          : re_hi, re_mid, re_lo, im_hi, im_mid, im_lo
//   tf32            : re, im
// Padding columns (k >= k) are written as zeros.
struct TcSplitArgs {
    uint64_t ptrSrc;                 // device array of n_inst source addresses (complex64)
    uint64_t planes;                 // plane base (device)
    uint64_t scales;                 // FP16X3: float 2^-s per [group][K chunk][row of the group] (else 0)
    int64_t rows, k, rows_group, k_pad;
    int32_t n_inst, n_planes;
    int32_t per_group, pair16;       // pair16: the fastest summed label (k_dim[0]) has stride 1,
                                     // so source entries 2c, 2c + 1 of a row are adjacent
    int32_t rank_r, rank_k;
    int32_t mode, fast_k;           // fast_k: the source's stride-1 label is a summed label
    int64_t r_dim[JET_MAXR], r_s[JET_MAXR];   // row labels, fastest first, source strides
    int64_t k_dim[JET_MAXR], k_s[JET_MAXR];   // summed labels, fastest first, source strides
    // row_perm: the row labels above are in the order that reads the source best
    // (tile rows along its fastest labels); a row's plane row is then the sum of
    // its digits times p_s (the labels' strides in the planes' row order)
    int64_t p_s[JET_MAXR];
    int32_t row_perm, pad2_;
};

// C[m][n] = sum_k A[m][k] B[n][k] over split planes, complex 4M form: the real
// accumulator takes Ar.Br + (-Ai).Bi, the imaginary one Ar.Bi + Ai.Br, each
// real product expanded into the split terms of the mode.
// A launch runs n_inst blocks.  Block b is one product of an A group of nA
// operand instances (rows j * Mi + m) and a B group of nB (columns l * Ni + n):
// M = nA * Mi rows, N = nB * Ni columns; its entry (j, m; l, n) belongs to node
// instance itab[(b * nA + j) * nB + l] (-1: not computed), element m * Ni + n
// of that instance's output.  Without itab (nA = nB = 1) block b is instance b.
struct TcGemmArgs {
    CUtensorMap tmA;                 // 3-D map over A planes: (k_pad, m_pad, planes)
    CUtensorMap tmB;                 // 3-D map over B planes: (k_pad, n_pad, planes)
    CUtensorMap tmC;                 // c_tma: 3-D map over the node's outputs as floats:
                                     // (2 Ni, Mi, c_inst), 32 x 32 boxes, 128-byte swizzle
    uint64_t baseC;                  // c_tma: the node's output buffer (instance i at i M N)
    uint64_t planesA, planesB;       // plane bases (device), used to encode the maps
    uint64_t zA, zB;                 // device int32[n_inst]: first plane index of each block's groups
    uint64_t ptrC;                   // device array of the node instances' output addresses (complex64)
    uint64_t status;                 // device uint32 error word (bounded-wait time-outs)
    uint64_t scaleA, scaleB;         // FP16X3: 2^-s per [group][K chunk][row] of each operand
    uint64_t itab;                   // device int32[n_inst * nA * nB], or 0
    int64_t M, N, K;                 // rows and columns of one block, summed extent
    int64_t m_pad, n_pad, k_pad;     // rows of an A group's planes, of a B group's, padded K
    int64_t Mi, Ni;                  // rows and columns of one node instance
    int64_t planesA_total, planesB_total;   // plane count along the maps' third dimension
    int32_t n_inst, mode;            // blocks
    int32_t n_kb, nA;
    int32_t nB, mi_shift;            // log2(Mi) and log2(Ni) when powers of two, else -1
    int32_t ni_shift, c_tma;         // c_tma: C leaves through tensor-map bulk stores (Ni even;
                                     // grouped blocks: Mi a multiple of 32, Ni of 16)
    int64_t c_inst;                  // c_tma: node instances (the map's third extent)
    // FP16X3 fused split (fz_planes != 0): instead of complex64 C, the epilogue
    // writes the node's output as its parent GEMM's operand planes and scales.
    // Node instance i, row m = (m_f, m_k) with m_k the lowest lmk bits, column
    // n = (n_f, n_k) with n_k the lowest lnk bits: parent row r = fz_pm[m_f] +
    // fz_pn[n_f], parent summed index k = m_k 2^lnk + n_k; element (r, k) of
    // plane q at fz_planes + 2 (fz_ibase[2 i] + q fz_plane_elems + r fz_kpad + k)
    // bytes, its 64-wide chunk scale at fz_scales + 4 (fz_ibase[2 i + 1] +
    // (k / 64) fz_rows_pad + r) (64 / 2^lnk lanes share a chunk; lnk is 2 or 3)
    uint64_t fz_planes, fz_scales, fz_ibase, fz_pm, fz_pn;
    int64_t fz_plane_elems, fz_kpad, fz_rows_pad;
    int32_t fz_lmk, fz_lnk;
    // Dot epilogue (dot_parts != 0): the parent contracts this output with a
    // sibling tensor A over every label (a dot product per parent instance).
    // Instead of C, the launch runs dot_nblk blocks of up to two node instances
    // that pair the same A instances (up to two): dot_pair[8 d ..] = {c0, c1,
    // p00, p01, p10, p11, 0, 0} (c1 = -1 for none; p_km the parent instance of
    // c_k with A instance m, or -1), A_m at dot_ptrA[2 d + m]; node instance c
    // is entry (j, l) of GEMM block b, (b, j, l) = dot_cpos[3 c ..].  A step is
    // one 128 x 128 tile position (Mi, Ni multiples of 128) of one dot block,
    // steps ordered block fastest; its two tiles (c0's and c1's, c0's again for
    // none) accumulate in the two TMEM buffers, and every tile entry (m, n) adds
    // C_k[m][n] A_m[x] to product p_km, x = the sum of dot_sm[b] over the set
    // bits b of m plus dot_xn[n]; a tile's sum goes to dot_parts[p dot_tiles +
    // the tile's index in the instance] (complex128), summed over tiles in FP64.
    // A's values of a warp's 32 rows x 8 columns are staged in shared memory by
    // 16-byte asynchronous copies of two values adjacent in A: two columns of a
    // row (dot_lcol = 1: A's stride-1 label is a column label) or two rows of a
    // column (0: a row label); every offset other than the stride-1 label's
    // digit is even and every A instance's address 16-byte aligned.
    uint64_t dot_parts, dot_ptrA, dot_pair, dot_xn, dot_cpos;
    int64_t dot_sm[JET_MAXR];
    int32_t dot_mbits, dot_tiles;
    int32_t dot_lcol, dot_nblk;
};
