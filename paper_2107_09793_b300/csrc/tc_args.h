// Argument blocks of the tensor-core route (split planes + tcgen05 GEMM).
#pragma once
#include <cuda.h>
#include <stdint.h>

#include "kernel_args.h"
#include "../../include/jet.h"

// Operand split: a complex64 operand, gathered from any strides into
// [rows_pad][k_pad] K-contiguous planes.  Plane order per instance:
//   bf16x3 / tf32x3 : re_hi, re_lo, im_hi, im_lo
//   bf16x6          : re_hi, re_mid, re_lo, im_hi, im_mid, im_lo
//   tf32            : re, im
// Padding rows/columns are written as zeros.
struct TcSplitArgs {
    uint64_t ptrSrc;                 // device array of n_inst source addresses (complex64)
    uint64_t planes;                 // plane base (device)
    uint64_t scales;                 // FP16X3: float 2^-s per [instance][K chunk][row] (else 0)
    int64_t rows, k, rows_pad, k_pad;
    int32_t n_inst, n_planes;
    int32_t rank_r, rank_k;
    int32_t mode, fast_k;           // fast_k: the source's stride-1 label is a summed label
    int64_t r_dim[JET_MAXR], r_s[JET_MAXR];   // row labels, fastest first, source strides
    int64_t k_dim[JET_MAXR], k_s[JET_MAXR];   // summed labels, fastest first, source strides
};

// C[m][n] = sum_k A[m][k] B[n][k] over split planes, complex 4M form with three
// FP32 accumulators in TMEM: P = Ar.Br, Q = Ai.Bi, I = Ar.Bi + Ai.Br;
// C = (P - Q) + i I.  Each real product expands into the split terms of the mode.
struct TcGemmArgs {
    CUtensorMap tmA;                 // 3-D map over A planes: (k_pad, m_pad, planes)
    CUtensorMap tmB;                 // 3-D map over B planes: (k_pad, n_pad, planes)
    uint64_t planesA, planesB;       // plane bases (device), used to encode the maps
    uint64_t zA, zB;                 // device int32[n_inst]: first plane index of each instance
    uint64_t ptrC;                   // device array of n_inst output addresses (complex64)
    uint64_t status;                 // device uint32 error word (bounded-wait time-outs)
    uint64_t scaleA, scaleB;         // FP16X3: 2^-s per [instance][K chunk][row] of each operand
    int64_t M, N, K;
    int64_t m_pad, n_pad, k_pad;
    int64_t planesA_total, planesB_total;   // plane count along the maps' third dimension
    int32_t n_inst, mode;
    int32_t n_kb, pad_;
};
