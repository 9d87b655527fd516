// Plain-old-data argument blocks of the device kernels.  Built on the host by
// the plan compiler, passed to the kernels by value (__grid_constant__).
// Pointer-table fields hold device addresses patched in when the plan is bound
// to its buffers.
#pragma once
#include <stdint.h>

#define JET_MAXR 40          // max labels decoded by loop (rows, outer K part)
#define JET_COLMAX 1024      // max entries of a column offset table
#define JET_KLOMAX 1024      // max entries of an inner-K offset table
#define JET_SPLITK_G 8       // outputs per block in the split-K direct kernel
#define JET_APPLY_MAXK 256   // small-operand application: max summed entries (streamed form)
#define JET_APPLY_STREAMB 4096 // streamed form: max entries of the small operand (free padded to 16)
#define JET_APPLY_HOLDK 32   // ... held in registers: max summed entries
#define JET_APPLY_MAXF 256   // small-operand application: max free entries of the small operand
#define JET_APPLY_MAXB 1024  // held form: max entries of the small operand (summed extent padded)
#define JET_APPLY_STREAMF 32 // streamed form: max free entries of the small operand
#define JET_APPLY_TC_MAXF 128 // tensor-core form: max free entries of the small operand (N <= 256 real columns)
#define JET_APPLY_TC_MAXF_MULTI 32 // ... when the summed extent is above one 32-entry chunk (FP32 promotion registers)
#define JET_APPLY_TC_WIDEF 64 // above this many free entries (at most 32 summed): the A chunk is staged in halves
#define JET_APPLY_TC_ABYTES 65536 // tensor-core form: one group's A chunk, hi + lo TF32 planes of 128 x 64
#define JET_APPLY_TC_SMEM_MAX 231424 // tensor-core form: dynamic shared memory cap (227 KiB less 1 KiB)

// Dynamic shared memory of the tensor-core application: 1 KiB alignment slack,
// one A chunk per thread group (half a chunk when staged in halves) and the hi /
// lo TF32 planes of the small operand (summed entries padded to blocks of 8,
// free entries to 8, two real rows each).
// Chunks staged in halves of 16 summed entries: above JET_APPLY_TC_WIDEF free
// entries, or when two groups' whole chunks and the operand planes do not fit.
static inline bool jet_apply_tc_half(int nk, int nf)
{
    const int nkb = (nk + 7) / 8, nr = 2 * ((nf + 7) / 8 * 8);
    return nf > JET_APPLY_TC_WIDEF || 1024 + 2 * JET_APPLY_TC_ABYTES + 2 * nkb * nr * 64 > JET_APPLY_TC_SMEM_MAX;
}
// (f16: the FP16 form's A planes take half the bytes; its small operand's
// exponents and their inverses follow the planes, 512 of each)
static inline int jet_apply_tc_smem(int groups, int nk, int nf, int f16 = 0)
{
    const int nkb = (nk + 7) / 8, nr = 2 * ((nf + 7) / 8 * 8);
    const int abytes = (jet_apply_tc_half(nk, nf) ? JET_APPLY_TC_ABYTES / 2 : JET_APPLY_TC_ABYTES) / (f16 ? 2 : 1);
    return 1024 + groups * abytes + 2 * nkb * nr * 64 + (f16 ? 512 * 8 : 0);
}

// Pairwise contraction C = sum_K A * B evaluated directly from strides
// (Section 2.3).  The output index is split as (row, col): col is the trailing
// group of output labels (offset tables colA/colB), row is decoded by loop.
// The summed index is split as (khi, klo): klo has offset tables kA/kB, khi is
// decoded by loop.  All offsets are in elements.
struct DirectArgs {
    uint64_t ptrA, ptrB, ptrC;      // device arrays of n_inst addresses (uint64)
    uint64_t colA, colB;            // device int32[n_cols]
    uint64_t kA, kB;                // device int32[n_klo]
    uint64_t partials;              // split-K scratch: complex[n_inst][ksplit][n_out] (or 0)
    int64_t n_rows, n_khi, n_out;
    int32_t n_cols, n_klo;
    int32_t n_inst, ksplit;
    int32_t row_rank, khi_rank;
    int32_t khi_per_part;           // split-K: khi values per part
    int32_t splitk_na;              // split-K: 0, or the outer-product pattern of every group of
                                    // 8 outputs, whose operand values are then read once per
                                    // summed entry: NA in {1, 2, 4, 8} = NA values of A (fastest)
                                    // x 8 / NA of B; 16 + NB (NB in {2, 4}) = NB of B fastest;
                                    // 32 = a single output (a dot product); 64 = dot
                                    // products of instance blocks (below; 65: blocks of at
                                    // most 2 x 2; 66: the same with B staged, below)
    uint64_t itab;                  // splitk_na 64, 65: block b (blockIdx.z) holds node instances
                                    // itab[(b blk_na + j) blk_nb + l], their A the A of
                                    // instance (j, 0), their B the B of instance (0, l): each
                                    // operand value is loaded once for blk_na x blk_nb outputs
    int32_t blk_na, blk_nb;
    uint64_t qB;                    // splitk_na 66 (2 x 2 blocks, B staged in shared memory): kB
                                    // lists B's inner entries in increasing B offset and
                                    // device int32[n_klo] qB their inner index q (A's kA order)
    int64_t row_dim[JET_MAXR], row_sA[JET_MAXR], row_sB[JET_MAXR];   // fastest label first
    int64_t khi_dim[JET_MAXR], khi_sA[JET_MAXR], khi_sB[JET_MAXR];   // fastest label first
};

// Small operand applied to a large one: C[r, f] = sum_q B[f, q] A[r, q], r over
// A's free labels (decoded fastest first), q over the summed labels, f over B's
// free labels.  Offsets are in elements.
struct ApplyArgs {
    uint64_t ptrA, ptrB, ptrC;      // device arrays of n_inst addresses (A large, B small)
    uint64_t status;                // device uint32 error word (tensor-core form: bounded-wait time-outs)
    int64_t n_fib;                  // fibers per instance: product of A's free dims
    int32_t n_inst, nk, nf, rank;   // nk <= nk_tmpl (entries nk..nk_tmpl-1 are padding)
    int32_t nk_tmpl;                // held form: compile-time summed extent
    int32_t nf_tmpl;                // streamed form (nf_tmpl > 0): free entries per register chunk
    int32_t tc_terms;               // tensor-core form: products per real product (1 or 3)
    int32_t tc_f16;                 // tensor-core form, 3 terms: FP16 hi + lo parts with a power-of-two
                                    // scale per row and 32-entry chunk (kind::f16, K = 16 per MMA)
                                    // instead of TF32 hi + lo (K = 8)
    int64_t kA[JET_APPLY_MAXK], bK[JET_APPLY_MAXK];   // summed entry q: offset in A, in B
    int64_t cF[JET_APPLY_MAXF], bF[JET_APPLY_MAXF];   // B-free entry f: offset in C, in B
    int64_t dim[JET_MAXR], sA[JET_MAXR], sC[JET_MAXR];
    int32_t shift[JET_MAXR];        // power-of-two dims: digit j of a fiber index starts at bit shift[j]
};

// Sum the split-K partials of each output in a fixed order (deterministic).
struct SplitKReduceArgs {
    uint64_t partials;              // complex[n_inst][ksplit][n_out] (parts64: complex128)
    uint64_t ptrC;                  // device array of n_inst addresses
    int64_t n_out;
    int32_t n_inst, ksplit;
    int32_t parts64, pad_;          // 1: FP64 partials summed in FP64 (a GEMM's dot epilogue)
};

// Gather a strided tensor into a dense one: dst[i] = src[off(i)], where the
// destination index is decoded fastest label first (Section 3.1: the transpose
// half of transpose-transpose-GEMM).
struct PermuteArgs {
    uint64_t ptrSrc, ptrDst;        // device arrays of n_inst addresses
    int64_t n;                      // elements per instance
    int32_t rank, n_inst;
    int64_t dim[JET_MAXR];          // destination labels, fastest first
    int64_t sstride[JET_MAXR];      // matching source strides
};

// Batched complex GEMM C[m][n] = sum_k A[m][k] B[k][n] (row-major C, ldc = N).
// a_kmajor: A stored [M][K] (else [K][M]); b_kmajor: B stored [N][K] (else [K][N]).
struct GemmArgs {
    uint64_t ptrA, ptrB, ptrC;      // device arrays of n_inst addresses
    int64_t M, N, K;
    int32_t n_inst;
    int32_t a_kmajor, b_kmajor;
    int32_t pad_;
};

// A small pairwise contraction inside a batched launch: full offset tables
// (output -> A/B offsets, summed index -> A/B offsets), no index decoding.
struct SmallTask {
    uint64_t ptrA, ptrB, ptrC;      // device arrays of n_inst addresses
    uint64_t offA, offB;            // device int32[n_out]
    uint64_t kA, kB;                // device int32[n_k]
    int32_t n_out, n_k, n_inst;
    int32_t block0;                 // first block of this task within the launch
};

// One launch over many independent small contractions of one tree level; or
// (chain, n_levels > 0) consecutive small levels in one cooperative launch of
// n_blocks blocks, level l being tasks [lv_end[l - 1], lv_end[l]) run after
// level l - 1 behind a grid barrier, each task's block0 then holding its first
// item within its level.
#define JET_CHAIN_LEVELS 32
#define JET_CHAIN_TASKS 1024   // tasks per chained level
struct SmallBatchArgs {
    uint64_t tasks;                 // device SmallTask[n_tasks], ordered by block0 (per level)
    int32_t n_tasks, n_blocks;
    int32_t n_levels, pad_;
    uint64_t barrier;               // chain: device uint32[2] (arrivals, departures), zero between launches
    uint64_t status;                // chain: device uint32 error word (bit 8: a grid barrier timed out)
    int32_t lv_end[JET_CHAIN_LEVELS];
};

// Adjoint accumulation: for each target instance t, env_t[off(e)] += sum over the
// source instances i mapped to t (ascending i) of src_i[e]; e runs over the
// dense source layout, off(e) decodes it with the target's strides.
struct AccumArgs {
    uint64_t src;                   // source base; instance i at src + i * n elements
    uint64_t tgt;                   // device array of n_tgt target addresses
    uint64_t csr_ptr, csr_src;      // int32[n_tgt + 1], int32[n_src]
    int64_t n;                      // elements per source instance
    int32_t n_tgt, rank;
    int32_t src_fp64, tgt_fp64;
    int64_t dim[JET_MAXR];          // source labels, fastest first
    int64_t tstride[JET_MAXR];      // matching target strides
};

// Several adjoint accumulations of one tree level in one launch: task t owns
// blocks [block0_t, block0_{t+1}); each task is an AccumArgs.
struct AccumTask {
    AccumArgs a;
    int32_t block0, pad_[3];
};
struct AccumBatchArgs {
    uint64_t tasks;                 // device AccumTask[n_tasks], ordered by block0
    int32_t n_tasks, n_blocks;
};

// cudaMemsetAsync(ptr, 0, bytes) as a plan step.
struct MemsetArgs {
    uint64_t ptr;
    int64_t bytes;
};

// amp[b] = sum over slices s (increasing s) of root[inst(b, s)], FP64
// (Section 2.4, Eq. sliced_sum; the single reduction over slices).
struct ReduceArgs {
    uint64_t roots;                 // device array of n_amps * n_slices root-instance addresses
    uint64_t amps;                  // complex128[n_amps][n_elem] (or [n_amps][n_slices][n_elem] partials)
    uint64_t eoff;                  // device int64[n_elem]: element offset in a root instance of
                                    // value e of the free open legs (0 when n_elem == 1)
    int32_t n_amps, n_slices;
    int32_t fp64_in;
    int32_t partials;               // 1: write every root value instead of the sums
    int32_t n_elem, pad_;           // values per amplitude row
};
