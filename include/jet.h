/*
 * jet.h - C ABI of the B300 sliced tensor-network contraction library.
 *
 * The problem these calls state (Section 3, "Overview of Jet"): a tensor network
 * of gate and state tensors with labelled indices, a pairwise contraction path,
 * and a set of sliced indices, reduced to one or more output amplitudes.
 *
 *   network  Section 2.1 / 2.2.1: tensors are nodes, shared labels are edges; a
 *            label carried by two tensors is summed over, a label carried by one
 *            tensor is an open leg (an output qudit).
 *   path     Section 2.3 (Eq. sequence, binary contraction tree): step k contracts
 *            two live tensors over the labels they share.
 *   slice    Section 2.4 (Eq. sliced_sum): a sliced label is fixed to each of its
 *            values in turn; the amplitude is the sum of the partial contractions.
 *   reuse    Section 3.2 (Eq. task_based_amplitude_flops): an intermediate that
 *            does not depend on a slice (or amplitude) value is computed once and
 *            read by every slice (amplitude) that needs it.
 *
 * Conventions shared by every call
 *   - Tensors are dense and row-major; labels[0] is the slowest index.
 *   - Every call returns JET_OK (0) or a negative JET_E* code; on error nothing
 *     has changed (all-or-nothing) and jet_last_error() describes the failure.
 *     A handle stays valid after an error.
 *   - Input buffers are copied; the caller keeps ownership of everything it
 *     passes.  Output buffers are caller-owned.
 *   - A handle is not thread-safe: one thread at a time per handle.
 *   - Complex numbers are interleaved (re, im).
 *   - Device work runs on the CUDA stream the caller passes (NULL = the legacy
 *     default stream) on the device named in jet_options.device.
 */
#ifndef JET_B300_H
#define JET_B300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define JET_OK        0
#define JET_EINVAL   -1   /* bad label, dim, path, slice, size or pointer         */
#define JET_ENOMEM   -2   /* device or host allocation failed, or workspace too small */
#define JET_ECUDA    -3   /* a CUDA runtime or driver call failed                 */
#define JET_ETIMEOUT -4   /* a bounded device-side wait ran out                   */
#define JET_ESTATE   -5   /* call out of order (e.g. contract before a path)      */

typedef struct jet_network jet_network;            /* opaque, owned by the library */

typedef struct { float re, im; } jet_c64;
typedef struct { double re, im; } jet_c128;

/* Arithmetic used for the large (GEMM-shaped) pairwise contractions and, in
 * the split modes (every mode but FP32 and FP64), for the application of a
 * small operand with at most 256 summed and 32 free entries (128 free when it
 * has at most 32 summed), and at least apply_tc_min_kf of them in all
 * (summed x free), to a large one (TF32 hi + lo,
 * three products; one in JET_PREC_TF32).  Other small contractions always run
 * on CUDA cores in FP32 (FP64 in JET_PREC_FP64).
 * Intermediates are complex64, except in JET_PREC_FP64 (complex128).  Slice
 * and amplitude sums are always FP64. */
typedef enum {
    JET_PREC_FP32   = 0,  /* FP32 FMA on CUDA cores (the plain reference path)         */
    JET_PREC_TF32   = 1,  /* one TF32 tcgen05 product per real product, FP32 accumulate */
    JET_PREC_TF32X3 = 2,  /* x = hi + lo in TF32; hi*hi + hi*lo + lo*hi                 */
    JET_PREC_BF16X3 = 3,  /* x = hi + lo in BF16; hi*hi + hi*lo + lo*hi                 */
    JET_PREC_BF16X6 = 4,  /* x = hi + mid + lo in BF16; the six products above 2^-24    */
    JET_PREC_FP64   = 5,  /* complex128 everywhere, FP64 on CUDA cores                  */
    JET_PREC_FP16X3 = 6   /* x * 2^s = hi + lo in FP16, one power-of-two scale s per
                             operand row and 32-wide K chunk (undone exactly when the
                             chunk is added up); hi*hi + hi*lo + lo*hi                   */
} jet_precision;

typedef struct {
    int32_t precision;        /* jet_precision, default JET_PREC_FP32                     */
    int32_t reuse;            /* 1 (default): shared intermediates computed once;
                                 0: every (slice, amplitude) recomputes its whole tree   */
    int32_t use_graph;        /* 1 (default): record the launch sequence in a CUDA graph */
    int32_t device;           /* CUDA device ordinal, default 0                          */
    int64_t gemm_min_k;       /* contractions with a summed extent >= this (and both free
                                 extents >= 64) take the GEMM route, except, in the split
                                 modes, those with a summed extent <= 32 and one free
                                 extent <= 128 that the tensor-core small-operand form
                                 takes; default 16                                        */
    int64_t workspace_limit;  /* bytes of device workspace a contraction may use; 0 = no
                                 limit.  When the plan for every slice needs more,
                                 jet_contract / jet_contract_async run the slices in
                                 ranges chosen to share work (see jet_plan_ranges),
                                 each range's shared intermediates computed once, and
                                 sum the per-slice partials in increasing slice id in
                                 FP64 (the order of one plan; a range's plan may route a
                                 node with fewer instances to another kernel form, so
                                 the values agree to the arithmetic's rounding).  A
                                 caller-provided workspace smaller than the plan caps
                                 it the same way. */
    int32_t profile;          /* 0 (default): off; 1: CUDA events around every GEMM, operand
                                 split and small-operand launch; 2: around every launch
                                 (read with jet_profile)                                  */
    int32_t apply_tc_min_kf;  /* split modes: small-operand applications whose small operand
                                 has at least this many entries (summed x free) run on the
                                 tensor cores, and from half as many those with at most 32
                                 summed entries and summed x free >= 10 (summed + free),
                                 where the CUDA-core forms are FMA-bound; default 1024,
                                 above 8192 none does                                     */
    int32_t gemm_group;       /* 1 (default): a GEMM-route node whose instances pair every
                                 instance of one operand with the same instances of the
                                 other runs those pairs as one wider product per block
                                 (a shared operand read once per tile row or column, short
                                 sides packed into full tiles); 0: one product per
                                 instance                                                 */
    int32_t fuse_split;       /* 1 (default): epilogue fusions of the tensor-core GEMMs
                                 where the shapes allow them: in FP16x3, a GEMM whose
                                 output is the larger operand of the next GEMM writes that
                                 GEMM's FP16 operand planes and chunk scales (no complex64
                                 intermediate, no operand split); a GEMM whose output is
                                 contracted with its sibling over every label, with its
                                 summed extent in one accumulator chunk, forms those dot
                                 products per tile (the parent only adds the tiles' parts;
                                 a choice that jet_autotune times); 0: complex64 output,
                                 contracted by the next step                              */
} jet_options;

typedef struct {
    int32_t rank;
    const int64_t *labels;    /* rank labels, any non-negative values                    */
    const int32_t *dims;      /* rank dims, each >= 1; a label has one dim everywhere     */
    const jet_c64 *data;      /* prod(dims) values, row-major, labels[0] slowest (host)   */
} jet_tensor_desc;

typedef struct {
    double   flop_planned;        /* algorithmic real FLOP of one amplitude, the path
                                     unsliced: 8 * prod(dims of the union) per step        */
    double   flop_sliced;         /* N_sl * FLOP_sl (Eq. sliced_flops), no reuse           */
    double   flop_executed;       /* FLOP of the unique instances the last plan executes  */
    double   reuse_fraction;      /* f_sl of Eq. task_based_amplitude_flops (last plan)   */
    double   bytes_executed;      /* algorithmic HBM bytes of the last plan               */
    int64_t  max_intermediate;    /* largest intermediate of one slice, elements          */
    int64_t  workspace_bytes;     /* device workspace the last plan needs                 */
    int64_t  n_instances;         /* unique contraction instances in the last plan        */
    int64_t  n_launches;          /* kernel launches per contract call                    */
    int32_t  n_slices;            /* N_sl                                                  */
    int32_t  n_sliced_labels;
    int32_t  n_gemm_nodes;        /* tree nodes routed to the GEMM kernels                */
    int32_t  n_direct_nodes;      /* tree nodes routed to the direct-contraction kernel   */
} jet_stats_t;

/* One launch of the plan run last, for jet_profile. */
typedef struct {
    int32_t kind;             /* 0 direct, 1 permute, 2 SIMT GEMM, 3 tensor-core GEMM,
                                 4 slice reduction, 5 split-K reduction, 6 operand split,
                                 7 batched small contractions of one tree level,
                                 8 adjoint accumulation, 9 memset, 10 small operand
                                 applied to a large one, 11 batched adjoint
                                 accumulations of one tree level                          */
    int32_t node;             /* tree node (SSA id) the launch belongs to               */
    int64_t n_inst;           /* instances the launch processes                         */
    double  flop;             /* algorithmic real FLOP of the launch                    */
    double  bytes;            /* algorithmic HBM bytes of the launch                    */
    float   ms;               /* device time of the last run, -1 if not timed           */
    int32_t block;            /* threads per block                                      */
    int32_t grid[3];          /* launch grid                                            */
    int32_t smem;             /* dynamic shared memory bytes (0 = kernel default)       */
    int32_t variant;          /* kernel variant selector (kind specific)                */
    int32_t pad_;
} jet_op_record;

/* Defaults listed in jet_options above. */
void jet_options_default(jet_options *opt);

/* Build a network from n tensors (Section 2.2.1).  Copies every tensor to the
 * device.  Each label must appear in one or two tensors, with the same dim in
 * both; labels appearing once are open legs.  opt may be NULL (defaults).
 * Errors: JET_EINVAL (n < 1, rank < 0, dim < 1, a label on three tensors or
 * repeated in one tensor, mismatched dims, NULL pointers), JET_ENOMEM, JET_ECUDA. */
int jet_network_create(const jet_tensor_desc *tensors, int32_t n, const jet_options *opt,
                       jet_network **out);

/* Declare the output legs, in the order the amplitude patterns of jet_contract
 * list their digits (the bras <a_i| of Section 2.2.1 attach here).  Every open
 * leg must be listed exactly once.  Clears the path-dependent plan.
 * Errors: JET_EINVAL (a label that is not an open leg, a duplicate, a missing leg). */
int jet_network_set_open(jet_network *net, int32_t n_out, const int64_t *out_labels);

/* Keep shared work for later contractions (Section 3.2: work shared between
 * contractions is done once; the paper's conclusion: it can be stored for any
 * later slice or amplitude calculation).  A sub-tree of the path whose tensors
 * carry no fixed label (no sliced label, no open leg fixed by a bra) has the
 * same value in every contraction of this network.  With min_elems > 0 every
 * maximal such sub-tree whose result has at least min_elems elements keeps its
 * result in a device pool after the first contraction computes it; later
 * contractions (any outputs or slices) read it instead of launching the
 * sub-tree.  A contraction that fills the pool synchronises its stream at the
 * end.  The pool starts afresh when the path, slicing, open or free legs or any
 * tensor value change; min_elems = 0 switches keeping off and frees the pool.
 * Gradients and networks planned without reuse do not keep.
 * Errors: JET_EINVAL (min_elems < 0). */
int jet_network_keep_shared(jet_network *net, int64_t min_elems);

/* Store the kept shared work in a file, and read it back into a network that
 * has the same tensors (by value), path, sliced labels, open and free legs,
 * precision and keep threshold -- in this process or another one (the
 * paper's conclusion: shared work stored on disk for any later slice or
 * amplitude calculation).  save writes every ready kept result (HOST file:
 * a key of what the results depend on, then the results).  load (keeping must
 * be on) checks that key against the network and marks the results ready; the
 * next contraction reads them instead of computing their sub-trees.
 * Errors: JET_ESTATE (nothing kept yet / keeping off), JET_EINVAL (file
 * unreadable or not written by save, or written for another network, path,
 * slicing, legs, precision, threshold or tensor values). */
int jet_network_save_shared(jet_network *net, const char *file);
int jet_network_load_shared(jet_network *net, const char *file);

/* Leave some output legs free (Section 2.2.1: an open leg without a bra stays
 * an index of the result; Section 3.2: a batch of amplitudes is one
 * multi-contraction whose shared work is done once).  Every contraction then
 * returns, for each row of outputs, all E = prod(dims of the free legs) values
 * of those legs at once, every intermediate that does not hold a free leg
 * computed once for all of them.  free_labels lists open legs (a subset of
 * jet_network_set_open's); their digits in outputs are ignored.  Value e of a
 * row is the mixed-radix number over the free legs in this order, the first
 * most significant: jet_contract writes amps_out[b * E + e], jet_contract_async
 * the same layout in device memory, jet_contract_slices
 * partials_out[(b * n_ids + j) * E + e].  The path planners count a free leg
 * with its dim (a fixed one counts as 1).  n_free = 0 fixes every open leg
 * again; jet_network_set_open clears the list; jet_contract_grad refuses free
 * legs.  Clears the plan.
 * Errors: JET_EINVAL (not an open leg, a duplicate, more than 2^24 values per
 * row), JET_ESTATE (open legs not declared yet). */
int jet_network_set_free(jet_network *net, int32_t n_free, const int64_t *free_labels);

/* Replace the values of tensor tensor_id (same shape).  Host pointer; the copy to
 * the device is ordered on the library's internal stream before the next
 * contraction.  Errors: JET_EINVAL (bad id / NULL), JET_ECUDA. */
int jet_tensor_update(jet_network *net, int32_t tensor_id, const jet_c64 *data);

/* Replace the values of all tensors at once: data holds every tensor's values
 * back to back in tensor order (jet_network_n_values() complex values).  One
 * host-to-device copy on `stream`, ordered before work later issued there.
 * Pass pinned host memory for an asynchronous copy. */
int jet_tensors_upload(jet_network *net, const jet_c64 *data, void *cuda_stream);
int64_t jet_network_n_values(const jet_network *net);

/* Set the contraction path (Section 2.3): n_steps = n_tensors - 1 pairs in SSA
 * form: ids 0..n-1 are the input tensors, step k creates id n+k; each id is
 * consumed exactly once.  Errors: JET_EINVAL (wrong count, an id used twice or
 * not yet created), JET_ESTATE (open legs not declared). */
int jet_path_set(jet_network *net, int32_t n_steps, const int32_t *pairs);

/* Read back the current path (2 * (n_tensors - 1) ints). */
int jet_path_get(const jet_network *net, int32_t *pairs_out);

/* The library's own planner (the paper delegates path search to an external
 * tool, Section 3).  Greedy: repeatedly contract the pair of tensors sharing a
 * label that minimises size(out) - size(A) - size(B), ties to smaller FLOP then
 * smaller ids; trial t > 0 perturbs the score with seeded noise; the path of
 * lowest total FLOP is kept.  It is then improved by sub-tree reconfiguration:
 * for every internal node, the sub-tree below it is opened down to at most 10
 * tensors (largest intermediate first) and re-ordered optimally by dynamic
 * programming over subsets, when that lowers the FLOP without an intermediate
 * above the path's largest (8 passes over the tree).  The result is set;
 * flop_out (may be NULL) receives its FLOP.  Open legs count as fixed (dim 1)
 * because every amplitude fixes them.  Networks of up to 10 tensors get an
 * optimal order under that size bound. */
int jet_path_greedy(jet_network *net, uint64_t seed, int32_t n_trials, double *flop_out);

/* Batch-aware form of jet_path_greedy for a batch of amplitudes contracted
 * together with shared work reused (Sections 3.2 and 4: several amplitudes
 * with one path, only the bras differ).  A tree node holding open legs L is
 * computed once per distinct restriction of the batch's output digits to L, so
 * every size and FLOP in the greedy score is weighted by that count: subtrees
 * without bras are shared by the whole batch and the planner keeps the bras
 * late when that is cheaper.  Besides the pairwise passes of jet_path_greedy it
 * runs linear passes (one tensor grows by absorbing the neighbouring leaf with
 * the smallest weighted result), from leaf 0 and, on odd trials, from a seeded
 * random leaf, and two leaf-order linear paths: leaves absorbed strictly in
 * index order (for a circuit listed initial states first, then gates in time
 * order: the state-vector order), and the lowest-index leaf sharing a label
 * with the growing tensor (initial states join when first touched).  Steps whose weighted result (instances x elements) exceeds
 * max_elems are taken only when no other step is left, and the kept path is
 * the one of lowest FLOP among those whose largest weighted intermediate fits
 * max_elems (none fits: the smallest such peak).  max_elems <= 0: no cap.
 * outputs: n_amps x n_out digits, HOST memory, the jet_contract layout (only
 * read during the call).  flop_out receives the batch's total FLOP (instances
 * x node FLOP, summed).  Errors: JET_EINVAL (NULL, n_amps < 1, digit out of
 * range), JET_ESTATE (open legs not declared). */
int jet_path_greedy_batch(jet_network *net, int32_t n_amps, const int32_t *outputs, int64_t max_elems,
                          uint64_t seed, int32_t n_trials, double *flop_out);

/* Improve the current path for its current slicing (Section 3.2: minimise
 * Eq. task_based_amplitude_flops itself rather than the FLOP of one slice).
 * Every node counts once per distinct assignment of the sliced labels under
 * it, and once per distinct restriction of the batch rows to the open legs
 * under it when outputs lists n_amps > 1 rows (NULL: one amplitude).  objective
 * 0: a node costs its FLOP (the sum is Eq. task_based_amplitude_flops);
 * 1: it costs max(FLOP / 100 TFLOP/s, 8 B x (|A| + |B| + |C|) / 4 TB/s), an
 * estimated time that weighs the HBM traffic of small-operand steps.  Every
 * sub-tree is opened down to at most 10 tensors and re-ordered optimally by
 * dynamic programming over subsets, `passes` times over the tree, and no
 * intermediate of one slice (times its batch instances) may grow above the
 * current path's largest, so the slicing stays valid.  The path is replaced
 * only when the cost falls.  cost_before / cost_after (may be NULL): the cost
 * before and after (FLOP, or seconds).
 * Errors: JET_ESTATE (no path, or a batch without declared open legs),
 * JET_EINVAL (passes outside [1, 64], objective not 0 or 1, digit out of range). */
int jet_path_reconfigure(jet_network *net, int32_t passes, int32_t objective, int32_t n_amps,
                         const int32_t *outputs, double *cost_before, double *cost_after);

/* Slice the given closed labels (Section 2.4); n = 0 clears the slicing.
 * Slice id s is the mixed-radix number over the sliced labels, the first label
 * most significant.  Errors: JET_EINVAL (open or unknown label, duplicate). */
int jet_slice(jet_network *net, int32_t n, const int64_t *labels);

/* Greedy slice finder along the current path: while an intermediate of one
 * slice exceeds max_elems, or fewer than min_n labels are sliced, slice the
 * closed label of the largest intermediate that minimises the reuse-aware FLOP
 * of Eq. task_based_amplitude_flops (ties: lower total FLOP, then smaller
 * label), at most max_n labels.  Writes the chosen labels (labels_out may be
 * NULL, else room for max_n) and their count, and applies them.
 * Errors: JET_ESTATE (no path), JET_EINVAL (cap not reachable within max_n). */
int jet_slice_auto(jet_network *net, int64_t max_elems, int32_t min_n, int32_t max_n, int32_t *n_out,
                   int64_t *labels_out);

/* Contract the network to n_amps amplitudes.  outputs holds n_amps rows of
 * n_out digits (the values of the open legs, in jet_network_set_open order).
 * amp_b = sum over slices s (increasing s, FP64) of the sliced contraction.
 * amps_out: n_amps complex128 values in HOST memory (n_amps * E with free legs,
 * see jet_network_set_free); the call copies them back and synchronises the
 * stream before returning.
 * Errors: JET_EINVAL (digit out of range, n_amps < 1), JET_ESTATE (no path),
 * JET_ENOMEM (workspace), JET_ECUDA, JET_ETIMEOUT. */
int jet_contract(jet_network *net, int32_t n_amps, const int32_t *outputs,
                 jet_c128 *amps_out, void *cuda_stream);

/* Contract only the listed slices and return each one's partial contraction
 * (the s_i of Eq. sliced_sum): partials_out[b * n_ids + j] is amplitude b's
 * network with the sliced labels fixed to the digits of slice id slice_ids[j]
 * (mixed radix, first sliced label most significant).  Intermediates shared by
 * the listed slices are computed once.  Summing the partials of every slice in
 * increasing id order gives jet_contract's amplitude; disjoint id ranges are
 * how independent processes (one per GPU) split one amplitude's work.
 * partials_out: n_amps * n_ids complex128 values of HOST memory (times E with
 * free legs, value e innermost); the call
 * synchronises the stream.  Errors as jet_contract, plus JET_EINVAL (empty list
 * or an id outside [0, number of slices)). */
int jet_contract_slices(jet_network *net, int32_t n_amps, const int32_t *outputs, int32_t n_ids,
                        const int64_t *slice_ids, jet_c128 *partials_out, void *cuda_stream);

/* Same as jet_contract but amps_dev is DEVICE memory (n_amps complex128, times
 * E with free legs; when workspace_limit splits the slices into ranges the call
 * synchronises) and
 * the call returns without synchronising: the amplitudes are ready when work
 * issued on cuda_stream before the next call completes. */
int jet_contract_async(jet_network *net, int32_t n_amps, const int32_t *outputs,
                       jet_c128 *amps_dev, void *cuda_stream);

/* The cross-slice reduction of Eq. sliced_sum on the host: sums_out[b * n_elem
 * + e] = sum over j = 0, 1, ..., n_ids - 1, in that order, in FP64, of
 * partials[(b * n_ids + j) * n_elem + e].  Partials gathered from processes
 * that each contracted a slice-id range (jet_contract_slices), concatenated in
 * increasing slice id, sum in the order of a single jet_contract, so the result
 * does not depend on how the slices were split.  HOST buffers; n_ids = 0 gives
 * zeros.  Errors: JET_EINVAL (negative sizes, n_elem < 1, NULL buffers). */
int jet_sum_partials(int32_t n_amps, int64_t n_ids, int64_t n_elem, const jet_c128 *partials, jet_c128 *sums_out);

/* Device workspace.  jet_plan prepares the plan for this batch of outputs and
 * reports the bytes of device workspace it needs.  jet_set_workspace hands the
 * library caller-owned device memory (at least that many bytes, 256-byte
 * aligned) to use instead of allocating its own; NULL releases it.  The caller
 * keeps the memory alive until the handle is destroyed or another workspace is
 * set.  Without a workspace the library allocates one itself. */
int jet_plan(jet_network *net, int32_t n_amps, const int32_t *outputs, size_t *bytes_out);
/* jet_plan for the plan jet_contract_slices runs with the same arguments (only
 * the listed slice ids, their shared intermediates computed once): builds and
 * keeps it, and writes the workspace bytes it needs.  Errors as
 * jet_contract_slices. */
int jet_plan_slices(jet_network *net, int32_t n_amps, const int32_t *outputs, int32_t n_ids,
                    const int64_t *slice_ids, size_t *bytes_out);
int jet_set_workspace(jet_network *net, void *dptr, size_t bytes);

/* Slice ranges for a workspace cap (Section 4: when the shared work of every
 * slice does not fit, a subset of the slices is held in memory at a time, its
 * size determined a priori).  A range fixes the digits of a set of the sliced
 * labels and holds every slice with those digits, so an intermediate with one
 * of those labels under it is still computed once in all, and one without is
 * computed again in each range.  The library takes, among the sets of the
 * fewest labels whose range plan fits max_bytes, the one that minimises the
 * FLOP of all ranges together.  jet_contract / jet_contract_async use the same
 * choice whenever the plan of every slice exceeds their cap
 * (jet_options.workspace_limit, a smaller caller workspace, or, with neither,
 * 90% of the free device memory): they run the ranges one after the other,
 * each range's plan kept (and replayed as its CUDA graph) for later calls with
 * the same outputs, and sum the per-slice partials in increasing slice id in
 * FP64.  This call plans (host only) and reports: the number of labels a range
 * fixes and those labels (fixed_labels_out: room for every sliced label, may
 * be NULL), the number of ranges, the FLOP of all ranges together and the
 * workspace bytes of one range; a plan that fits max_bytes reports 0 labels, 1
 * range and its own FLOP and size.  Any output pointer may be NULL.
 * Errors: as jet_plan, JET_EINVAL (max_bytes 0), JET_ENOMEM (one slice does
 * not fit). */
int jet_plan_ranges(jet_network *net, int32_t n_amps, const int32_t *outputs, size_t max_bytes,
                    int32_t *n_fixed_out, int64_t *fixed_labels_out, int64_t *n_ranges_out, double *flop_out,
                    size_t *bytes_out);

/* Adjoint (environment) contraction; not in the paper.
 * env_G = sum_b cot_b * d amp_b / d G for each requested input tensor G
 * (holomorphic: G is not conjugated; env_G has G's shape and layout).
 * For loss = sum_b |amp_b|^2 pass cot_b = conj(amp_b); then
 * d loss / d theta = 2 Re sum_G <env_G, dG/dtheta>, <X,Y> = sum_i X_i Y_i.
 * Slice by slice the forward tree is recomputed (intermediates shared by the
 * amplitudes of the batch are computed once; nothing is kept across slices),
 * then swept backwards: for C = sum_K A B, env(A) = env(C) contracted with B
 * over B's free labels.  Environments accumulate over slices in FP64.
 * env_out[i] points to prod(dims) complex64 values of HOST memory for tensor
 * tensor_ids[i]; amps_out (may be NULL) receives the amplitudes.  Synchronises
 * cuda_stream before returning.  An unsliced network keeps its adjoint plan
 * (replayed as a CUDA graph): a later call with the same outputs and tensor ids
 * only rewrites the cotangent seed; a sliced network plans and runs its slices
 * one after the other.
 * Errors as jet_contract, plus JET_EINVAL (bad or repeated tensor id,
 * a network of one tensor, free output legs). */
int jet_contract_grad(jet_network *net, int32_t n_amps, const int32_t *outputs,
                      const jet_c128 *cot, int32_t n_req, const int32_t *tensor_ids,
                      jet_c64 *const *env_out, jet_c128 *amps_out, void *cuda_stream);

/* The launches of the plan run last (a contraction, a slice subset or an
 * unsliced adjoint; otherwise the current forward plan) in issue order, with
 * the device time of each timed launch in that run (jet_options.profile).
 * Waits for that run to finish.  Writes min(cap, count) records and the count.
 * Errors: JET_ESTATE (no plan yet). */
int jet_profile(const jet_network *net, jet_op_record *out, int32_t cap, int32_t *n_out);

/* One device-workspace allocation of a plan, for jet_plan_buffers.  Times
 * count launches in issue order: an allocation made with t launches issued is
 * first usable by launch t, and a release made with t launches issued frees
 * the bytes for launches t and later. */
typedef struct {
    int32_t node;             /* tree node (SSA id) whose instances it holds; -1 = scratch
                                 of one node's launches (split-K partials, operand planes) */
    int32_t t_alloc;          /* launches issued when it was allocated                   */
    int32_t t_release;        /* launches issued when it was released; -1 = never (held
                                 to the end, e.g. by an adjoint sweep)                    */
    int32_t first_use;        /* node buffers: first launch of the node (it writes them)  */
    int32_t last_use;         /* node buffers: last launch of the node or of its parent
                                 (the reader); -1 for scratch                             */
    int32_t pad_;
    int64_t offset;           /* byte offset in the workspace                           */
    int64_t bytes;            /* bytes (rounded up to 256)                               */
} jet_buffer_record;

/* Intermediate deletion (Section 4: an intermediate is deleted once every
 * task that reads it has run): the liveness record of the device workspace of
 * the plan run last (else the current forward plan), one record per
 * allocation in allocation order.  A correct plan releases a node's buffer
 * only after its last reader was issued (last_use < t_release), and never
 * gives overlapping bytes to two allocations whose [t_alloc, t_release)
 * windows meet.  Host only; writes min(cap, count) records and the count.
 * Errors: JET_ESTATE (no plan yet), JET_EINVAL (net NULL). */
int jet_plan_buffers(const jet_network *net, jet_buffer_record *out, int32_t cap, int32_t *n_out);

/* Statistics of the network and the last plan (see jet_stats_t). */
int jet_stats(const jet_network *net, jet_stats_t *out);

/* Autotuner (not in the paper): for the contraction of these outputs, choose
 * per tree node between the kernel forms that both take the node's shape --
 * the GEMM route's instance blocks or one product per instance, a small
 * operand's tensor-core application or its CUDA-core form, and a GEMM whose
 * parent is a dot product forming those products in its epilogue or writing
 * its output (timed together with the parent) -- by timing them on the
 * device.  Two timed runs (each the second of two, CUDA events around every
 * launch): every tunable node in its default form, then every one in its
 * other form; a node takes the other form where that ran at least 3% faster,
 * and the choices are kept only if a third run of the whole plan is not slower
 * than the defaults by more than 2%.  A contraction that runs in slice ranges
 * is tuned on its first range (every range has the same launches).  The
 * choices hold for the current path and slicing (any contraction plans with
 * them from then on) and are stored in cache_file (HOST path, may be NULL; one
 * "signature choice" line per node shape: precision, form kind and the node's
 * extents and instance counts), which a later call reads first: when every
 * tunable node's shape is there, no alternative is timed.  default_ms /
 * tuned_ms (may be NULL): device time of the default and the tuned plan;
 * n_changed: nodes that left their default form.  Synchronises cuda_stream.
 * Errors: as jet_contract. */
int jet_autotune(jet_network *net, int32_t n_amps, const int32_t *outputs, const char *cache_file,
                 void *cuda_stream, double *default_ms, double *tuned_ms, int32_t *n_changed);

/* Self-test of the bounded device-side waits (the tensor-core kernels give up
 * a wait after ~2 s, record it in the network's status word, release their
 * tensor memory and return; a contraction then fails with JET_ETIMEOUT).  One
 * CTA on the network's device, on cuda_stream, allocates tensor memory, waits
 * with the same bounded-wait helper on an mbarrier that nothing arrives on,
 * gives up after limit_us microseconds, records the time-out, then waits at
 * the chained small levels' grid barrier for a block that does not exist and
 * gives up likewise, frees the tensor memory and returns; the call reads and
 * clears the status word.  Nothing is
 * left in flight and the handle stays usable.  Returns JET_ETIMEOUT (the
 * expected outcome: the wait ran out and was reported), JET_ECUDA if the wait
 * did not run out or the launch failed, JET_EINVAL (limit_us outside
 * [1, 10^7]).  Synchronises cuda_stream.  Not in the paper. */
int jet_selftest_wait(jet_network *net, int64_t limit_us, void *cuda_stream);

/* Pairwise contraction of two dense tensors that allocates no device memory.
 * The paper has no counterpart; it serves callers that cannot call cudaMalloc:
 * a process whose GPU memory is pre-reserved by its own allocator (an
 * allocation behind that allocator's back can fail or fragment its pool), or a
 * latency-critical loop where cudaMalloc / cudaFree would add implicit device
 * synchronisation.  a_dev and b_dev are row-major complex64 tensors in DEVICE
 * memory (labels[0] slowest); labels shared by the two tensors are summed;
 * c_dev (DEVICE, caller-allocated) receives the result with A's unshared labels
 * in A's order followed by B's unshared labels in B's order, row-major.
 * Scratch (split-K partial sums and offset tables) lives in one fixed 16 MiB
 * device array inside the library, held by every GPU that loads the library
 * until the process exits; the output may have at most 524280 elements
 * (larger outputs are rejected with JET_EINVAL), each tensor fewer than 2^31
 * elements, at most 40 labels each (labels of dim 1 are accepted and ignored).
 * The offset tables are written into the scratch by a small kernel on
 * cuda_stream (three launches per call, no host-to-device copy).  A CUDA error
 * already pending on the calling thread is reported as JET_ECUDA and left
 * pending.  The first call on a device looks up that
 * array's device address (cudaGetSymbolAddress); make that first call before
 * any stream capture on the device.  Every call shares the array: calls that
 * overlap on the GPU (different streams, or different host threads) race, so
 * order them on one stream.  Runs asynchronously on cuda_stream on `device`.
 * Errors: JET_EINVAL (NULL pointer, bad rank/dim, repeated label, size limit),
 * JET_ECUDA. */
int jet_pair_contract_noalloc(int32_t rank_a, const int64_t *labels_a, const int32_t *dims_a,
                              const jet_c64 *a_dev, int32_t rank_b, const int64_t *labels_b,
                              const int32_t *dims_b, const jet_c64 *b_dev, jet_c64 *c_dev,
                              int32_t device, void *cuda_stream);

/* Release the handle and every device buffer the library allocated. */
void jet_network_destroy(jet_network *net);

/* Thread-local description of the last error on this thread ("" if none). */
const char *jet_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* JET_B300_H */
