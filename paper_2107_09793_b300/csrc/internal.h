// Internal data structures of the library (host side).
#pragma once

#include <cstdint>
#include <map>
#include <memory>
#include <string>
#include <unordered_map>
#include <utility>
#include <vector>

#include "../../include/jet.h"

namespace jet {

// Error carrying a JET_E* code; caught at the C boundary.
struct Error {
    int code;
    std::string msg;
};
[[noreturn]] void fail(int code, const std::string &msg);
void set_last_error(const std::string &msg);

struct Leaf {
    std::vector<int64_t> labels;
    std::vector<int32_t> dims;
    int64_t size = 1;
    int64_t offset = 0;      // element offset in the packed leaf buffer
};

struct LabelInfo {
    int32_t dim = 0;
    int32_t owner[2] = {-1, -1};
    int32_t n_owner = 0;
};

// ---------------------------------------------------------------- planner
// Contraction tree derived from an SSA path (Section 2.3, binary tree).
struct Tree {
    int32_t n_leaves = 0;
    std::vector<std::pair<int32_t, int32_t>> children;   // internal node k -> (a, b), ids are SSA ids
    // per SSA id: remaining labels (fixed ones removed), in no particular order
    std::vector<std::vector<int64_t>> labels;
    int32_t root() const { return n_leaves + (int32_t)children.size() - 1; }
};

// FLOP / size model of a path with a given set of fixed labels (dim 1).
struct PathCost {
    double flop = 0;                 // sum over steps of 8 * prod(dims of the union)
    double max_size = 0;             // largest intermediate (elements)
    std::vector<double> step_flop;   // per internal node
    std::vector<double> node_size;   // per SSA id
};

// -------------------------------------------------------------- plan / ops
enum class OpKind : int32_t { Direct = 0, Permute = 1, GemmSimt = 2, GemmTc = 3, Reduce = 4, SplitKReduce = 5, TcSplit = 6, SmallBatch = 7, Accum = 8, Memset = 9, Apply = 10, AccumBatch = 11 };

struct Op {
    OpKind kind;
    int32_t node = -1;
    int64_t n_inst = 0;
    size_t args_off = 0;      // byte offset of this op's argument block in the plan's constant buffer
    size_t args_bytes = 0;
    double flop = 0;          // algorithmic real FLOP of this launch (all instances)
    double bytes = 0;         // algorithmic HBM bytes of this launch
    int32_t grid_x = 1, grid_y = 1, grid_z = 1, block = 256;
    int32_t smem = 0;
    int32_t variant = 0;      // kernel-specific variant selector
    int32_t batch_first = -1; // batched small contractions: their nodes in Plan::batch_nodes
    int32_t batch_count = 0;
};

struct Network;

// What an adjoint plan needs besides the forward plan: the cotangent of every
// amplitude and, per input tensor, where its FP64 environment accumulates
// (complex128 element offset in the environment buffer, -1 = not requested).
struct GradRequest {
    std::vector<double> cot;          // 2 * n_amps (re, im)
    std::vector<int64_t> env_off;     // per tensor id
    std::vector<int32_t> leaves;      // requested tensor ids
};

struct Plan {
    // key
    std::vector<int32_t> outputs;
    int32_t n_amps = 0;
    uint64_t path_version = 0;
    uint64_t slice_version = 0;
    int32_t precision = 0;
    int32_t reuse = 1;
    std::vector<int64_t> slice_ids;  // listed slices only (partials mode), else all
    bool partials = false;

    // sizes
    int64_t n_slices = 1;
    int64_t n_elem = 1;              // values per amplitude row (product of the free legs' dims)
    std::vector<int32_t> kept_fill;  // kept entries this plan computes (ready once it has run)
    bool superseded = false;         // its kept entries are ready: the next call plans afresh
    size_t kept_pool_bytes = 0;      // device pool the plan's kept entries need
    size_t arena_bytes = 0;          // intermediates + scratch (device workspace)
    std::vector<Op> ops;
    std::vector<int32_t> batch_nodes;  // nodes of the batched small-contraction launches
    // arena liveness record: one entry per allocation, times in launches issued
    struct BufferRec {
        int32_t node;             // tree node whose result it holds, -1 = scratch
        int64_t offset, bytes;
        int32_t t_alloc, t_release;   // launches issued before the allocation / the release (-1: never)
    };
    std::vector<BufferRec> buffers;
    std::vector<int32_t> parent;       // per tree node (SSA id), -1 for the root
    // nodes with two feasible forms the autotuner may choose between: (node,
    // kind 0 = GEMM grouping / 1 = application form, the form taken) and a
    // signature of the node's shape that keys the tuner's cache
    // (node2: a second node whose time the choice also moves, or -1)
    struct Tunable { int32_t node, kind, taken; std::string sig; int32_t node2 = -1; };
    std::vector<Tunable> tunables;
    std::vector<uint8_t> host_args;   // argument blocks (pointers patched at bind time)
    // pointer patch list: (byte offset in host_args, buffer id, element/byte offset)
    struct Patch { size_t at; int32_t base; int64_t byte_off; };
    std::vector<Patch> patches;       // base: 0 = leaf buffer, 1 = arena, 2 = args buffer itself, 3 = amps out
    size_t amps_patch_count = 0;

    // statistics
    double flop_executed = 0, bytes_executed = 0;
    int64_t n_instances = 0;
    int32_t n_gemm = 0, n_direct = 0;
    int64_t max_intermediate = 0;

    // device state (owned)
    void *d_args = nullptr;
    size_t d_args_bytes = 0;
    void *bound_arena = nullptr;
    void *bound_leaves = nullptr;
    void *bound_amps = nullptr;
    void *bound_env = nullptr;
    void *bound_kept = nullptr;

    // adjoint plans: where the root's cotangent seed sits in the argument buffer,
    // so that a cached plan takes new cotangents without being rebuilt
    bool grad = false;
    std::vector<int32_t> grad_leaves;    // requested tensor ids, in request order
    std::vector<int64_t> grad_env_off;   // their environment offsets
    size_t seed_off = 0;                 // byte offset of the seed values in host_args
    std::vector<int32_t> seed_inst;      // root instance of each (amplitude, slice) assignment
    int64_t seed_n_inst = 0, seed_n_sl = 1;
    bool seed_dirty = false;
    std::vector<void *> ev_begin, ev_end;   // per op: cudaEvent_t pair when profiled
    int32_t profile_level = 0;
    void *graph_exec = nullptr;       // cudaGraphExec_t
    void *graph_stream = nullptr;
    bool dirty_args = true;
};

// Slice ranges (Section 4: a subset of the slices held in memory at a time,
// its size determined a priori) for a workspace cap below the plan of every
// slice: a range fixes the digits of the sliced labels at `fixed_pos` and runs
// every slice with those digits, so an intermediate with one of those labels
// under it is computed once in all, and one without once per range.  The
// labels are chosen to minimise the FLOP of all ranges together; each range's
// plan is kept (and replayed as its CUDA graph) while the key holds.
struct RangeSet {
    // key
    std::vector<int32_t> outputs;
    int32_t n_amps = 0;
    uint64_t path_version = 0, slice_version = 0;
    int32_t precision = 0, reuse = 1;
    size_t cap = 0;
    // partition
    std::vector<int32_t> fixed_pos;            // positions in Network::sliced
    std::vector<std::vector<int64_t>> ids;     // slice ids of each range, increasing
    double flop = 0;                           // FLOP of all ranges together
    size_t arena = 0;                          // workspace of one range
    std::vector<std::unique_ptr<Plan>> plans;  // per range, built on first use
};

// Route choice of the autotuner for one tree node; -1 leaves the planner's own.
struct TuneChoice {
    int8_t group = -1;      // GEMM route: instance blocks (1) or one product per instance (0)
    int8_t apply_tc = -1;   // small-operand application: tensor-core form (1) or CUDA-core form (0)
    int8_t dot = -1;        // a GEMM whose parent is a dot product: dot epilogue (1) or its output (0)
};

struct Network {
    jet_options opt;
    std::vector<Leaf> leaves;
    std::unordered_map<int64_t, LabelInfo> labels;
    std::vector<int64_t> open;        // declared output legs (order = pattern digit order)
    bool open_set = false;
    std::vector<int64_t> free_open;   // open legs left unfixed: every value of them per row
                                      // (order = digit order of the values, first slowest)
    // kept shared work: results of sub-trees without fixed labels, kept on the
    // device across contractions while `kept_key` (path, slicing, tensors, legs) holds
    struct KeptEntry {
        size_t off = 0, bytes = 0;
        bool ready = false;
    };
    int64_t keep_min = 0;             // keep such results of at least this many elements; 0: off
    uint64_t tensors_version = 0;     // bumped by every tensor update
    std::unordered_map<int32_t, KeptEntry> kept;   // tree node -> its result in d_kept
    std::vector<int64_t> kept_key;
    void *d_kept = nullptr;
    size_t d_kept_bytes = 0;
    std::vector<std::pair<int32_t, int32_t>> path;
    uint64_t path_version = 0;
    std::vector<int64_t> sliced;
    uint64_t slice_version = 0;

    int64_t n_values = 0;            // total complex values of all leaves
    std::vector<jet_c64> host_values;
    void *d_leaves = nullptr;        // complex64, packed
    void *d_leaves64 = nullptr;      // complex128 copy for the FP64 path (lazy)
    bool leaves64_stale = true;
    void *stream = nullptr;          // library-internal stream for uploads

    std::unique_ptr<Plan> plan;
    std::unique_ptr<RangeSet> ranges;    // slice ranges under a workspace cap
    // autotuned route choices, valid for the path and slicing they were tuned on
    std::unordered_map<int32_t, TuneChoice> tune;
    uint64_t tune_path_version = 0, tune_slice_version = 0;
    int32_t tune_flip = 0;               // while tuning: every tunable node takes its other choice
    std::unique_ptr<Plan> grad_plan;     // cached adjoint plan (unsliced networks)
    const Plan *last_run = nullptr;      // the plan jet_profile reports
    void *own_arena = nullptr;
    size_t own_arena_bytes = 0;
    void *user_arena = nullptr;
    size_t user_arena_bytes = 0;
    void *d_amps = nullptr;          // device amplitude buffer (complex128)
    void *d_status = nullptr;        // device status word (bounded-wait time-outs)
    void *d_env = nullptr;           // complex128 environments of requested tensors (adjoint)
    int64_t d_env_cap = 0;
    int64_t d_amps_cap = 0;

    // planner results
    double flop_planned = 0;
};

// planner.cpp
Tree build_tree(const Network &net, const std::vector<std::pair<int32_t, int32_t>> &path);
PathCost path_cost(const Network &net, const std::vector<std::pair<int32_t, int32_t>> &path,
                   const std::vector<int64_t> &fixed);
// outputs != NULL selects the batch planner: every node is costed once per
// distinct restriction of the outputs (n_amps x n_open digits) to the open legs
// under it, linear passes join the pairwise ones, and paths whose largest
// instance-weighted intermediate exceeds max_elems (> 0) lose to those under it.
std::vector<std::pair<int32_t, int32_t>> greedy_path(const Network &net, uint64_t seed, int32_t n_trials,
                                                     double *flop_out, int32_t n_amps = 1,
                                                     const int32_t *outputs = nullptr, double max_elems = 0);
std::vector<int64_t> slice_auto(const Network &net, int64_t max_elems, int32_t min_n, int32_t max_n);
std::vector<std::pair<int32_t, int32_t>> reconfigure_sliced(const Network &net, int32_t passes, int32_t n_amps,
                                                            const int32_t *outputs, double *before, double *after,
                                                            bool time_model);
double reuse_aware_flop(const Network &net, const std::vector<std::pair<int32_t, int32_t>> &path,
                        const std::vector<int64_t> &sliced);
void validate_path(const Network &net, const std::vector<std::pair<int32_t, int32_t>> &path);

// plan.cpp
std::unique_ptr<Plan> build_plan(Network &net, int32_t n_amps, const int32_t *outputs,
                                 const std::vector<int64_t> *slice_ids = nullptr,
                                 const GradRequest *grad = nullptr);

// exec.cu
void ensure_leaves_on_device(Network &net);
void bind_and_run(Network &net, Plan &plan, void *amps_dev, void *stream, bool allow_graph = true);
void release_plan_device(Plan &plan);
void free_network_device(Network &net);
void upload_leaf(Network &net, int32_t tensor_id, void *stream);
void upload_all(Network &net, const jet_c64 *data, void *stream);
void *device_alloc(size_t bytes);
size_t device_free_bytes(Network &net);         // free device memory on the network's device
void ensure_workspace(Network &net, size_t bytes, void *stream);   // grow the library's own arena
void device_free(void *p);
void sync_stream(Network &net, void *stream);   // the given stream, or the library's own when NULL
void copy_d2h(void *dst, const void *src, size_t bytes, void *stream);
void copy_d2d_async(void *dst, const void *src, size_t bytes, void *stream);
void copy_h2d_sync(void *dst, const void *src, size_t bytes, void *stream);
void device_memset_async(void *dst, size_t bytes, void *stream);
bool gemm_available(int32_t precision);
int read_clear_status(Network &net, void *stream);
float op_elapsed_ms(const Plan &plan, size_t i);

// selftest.cu: the bounded-wait self-test; returns the status word it left (and clears it)
int selftest_wait(Network &net, int64_t limit_us, void *stream);

// noalloc.cu
void pair_contract_noalloc(int32_t rank_a, const int64_t *labels_a, const int32_t *dims_a, const void *a_dev,
                           int32_t rank_b, const int64_t *labels_b, const int32_t *dims_b, const void *b_dev,
                           void *c_dev, int32_t device, void *stream);

}  // namespace jet
