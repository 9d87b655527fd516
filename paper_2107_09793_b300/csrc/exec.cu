// Executor: binds a plan to its device buffers (leaves, arena, amplitudes),
// issues its launches in tree order on the caller's stream, and records the
// whole launch sequence once into a CUDA graph that later calls replay.
#include <cuda_runtime.h>

#include <cstring>
#include <string>

#include "internal.h"
#include "kernel_args.h"
#include "kernels.cuh"

namespace jet {

#define JET_CUDA(call)                                                                          \
    do {                                                                                        \
        cudaError_t e_ = (call);                                                                \
        if (e_ != cudaSuccess) fail(JET_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

void *device_alloc(size_t bytes)
{
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, std::max<size_t>(bytes, 256));
    if (e != cudaSuccess) {
        cudaGetLastError();
        fail(e == cudaErrorMemoryAllocation ? JET_ENOMEM : JET_ECUDA,
             std::string("cudaMalloc(") + std::to_string(bytes) + "): " + cudaGetErrorString(e));
    }
    return p;
}

void device_free(void *p)
{
    if (p) cudaFree(p);
}

static void set_device(const Network &net) { JET_CUDA(cudaSetDevice(net.opt.device)); }

static bool g_smem_set[64] = {false};

static void init_device_once(const Network &net)
{
    int dev = net.opt.device;
    if (dev >= 0 && dev < 64 && !g_smem_set[dev]) {
        JET_CUDA(set_direct_smem_limits());
        JET_CUDA(set_tc_smem_limits());
        JET_CUDA(set_apply_tc_smem_limits());
        g_smem_set[dev] = true;
    }
}

void ensure_leaves_on_device(Network &net)
{
    set_device(net);
    init_device_once(net);
    if (!net.stream) {
        cudaStream_t s;
        JET_CUDA(cudaStreamCreate(&s));
        net.stream = s;
    }
    if (!net.d_status) {
        net.d_status = device_alloc(256);
        JET_CUDA(cudaMemset(net.d_status, 0, 256));
    }
    if (!net.d_leaves) {
        net.d_leaves = device_alloc((size_t)net.n_values * sizeof(jet_c64));
        JET_CUDA(cudaMemcpy(net.d_leaves, net.host_values.data(), (size_t)net.n_values * sizeof(jet_c64),
                            cudaMemcpyHostToDevice));
        net.leaves64_stale = true;
    }
    if (net.opt.precision == JET_PREC_FP64) {
        if (!net.d_leaves64) {
            net.d_leaves64 = device_alloc((size_t)net.n_values * sizeof(jet_c128));
            net.leaves64_stale = true;
        }
        if (net.leaves64_stale) {
            JET_CUDA(launch_c64_to_c128(net.d_leaves, net.d_leaves64, net.n_values, (cudaStream_t)net.stream));
            JET_CUDA(cudaStreamSynchronize((cudaStream_t)net.stream));
            net.leaves64_stale = false;
        }
    }
}

void upload_leaf(Network &net, int32_t tensor_id, void *)
{
    if (!net.d_leaves) return;  // uploaded in full on first use
    set_device(net);
    const Leaf &L = net.leaves[tensor_id];
    JET_CUDA(cudaMemcpy((jet_c64 *)net.d_leaves + L.offset, net.host_values.data() + L.offset,
                        (size_t)L.size * sizeof(jet_c64), cudaMemcpyHostToDevice));
    net.leaves64_stale = true;
}

void upload_all(Network &net, const jet_c64 *data, void *stream)
{
    ensure_leaves_on_device(net);
    cudaStream_t s = (cudaStream_t)stream;
    JET_CUDA(cudaMemcpyAsync(net.d_leaves, data, (size_t)net.n_values * sizeof(jet_c64), cudaMemcpyHostToDevice, s));
    if (net.opt.precision == JET_PREC_FP64) {
        JET_CUDA(launch_c64_to_c128(net.d_leaves, net.d_leaves64, net.n_values, s));
        net.leaves64_stale = false;
    } else {
        net.leaves64_stale = true;
    }
}

void copy_d2h(void *dst, const void *src, size_t bytes, void *stream)
{
    JET_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, (cudaStream_t)stream));
    JET_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
}

void device_memset_async(void *dst, size_t bytes, void *stream)
{
    JET_CUDA(cudaMemsetAsync(dst, 0, bytes, (cudaStream_t)stream));
}

void copy_d2d_async(void *dst, const void *src, size_t bytes, void *stream)
{
    JET_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
}

void sync_stream(Network &net, void *stream)
{
    if (stream || net.stream) JET_CUDA(cudaStreamSynchronize((cudaStream_t)(stream ? stream : net.stream)));
}

void copy_h2d_sync(void *dst, const void *src, size_t bytes, void *stream)
{
    JET_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, (cudaStream_t)stream));
    JET_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
}

bool gemm_available(int32_t) { return true; }

int read_clear_status(Network &net, void *stream)
{
    if (!net.d_status) return 0;
    uint32_t st = 0;
    cudaStream_t s = stream ? (cudaStream_t)stream : (cudaStream_t)net.stream;
    JET_CUDA(cudaMemcpyAsync(&st, net.d_status, 4, cudaMemcpyDeviceToHost, s));
    JET_CUDA(cudaStreamSynchronize(s));
    if (st) JET_CUDA(cudaMemsetAsync(net.d_status, 0, 4, s));
    return (int)st;
}

static void destroy_events(Plan &plan)
{
    for (void *e : plan.ev_begin)
        if (e) cudaEventDestroy((cudaEvent_t)e);
    for (void *e : plan.ev_end)
        if (e) cudaEventDestroy((cudaEvent_t)e);
    plan.ev_begin.clear();
    plan.ev_end.clear();
    plan.profile_level = 0;
}

float op_elapsed_ms(const Plan &plan, size_t i)
{
    if (i >= plan.ev_begin.size() || !plan.ev_begin[i]) return -1.f;
    if (cudaEventSynchronize((cudaEvent_t)plan.ev_end[i]) != cudaSuccess) return -1.f;
    float ms = -1.f;
    if (cudaEventElapsedTime(&ms, (cudaEvent_t)plan.ev_begin[i], (cudaEvent_t)plan.ev_end[i]) != cudaSuccess) {
        cudaGetLastError();
        return -1.f;
    }
    return ms;
}

void release_plan_device(Plan &plan)
{
    destroy_events(plan);
    if (plan.graph_exec) cudaGraphExecDestroy((cudaGraphExec_t)plan.graph_exec);
    plan.graph_exec = nullptr;
    device_free(plan.d_args);
    plan.d_args = nullptr;
    plan.d_args_bytes = 0;
}

size_t device_free_bytes(Network &net)
{
    int prev = 0;
    JET_CUDA(cudaGetDevice(&prev));
    JET_CUDA(cudaSetDevice(net.opt.device));
    size_t fr = 0, tot = 0;
    const cudaError_t e = cudaMemGetInfo(&fr, &tot);
    cudaSetDevice(prev);
    JET_CUDA(e);
    return fr;
}

void ensure_workspace(Network &net, size_t bytes, void *stream)
{
    if (net.user_arena || net.own_arena_bytes >= bytes) return;
    cudaStream_t s = stream ? (cudaStream_t)stream : (cudaStream_t)net.stream;
    JET_CUDA(cudaStreamSynchronize(s));
    device_free(net.own_arena);
    net.own_arena = nullptr;
    net.own_arena_bytes = 0;
    net.own_arena = device_alloc(bytes);
    net.own_arena_bytes = bytes;
}

void free_network_device(Network &net)
{
    if (net.plan) release_plan_device(*net.plan);
    if (net.ranges)
        for (auto &p : net.ranges->plans)
            if (p) release_plan_device(*p);
    if (net.grad_plan) release_plan_device(*net.grad_plan);
    net.last_run = nullptr;
    device_free(net.d_leaves);
    device_free(net.d_leaves64);
    device_free(net.own_arena);
    device_free(net.d_amps);
    device_free(net.d_status);
    net.d_status = nullptr;
    device_free(net.d_env);
    net.d_env = nullptr;
    net.d_env_cap = 0;
    device_free(net.d_kept);
    net.d_kept = nullptr;
    net.d_kept_bytes = 0;
    if (net.stream) cudaStreamDestroy((cudaStream_t)net.stream);
    net.d_leaves = net.d_leaves64 = net.own_arena = net.d_amps = nullptr;
    net.stream = nullptr;
}

static void launch_op(const Plan &P, const std::vector<uint8_t> &args, const Op &op, cudaStream_t s)
{
    LaunchCfg c{op.grid_x, op.grid_y, op.grid_z, op.block, op.smem, op.variant};
    const uint8_t *p = args.data() + op.args_off;
    cudaGetLastError();   // drop any stale error so the check below sees this launch only
    cudaError_t e = cudaSuccess;
    switch (op.kind) {
    case OpKind::Direct: {
        DirectArgs a;
        std::memcpy(&a, p, sizeof a);
        e = launch_direct(a, c, s);
        break;
    }
    case OpKind::Apply: {
        ApplyArgs a;
        std::memcpy(&a, p, sizeof a);
        e = launch_apply(a, c, s);
        break;
    }
    case OpKind::SplitKReduce: {
        SplitKReduceArgs a;
        std::memcpy(&a, p, sizeof a);
        e = launch_splitk_reduce(a, c, s);
        break;
    }
    case OpKind::SmallBatch: {
        SmallBatchArgs a;
        std::memcpy(&a, p, sizeof a);
        e = launch_small_batch(a, c, s);
        break;
    }
    case OpKind::Accum: {
        AccumArgs a;
        std::memcpy(&a, p, sizeof a);
        e = launch_accum(a, c, s);
        break;
    }
    case OpKind::AccumBatch: {
        AccumBatchArgs a;
        std::memcpy(&a, p, sizeof a);
        e = launch_accum_batch(a, c, s);
        break;
    }
    case OpKind::Memset: {
        MemsetArgs a;
        std::memcpy(&a, p, sizeof a);
        e = cudaMemsetAsync((void *)a.ptr, 0, (size_t)a.bytes, s);
        break;
    }
    case OpKind::Permute: {
        PermuteArgs a;
        std::memcpy(&a, p, sizeof a);
        e = launch_permute(a, c, s);
        break;
    }
    case OpKind::GemmSimt: {
        GemmArgs a;
        std::memcpy(&a, p, sizeof a);
        e = launch_gemm_simt(a, c, s);
        break;
    }
    case OpKind::TcSplit: {
        TcSplitArgs a;
        std::memcpy(&a, p, sizeof a);
        e = launch_tc_split(a, c, s);
        break;
    }
    case OpKind::GemmTc: {
        TcGemmArgs a;
        std::memcpy(&a, p, sizeof a);
        e = launch_tc_gemm(a, c, s);
        break;
    }
    case OpKind::Reduce: {
        ReduceArgs a;
        std::memcpy(&a, p, sizeof a);
        e = launch_slice_reduce(a, c, s);
        break;
    }
    default:
        fail(JET_EINVAL, "internal: unknown op kind");
    }
    if (e != cudaSuccess)
        fail(JET_ECUDA, std::string("kernel launch (op kind ") + std::to_string((int)op.kind) + ", node " +
                            std::to_string(op.node) + ", grid " + std::to_string(op.grid_x) + "x" +
                            std::to_string(op.grid_y) + "x" + std::to_string(op.grid_z) + ", smem " +
                            std::to_string(op.smem) + ", variant " + std::to_string(op.variant) +
                            "): " + cudaGetErrorString(e));
    (void)P;
}

void bind_and_run(Network &net, Plan &P, void *, void *stream, bool allow_graph)
{
    ensure_leaves_on_device(net);
    cudaStream_t s = stream ? (cudaStream_t)stream : (cudaStream_t)net.stream;

    // workspace
    void *arena = nullptr;
    if (net.user_arena) {
        if (net.user_arena_bytes < P.arena_bytes)
            fail(JET_ENOMEM, "workspace too small: need " + std::to_string(P.arena_bytes) + " bytes, have " +
                                 std::to_string(net.user_arena_bytes));
        arena = net.user_arena;
    } else {
        if (net.own_arena_bytes < P.arena_bytes) {
            JET_CUDA(cudaStreamSynchronize(s));
            device_free(net.own_arena);
            net.own_arena = nullptr;
            net.own_arena_bytes = 0;
            net.own_arena = device_alloc(P.arena_bytes);
            net.own_arena_bytes = P.arena_bytes;
        }
        arena = net.own_arena;
    }
    const int64_t n_out_vals = (P.partials ? (int64_t)P.n_amps * P.n_slices : P.n_amps) * P.n_elem;
    if (net.d_amps_cap < n_out_vals) {
        JET_CUDA(cudaStreamSynchronize(s));
        device_free(net.d_amps);
        net.d_amps = nullptr;
        net.d_amps = device_alloc((size_t)n_out_vals * sizeof(jet_c128));
        net.d_amps_cap = n_out_vals;
    }
    void *leaves = net.opt.precision == JET_PREC_FP64 ? net.d_leaves64 : net.d_leaves;
    // kept shared results: grow the pool, carrying over the ready ones
    if (net.d_kept_bytes < P.kept_pool_bytes) {
        JET_CUDA(cudaStreamSynchronize(s));
        void *pool = device_alloc(P.kept_pool_bytes);
        if (net.d_kept && net.d_kept_bytes) JET_CUDA(cudaMemcpy(pool, net.d_kept, net.d_kept_bytes, cudaMemcpyDeviceToDevice));
        device_free(net.d_kept);
        net.d_kept = pool;
        net.d_kept_bytes = P.kept_pool_bytes;
    }

    // (re)bind pointers
    bool rebind = P.dirty_args || P.bound_arena != arena || P.bound_leaves != leaves || P.bound_amps != net.d_amps ||
                  P.bound_env != net.d_env || P.bound_kept != net.d_kept;
    if (rebind) {
        if (P.graph_exec) {
            JET_CUDA(cudaStreamSynchronize(s));
            cudaGraphExecDestroy((cudaGraphExec_t)P.graph_exec);
            P.graph_exec = nullptr;
        }
        if (P.d_args_bytes < P.host_args.size()) {
            device_free(P.d_args);
            P.d_args = nullptr;
            P.d_args = device_alloc(P.host_args.size());
            P.d_args_bytes = P.host_args.size();
        }
        uintptr_t bases[7] = {(uintptr_t)leaves, (uintptr_t)arena, (uintptr_t)P.d_args, (uintptr_t)net.d_amps,
                              (uintptr_t)net.d_status, (uintptr_t)net.d_env, (uintptr_t)net.d_kept};
        for (const auto &pt : P.patches) {
            uint64_t v = (uint64_t)(bases[pt.base] + (uintptr_t)pt.byte_off);
            std::memcpy(P.host_args.data() + pt.at, &v, 8);
        }
        // tensor maps of the tensor-core GEMMs point into the (re)bound arena
        for (const Op &op : P.ops)
            if (op.kind == OpKind::GemmTc) {
                TcGemmArgs g;
                std::memcpy(&g, P.host_args.data() + op.args_off, sizeof g);
                int rc = encode_tc_maps(g);
                if (rc != 0) fail(JET_ECUDA, "cuTensorMapEncodeTiled failed (" + std::to_string(rc) + ")");
                std::memcpy(P.host_args.data() + op.args_off, &g, sizeof g);
            }
        JET_CUDA(cudaMemcpy(P.d_args, P.host_args.data(), P.host_args.size(), cudaMemcpyHostToDevice));
        P.bound_arena = arena;
        P.bound_leaves = leaves;
        P.bound_amps = net.d_amps;
        P.bound_env = net.d_env;
        P.bound_kept = net.d_kept;
        P.dirty_args = false;
        P.seed_dirty = false;
    } else if (P.seed_dirty) {   // new cotangents of a cached adjoint plan: only the seed bytes change
        const size_t es = net.opt.precision == JET_PREC_FP64 ? 16 : 8;
        JET_CUDA(cudaMemcpyAsync((uint8_t *)P.d_args + P.seed_off, P.host_args.data() + P.seed_off,
                                 (size_t)P.seed_n_inst * es, cudaMemcpyHostToDevice, s));
        JET_CUDA(cudaStreamSynchronize(s));   // the pageable source may change before a later call
        P.seed_dirty = false;
    }
    net.last_run = &P;

    // optional per-launch timing: event records become nodes of the captured graph
    if (P.profile_level != net.opt.profile) {
        if (P.graph_exec) {
            JET_CUDA(cudaStreamSynchronize(s));
            cudaGraphExecDestroy((cudaGraphExec_t)P.graph_exec);
            P.graph_exec = nullptr;
        }
        destroy_events(P);
        if (net.opt.profile > 0) {
            P.ev_begin.assign(P.ops.size(), nullptr);
            P.ev_end.assign(P.ops.size(), nullptr);
            for (size_t i = 0; i < P.ops.size(); ++i) {
                OpKind k = P.ops[i].kind;
                bool want = net.opt.profile >= 2 || k == OpKind::GemmTc || k == OpKind::GemmSimt ||
                            k == OpKind::Apply || k == OpKind::TcSplit;
                if (!want) continue;
                cudaEvent_t a, b;
                JET_CUDA(cudaEventCreate(&a));
                JET_CUDA(cudaEventCreate(&b));
                P.ev_begin[i] = a;
                P.ev_end[i] = b;
            }
        }
        P.profile_level = net.opt.profile;
    }
    auto issue_all = [&](cudaStream_t st, bool capturing) {
        // while capturing, external event records become real timestamp nodes of the
        // graph; issued directly, they are plain records
        auto record = [&](void *ev) {
            if (capturing) JET_CUDA(cudaEventRecordWithFlags((cudaEvent_t)ev, st, cudaEventRecordExternal));
            else JET_CUDA(cudaEventRecord((cudaEvent_t)ev, st));
        };
        for (size_t i = 0; i < P.ops.size(); ++i) {
            const bool timed = i < P.ev_begin.size() && P.ev_begin[i];
            if (timed) record(P.ev_begin[i]);
            launch_op(P, P.host_args, P.ops[i], st);
            if (timed) record(P.ev_end[i]);
        }
    };

    if (net.opt.use_graph && allow_graph) {
        if (!P.graph_exec) {
            if (P.graph_exec) {
                cudaGraphExecDestroy((cudaGraphExec_t)P.graph_exec);
                P.graph_exec = nullptr;
            }
            // capture on a private stream, then replay on the caller's
            cudaStream_t cap;
            JET_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
            cudaGraph_t g = nullptr;
            cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                try {
                    issue_all(cap, true);
                } catch (...) {
                    cudaStreamEndCapture(cap, &g);
                    if (g) cudaGraphDestroy(g);
                    cudaStreamDestroy(cap);
                    throw;
                }
                e = cudaStreamEndCapture(cap, &g);
            }
            cudaStreamDestroy(cap);
            if (e != cudaSuccess) fail(JET_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
            cudaGraphExec_t ge;
            e = cudaGraphInstantiate(&ge, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) fail(JET_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
            P.graph_exec = ge;
            P.graph_stream = (void *)s;
        }
        JET_CUDA(cudaGraphLaunch((cudaGraphExec_t)P.graph_exec, s));
    } else {
        issue_all(s, false);
    }
}

}  // namespace jet
