// Plan compiler: turns (network, path, sliced labels, batch of output patterns)
// into a fixed list of kernel launches over a liveness-planned device arena.
//
// Reuse DAG (Section 3.2): an assignment alpha = (amplitude b, slice s) gives a
// value to every fixed label (open legs take the pattern's digits, sliced
// labels the slice id's digits, Section 2.4).  A tree node's result depends
// only on the fixed labels under it, so its distinct instances are the
// distinct restrictions of alpha to those labels - the paper's task naming
// "<path step> + <indices> + <slice values>" made into integer keys.  Each
// instance is computed once (reuse on) and read by every alpha that needs it.
// With reuse off every alpha gets its own copy of every internal node (the
// no-shared-work baseline of Section 4).
//
// Intermediate deletion (Section 4, peak memory): a node's buffer lives from
// its own launch until its parent's launch has been issued; offsets come from
// a best-fit allocator simulated in launch order, so the arena size is the
// peak of live intermediates.
#include <algorithm>
#include <map>
#include <cstring>
#include <numeric>
#include <unordered_map>

#include "internal.h"
#include "kernel_args.h"
#include "tc_args.h"

namespace jet {

namespace {

enum Base : int32_t {
    BASE_LEAVES = 0, BASE_ARENA = 1, BASE_BLOB = 2, BASE_AMPS = 3, BASE_STATUS = 4, BASE_ENV = 5, BASE_KEPT = 6
};

struct View {
    std::vector<int64_t> labels;   // layout order, slowest first
    std::vector<int64_t> strides;  // elements
    std::vector<int64_t> dims;
    int64_t size = 1;
};

struct NodeInfo {
    View view;
    int64_t n_inst = 0;
    std::vector<int64_t> inst_off;   // element offset of each instance from its base
    int32_t base = BASE_ARENA;
    int64_t buf_off = 0;             // arena byte offset of instance 0 (internal nodes)
    std::vector<int32_t> ia, ib;     // child instances of each instance (internal nodes)
    int32_t a = -1, b = -1;          // children (internal nodes)
    std::vector<int64_t> K, fa, fb;  // summed labels, free labels of a, free labels of b
    bool use_gemm = false, a_big = false, small = false;
    bool a_is_m = true;              // GEMM route: child a is the M operand
    std::vector<int64_t> fM, fN;     // GEMM route: output = fM ++ fN, in these orders
    int32_t depth = 0;               // tree level (leaves 0)
    // FP16X3 fused split (pass 1: candidate; pass 2: fz_ok once its parent's
    // planes layout is known): this GEMM's epilogue writes its parent GEMM's
    // operand planes; fz_mk / fz_nk are the parent's summed labels among fM / fN
    // (the lowest labels of each), fz_kappa the parent's summed-label order
    bool fuse = false, fz_ok = false;
    std::vector<int64_t> fz_mk, fz_nk, fz_kappa;
    size_t alloc_bytes = 0;          // arena bytes of buf_off (0: n_inst view.size elements)
    size_t fz_scales_off = 0;        // fz_ok: arena offset of the scales (the planes at buf_off)
    // dot epilogue (pass 1: candidate; pass 2: dot_ok): the parent is a full dot
    // product of this GEMM's output with its sibling; this node's epilogue adds
    // each tile's part of the parent's products into partials at buf_off
    // ([parent instance][dot_tiles] complex128), the parent only sums them
    bool dot = false, dot_ok = false;
    int32_t dot_tiles = 0;
};

struct Blob {
    std::vector<uint8_t> bytes;
    std::vector<Plan::Patch> patches;
    size_t reserve(size_t n, size_t align = 16)
    {
        size_t off = (bytes.size() + align - 1) / align * align;
        bytes.resize(off + n, 0);
        return off;
    }
    size_t put_i32(const std::vector<int32_t> &v)
    {
        size_t off = reserve(std::max<size_t>(v.size(), 1) * 4);
        if (!v.empty()) std::memcpy(bytes.data() + off, v.data(), v.size() * 4);
        return off;
    }
    size_t put_ptrs(const std::vector<std::pair<int32_t, int64_t>> &refs)
    {
        size_t off = reserve(std::max<size_t>(refs.size(), 1) * 8);
        for (size_t i = 0; i < refs.size(); ++i) patches.push_back({off + 8 * i, refs[i].first, refs[i].second});
        return off;
    }
    void patch_field(size_t struct_off, size_t field_off, int32_t base, int64_t byte_off)
    {
        patches.push_back({struct_off + field_off, base, byte_off});
    }
};

// Best-fit allocator over a linear arena, 256-byte granules.  Every allocation
// is logged with the launch count at the time it was made and released (the
// plan's liveness record, read back by jet_plan_buffers).
struct Arena {
    std::map<size_t, size_t> free_;   // offset -> size
    size_t top = 0, peak = 0;
    const std::vector<Op> *clock = nullptr;
    std::vector<Plan::BufferRec> log;
    static size_t round(size_t b) { return (b + 255) / 256 * 256; }
    int32_t now() const { return clock ? (int32_t)clock->size() : 0; }
    size_t alloc(size_t bytes)
    {
        const size_t off = alloc_(bytes);
        log.push_back({-1, (int64_t)off, (int64_t)round(std::max<size_t>(bytes, 1)), now(), -1});
        return off;
    }
    size_t alloc_(size_t bytes)
    {
        bytes = round(std::max<size_t>(bytes, 1));
        auto best = free_.end();
        for (auto it = free_.begin(); it != free_.end(); ++it)
            if (it->second >= bytes && (best == free_.end() || it->second < best->second)) best = it;
        if (best != free_.end()) {
            size_t off = best->first, sz = best->second;
            free_.erase(best);
            if (sz > bytes) free_[off + bytes] = sz - bytes;
            return off;
        }
        size_t off = top;
        top += bytes;
        peak = std::max(peak, top);
        return off;
    }
    void release(size_t off, size_t bytes)
    {
        for (auto r = log.rbegin(); r != log.rend(); ++r)
            if (r->offset == (int64_t)off && r->t_release < 0) {
                r->t_release = now();
                break;
            }
        bytes = round(std::max<size_t>(bytes, 1));
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
                it = pv;
            }
        }
        if (it->first + it->second == top) {
            top = it->first;
            free_.erase(it);
        }
    }
};

int64_t prod(const std::vector<int64_t> &d, size_t from = 0, size_t to = SIZE_MAX)
{
    int64_t p = 1;
    for (size_t i = from; i < std::min(to, d.size()); ++i) p *= d[i];
    return p;
}

View dense_view(const std::vector<int64_t> &labels, const Network &net)
{
    View v;
    v.labels = labels;
    for (int64_t l : labels) v.dims.push_back(net.labels.at(l).dim);
    v.strides.assign(labels.size(), 1);
    for (int i = (int)labels.size() - 2; i >= 0; --i) v.strides[i] = v.strides[i + 1] * v.dims[i + 1];
    v.size = prod(v.dims);
    return v;
}

int find_pos(const std::vector<int64_t> &v, int64_t x)
{
    auto it = std::find(v.begin(), v.end(), x);
    return it == v.end() ? -1 : (int)(it - v.begin());
}

// Blocks of a GEMM node's instances.  Instance i pairs M-side child instance
// mi[i] with N-side child instance ni[i].  Grouping by one side: the instances
// of that side that pair with the same set of the other side's instances form
// one group, that set another, and the two make a block whose product covers
// each of those pairs once; blocks of equal shape run as one launch of wider
// products (a shared operand instance is read once per tile row or column
// instead of once per pair, and short sides fill the tiles).
struct GemmGroups {
    std::vector<std::vector<int32_t>> gM, gN;   // child instances of each group
    std::vector<int32_t> bM, bN;                // per block: its M group and N group
    std::vector<int32_t> itab;                  // per block: [j][l] -> node instance
    int32_t nA = 1, nB = 1;                     // instances per M group, per N group
    int64_t dup = 0;                            // child instances split into more than one group
};

bool group_instances(const std::vector<int32_t> &mi, const std::vector<int32_t> &ni, bool by_m, GemmGroups &G)
{
    const std::vector<int32_t> &p = by_m ? mi : ni, &q = by_m ? ni : mi;
    std::map<int32_t, std::vector<std::pair<int32_t, int32_t>>> byp;   // p instance -> (q instance, node instance)
    for (size_t i = 0; i < p.size(); ++i) byp[p[i]].push_back({q[i], (int32_t)i});
    std::map<std::vector<int32_t>, int32_t> block_of;
    std::vector<std::vector<int32_t>> bp, bq;
    std::vector<std::vector<std::vector<int32_t>>> binst;   // block -> [j] -> node instance per l
    for (auto &kv : byp) {
        auto &lst = kv.second;
        std::sort(lst.begin(), lst.end());
        std::vector<int32_t> key;
        for (auto &x : lst) key.push_back(x.first);
        if (std::adjacent_find(key.begin(), key.end()) != key.end()) return false;   // a repeated pair
        auto it = block_of.find(key);
        if (it == block_of.end()) {
            it = block_of.emplace(key, (int32_t)bp.size()).first;
            bp.emplace_back();
            bq.push_back(key);
            binst.emplace_back();
        }
        bp[it->second].push_back(kv.first);
        std::vector<int32_t> row;
        for (auto &x : lst) row.push_back(x.second);
        binst[it->second].push_back(row);
    }
    const size_t np = bp[0].size(), nq = bq[0].size();
    for (size_t b = 0; b < bp.size(); ++b)
        if (bp[b].size() != np || bq[b].size() != nq) return false;
    G = GemmGroups();
    std::map<int32_t, int> seen_q;
    for (auto &k : bq)
        for (int32_t x : k) ++seen_q[x];
    for (auto &kv : seen_q) G.dup += kv.second - 1;
    for (size_t b = 0; b < bp.size(); ++b) {
        (by_m ? G.gM : G.gN).push_back(bp[b]);
        (by_m ? G.gN : G.gM).push_back(bq[b]);
        G.bM.push_back((int32_t)b);
        G.bN.push_back((int32_t)b);
        for (size_t jm = 0; jm < (by_m ? np : nq); ++jm)
            for (size_t ln = 0; ln < (by_m ? nq : np); ++ln)
                G.itab.push_back(by_m ? binst[b][jm][ln] : binst[b][ln][jm]);
    }
    G.nA = (int32_t)(by_m ? np : nq);
    G.nB = (int32_t)(by_m ? nq : np);
    return true;
}

}  // namespace

// tensor-core route geometry (gemm_tc.cu)
int tc_planes(int mode);
int tc_elem_bytes(int mode);
int tc_k_block(int mode);
int tc_tile();
int tc_dot_max_k(int mode);

std::unique_ptr<Plan> build_plan(Network &net, int32_t n_amps, const int32_t *outputs,
                                 const std::vector<int64_t> *slice_ids, const GradRequest *grad)
{
    if (net.path.size() + 1 != net.leaves.size()) fail(JET_ESTATE, "no contraction path set");
    if (!net.open_set) fail(JET_ESTATE, "open legs not declared (jet_network_set_open)");
    if (n_amps < 1) fail(JET_EINVAL, "n_amps must be >= 1");
    const int32_t n_open = (int32_t)net.open.size();
    for (int32_t b = 0; b < n_amps; ++b)
        for (int32_t j = 0; j < n_open; ++j) {
            int32_t v = outputs[(int64_t)b * n_open + j];
            if (v < 0 || v >= net.labels.at(net.open[j]).dim)
                fail(JET_EINVAL, "output digit out of range at amplitude " + std::to_string(b));
        }

    auto plan = std::make_unique<Plan>();
    Plan &P = *plan;
    P.outputs.assign(outputs, outputs + (int64_t)n_amps * n_open);
    P.n_amps = n_amps;
    P.path_version = net.path_version;
    P.slice_version = net.slice_version;
    P.precision = net.opt.precision;
    P.reuse = net.opt.reuse;
    const bool fp64 = net.opt.precision == JET_PREC_FP64;
    const int64_t es = fp64 ? 16 : 8;
    // the form a tunable node takes: the autotuner's choice, else the default
    // (the other one while the tuner times the alternatives)
    const bool tune_valid = net.tune_path_version == net.path_version && net.tune_slice_version == net.slice_version;
    auto tuned = [&](int32_t v, int kind, bool deflt) -> bool {
        if (tune_valid) {
            auto it = net.tune.find(v);
            if (it != net.tune.end()) {
                const int c = kind == 0 ? it->second.group : kind == 1 ? it->second.apply_tc : it->second.dot;
                if (c >= 0) return c != 0;
            }
        }
        return net.tune_flip ? !deflt : deflt;
    };
    auto sig_of = [&](int kind, std::initializer_list<int64_t> xs) {
        std::string sg = "k" + std::to_string(kind) + ".p" + std::to_string(net.opt.precision);
        for (int64_t x : xs) sg += "." + std::to_string(x);
        return sg;
    };

    // ---- fixed labels and their values under an assignment alpha = b * n_sl + s
    std::unordered_map<int64_t, int32_t> open_pos, slice_pos;
    for (int32_t j = 0; j < n_open; ++j)   // free open legs stay in the tensors: every value is computed
        if (std::find(net.free_open.begin(), net.free_open.end(), net.open[j]) == net.free_open.end())
            open_pos[net.open[j]] = j;
    std::vector<int64_t> sl_dim, sl_w;
    for (size_t j = 0; j < net.sliced.size(); ++j) {
        slice_pos[net.sliced[j]] = (int32_t)j;
        sl_dim.push_back(net.labels.at(net.sliced[j]).dim);
    }
    sl_w.assign(sl_dim.size(), 1);
    for (int j = (int)sl_dim.size() - 2; j >= 0; --j) sl_w[j] = sl_w[j + 1] * sl_dim[j + 1];
    // all slices, or only the listed slice ids (per-slice partials, Eq. sliced_sum's s_i)
    const int64_t n_sl_all = prod(sl_dim);
    if (slice_ids) {
        if (slice_ids->empty()) fail(JET_EINVAL, "empty slice-id list");
        for (int64_t sid : *slice_ids)
            if (sid < 0 || sid >= n_sl_all)
                fail(JET_EINVAL, "slice id " + std::to_string(sid) + " out of range [0, " + std::to_string(n_sl_all) + ")");
        P.slice_ids = *slice_ids;
        P.partials = true;
    }
    const int64_t n_sl = slice_ids ? (int64_t)slice_ids->size() : n_sl_all;
    P.n_slices = n_sl;
    for (int64_t l : net.free_open) P.n_elem *= net.labels.at(l).dim;
    const int64_t n_assign = (int64_t)n_amps * n_sl;
    if (n_assign > (int64_t)1 << 30) fail(JET_EINVAL, "too many (amplitude, slice) assignments");
    if (n_assign * P.n_elem > (int64_t)1 << 31) fail(JET_EINVAL, "too many output values");
    auto value = [&](int64_t l, int64_t alpha) -> int64_t {
        auto o = open_pos.find(l);
        int64_t b = alpha / n_sl, s = alpha % n_sl;
        if (o != open_pos.end()) return outputs[b * n_open + o->second];
        if (slice_ids) s = (*slice_ids)[s];
        int32_t j = slice_pos.at(l);
        return (s / sl_w[j]) % sl_dim[j];
    };
    auto is_fixed = [&](int64_t l) { return open_pos.count(l) || slice_pos.count(l); };

    const int32_t n_leaves = (int32_t)net.leaves.size();
    const int32_t n_nodes = 2 * n_leaves - 1;
    std::vector<NodeInfo> node(n_nodes);
    std::vector<std::vector<int32_t>> inst_of(n_nodes);   // per node: instance id for each alpha

    std::vector<char> leaf_fixed(n_leaves, 0);   // the leaf carries a fixed (sliced or bra) label
    // ---- leaves: strided views with the fixed labels removed
    for (int32_t i = 0; i < n_leaves; ++i) {
        const Leaf &L = net.leaves[i];
        NodeInfo &N = node[i];
        N.base = BASE_LEAVES;
        std::vector<int64_t> full_stride(L.labels.size(), 1);
        for (int k = (int)L.labels.size() - 2; k >= 0; --k) full_stride[k] = full_stride[k + 1] * L.dims[k + 1];
        std::vector<int64_t> fx, fx_stride, fx_dim;
        for (size_t k = 0; k < L.labels.size(); ++k) {
            if (is_fixed(L.labels[k])) {
                fx.push_back(L.labels[k]);
                fx_stride.push_back(full_stride[k]);
                fx_dim.push_back(L.dims[k]);
            } else {
                N.view.labels.push_back(L.labels[k]);
                N.view.strides.push_back(full_stride[k]);
                N.view.dims.push_back(L.dims[k]);
            }
        }
        N.view.size = prod(N.view.dims);
        leaf_fixed[i] = !fx.empty();
        auto &ids = inst_of[i];
        ids.resize(n_assign);
        if (fx.empty()) {
            N.n_inst = 1;
            N.inst_off.push_back(L.offset);
            std::fill(ids.begin(), ids.end(), 0);
        } else {
            std::unordered_map<int64_t, int32_t> key2id;
            for (int64_t a = 0; a < n_assign; ++a) {
                int64_t key = 0, off = 0;
                for (size_t k = 0; k < fx.size(); ++k) {
                    int64_t v = value(fx[k], a);
                    key = key * fx_dim[k] + v;
                    off += v * fx_stride[k];
                }
                auto it = key2id.find(key);
                if (it == key2id.end()) {
                    it = key2id.emplace(key, (int32_t)N.inst_off.size()).first;
                    N.inst_off.push_back(L.offset + off);
                }
                ids[a] = it->second;
            }
            N.n_inst = (int64_t)N.inst_off.size();
        }
    }

    // ---- internal nodes: instances, layouts, routing
    Arena arena;
    arena.clock = &P.ops;
    Blob blob;
    const bool gemm_ok = gemm_available(net.opt.precision);
    const bool tc_mode = tc_planes(net.opt.precision) > 0;
    int64_t max_inter = 0;

    auto base_ref = [&](int32_t id, int32_t inst) -> std::pair<int32_t, int64_t> {
        const NodeInfo &N = node[id];
        if (N.base == BASE_LEAVES) return {BASE_LEAVES, N.inst_off[inst] * es};
        return {N.base, N.buf_off + (int64_t)inst * N.view.size * es};
    };

    auto dimprod = [&](const std::vector<int64_t> &ls) {
        int64_t p = 1;
        for (int64_t l : ls) p *= net.labels.at(l).dim;
        return p;
    };

    // label sets of every tree node (fixed labels removed) and each node's parent
    // and sibling: a GEMM node shapes its output for the contraction that reads it
    std::vector<std::vector<int64_t>> labset(n_nodes);
    std::vector<int32_t> parent(n_nodes, -1), sibling(n_nodes, -1);
    for (int32_t i = 0; i < n_leaves; ++i) labset[i] = node[i].view.labels;
    for (int32_t k = 0; k < (int32_t)net.path.size(); ++k) {
        const int32_t a = net.path[k].first, b = net.path[k].second, v = n_leaves + k;
        for (int64_t l : labset[a])
            if (find_pos(labset[b], l) < 0) labset[v].push_back(l);
        for (int64_t l : labset[b])
            if (find_pos(labset[a], l) < 0) labset[v].push_back(l);
        parent[a] = parent[b] = v;
        sibling[a] = b;
        sibling[b] = a;
    }

    // Small-operand application route: the small operand holds at most
    // JET_APPLY_MAXK summed and JET_APPLY_MAXF free entries (at most
    // JET_APPLY_MAXB in all) and the large one has enough fibers to fill the GPU.
    // free labels of a view: those not summed
    auto free_of = [&](const View &V, const std::vector<int64_t> &K) {
        std::vector<int64_t> f;
        for (int64_t l : V.labels)
            if (find_pos(K, l) < 0) f.push_back(l);
        return f;
    };
    // tensor-core form (split modes), for small operands of at least
    // apply_tc_min_kf entries (where the CUDA-core forms run out of FMA issue
    // slots before HBM bandwidth): thread groups per CTA that fit the operand
    // planes in shared memory (three for one chunk of summed entries, else
    // two), 0 when the form does not apply
    // A small operand of one chunk (at most 32 summed entries) qualifies from half
    // the threshold on when the CUDA-core forms are FMA-bound on it: at least 10
    // complex multiply-adds per operand entry loaded or stored, nk nf >= 10 (nk + nf).
    auto apply_tc_groups = [&](int64_t nk, int64_t nf) -> int {
        const int64_t kf = nk * nf, min_kf = net.opt.apply_tc_min_kf;
        const bool big = kf >= min_kf || (nk <= 32 && 2 * kf >= min_kf && kf >= 10 * (nk + nf));
        if (!tc_mode || fp64 || !big || nk > JET_APPLY_MAXK || nf < 1 || nf > JET_APPLY_TC_MAXF ||
            (nk > 32 && nf > JET_APPLY_TC_MAXF_MULTI))
            return 0;
        if (nk <= 32 && !jet_apply_tc_half((int)nk, (int)nf) &&
            jet_apply_tc_smem(3, (int)nk, (int)nf) <= JET_APPLY_TC_SMEM_MAX)
            return 3;   // (chunks staged in halves take two groups: up to 256 TMEM columns each)
        if (jet_apply_tc_smem(2, (int)nk, (int)nf) <= JET_APPLY_TC_SMEM_MAX) return 2;
        return 0;
    };
    // the tensor-core form's groups for a shape whatever its size (the tuner's alternative)
    auto apply_tc_groups_any = [&](int64_t nk, int64_t nf) -> int {
        if (!tc_mode || fp64 || nk > JET_APPLY_MAXK || nf < 1 || nf > JET_APPLY_TC_MAXF ||
            (nk > 32 && nf > JET_APPLY_TC_MAXF_MULTI))
            return 0;
        if (nk <= 32 && !jet_apply_tc_half((int)nk, (int)nf) &&
            jet_apply_tc_smem(3, (int)nk, (int)nf) <= JET_APPLY_TC_SMEM_MAX)
            return 3;
        if (jet_apply_tc_smem(2, (int)nk, (int)nf) <= JET_APPLY_TC_SMEM_MAX) return 2;
        return 0;
    };
    // The GEMM route: a summed extent of at least gemm_min_k and both free
    // extents of 64 or more, except where the summed extent is one chunk (<= 32)
    // and one free side has at most 64 entries: the tensor-core small-operand
    // form then reads the large operand once, where the GEMM route first splits
    // it into planes (reading it once and writing it twice over).
    auto tc_apply_short = [&](int64_t nK, int64_t nFa, int64_t nFb) {
        const int64_t nfs = std::min(nFa, nFb);
        return nK <= 32 && nfs <= JET_APPLY_TC_MAXF && apply_tc_groups(nK, nfs) > 0;
    };
    auto gemm_route = [&](int64_t nK, int64_t nFa, int64_t nFb) {
        return gemm_ok && nK >= net.opt.gemm_min_k && nFa >= 64 && nFb >= 64 && !tc_apply_short(nK, nFa, nFb);
    };
    // a small operand of nk summed and nf free entries that some application form takes
    auto apply_shape_ok = [&](int64_t nk, int64_t nf) {
        int64_t nk2 = 1;   // the kernel's compile-time summed extent (power of two >= nk)
        while (nk2 < nk) nk2 *= 2;
        // held in registers: up to 16 summed entries (complex128 too), or 32 (complex64)
        const bool held = nk <= (fp64 ? 16 : JET_APPLY_HOLDK) && nk2 * nf <= JET_APPLY_MAXB;
        const int64_t nfp = nf <= 4 ? nf : (nf + 15) / 16 * 16;
        const bool streamed = !fp64 && nk <= JET_APPLY_MAXK && nf <= JET_APPLY_STREAMF &&
                              (nf <= 4 || nk * nfp <= JET_APPLY_STREAMB);
        const bool tc = apply_tc_groups(nk, nf) > 0;
        return nk >= 1 && (held || streamed || tc) && nf <= JET_APPLY_MAXF;
    };
    auto apply_ok_views = [&](const View &VA, const View &VB, const std::vector<int64_t> &K, bool a_big,
                              int64_t n_inst) {
        const View &VS = a_big ? VB : VA, &VL = a_big ? VA : VB;
        const std::vector<int64_t> fs = free_of(VS, K), fl = free_of(VL, K);
        const int64_t nk = dimprod(K), nf = dimprod(fs), nfib = dimprod(fl);
        return apply_shape_ok(nk, nf) && nfib * n_inst >= (1 << 15) && (int64_t)fl.size() <= JET_MAXR &&
               VS.size == nk * nf && VL.size == nk * nfib;
    };
    auto apply_ok = [&](const NodeInfo &N, const View &VA, const View &VB) {
        return apply_ok_views(VA, VB, N.K, N.a_big, N.n_inst);
    };
    // The summed labels of v's parent when the parent applies a small operand
    // (up to 2048 entries or a shape an application form takes, not the GEMM
    // route) to v as its large operand:
    // laying them out slowest in v lets the parent read, for each summed
    // entry, runs of consecutive fibers (whole sectors per warp) and write its
    // own small operand's labels in their place, again slowest.
    auto consumer_summed = [&](int32_t v) -> std::vector<int64_t> {
        const int32_t pp = parent[v];
        if (pp < 0) return {};
        const auto &ls = labset[sibling[v]];
        std::vector<int64_t> Kp, Fp, Fs;
        for (int64_t l : labset[v]) (find_pos(ls, l) >= 0 ? Kp : Fp).push_back(l);
        for (int64_t l : ls)
            if (find_pos(labset[v], l) < 0) Fs.push_back(l);
        const int64_t sv = dimprod(labset[v]), ss = dimprod(ls);
        const bool p_gemm = !Kp.empty() && gemm_route(dimprod(Kp), dimprod(Fp), dimprod(Fs));
        if (p_gemm || Kp.empty() || sv <= ss || (ss > 2048 && !apply_shape_ok(dimprod(Kp), dimprod(Fs)))) return {};
        return Kp;
    };

    // ---- pass 1, tree order: instances (reuse DAG), label classes, route, layout, depth
    for (int32_t k = 0; k < (int32_t)net.path.size(); ++k) {
        const int32_t a = net.path[k].first, b = net.path[k].second, v = n_leaves + k;
        NodeInfo &N = node[v];
        N.a = a;
        N.b = b;
        auto &ids = inst_of[v];
        ids.resize(n_assign);
        const NodeInfo &NA = node[a], &NB = node[b];
        if (!P.reuse) {
            for (int64_t x = 0; x < n_assign; ++x) {
                ids[x] = (int32_t)x;
                N.ia.push_back(inst_of[a][x]);
                N.ib.push_back(inst_of[b][x]);
            }
        } else if (NA.n_inst == 1 && NB.n_inst == 1) {
            std::fill(ids.begin(), ids.end(), 0);
            N.ia.push_back(0);
            N.ib.push_back(0);
        } else {
            std::unordered_map<int64_t, int32_t> key2id;
            for (int64_t x = 0; x < n_assign; ++x) {
                int64_t key = (int64_t)inst_of[a][x] * NB.n_inst + inst_of[b][x];
                auto it = key2id.find(key);
                if (it == key2id.end()) {
                    it = key2id.emplace(key, (int32_t)N.ia.size()).first;
                    N.ia.push_back(inst_of[a][x]);
                    N.ib.push_back(inst_of[b][x]);
                }
                ids[x] = it->second;
            }
        }
        N.n_inst = (int64_t)N.ia.size();
        std::vector<int32_t>().swap(inst_of[a]);
        std::vector<int32_t>().swap(inst_of[b]);

        const View &VA = NA.view, &VB = NB.view;
        for (int64_t l : VA.labels) (find_pos(VB.labels, l) >= 0 ? N.K : N.fa).push_back(l);
        for (int64_t l : VB.labels)
            if (find_pos(VA.labels, l) < 0) N.fb.push_back(l);
        const int64_t nK = dimprod(N.K), nFa = dimprod(N.fa), nFb = dimprod(N.fb);
        N.use_gemm = gemm_route(nK, nFa, nFb) ||
                     (gemm_ok && nK >= net.opt.gemm_min_k && nFa >= 64 && nFb >= 64 &&
                      !apply_ok_views(VA, VB, N.K, VA.size >= VB.size, N.n_inst));
        // a skinny product (one free side of 8..63 entries, the other large) that no
        // small-operand form takes: the GEMM route with partly filled tiles still runs
        // far faster than the strided direct contraction
        if (!N.use_gemm && gemm_ok && nK >= net.opt.gemm_min_k && std::min(nFa, nFb) >= 8 &&
            std::max(nFa, nFb) >= 4096 && !apply_ok_views(VA, VB, N.K, VA.size >= VB.size, N.n_inst))
            N.use_gemm = true;

        // output layout
        std::vector<int64_t> out;
        N.a_big = VA.size >= VB.size;
        const View &VBig = N.a_big ? VA : VB;
        const View &VSmall = N.a_big ? VB : VA;
        const std::vector<int64_t> &fbig = N.a_big ? N.fa : N.fb, &fsmall = N.a_big ? N.fb : N.fa;
        // in-place pairing: the small operand's j-th free label (in its own
        // order) takes the place of its j-th summed label, when the counts and
        // dims agree (a gate [outs..., ins...] then maps each output wire onto
        // its input wire and the large operand's layout is kept)
        std::vector<int64_t> ks_small, fs_small_order;
        for (int64_t l : VSmall.labels) (find_pos(N.K, l) >= 0 ? ks_small : fs_small_order).push_back(l);
        // this node applies its small operand to the large one (a small operand of
        // up to 2048 entries, or one that an application form takes)
        const bool v_applies = !N.use_gemm && VBig.size > VSmall.size &&
                               (VSmall.size <= 2048 || apply_ok_views(VA, VB, N.K, N.a_big, N.n_inst));
        bool pairable = v_applies && !ks_small.empty() &&
                        ks_small.size() == fs_small_order.size();
        for (size_t j = 0; pairable && j < ks_small.size(); ++j)
            pairable = net.labels.at(ks_small[j]).dim == net.labels.at(fs_small_order[j]).dim;
        if (pairable) {
            for (int64_t l : VBig.labels) {
                const int p = find_pos(ks_small, l);
                out.push_back(p >= 0 ? fs_small_order[p] : l);
            }
        } else if (v_applies) {
            // keep the big operand's order; the small operand's free labels take
            // the place of the first summed label (gate application in place)
            int ins = -1;
            for (size_t i = 0; i < VBig.labels.size(); ++i)
                if (find_pos(N.K, VBig.labels[i]) >= 0) { ins = (int)i; break; }
            for (size_t i = 0; i < VBig.labels.size(); ++i) {
                if ((int)i == ins) out.insert(out.end(), fsmall.begin(), fsmall.end());
                if (find_pos(N.K, VBig.labels[i]) < 0) out.push_back(VBig.labels[i]);
            }
            if (ins < 0) out.insert(out.begin(), fsmall.begin(), fsmall.end());
        } else if (N.use_gemm) {
            N.a_is_m = nFa >= nFb;
            N.fM = N.a_is_m ? N.fa : N.fb;
            N.fN = N.a_is_m ? N.fb : N.fa;
            const int32_t pp = parent[v];
            // FP16x3 with a GEMM parent that sums labels of both of this node's
            // sides: this node's epilogue can write the parent's operand planes
            // (fused split) when the parent's summed labels from the N side number
            // 4 or 8 entries and, with those from the M side, fill whole 64-entry
            // chunks; they go lowest on each side (fM = [m_f, m_k], fN = [n_f, n_k])
            if (tc_mode && net.opt.precision == JET_PREC_FP16X3 && net.opt.fuse_split && !grad && pp >= 0) {
                const auto &ls = labset[sibling[v]];
                std::vector<int64_t> Kp, Fp, Fs;
                for (int64_t l : labset[v]) (find_pos(ls, l) >= 0 ? Kp : Fp).push_back(l);
                for (int64_t l : ls)
                    if (find_pos(labset[v], l) < 0) Fs.push_back(l);
                // (a GEMM parent, or a skinny product the GEMM route also takes; pass 2
                // checks the parent's route)
                const int64_t kp = dimprod(Kp), fp_ = dimprod(Fp), fs_ = dimprod(Fs);
                const bool p_gemm = !Kp.empty() && (gemm_route(kp, fp_, fs_) ||
                                                    (gemm_ok && kp >= net.opt.gemm_min_k && std::min(fp_, fs_) >= 8 &&
                                                     std::max(fp_, fs_) >= 4096));
                bool pow2 = true;
                for (int64_t l : labset[v]) pow2 = pow2 && (net.labels.at(l).dim & (net.labels.at(l).dim - 1)) == 0;
                for (int flip = 0; flip < 2 && p_gemm && pow2 && dimprod(Kp) % 64 == 0 && !N.fuse; ++flip) {
                    const bool am = flip ? !N.a_is_m : N.a_is_m;
                    const auto &sM = am ? N.fa : N.fb, &sN = am ? N.fb : N.fa;
                    std::vector<int64_t> mk, nk, mf, nf;
                    for (int64_t l : sM) (find_pos(Kp, l) >= 0 ? mk : mf).push_back(l);
                    for (int64_t l : sN) (find_pos(Kp, l) >= 0 ? nk : nf).push_back(l);
                    const int64_t NKd = dimprod(nk), MKd = dimprod(mk);
                    // within each group, the label of smallest stride in the child that
                    // holds it last: this node's own operand splits keep reading along
                    // the children's fastest labels
                    auto by_stride = [&](std::vector<int64_t> &ls, int32_t child) {
                        const View &Vc = node[child].view;
                        std::stable_sort(ls.begin(), ls.end(), [&](int64_t x, int64_t y) {
                            return Vc.strides[find_pos(Vc.labels, x)] > Vc.strides[find_pos(Vc.labels, y)];
                        });
                    };
                    const int32_t cM = am ? a : b, cN = am ? b : a;
                    by_stride(mf, cM);
                    by_stride(mk, cM);
                    by_stride(nf, cN);
                    by_stride(nk, cN);
                    if ((NKd == 4 || NKd == 8) && MKd >= 64 / NKd && MKd * NKd == dimprod(Kp) && !mf.empty() &&
                        !nf.empty()) {
                        N.a_is_m = am;
                        N.fM = mf;
                        N.fM.insert(N.fM.end(), mk.begin(), mk.end());
                        N.fN = nf;
                        N.fN.insert(N.fN.end(), nk.begin(), nk.end());
                        N.fz_mk = mk;
                        N.fz_nk = nk;
                        N.fuse = true;
                    }
                }
            }
            // a parent that contracts this output with its sibling over every label
            // (a dot product per instance): the epilogue computes the products
            // itself; each side's labels in decreasing stride in the sibling (when
            // its view is known), so a warp's reads of the sibling run along it
            if (tc_mode && net.opt.fuse_split && dimprod(N.K) <= tc_dot_max_k(net.opt.precision) && !grad && pp >= 0 &&
                !N.fuse) {
                const int32_t sb = sibling[v];
                bool full = labset[pp].empty() && labset[sb].size() == labset[v].size();
                for (int64_t l : labset[v]) full = full && find_pos(labset[sb], l) >= 0;
                // (a tunable choice, taken by default: its time is this GEMM's and
                // its parent's)
                if (full) {
                    N.dot = tuned(v, 2, true);
                    P.tunables.push_back({v, 2, N.dot ? 1 : 0,
                                          sig_of(2, {dimprod(N.K), dimprod(labset[v]), N.n_inst, node[sb].n_inst,
                                                     node[pp].n_inst}),
                                          pp});
                }
                if (N.dot) {
                    if (sb < v) {
                        const View &Vs = node[sb].view;
                        auto by_sib = [&](std::vector<int64_t> &ls) {
                            std::stable_sort(ls.begin(), ls.end(), [&](int64_t x, int64_t y) {
                                return Vs.strides[find_pos(Vs.labels, x)] > Vs.strides[find_pos(Vs.labels, y)];
                            });
                        };
                        by_sib(N.fM);
                        by_sib(N.fN);
                    }
                }
            }
            // for a tensor-core parent, lay the output out as [parent-free, parent-summed]
            // when the parent's summed labels all come from one side: the parent's
            // operand split is then a plain format conversion
            if (tc_mode && pp >= 0 && !N.fuse && !N.dot) {
                const auto &ls = labset[sibling[v]];
                std::vector<int64_t> Kp, Fp, Fs;
                for (int64_t l : labset[v]) (find_pos(ls, l) >= 0 ? Kp : Fp).push_back(l);
                for (int64_t l : ls)
                    if (find_pos(labset[v], l) < 0) Fs.push_back(l);
                const bool p_gemm = !Kp.empty() && gemm_route(dimprod(Kp), dimprod(Fp), dimprod(Fs));
                auto holds_all = [&](const std::vector<int64_t> &X) {
                    for (int64_t l : Kp)
                        if (find_pos(X, l) < 0) return false;
                    return true;
                };
                const int side = !p_gemm ? -1 : holds_all(N.fb) ? 1 : holds_all(N.fa) ? 0 : -1;
                if (side >= 0) {
                    N.a_is_m = side == 1;
                    N.fM = N.a_is_m ? N.fa : N.fb;
                    const auto &fNs = N.a_is_m ? N.fb : N.fa;
                    N.fN.clear();
                    for (int64_t l : fNs)
                        if (find_pos(Kp, l) < 0) N.fN.push_back(l);
                    for (int64_t l : fNs)
                        if (find_pos(Kp, l) >= 0) N.fN.push_back(l);
                }
            }
            // for a parent that applies a small operand: its summed labels slowest,
            // when one side holds them all (that side becomes M, their rows first)
            // (tensor-core route: the operand split gathers rows in any order)
            const std::vector<int64_t> Kc = tc_mode && !N.fuse && !N.dot ? consumer_summed(v) : std::vector<int64_t>();
            if (!Kc.empty()) {
                auto holds_all = [&](const std::vector<int64_t> &X) {
                    for (int64_t l : Kc)
                        if (find_pos(X, l) < 0) return false;
                    return true;
                };
                const int side = holds_all(N.fa) ? 0 : holds_all(N.fb) ? 1 : -1;
                if (side >= 0) {
                    N.a_is_m = side == 0;
                    const auto &fMs = N.a_is_m ? N.fa : N.fb;
                    N.fM = Kc;
                    for (int64_t l : fMs)
                        if (find_pos(Kc, l) < 0) N.fM.push_back(l);
                    N.fN = N.a_is_m ? N.fb : N.fa;
                }
            }
            out = N.fM;
            out.insert(out.end(), N.fN.begin(), N.fN.end());
        } else {
            out = fbig;
            out.insert(out.end(), fsmall.begin(), fsmall.end());
        }
        if (!N.use_gemm) {
            // A parent that applies a small operand reads, per summed entry, runs of
            // its fibers: with its summed labels slowest those runs are contiguous.
            // Moving them can break up this node's own writes when they were among
            // its fastest labels, so the reordered layout is taken only when it
            // touches fewer 32-byte sectors per warp access, counting both this
            // node's writes (32 consecutive fibers of a small-operand application,
            // one free entry) and the parent's reads (32 consecutive fibers, one
            // summed entry); both touch every element of the intermediate once.
            // A write sector weighs 4 reads: partly written sectors are merged in
            // L2, while the parent's other summed entries find a partly read
            // sector in L1 (measured on the bosonic lattice: twice the write
            // sectors cost 3.8x the time, four times the read sectors 2.7x).
            const std::vector<int64_t> Kc = consumer_summed(v);
            if (!Kc.empty()) {
                std::vector<int64_t> re;
                for (int64_t l : out)
                    if (find_pos(Kc, l) >= 0) re.push_back(l);
                for (int64_t l : out)
                    if (find_pos(Kc, l) < 0) re.push_back(l);
                const bool v_apply = v_applies;
                std::vector<int64_t> vfib;   // this node's fibers in its decode order (large operand's strides)
                if (v_apply) {
                    for (size_t i = VBig.labels.size(); i-- > 0;)
                        if (find_pos(N.K, VBig.labels[i]) < 0) vfib.push_back(VBig.labels[i]);
                    std::stable_sort(vfib.begin(), vfib.end(), [&](int64_t x, int64_t y) {
                        return VBig.strides[find_pos(VBig.labels, x)] < VBig.strides[find_pos(VBig.labels, y)];
                    });
                }
                // distinct 32-byte sectors of 32 consecutive indices over `order` (fastest first)
                auto sectors32 = [&](const std::vector<int64_t> &order, const View &L) {
                    std::vector<int64_t> sec;
                    for (int64_t r = 0; r < 32; ++r) {
                        int64_t x = r, off = 0;
                        for (int64_t l : order) {
                            const int64_t dm = net.labels.at(l).dim;
                            off += (x % dm) * L.strides[find_pos(L.labels, l)];
                            x /= dm;
                        }
                        sec.push_back(off * es / 32);
                    }
                    std::sort(sec.begin(), sec.end());
                    return (int64_t)(std::unique(sec.begin(), sec.end()) - sec.begin());
                };
                auto cost = [&](const std::vector<int64_t> &lay) {
                    const View L = dense_view(lay, net);
                    std::vector<int64_t> pfib;   // the parent's fibers, fastest first
                    for (size_t i = lay.size(); i-- > 0;)
                        if (find_pos(Kc, lay[i]) < 0) pfib.push_back(lay[i]);
                    return (v_apply ? 4 * sectors32(vfib, L) : 0) + sectors32(pfib, L);
                };
                if (cost(re) < cost(out)) out = re;
            }
        }
        N.view = dense_view(out, net);
        max_inter = std::max(max_inter, N.view.size);
        // small direct contractions are batched per tree level into one launch
        // (their full offset tables are int32: operands below 2^31 elements)
        // (also those of at most 131072 outputs over all instances and 2^20
        // multiply-adds, which the chained small levels take)
        N.small = !N.use_gemm && nK <= 2048 &&
                  (N.view.size <= 4096 || ((double)N.n_inst * (double)N.view.size <= 131072.0 &&
                                           (double)N.n_inst * (double)N.view.size * (double)nK <= (double)(1 << 20))) &&
                  (double)N.n_inst * (double)N.view.size * (double)nK <= (double)(1 << 24) &&
                  VA.size <= INT32_MAX && VB.size <= INT32_MAX;
        N.depth = 1 + std::max(node[a].depth, node[b].depth);
    }

    // ---- launch order: by tree level, a level's small contractions first (one
    // batched launch), then its large ones in tree order
    std::vector<int32_t> order;
    for (int32_t k = 0; k < (int32_t)net.path.size(); ++k) order.push_back(n_leaves + k);
    std::stable_sort(order.begin(), order.end(), [&](int32_t x, int32_t y) {
        if (node[x].depth != node[y].depth) return node[x].depth < node[y].depth;
        return (int)node[x].small > (int)node[y].small;
    });

    // ---- kept shared work: a sub-tree whose leaves carry no fixed label has the
    // same value in every contraction of this network (Section 3.2's shared work,
    // kept for later use).  Its maximal such nodes of at least keep_min elements
    // keep their results in a device pool: a ready result replaces its sub-tree
    // (no launches), a missing one is computed into the pool by this plan.
    std::vector<char> skip(n_nodes, 0);
    if (net.keep_min > 0 && !grad && P.reuse) {
        std::vector<char> inv(n_nodes, 0);
        for (int32_t i = 0; i < n_leaves; ++i) inv[i] = !leaf_fixed[i];
        for (int32_t k = 0; k < (int32_t)net.path.size(); ++k) {
            const int32_t v = n_leaves + k;
            inv[v] = inv[node[v].a] && inv[node[v].b];
        }
        size_t pool = 0;
        for (auto &kv : net.kept) pool = std::max(pool, kv.second.off + kv.second.bytes);
        for (int32_t k = 0; k < (int32_t)net.path.size(); ++k) {
            const int32_t v = n_leaves + k;
            if (!inv[v] || (parent[v] >= 0 && inv[parent[v]]) || node[v].view.size < net.keep_min) continue;
            auto it = net.kept.find(v);
            if (it == net.kept.end()) {
                Network::KeptEntry e;
                e.off = (pool + 255) / 256 * 256;
                e.bytes = (size_t)node[v].view.size * es;
                pool = e.off + e.bytes;
                it = net.kept.emplace(v, e).first;
            }
            if (it->second.ready) {   // the sub-tree's work is done: read the kept result
                std::vector<int32_t> st{v};
                while (!st.empty()) {
                    const int32_t x = st.back();
                    st.pop_back();
                    if (x < n_leaves) continue;
                    skip[x] = 1;
                    st.push_back(node[x].a);
                    st.push_back(node[x].b);
                }
                node[v].base = BASE_KEPT;
                node[v].buf_off = (int64_t)it->second.off;
            } else {
                P.kept_fill.push_back(v);
            }
        }
        P.kept_pool_bytes = pool;
    }

    // pending batch of small contractions (one tree level)
    std::vector<Plan::Patch> batch_patches;   // offsets relative to the batch's task array
    std::vector<SmallTask> batch;
    std::vector<int32_t> batch_nodes;
    double batch_flop = 0, batch_bytes = 0;
    auto release_children = [&](int32_t v) {
        if (grad) return;   // the adjoint sweep reads every forward intermediate
        for (int32_t c : {node[v].a, node[v].b})
            if (node[c].base == BASE_ARENA)
                arena.release((size_t)node[c].buf_off, node[c].alloc_bytes ? node[c].alloc_bytes
                                                                            : (size_t)node[c].n_inst * node[c].view.size * es);
    };
    // consecutive tiny levels of the forward sweep run as one chain launch (one
    // block, a barrier between levels); their children are released when the
    // chain is issued
    bool chain_on = true;
    std::vector<SmallTask> chain;
    std::vector<Plan::Patch> chain_patches;
    std::vector<int32_t> chain_nodes, chain_lv_end;
    double chain_flop = 0, chain_bytes = 0;
    auto flush_chain = [&]() {
        if (chain.empty()) return;
        size_t o_tasks = blob.reserve(sizeof(SmallTask) * chain.size(), 64);
        for (size_t i = 0; i < chain.size(); ++i)
            std::memcpy(blob.bytes.data() + o_tasks + i * sizeof(SmallTask), &chain[i], sizeof(SmallTask));
        for (auto &pt : chain_patches) blob.patches.push_back({o_tasks + pt.at, pt.base, pt.byte_off});
        // one block per 256 items of the widest level, at most one per SM
        int64_t widest = 0, lv0 = 0;
        for (int32_t e : chain_lv_end) {
            const SmallTask &tl = chain[(size_t)e - 1];
            widest = std::max<int64_t>(widest, (int64_t)tl.block0 + (int64_t)tl.n_inst * tl.n_out);
            lv0 = e;
        }
        (void)lv0;
        const int32_t G = (int32_t)std::max<int64_t>(1, std::min<int64_t>(148, (widest + 255) / 256));
        SmallBatchArgs sb;
        std::memset(&sb, 0, sizeof sb);
        sb.n_tasks = (int32_t)chain.size();
        sb.n_blocks = G;
        sb.n_levels = (int32_t)chain_lv_end.size();
        for (size_t l = 0; l < chain_lv_end.size(); ++l) sb.lv_end[l] = chain_lv_end[l];
        const size_t o_bar = blob.reserve(8, 8);   // the grid barrier's counters (zero)
        size_t so = blob.reserve(sizeof sb);
        std::memcpy(blob.bytes.data() + so, &sb, sizeof sb);
        blob.patch_field(so, offsetof(SmallBatchArgs, tasks), BASE_BLOB, (int64_t)o_tasks);
        blob.patch_field(so, offsetof(SmallBatchArgs, barrier), BASE_BLOB, (int64_t)o_bar);
        blob.patch_field(so, offsetof(SmallBatchArgs, status), BASE_STATUS, 0);
        Op op;
        op.kind = OpKind::SmallBatch;
        op.node = chain_nodes.front();
        op.n_inst = (int64_t)chain.size();
        op.args_off = so;
        op.args_bytes = sizeof sb;
        op.flop = chain_flop;
        op.bytes = chain_bytes;
        op.variant = (fp64 ? 1 : 0) | 2;
        op.grid_x = G;
        op.block = 256;
        op.batch_first = (int32_t)P.batch_nodes.size();
        op.batch_count = (int32_t)chain_nodes.size();
        P.batch_nodes.insert(P.batch_nodes.end(), chain_nodes.begin(), chain_nodes.end());
        P.ops.push_back(op);
        for (int32_t v : chain_nodes) release_children(v);
        chain.clear();
        chain_patches.clear();
        chain_nodes.clear();
        chain_lv_end.clear();
        chain_flop = chain_bytes = 0;
    };
    auto flush_batch = [&]() {
        if (batch.empty()) return;
        {   // a small level (at most 262144 outputs, about seven per thread of a full
            // grid, and 8 MFLOP) joins the chain
            int64_t items = 0;
            for (auto &t : batch) items += (int64_t)t.n_inst * t.n_out;
            if (chain_on && items <= 262144 && batch_flop <= 8e6 && (int64_t)batch.size() <= JET_CHAIN_TASKS) {
                if ((int)chain_lv_end.size() == JET_CHAIN_LEVELS) flush_chain();
                const size_t base = chain.size() * sizeof(SmallTask);
                int64_t item0 = 0;
                for (auto &t : batch) {
                    SmallTask u = t;
                    u.block0 = (int32_t)item0;   // first item within the level
                    item0 += (int64_t)t.n_inst * t.n_out;
                    chain.push_back(u);
                }
                for (auto &pt : batch_patches) chain_patches.push_back({base + pt.at, pt.base, pt.byte_off});
                chain_lv_end.push_back((int32_t)chain.size());
                chain_nodes.insert(chain_nodes.end(), batch_nodes.begin(), batch_nodes.end());
                chain_flop += batch_flop;
                chain_bytes += batch_bytes;
                batch.clear();
                batch_nodes.clear();
                batch_patches.clear();
                batch_flop = batch_bytes = 0;
                return;
            }
        }
        flush_chain();
        int32_t blocks = 0;
        for (auto &t : batch) {
            t.block0 = blocks;
            int64_t items = (int64_t)t.n_inst * t.n_out;
            blocks += (int32_t)std::max<int64_t>(1, std::min<int64_t>((items + 255) / 256, 256));
        }
        // task records (their table pointers are patched like every other pointer)
        size_t o_tasks = blob.reserve(sizeof(SmallTask) * batch.size(), 64);
        for (size_t i = 0; i < batch.size(); ++i)
            std::memcpy(blob.bytes.data() + o_tasks + i * sizeof(SmallTask), &batch[i], sizeof(SmallTask));
        for (auto &pt : batch_patches) blob.patches.push_back({o_tasks + pt.at, pt.base, pt.byte_off});
        SmallBatchArgs sb;
        std::memset(&sb, 0, sizeof sb);
        sb.n_tasks = (int32_t)batch.size();
        sb.n_blocks = blocks;
        size_t so = blob.reserve(sizeof sb);
        std::memcpy(blob.bytes.data() + so, &sb, sizeof sb);
        blob.patch_field(so, offsetof(SmallBatchArgs, tasks), BASE_BLOB, (int64_t)o_tasks);
        Op op;
        op.kind = OpKind::SmallBatch;
        op.node = batch_nodes.empty() ? -1 : batch_nodes.front();
        op.n_inst = (int64_t)batch.size();
        op.args_off = so;
        op.args_bytes = sizeof sb;
        op.flop = batch_flop;
        op.bytes = batch_bytes;
        op.variant = fp64 ? 1 : 0;
        op.grid_x = blocks;
        op.batch_first = (int32_t)P.batch_nodes.size();
        op.batch_count = (int32_t)batch_nodes.size();
        P.batch_nodes.insert(P.batch_nodes.end(), batch_nodes.begin(), batch_nodes.end());
        P.ops.push_back(op);
        for (int32_t v : batch_nodes) release_children(v);
        batch.clear();
        batch_nodes.clear();
        batch_patches.clear();
        batch_flop = batch_bytes = 0;
    };

    // A small contraction C (dense layout Cv) = sum over K of A (view VA) * B
    // (view VB) as one task of the current level batch: full offset tables.
    auto add_small_task = [&](const View &VA, const View &VB, const View &Cv, const std::vector<int64_t> &K, bool a_big,
                              const std::vector<std::pair<int32_t, int64_t>> &pa,
                              const std::vector<std::pair<int32_t, int64_t>> &pb,
                              const std::vector<std::pair<int32_t, int64_t>> &pc, int64_t n_inst) {
        auto strideOf = [&](const View &V, int64_t l) {
            int p = find_pos(V.labels, l);
            return p < 0 ? (int64_t)0 : V.strides[p];
        };
        const auto &C = Cv;
        const int64_t nK = dimprod(K);
        std::vector<int32_t> oA(C.size), oB(C.size), kA(nK), kB(nK);
        for (int64_t o = 0; o < C.size; ++o) {
            int64_t r = o, x = 0, y = 0;
            for (int j = (int)C.labels.size() - 1; j >= 0; --j) {
                int64_t dg = r % C.dims[j];
                r /= C.dims[j];
                x += dg * strideOf(VA, C.labels[j]);
                y += dg * strideOf(VB, C.labels[j]);
            }
            oA[o] = (int32_t)x;
            oB[o] = (int32_t)y;
        }
        // summed labels in the direct kernel's order (slowest first by stride in the
        // larger operand), so both kernels add the terms in the same sequence
        const View &VX = a_big ? VA : VB;
        std::vector<int64_t> Ks = K;
        std::stable_sort(Ks.begin(), Ks.end(), [&](int64_t x, int64_t y) { return strideOf(VX, x) > strideOf(VX, y); });
        std::vector<int64_t> Kd;
        for (int64_t l : Ks) Kd.push_back(net.labels.at(l).dim);
        for (int64_t q = 0; q < nK; ++q) {
            int64_t r = q, x = 0, y = 0;
            for (int j = (int)Ks.size() - 1; j >= 0; --j) {
                int64_t dg = r % Kd[j];
                r /= Kd[j];
                x += dg * strideOf(VA, Ks[j]);
                y += dg * strideOf(VB, Ks[j]);
            }
            kA[q] = (int32_t)x;
            kB[q] = (int32_t)y;
        }
        SmallTask t;
        std::memset(&t, 0, sizeof t);
        t.n_out = (int32_t)C.size;
        t.n_k = (int32_t)nK;
        t.n_inst = (int32_t)n_inst;
        const size_t i0 = batch.size() * sizeof(SmallTask);
        size_t o_pa = blob.put_ptrs(pa), o_pb = blob.put_ptrs(pb), o_pc = blob.put_ptrs(pc);
        size_t o_oa = blob.put_i32(oA), o_ob = blob.put_i32(oB), o_ka = blob.put_i32(kA), o_kb = blob.put_i32(kB);
        batch_patches.push_back({i0 + offsetof(SmallTask, ptrA), BASE_BLOB, (int64_t)o_pa});
        batch_patches.push_back({i0 + offsetof(SmallTask, ptrB), BASE_BLOB, (int64_t)o_pb});
        batch_patches.push_back({i0 + offsetof(SmallTask, ptrC), BASE_BLOB, (int64_t)o_pc});
        batch_patches.push_back({i0 + offsetof(SmallTask, offA), BASE_BLOB, (int64_t)o_oa});
        batch_patches.push_back({i0 + offsetof(SmallTask, offB), BASE_BLOB, (int64_t)o_ob});
        batch_patches.push_back({i0 + offsetof(SmallTask, kA), BASE_BLOB, (int64_t)o_ka});
        batch_patches.push_back({i0 + offsetof(SmallTask, kB), BASE_BLOB, (int64_t)o_kb});
        batch.push_back(t);
    };

    // Direct strided contraction of every instance: C (dense, layout Cv) = sum over
    // K of A (view VA) * B (view VB); pa/pb/pc: per-instance addresses.
    auto emit_direct = [&](int32_t v, const View &VA, const View &VB, const View &Cv, const std::vector<int64_t> &K,
                           bool a_big, int64_t n_inst, const std::vector<std::pair<int32_t, int64_t>> &pa,
                           const std::vector<std::pair<int32_t, int64_t>> &pb,
                           const std::vector<std::pair<int32_t, int64_t>> &pc, double flop, double bytes,
                           std::vector<size_t> &scratch, std::vector<size_t> &scratch_bytes, bool group = true) {
            const View &VX = a_big ? VA : VB;   // operand whose strides order the summed labels
            auto strideA = [&](int64_t l) { int p = find_pos(VA.labels, l); return p < 0 ? 0 : VA.strides[p]; };
            auto strideB = [&](int64_t l) { int p = find_pos(VB.labels, l); return p < 0 ? 0 : VB.strides[p]; };
            DirectArgs d;
            std::memset(&d, 0, sizeof d);
            // output split: cols = longest suffix with product <= JET_COLMAX whose
            // offsets fit the int32 tables (labels with larger strides are decoded)
            const auto &C = Cv;
            size_t ncol_labels = 0;
            int64_t ncols = 1, col_maxA = 0, col_maxB = 0;
            while (ncol_labels < C.labels.size()) {
                const size_t li = C.labels.size() - 1 - ncol_labels;
                const int64_t dm = C.dims[li] - 1;
                if (ncols * C.dims[li] > JET_COLMAX || col_maxA + dm * strideA(C.labels[li]) > INT32_MAX ||
                    col_maxB + dm * strideB(C.labels[li]) > INT32_MAX)
                    break;
                ncols *= C.dims[li];
                col_maxA += dm * strideA(C.labels[li]);
                col_maxB += dm * strideB(C.labels[li]);
                ++ncol_labels;
            }
            size_t nrow_labels = C.labels.size() - ncol_labels;
            if (nrow_labels > JET_MAXR) fail(JET_EINVAL, "intermediate rank too large");
            std::vector<int32_t> colA(ncols), colB(ncols);
            for (int64_t c = 0; c < ncols; ++c) {
                int64_t r = c, oa = 0, ob = 0;
                for (size_t j = 0; j < ncol_labels; ++j) {
                    size_t li = C.labels.size() - 1 - j;
                    int64_t dg = r % C.dims[li];
                    r /= C.dims[li];
                    oa += dg * strideA(C.labels[li]);
                    ob += dg * strideB(C.labels[li]);
                }
                if (oa > INT32_MAX || ob > INT32_MAX) fail(JET_EINVAL, "column offset overflow");
                colA[c] = (int32_t)oa;
                colB[c] = (int32_t)ob;
            }
            d.n_cols = (int32_t)ncols;
            d.n_rows = prod(C.dims, 0, nrow_labels);
            d.row_rank = (int32_t)nrow_labels;
            for (size_t j = 0; j < nrow_labels; ++j) {
                size_t li = nrow_labels - 1 - j;
                d.row_dim[j] = C.dims[li];
                d.row_sA[j] = strideA(C.labels[li]);
                d.row_sB[j] = strideB(C.labels[li]);
            }
            // summed labels, slowest first.  The inner part (a table of up to
            // JET_KLOMAX entries whose entries a block's threads share out) takes
            // the fastest summed labels of the two operands in turn, so that both
            // read whole sectors within a block when they order these labels
            // differently; inside each part, slowest first by stride in the larger
            // operand.
            const View &VY = a_big ? VB : VA;
            auto slower_in = [&](const View &V) {
                return [&V](int64_t x, int64_t y) {
                    return V.strides[find_pos(V.labels, x)] > V.strides[find_pos(V.labels, y)];
                };
            };
            std::vector<int64_t> fx = K, fy = K, lo, hi;
            std::stable_sort(fx.begin(), fx.end(), slower_in(VX));
            std::stable_sort(fy.begin(), fy.end(), slower_in(VY));
            {
                int64_t n_lo = 1, mA = 0, mB = 0;
                auto take = [&](int64_t l) {
                    const int64_t d = net.labels.at(l).dim;
                    if (find_pos(lo, l) >= 0 || n_lo * d > JET_KLOMAX || mA + (d - 1) * strideA(l) > INT32_MAX ||
                        mB + (d - 1) * strideB(l) > INT32_MAX)
                        return;
                    lo.push_back(l);
                    n_lo *= d;
                    mA += (d - 1) * strideA(l);
                    mB += (d - 1) * strideB(l);
                };
                for (size_t i = K.size(); i-- > 0;) {   // fastest first in each operand, in turn
                    take(fx[i]);
                    take(fy[i]);
                }
            }
            for (int64_t l : fx)
                if (find_pos(lo, l) < 0) hi.push_back(l);
            std::stable_sort(lo.begin(), lo.end(), slower_in(VX));
            std::vector<int64_t> Ks = hi;   // hi already slowest first in VX
            Ks.insert(Ks.end(), lo.begin(), lo.end());
            std::vector<int64_t> Kd;
            for (int64_t l : Ks) Kd.push_back(net.labels.at(l).dim);
            size_t nklo_labels = 0;
            int64_t nklo = 1, klo_maxA = 0, klo_maxB = 0;
            while (nklo_labels < Ks.size()) {
                const size_t li = Ks.size() - 1 - nklo_labels;
                const int64_t dm = Kd[li] - 1;
                if (nklo * Kd[li] > JET_KLOMAX || klo_maxA + dm * strideA(Ks[li]) > INT32_MAX ||
                    klo_maxB + dm * strideB(Ks[li]) > INT32_MAX)
                    break;
                nklo *= Kd[li];
                klo_maxA += dm * strideA(Ks[li]);
                klo_maxB += dm * strideB(Ks[li]);
                ++nklo_labels;
            }
            size_t nkhi_labels = Ks.size() - nklo_labels;
            if (nkhi_labels > JET_MAXR) fail(JET_EINVAL, "summed rank too large");
            std::vector<int32_t> kA(nklo), kB(nklo);
            for (int64_t q = 0; q < nklo; ++q) {
                int64_t r = q, oa = 0, ob = 0;
                for (size_t j = 0; j < nklo_labels; ++j) {
                    size_t li = Ks.size() - 1 - j;
                    int64_t dg = r % Kd[li];
                    r /= Kd[li];
                    oa += dg * strideA(Ks[li]);
                    ob += dg * strideB(Ks[li]);
                }
                if (oa > INT32_MAX || ob > INT32_MAX) fail(JET_EINVAL, "summed offset overflow");
                kA[q] = (int32_t)oa;
                kB[q] = (int32_t)ob;
            }
            d.n_klo = (int32_t)nklo;
            d.khi_rank = (int32_t)nkhi_labels;
            d.n_khi = 1;
            for (size_t j = 0; j < nkhi_labels; ++j) {
                size_t li = nkhi_labels - 1 - j;
                d.khi_dim[j] = Kd[li];
                d.khi_sA[j] = strideA(Ks[li]);
                d.khi_sB[j] = strideB(Ks[li]);
                d.n_khi *= Kd[li];
            }
            d.n_out = d.n_rows * d.n_cols;
            d.n_inst = (int32_t)n_inst;
            // split the summed index across blocks when there are few outputs
            const int64_t total_out = d.n_out * n_inst;
            const int64_t n_k = d.n_khi * d.n_klo;
            d.ksplit = 1;
            // the split form (8 outputs per block, the block's threads sharing the
            // summed index) also when the one-output-per-thread form would launch
            // fewer than 4 blocks per SM: at least two parts then
            const int64_t plain_blocks = (d.n_out + 255) / 256 * n_inst;
            const bool few_blocks = plain_blocks < 148 * 4;
            if ((total_out < 16384 || few_blocks) && n_k >= 4096 && d.n_khi > 1) {
                // one wave of 8 blocks per SM, four for summed extents of 2^20 or more
                // (whose parts stay long; more parts for shorter ones cost more in
                // partials and launch tails than they gain: the adjoint's environments)
                int64_t groups = (d.n_out + JET_SPLITK_G - 1) / JET_SPLITK_G * n_inst;
                const int64_t waves = n_k >= (1 << 20) ? 4 : 1;
                int64_t want = std::max<int64_t>(few_blocks ? 2 : 1, (148 * 8 * waves + groups - 1) / groups);
                int64_t parts = std::min<int64_t>(want, d.n_khi);
                d.khi_per_part = (int32_t)((d.n_khi + parts - 1) / parts);
                d.ksplit = (int32_t)((d.n_khi + d.khi_per_part - 1) / d.khi_per_part);
            }
            // split form: when every group of 8 outputs is an outer product of NA
            // values of A and NB = 8 / NA of B, each is loaded once per summed entry
            // (fewest loads first: NA = 2 or 4 take 6, NA = 1 or 8 take 9); A's
            // values fastest (pattern NA) or B's (pattern 16 + NB)
            if (d.ksplit > 1 && d.n_out == 1) d.splitk_na = 32;   // a dot product
            // dot products whose instances pair every A instance of a block with the
            // same B instances (at most 4 x 4, 8 products): one block of threads
            // loads each operand value once for all of the block's products
            std::vector<int32_t> blk_itab;
            int64_t n_launch_inst = n_inst;
            if (group && d.splitk_na == 32 && n_inst > 1) {
                GemmGroups G;
                const std::vector<int32_t> &ia = node[v].ia, &ib = node[v].ib;
                bool ok = (int64_t)ia.size() == n_inst && group_instances(ia, ib, true, G) && G.dup == 0;
                if (!ok && (int64_t)ia.size() == n_inst) ok = group_instances(ia, ib, false, G) && G.dup == 0;
                if (ok && G.nA * G.nB >= 2 && G.nA <= 4 && G.nB <= 4 && G.nA * G.nB <= JET_SPLITK_G) {
                    d.splitk_na = G.nA <= 2 && G.nB <= 2 ? 65 : 64;   // (65: at most 2 x 2, fewer registers)
                    d.blk_na = G.nA;
                    d.blk_nb = G.nB;
                    blk_itab = G.itab;
                    n_launch_inst = (int64_t)G.bM.size();
                    // as many parts again as the blocks need to fill the same waves
                    const int64_t waves = n_k >= (1 << 20) ? 4 : 1;
                    const int64_t want = std::max<int64_t>(2, (148 * 8 * waves + n_launch_inst - 1) / n_launch_inst);
                    const int64_t parts = std::min<int64_t>(want, d.n_khi);
                    d.khi_per_part = (int32_t)((d.n_khi + parts - 1) / parts);
                    d.ksplit = (int32_t)((d.n_khi + d.khi_per_part - 1) / d.khi_per_part);
                }
            }
            if (d.ksplit > 1 && d.n_out % JET_SPLITK_G == 0 && d.n_out <= (1 << 16)) {
                std::vector<int64_t> eA(d.n_out), eB(d.n_out);
                for (int64_t e = 0; e < d.n_out; ++e) {
                    int64_t r = e / ncols, c = e - r * ncols, oa = colA[c], ob = colB[c];
                    for (int j = 0; j < d.row_rank; ++j) {
                        const int64_t dg = r % d.row_dim[j];
                        r /= d.row_dim[j];
                        oa += dg * d.row_sA[j];
                        ob += dg * d.row_sB[j];
                    }
                    eA[e] = oa;
                    eB[e] = ob;
                }
                for (int pat : {2, 4, 18, 20, 1, 8}) {
                    const bool bf = pat & 16;
                    const int nf = pat & 15;   // values of the fastest side
                    bool ok = true;
                    for (int64_t e = 0; ok && e < d.n_out; ++e) {
                        const int64_t g0 = e - e % JET_SPLITK_G, j = e - g0;
                        const int64_t fast = g0 + j % nf, slow = g0 + nf * (j / nf);
                        ok = bf ? (eB[e] == eB[fast] && eA[e] == eA[slow]) : (eA[e] == eA[fast] && eB[e] == eB[slow]);
                    }
                    if (ok) {
                        d.splitk_na = pat;
                        break;
                    }
                }
            }
            // 2 x 2 block dot products whose operands order the inner entries
            // differently (B's entries of 32 consecutive q not adjacent): B is read in
            // its own order (kB sorted by offset, qB each entry's q) and staged in
            // shared memory, so that both operands' warp loads cover whole lines
            std::vector<int32_t> qB;
            if (d.splitk_na == 65 && !fp64 && nklo >= 64) {
                bool adjacent = true;
                for (int64_t q = 1; q < 32 && adjacent; ++q) adjacent = kB[q] == kB[0] + q;
                if (!adjacent) {
                    std::vector<int32_t> js(nklo);
                    for (int64_t j = 0; j < nklo; ++j) js[j] = (int32_t)j;
                    std::stable_sort(js.begin(), js.end(), [&](int32_t x, int32_t y) { return kB[x] < kB[y]; });
                    std::vector<int32_t> kB2(nklo);
                    qB.resize(nklo);
                    for (int64_t j = 0; j < nklo; ++j) {
                        kB2[j] = kB[js[j]];
                        qB[j] = js[j];
                    }
                    kB.swap(kB2);
                    d.splitk_na = 66;
                }
            }
            size_t off_colA = blob.put_i32(colA), off_colB = blob.put_i32(colB);
            size_t off_kA = blob.put_i32(kA), off_kB = blob.put_i32(kB);
            size_t off_qB = qB.empty() ? 0 : blob.put_i32(qB);
            size_t off_pa = blob.put_ptrs(pa), off_pb = blob.put_ptrs(pb), off_pc = blob.put_ptrs(pc);
            size_t off_itab = blk_itab.empty() ? 0 : blob.put_i32(blk_itab);
            if (!blk_itab.empty()) d.n_inst = (int32_t)n_launch_inst;   // the kernel's blocks
            // bytes the launch must move: every distinct operand instance once (an
            // instance block reads a shared operand once for all its pairs)
            double op_bytes = bytes;
            if (!blk_itab.empty()) {
                const NodeInfo &N = node[v];
                op_bytes = (double)es * ((double)node[N.a].n_inst * (double)node[N.a].view.size +
                                         (double)node[N.b].n_inst * (double)node[N.b].view.size +
                                         (double)n_inst * (double)Cv.size);
            }
            size_t part_off = 0, part_bytes = 0;
            if (d.ksplit > 1) {
                part_bytes = (size_t)n_inst * d.ksplit * d.n_out * es;
                part_off = arena.alloc(part_bytes);
                scratch.push_back(part_off);
                scratch_bytes.push_back(part_bytes);
            }
            size_t so = blob.reserve(sizeof(DirectArgs));
            std::memcpy(blob.bytes.data() + so, &d, sizeof d);
            blob.patch_field(so, offsetof(DirectArgs, ptrA), BASE_BLOB, (int64_t)off_pa);
            blob.patch_field(so, offsetof(DirectArgs, ptrB), BASE_BLOB, (int64_t)off_pb);
            blob.patch_field(so, offsetof(DirectArgs, ptrC), BASE_BLOB, (int64_t)off_pc);
            blob.patch_field(so, offsetof(DirectArgs, colA), BASE_BLOB, (int64_t)off_colA);
            blob.patch_field(so, offsetof(DirectArgs, colB), BASE_BLOB, (int64_t)off_colB);
            blob.patch_field(so, offsetof(DirectArgs, kA), BASE_BLOB, (int64_t)off_kA);
            blob.patch_field(so, offsetof(DirectArgs, kB), BASE_BLOB, (int64_t)off_kB);
            if (d.ksplit > 1) blob.patch_field(so, offsetof(DirectArgs, partials), BASE_ARENA, (int64_t)part_off);
            if (!blk_itab.empty()) blob.patch_field(so, offsetof(DirectArgs, itab), BASE_BLOB, (int64_t)off_itab);
            if (!qB.empty()) blob.patch_field(so, offsetof(DirectArgs, qB), BASE_BLOB, (int64_t)off_qB);
            Op op;
            op.kind = OpKind::Direct;
            op.node = v;
            op.n_inst = n_inst;
            op.args_off = so;
            op.args_bytes = sizeof(DirectArgs);
            op.flop = flop;
            op.bytes = op_bytes;
            op.variant = fp64 ? 1 : 0;
            bool pow2 = true;
            for (int j = 0; j < d.row_rank; ++j) pow2 = pow2 && (d.row_dim[j] & (d.row_dim[j] - 1)) == 0;
            for (int j = 0; j < d.khi_rank; ++j) pow2 = pow2 && (d.khi_dim[j] & (d.khi_dim[j] - 1)) == 0;
            if (pow2) op.variant |= 4;
            op.block = 256;
            if (d.ksplit > 1) {
                op.grid_x = d.ksplit;
                op.grid_y = (int32_t)((d.n_out + JET_SPLITK_G - 1) / JET_SPLITK_G);
                op.grid_z = (int32_t)std::min<int64_t>(n_launch_inst, 65535);
                op.variant |= 2 | (d.splitk_na << 8);   // the outer-product factor, for the launch records
            } else {
                int64_t blocks = (d.n_out + 255) / 256;
                int64_t gy = std::min<int64_t>(n_inst, 65535);
                int64_t gx = std::min<int64_t>(blocks, std::max<int64_t>(1, 148 * 16 / std::max<int64_t>(1, gy)));
                op.grid_x = (int32_t)std::max<int64_t>(gx, 1);
                op.grid_y = (int32_t)gy;
            }
            op.smem = (int32_t)(8 * ncols + 8 * nklo);
            if (d.splitk_na == 66)   // tables kA, kB, qB; two buffers of 2 B vectors, one padding entry per 32
                op.smem = (int32_t)(((3 * nklo * 4 + 15) & ~(int64_t)15) + 2 * 2 * (nklo + (nklo >> 5)) * 8);
            P.ops.push_back(op);
            if (d.ksplit > 1) {
                SplitKReduceArgs r;
                std::memset(&r, 0, sizeof r);
                r.n_out = d.n_out;
                r.n_inst = (int32_t)n_inst;   // partials are per node instance in every form
                r.ksplit = d.ksplit;
                size_t ro = blob.reserve(sizeof r);
                std::memcpy(blob.bytes.data() + ro, &r, sizeof r);
                blob.patch_field(ro, offsetof(SplitKReduceArgs, partials), BASE_ARENA, (int64_t)part_off);
                blob.patch_field(ro, offsetof(SplitKReduceArgs, ptrC), BASE_BLOB, (int64_t)off_pc);
                Op rop;
                rop.kind = OpKind::SplitKReduce;
                rop.node = v;
                rop.n_inst = n_inst;
                rop.args_off = ro;
                rop.args_bytes = sizeof r;
                rop.variant = fp64 ? 1 : 0;
                int64_t tot = d.n_out * n_inst;
                rop.grid_x = (int32_t)std::min<int64_t>((tot + 255) / 256, 65535);
                P.ops.push_back(rop);
            }
    };

    // group: instance i pairs node v's child instances ia[i], ib[i] (the forward
    // contraction of v), so instances that share an operand instance may run as
    // one block; the adjoint sweep's launches pair other operands and pass false
    auto emit_apply = [&](int32_t v, const View &VA, const View &VB, const View &Cv, const std::vector<int64_t> &K,
                          bool a_big, int64_t n_inst, const std::vector<std::pair<int32_t, int64_t>> &pa,
                          const std::vector<std::pair<int32_t, int64_t>> &pb,
                          const std::vector<std::pair<int32_t, int64_t>> &pc, double flop, double bytes,
                          bool group = true) {
        const View &VL = a_big ? VA : VB, &VS = a_big ? VB : VA;
        const std::vector<int64_t> fs = free_of(VS, K), fl = free_of(VL, K);
        auto stride = [&](const View &V, int64_t l) {
            const int p = find_pos(V.labels, l);
            return p < 0 ? (int64_t)0 : V.strides[p];
        };
        ApplyArgs d;
        std::memset(&d, 0, sizeof d);
        const int64_t nk = dimprod(K), nf0 = std::max<int64_t>(1, dimprod(fs));
        // Instances that apply several small operands to one large operand
        // instance run as one application of those small operands side by side
        // (free entry l nf + f is small instance l's entry f): the large operand
        // is read once for all of them.  Taken when every large instance pairs
        // with the same number of small ones, their entries and outputs lie at
        // the same element distances from the first pair's, and the CUDA-core
        // form held in registers takes the wider operand (each output's sum is
        // the same sequence of multiply-adds, so the values do not change).
        int64_t nB = 1;
        std::vector<int64_t> dB, dC;   // per small slot l: element offset of its entries, of its outputs
        std::vector<std::pair<int32_t, int64_t>> gl, gs, gc;   // per large instance: the l = 0 pair's refs
        {
            const std::vector<int32_t> &il = a_big ? node[v].ia : node[v].ib, &is = a_big ? node[v].ib : node[v].ia;
            const std::vector<std::pair<int32_t, int64_t>> &pl = a_big ? pa : pb, &ps = a_big ? pb : pa;
            std::map<int32_t, std::vector<std::pair<int32_t, int32_t>>> by;
            if ((int64_t)il.size() == n_inst)
                for (int64_t i = 0; i < n_inst; ++i) by[il[i]].push_back({is[i], (int32_t)i});
            bool ok = group && net.opt.gemm_group && !fp64 && n_inst > 1 && !by.empty() && by.size() < (size_t)n_inst;
            int64_t nb = 0;
            for (auto &kv : by) {
                if (!ok) break;
                auto &lst = kv.second;
                std::sort(lst.begin(), lst.end());
                if (nb == 0) nb = (int64_t)lst.size();
                if ((int64_t)lst.size() != nb) {
                    ok = false;
                    break;
                }
                std::vector<int64_t> b_off, c_off;
                for (auto &e : lst) {
                    const auto &rb = ps[e.second], &rc = pc[e.second], &rb0 = ps[lst[0].second], &rc0 = pc[lst[0].second];
                    if (rb.first != rb0.first || rc.first != rc0.first) ok = false;
                    b_off.push_back((rb.second - rb0.second) / es);
                    c_off.push_back((rc.second - rc0.second) / es);
                }
                if (dB.empty()) {
                    dB = b_off;
                    dC = c_off;
                } else if (b_off != dB || c_off != dC) {
                    ok = false;
                }
                gl.push_back(pl[lst[0].second]);
                gs.push_back(ps[lst[0].second]);
                gc.push_back(pc[lst[0].second]);
            }
            int64_t nkt = 1;
            while (nkt < nk) nkt *= 2;
            ok = ok && nb > 1 && apply_tc_groups(nk, nf0) == 0 && nk <= JET_APPLY_HOLDK && nkt * nf0 * nb <= JET_APPLY_MAXB &&
                 nf0 * nb <= JET_APPLY_MAXF;
            if (ok) nB = nb;
        }
        const int64_t nf = nf0 * nB;
        d.nk = (int32_t)nk;
        d.nf = (int32_t)nf;
        d.nk_tmpl = 1;
        while (d.nk_tmpl < d.nk) d.nk_tmpl *= 2;
        if (!(d.nk <= (fp64 ? 16 : JET_APPLY_HOLDK) && d.nk_tmpl * d.nf <= JET_APPLY_MAXB)) {   // streamed form
            d.nf_tmpl = 1;   // register chunk of free entries; above 4: lane groups (16 per pass)
            while (d.nf_tmpl < d.nf && d.nf_tmpl < 4) d.nf_tmpl *= 2;
            if (d.nf > 4) d.nf_tmpl = 16;
        }
        // summed entries: mixed radix over K, the label of smallest stride in A
        // fastest; B's free entries: the label of smallest stride in C fastest
        std::vector<int64_t> Ks = K, Fs = fs;
        std::stable_sort(Ks.begin(), Ks.end(), [&](int64_t x, int64_t y) { return stride(VL, x) > stride(VL, y); });
        std::stable_sort(Fs.begin(), Fs.end(), [&](int64_t x, int64_t y) { return stride(Cv, x) > stride(Cv, y); });
        for (int64_t q = 0; q < nk; ++q) {
            int64_t r = q;
            for (int j = (int)Ks.size() - 1; j >= 0; --j) {
                const int64_t dm = net.labels.at(Ks[j]).dim, dg = r % dm;
                r /= dm;
                d.kA[q] += dg * stride(VL, Ks[j]);
                d.bK[q] += dg * stride(VS, Ks[j]);
            }
        }
        for (int64_t f = 0; f < nf; ++f) {
            int64_t r = f % nf0;
            for (int j = (int)Fs.size() - 1; j >= 0; --j) {
                const int64_t dm = net.labels.at(Fs[j]).dim, dg = r % dm;
                r /= dm;
                d.cF[f] += dg * stride(Cv, Fs[j]);
                d.bF[f] += dg * stride(VS, Fs[j]);
            }
            if (nB > 1) {   // small slot f / nf0: its entries and outputs
                d.cF[f] += dC[f / nf0];
                d.bF[f] += dB[f / nf0];
            }
        }
        // fibers: A's free labels, smallest A stride decoded first
        std::vector<int64_t> rl = fl;
        std::stable_sort(rl.begin(), rl.end(), [&](int64_t x, int64_t y) { return stride(VL, x) < stride(VL, y); });
        d.rank = (int32_t)rl.size();
        d.n_fib = 1;
        bool pow2 = true;
        int32_t bit = 0;
        for (int j = 0; j < d.rank; ++j) {
            d.dim[j] = net.labels.at(rl[j]).dim;
            d.sA[j] = stride(VL, rl[j]);
            d.sC[j] = stride(Cv, rl[j]);
            d.n_fib *= d.dim[j];
            pow2 = pow2 && (d.dim[j] & (d.dim[j] - 1)) == 0;
            d.shift[j] = bit;
            while (((int64_t)1 << bit) < d.n_fib) ++bit;   // power-of-two dims: log2 of the running product
        }
        const int64_t n_launch = nB > 1 ? (int64_t)gl.size() : n_inst;   // one unit per large instance
        d.n_inst = (int32_t)n_launch;
        d.tc_terms = net.opt.precision == JET_PREC_TF32 ? 1 : 3;
        d.tc_f16 = net.opt.precision == JET_PREC_FP16X3 ? 1 : 0;   // (tensor-core form: FP16 hi + lo parts)
        size_t off_pl = blob.put_ptrs(nB > 1 ? gl : (a_big ? pa : pb)), off_ps = blob.put_ptrs(nB > 1 ? gs : (a_big ? pb : pa));
        size_t off_pc = blob.put_ptrs(nB > 1 ? gc : pc);
        size_t so = blob.reserve(sizeof d);
        std::memcpy(blob.bytes.data() + so, &d, sizeof d);
        blob.patch_field(so, offsetof(ApplyArgs, ptrA), BASE_BLOB, (int64_t)off_pl);
        blob.patch_field(so, offsetof(ApplyArgs, ptrB), BASE_BLOB, (int64_t)off_ps);
        blob.patch_field(so, offsetof(ApplyArgs, ptrC), BASE_BLOB, (int64_t)off_pc);
        Op op;
        op.kind = OpKind::Apply;
        op.node = v;
        op.n_inst = n_inst;
        op.args_off = so;
        op.args_bytes = sizeof d;
        op.flop = flop;
        // grouped: every large instance read once, every small one and every output once
        op.bytes = nB > 1 ? (double)es * ((double)n_launch * VL.size + (double)n_inst * (VS.size + Cv.size)) : bytes;
        op.variant = (fp64 ? 1 : 0) | (pow2 ? 4 : 0);
        // the tensor-core form or a CUDA-core one, where both take the shape
        const int G_def = apply_tc_groups(nk, nf), G_any = apply_tc_groups_any(nk, nf);
        const bool cuda_ok = (d.nk <= (fp64 ? 16 : JET_APPLY_HOLDK) && d.nk_tmpl * d.nf <= JET_APPLY_MAXB &&
                              d.nf <= JET_APPLY_MAXF) ||
                             (!fp64 && d.nk <= JET_APPLY_MAXK && d.nf <= JET_APPLY_STREAMF &&
                              (d.nf <= 4 || d.nk * ((d.nf + 15) / 16 * 16) <= JET_APPLY_STREAMB));
        int G = G_def;
        if (group && G_any > 0 && cuda_ok && nB == 1) {   // (forward launches only: the tuner's)
            G = tuned(v, 1, G_def > 0) ? G_any : 0;
            P.tunables.push_back({v, 1, G > 0 ? 1 : 0, sig_of(1, {nk, nf, d.n_fib, n_inst, (int64_t)pow2})});
        }
        if (G) {
            // tensor-core form: one CTA per SM over contiguous ranges of (instance,
            // G tiles of 128 fibers); the status word takes its wait time-outs
            blob.patch_field(so, offsetof(ApplyArgs, status), BASE_STATUS, 0);
            const int64_t units = n_launch * (((d.n_fib + 127) / 128 + G - 1) / G);
            op.variant |= 8;
            op.block = 128 * G;
            op.smem = jet_apply_tc_smem(G, (int)nk, (int)nf, d.tc_f16);
            op.grid_x = (int32_t)std::min<int64_t>(148, units);
            op.grid_y = 1;
            P.ops.push_back(op);
            return;
        }
        // 256-thread blocks; complex64 threads take two fibers, complex128 one
        op.block = 256;
        const int64_t gy = std::min<int64_t>(n_launch, 65535);
        const int64_t per_block = fp64 ? 256 : 512;
        const int64_t blocks = (d.n_fib + per_block - 1) / per_block;
        const int64_t per_sm = 8;
        op.grid_y = (int32_t)gy;
        op.grid_x = (int32_t)std::max<int64_t>(1, std::min<int64_t>(blocks, std::max<int64_t>(1, 148 * per_sm / gy)));
        P.ops.push_back(op);
    };

    // GEMM route, tensor cores: the instance blocks of node pv (full products of
    // M-side and N-side child instance groups when every block has the same shape
    // and (nearly) no child instance is split twice; else one block per instance).
    // record: add the choice to the tuner's list (the node's own emission)
    auto gemm_groups_of = [&](int32_t pv, bool record) {
        const NodeInfo &Q = node[pv];
        const int32_t qM = Q.a_is_m ? Q.a : Q.b, qN = Q.a_is_m ? Q.b : Q.a;
        const std::vector<int32_t> &iM = Q.a_is_m ? Q.ia : Q.ib, &iN = Q.a_is_m ? Q.ib : Q.ia;
        const View &WM = node[qM].view, &WN = node[qN].view;
        GemmGroups G, gm, gn;
        const bool okm = group_instances(iM, iN, true, gm);
        const bool okn = group_instances(iM, iN, false, gn);
        const double vm = (double)WM.size, vn = (double)WN.size;
        const double cm = okm ? gm.dup * vn : 1e300, cn = okn ? gn.dup * vm : 1e300;
        const double budget = 0.25 * ((double)node[qM].n_inst * vm + (double)node[qN].n_inst * vn);
        const bool can_merge = (okm || okn) && std::min(cm, cn) <= budget &&
                               (okm && cm <= cn ? gm : gn).bM.size() < (size_t)Q.n_inst;
        const bool merge = can_merge && tuned(pv, 0, net.opt.gemm_group != 0);
        if (can_merge && record)
            P.tunables.push_back({pv, 0, merge ? 1 : 0,
                                  sig_of(0, {dimprod(Q.K), dimprod(Q.fM), dimprod(Q.fN), Q.n_inst, node[qM].n_inst,
                                             node[qN].n_inst, WM.size, WN.size})});
        if (merge) {
            G = okm && cm <= cn ? gm : gn;
        } else {   // one block per instance; every child instance one group
            for (int64_t j = 0; j < node[qM].n_inst; ++j) G.gM.push_back({(int32_t)j});
            for (int64_t j = 0; j < node[qN].n_inst; ++j) G.gN.push_back({(int32_t)j});
            G.bM.assign(iM.begin(), iM.end());
            G.bN.assign(iN.begin(), iN.end());
        }
        return G;
    };

    // ---- pass 2, launch order: arena offsets, pointer tables, launches
    std::vector<char> emitted(n_nodes, 0);
    for (int32_t i = 0; i < n_leaves; ++i) emitted[i] = 1;
    for (int32_t v : order) {
        if (skip[v]) continue;   // a kept result stands for this sub-tree
        emitted[v] = 1;          // (its launches precede every later node's)
        NodeInfo &N = node[v];
        const int32_t a = N.a, b = N.b;
        const NodeInfo &NA = node[a], &NB = node[b];
        const View &VA = NA.view, &VB = NB.view;
        const std::vector<int64_t> &K = N.K, &fa = N.fa, &fb = N.fb;
        const int64_t nK = dimprod(K), nFa = dimprod(fa), nFb = dimprod(fb);
        const bool use_gemm = N.use_gemm, a_big = N.a_big;
        if (!N.small || (!batch_nodes.empty() && node[batch_nodes.front()].depth != N.depth)) flush_batch();
        if (!N.small) flush_chain();   // the chain's levels run before this node's launches

        // fused split: this GEMM's epilogue writes its parent GEMM's FP16 planes
        // for this node's side (the parent's instance blocks and row order decide
        // the layout), allocated in place of the complex64 output
        std::vector<int64_t> fz_ibase;
        std::vector<int32_t> fz_pm, fz_pn;
        int64_t fz_plane_elems = 0, fz_kpad = 0, fz_rows_pad = 0;
        size_t fz_planes_bytes = 0, fz_scales_bytes = 0;
        N.fz_ok = false;
        const bool kept_v = std::find(P.kept_fill.begin(), P.kept_fill.end(), v) != P.kept_fill.end();
        if (N.fuse && use_gemm && tc_mode && !grad && !kept_v && parent[v] >= 0 && !skip[parent[v]]) {
            const int32_t pv = parent[v], sib = sibling[v];
            NodeInfo &Q = node[pv];
            bool ok = Q.use_gemm && !Q.small && std::find(P.kept_fill.begin(), P.kept_fill.end(), pv) == P.kept_fill.end();
            // one fused operand per parent: the larger one (child a on a tie)
            const double sz = (double)N.n_inst * N.view.size, szs = (double)node[sib].n_inst * node[sib].view.size;
            if (ok && node[sib].fuse && (szs > sz || (szs == sz && Q.a == sib))) ok = false;
            const bool vM = (Q.a_is_m ? Q.a : Q.b) == v;
            const std::vector<int64_t> &fp = vM ? Q.fM : Q.fN;
            const size_t nmf = N.fM.size() - N.fz_mk.size(), nnf = N.fN.size() - N.fz_nk.size();
            std::vector<int64_t> mf(N.fM.begin(), N.fM.begin() + nmf), nf(N.fN.begin(), N.fN.begin() + nnf);
            if (ok) {   // the parent's rows are this node's m_f and n_f labels, its summed labels m_k and n_k
                ok = fp.size() == nmf + nnf && Q.K.size() == N.fz_mk.size() + N.fz_nk.size();
                for (int64_t l : mf) ok = ok && find_pos(fp, l) >= 0;
                for (int64_t l : nf) ok = ok && find_pos(fp, l) >= 0;
                for (int64_t l : N.fz_mk) ok = ok && find_pos(Q.K, l) >= 0;
                for (int64_t l : N.fz_nk) ok = ok && find_pos(Q.K, l) >= 0;
            }
            const int64_t kblk = tc_k_block(net.opt.precision), T = tc_tile(), NP = tc_planes(net.opt.precision);
            const int64_t Kp = dimprod(Q.K);
            ok = ok && Kp % 64 == 0 && Kp % kblk == 0 && (dimprod(N.fz_nk) == 4 || dimprod(N.fz_nk) == 8) &&
                 Kp < ((int64_t)1 << 16);
            if (ok) {   // this node's own tiles: whole (rows in 32s per instance, columns in 64s)
                const GemmGroups Gv = gemm_groups_of(v, false);
                const int64_t mr = Gv.nA * dimprod(N.fM), nr = Gv.nB * dimprod(N.fN);
                ok = mr % T == 0 && nr % 64 == 0 && dimprod(N.fM) % 32 == 0 && dimprod(N.fN) % 16 == 0;
            }
            if (ok) {
                const GemmGroups Gp = gemm_groups_of(pv, false);
                const std::vector<std::vector<int32_t>> &groups = vM ? Gp.gM : Gp.gN;
                const int64_t per = vM ? Gp.nA : Gp.nB, rows = dimprod(fp);
                fz_rows_pad = (per * rows + T - 1) / T * T;
                fz_kpad = Kp;
                fz_plane_elems = fz_rows_pad * fz_kpad;
                fz_ibase.assign((size_t)N.n_inst * 2, -1);
                const int64_t n_ch = fz_kpad / 64;
                for (size_t g = 0; g < groups.size() && ok; ++g)
                    for (size_t j = 0; j < groups[g].size() && ok; ++j) {
                        const int32_t i = groups[g][j];
                        if (i < 0 || i >= N.n_inst || fz_ibase[2 * (size_t)i] >= 0) {
                            ok = false;   // each instance in exactly one block group
                            break;
                        }
                        fz_ibase[2 * (size_t)i] = (int64_t)g * NP * fz_plane_elems + (int64_t)j * rows * fz_kpad;
                        fz_ibase[2 * (size_t)i + 1] = (int64_t)g * n_ch * fz_rows_pad + (int64_t)j * rows;
                    }
                for (size_t i = 0; i < (size_t)N.n_inst && ok; ++i) ok = fz_ibase[2 * i] >= 0;
                if (ok) {
                    fz_planes_bytes = (size_t)groups.size() * NP * fz_plane_elems * 2;
                    fz_scales_bytes = (size_t)groups.size() * n_ch * fz_rows_pad * 4;
                    // parent-row contributions of the m_f and n_f digits (mixed radix,
                    // last label fastest, in this node's and in the parent's orders)
                    auto contrib = [&](const std::vector<int64_t> &ls, std::vector<int32_t> &tab) {
                        const int64_t n = dimprod(ls);
                        tab.assign((size_t)n, 0);
                        for (int64_t x = 0; x < n; ++x) {
                            int64_t r = x, off = 0;
                            for (int j = (int)ls.size() - 1; j >= 0; --j) {
                                const int64_t dm = net.labels.at(ls[j]).dim, dg = r % dm;
                                r /= dm;
                                int64_t st = 1;
                                for (size_t q = (size_t)find_pos(fp, ls[j]) + 1; q < fp.size(); ++q) st *= net.labels.at(fp[q]).dim;
                                off += dg * st;
                            }
                            tab[(size_t)x] = (int32_t)off;
                        }
                    };
                    contrib(mf, fz_pm);
                    contrib(nf, fz_pn);
                    N.fz_ok = true;
                    Q.fz_kappa = N.fz_mk;
                    Q.fz_kappa.insert(Q.fz_kappa.end(), N.fz_nk.begin(), N.fz_nk.end());
                }
            }
        }

        // dot epilogue: the parent's dot products of this output with its sibling
        // (already computed: it launched before this node) are formed in this
        // GEMM's epilogue, per tile, into partials in place of the output
        // (dot blocks: up to two instances of this node that pair the same sibling
        // instances, up to two; per block dot_pr holds {c0, c1, p00, p01, p10, p11,
        // 0, 0}, c1 = -1 for none, p_km the parent instance of (c_k, sibling m) or
        // -1, and dot_a its two sibling instances)
        std::vector<std::pair<int32_t, int64_t>> dot_a;
        std::vector<int32_t> dot_pr, dot_xn;
        std::vector<int64_t> dot_sm;
        int32_t dot_lcol = 0;
        N.dot_ok = false;
        if (N.dot && use_gemm && tc_mode && dimprod(N.K) <= tc_dot_max_k(net.opt.precision) && !grad && !kept_v && !N.fz_ok &&
            parent[v] >= 0 && !skip[parent[v]]) {
            const int32_t pv = parent[v], sb = sibling[v];
            const NodeInfo &Q = node[pv], &S_ = node[sb];
            const int64_t Mv = dimprod(N.fM), Nv = dimprod(N.fN);
            bool ok = emitted[sb] && !Q.use_gemm && Q.view.size == 1 && Mv % 128 == 0 && Nv % 128 == 0 &&
                      Nv <= INT32_MAX && S_.view.size <= INT32_MAX &&
                      std::find(P.kept_fill.begin(), P.kept_fill.end(), pv) == P.kept_fill.end();
            for (int64_t l : N.view.labels) ok = ok && find_pos(S_.view.labels, l) >= 0 &&
                                                 (net.labels.at(l).dim & (net.labels.at(l).dim - 1)) == 0;
            ok = ok && S_.view.labels.size() == N.view.labels.size();
            if (ok) {
                // each instance's (sibling instance, parent instance) pairs, at most two
                std::vector<std::vector<std::pair<int32_t, int32_t>>> sl((size_t)N.n_inst);
                const bool v_is_a = Q.a == v;
                for (int64_t i = 0; i < Q.n_inst && ok; ++i) {
                    const int32_t vi = v_is_a ? Q.ia[i] : Q.ib[i], si = v_is_a ? Q.ib[i] : Q.ia[i];
                    if (vi < 0 || vi >= N.n_inst || sl[(size_t)vi].size() >= 2) {
                        ok = false;   // at most two parent instances per instance of this node
                        break;
                    }
                    sl[(size_t)vi].push_back({si, (int32_t)i});
                }
                // instances with equal sibling sets, two to a block (in instance order)
                std::map<std::vector<int32_t>, std::vector<int32_t>> by_set;
                for (int32_t vi = 0; ok && vi < (int32_t)N.n_inst; ++vi) {
                    auto &x = sl[(size_t)vi];
                    if (x.empty()) continue;   // no product to form
                    std::sort(x.begin(), x.end());
                    std::vector<int32_t> key;
                    for (const auto &pq : x) key.push_back(pq.first);
                    by_set[key].push_back(vi);
                }
                for (const auto &kv : by_set) {
                    const auto &key = kv.first;
                    const auto &cs = kv.second;
                    for (size_t q = 0; q < cs.size(); q += 2) {
                        const int32_t c0 = cs[q], c1 = q + 1 < cs.size() ? cs[q + 1] : -1;
                        auto pr = [&](int32_t c, size_t m) { return c >= 0 && m < key.size() ? sl[(size_t)c][m].second : -1; };
                        const int32_t row[8] = {c0, c1, pr(c0, 0), pr(c0, 1), pr(c1, 0), pr(c1, 1), 0, 0};
                        dot_pr.insert(dot_pr.end(), row, row + 8);
                        for (size_t m = 0; m < 2; ++m) dot_a.push_back(base_ref(sb, key[m < key.size() ? m : 0]));
                    }
                }
                ok = ok && !dot_pr.empty() && dot_pr.size() / 8 <= INT32_MAX;
            }
            auto sstride = [&](int64_t l) { return S_.view.strides[find_pos(S_.view.labels, l)]; };
            if (ok) {   // the sibling's offset of a row: per bit; of a column: by table
                int bit = 0;
                for (size_t q = N.fM.size(); q-- > 0 && ok;) {
                    const int64_t d = net.labels.at(N.fM[q]).dim;
                    for (int64_t w = 1; w < d; w *= 2) {
                        if (bit >= JET_MAXR) {
                            ok = false;
                            break;
                        }
                        dot_sm.push_back(w * sstride(N.fM[q]));
                        ++bit;
                    }
                }
                dot_xn.assign((size_t)Nv, 0);
                for (int64_t n = 0; n < Nv && ok; ++n) {
                    int64_t r = n, off = 0;
                    for (size_t q = N.fN.size(); q-- > 0;) {
                        const int64_t d = net.labels.at(N.fN[q]).dim;
                        off += (r % d) * sstride(N.fN[q]);
                        r /= d;
                    }
                    dot_xn[(size_t)n] = (int32_t)off;
                }
            }
            if (ok) {
                N.dot_ok = true;
                N.dot_tiles = (int32_t)((Mv / 128) * (Nv / 128));
                // the epilogue copies pairs of values adjacent in the sibling: along
                // the side that holds its stride-1 label (the lowest digit of the
                // row or column index), all other offsets even, every sibling
                // instance 16-byte aligned (the buffers are: the offsets decide)
                if (Nv > 1 && dot_xn[1] == 1) dot_lcol = 1;
                else if (!dot_sm.empty() && dot_sm[0] == 1) dot_lcol = 0;
                else N.dot_ok = false;
                for (size_t q = 0; q < dot_sm.size(); ++q)
                    if (!(dot_lcol == 0 && q == 0) && dot_sm[q] % 2 != 0) N.dot_ok = false;
                for (size_t n = 0; n < dot_xn.size(); ++n) {
                    if ((dot_lcol == 0 || n % 2 == 0) && dot_xn[n] % 2 != 0) N.dot_ok = false;
                    if (dot_lcol == 1 && n % 2 == 1 && dot_xn[n] != dot_xn[n - 1] + 1) N.dot_ok = false;
                }
                for (const auto &r : dot_a)
                    if (r.second % 16 != 0) N.dot_ok = false;
                if (!N.dot_ok) N.dot_tiles = 0;
            }
        }

        // arena buffer for all instances (a kept result: its slot in the pool)
        size_t nbytes = N.fz_ok ? fz_planes_bytes + fz_scales_bytes : (size_t)N.n_inst * N.view.size * es;
        if (N.dot_ok) nbytes = (size_t)node[parent[v]].n_inst * N.dot_tiles * 16;   // complex128 partials
        N.alloc_bytes = nbytes;
        if (kept_v) {
            N.base = BASE_KEPT;
            N.buf_off = (int64_t)net.kept.at(v).off;
        } else {
            N.buf_off = (int64_t)arena.alloc(nbytes);
            arena.log.back().node = v;
            N.base = BASE_ARENA;
            if (N.fz_ok) N.fz_scales_off = (size_t)N.buf_off + fz_planes_bytes;
        }

        // per-instance pointer tables
        std::vector<std::pair<int32_t, int64_t>> pa, pb, pc;
        for (int64_t i = 0; i < N.n_inst; ++i) {
            pa.push_back(base_ref(a, N.ia[i]));
            pb.push_back(base_ref(b, N.ib[i]));
            pc.push_back({N.base, N.buf_off + i * N.view.size * es});
        }
        std::vector<int64_t> un = VA.labels;
        for (int64_t l : fb) un.push_back(l);
        const double flop = 8.0 * (double)dimprod(un) * (double)N.n_inst;
        const double bytes = (double)es * (double)N.n_inst * (double)(VA.size + VB.size + N.view.size);
        P.flop_executed += flop;
        P.bytes_executed += bytes;
        P.n_instances += N.n_inst;

        if (N.small) {
            ++P.n_direct;
            add_small_task(VA, VB, N.view, K, a_big, pa, pb, pc, N.n_inst);
            batch_nodes.push_back(v);
            batch_flop += flop;
            batch_bytes += bytes;
            continue;   // children are released when the batch is issued
        }

        std::vector<size_t> scratch;   // arena scratch freed after this node
        std::vector<size_t> scratch_bytes;

        // ------------------------------------------------ dot products formed by a child's epilogue
        const int32_t dot_child = node[a].dot_ok ? a : node[b].dot_ok ? b : -1;
        if (dot_child >= 0) {
            ++P.n_direct;
            SplitKReduceArgs r;
            std::memset(&r, 0, sizeof r);
            r.n_out = 1;
            r.n_inst = (int32_t)N.n_inst;
            r.ksplit = node[dot_child].dot_tiles;   // the child's tiles, added in tile order in FP64
            r.parts64 = 1;
            size_t ro = blob.reserve(sizeof r);
            std::memcpy(blob.bytes.data() + ro, &r, sizeof r);
            blob.patch_field(ro, offsetof(SplitKReduceArgs, partials), BASE_ARENA, node[dot_child].buf_off);
            blob.patch_field(ro, offsetof(SplitKReduceArgs, ptrC), BASE_BLOB, (int64_t)blob.put_ptrs(pc));
            Op rop;
            rop.kind = OpKind::SplitKReduce;
            rop.node = v;
            rop.n_inst = N.n_inst;
            rop.args_off = ro;
            rop.args_bytes = sizeof r;
            rop.flop = 0;
            rop.bytes = (double)N.n_inst * (double)r.ksplit * 16.0;
            rop.variant = 0;
            rop.grid_x = (int32_t)std::min<int64_t>((N.n_inst + 255) / 256, 65535);
            P.ops.push_back(rop);
        }
        // ------------------------------------------------ GEMM route (Section 3.1)
        else if (use_gemm) {
            ++P.n_gemm;
            const bool a_is_m = N.a_is_m;       // the output layout's choice (pass 1)
            const int32_t idM = a_is_m ? a : b, idN = a_is_m ? b : a;
            const View &VM = node[idM].view, &VN = node[idN].view;
            const std::vector<int64_t> &fM = N.fM, &fN = N.fN;
            const std::vector<int32_t> &instM = a_is_m ? N.ia : N.ib, &instN = a_is_m ? N.ib : N.ia;
            auto is_dense = [](const View &V) {
                int64_t s = 1;
                for (int i = (int)V.labels.size() - 1; i >= 0; --i) {
                    if (V.strides[i] != s) return false;
                    s *= V.dims[i];
                }
                return true;
            };
            auto cat = [](std::vector<int64_t> x, const std::vector<int64_t> &y) {
                x.insert(x.end(), y.begin(), y.end());
                return x;
            };
            // summed-label order: take it from an operand that is already [free, K] or [K, free]
            auto split_order = [&](const View &V, const std::vector<int64_t> &f, bool k_last) {
                std::vector<int64_t> kap;
                if (!is_dense(V) || V.labels.size() != f.size() + K.size()) return kap;
                size_t nf = f.size();
                std::vector<int64_t> head(V.labels.begin(), V.labels.begin() + (k_last ? nf : K.size()));
                std::vector<int64_t> tail(V.labels.begin() + (k_last ? nf : K.size()), V.labels.end());
                if ((k_last ? head : tail) != f) return kap;
                return k_last ? tail : head;
            };
            // the larger operand decides the summed-label order (its split is the costly one)
            const bool m_big = VM.size >= VN.size;
            // a fused child writes its planes with the summed labels in its own order
            const bool fzM = tc_mode && node[idM].fz_ok, fzN = tc_mode && node[idN].fz_ok;
            std::vector<int64_t> kappa = (fzM || fzN) ? N.fz_kappa
                                         : m_big      ? split_order(VM, fM, true)
                                                      : split_order(VN, fN, true);
            if (kappa.empty()) kappa = m_big ? split_order(VM, fM, false) : split_order(VN, fN, false);
            if (kappa.empty()) kappa = m_big ? split_order(VN, fN, true) : split_order(VM, fM, true);
            if (kappa.empty()) kappa = m_big ? split_order(VN, fN, false) : split_order(VM, fM, false);
            if (kappa.empty())
                for (int64_t l : VM.labels)
                    if (find_pos(K, l) >= 0) kappa.push_back(l);
            auto form = [&](const View &V, const std::vector<int64_t> &f) {
                if (!is_dense(V)) return -1;
                if (V.labels == cat(f, kappa)) return 1;   // [free][K]: K-major
                if (V.labels == cat(kappa, f)) return 0;   // [K][free]
                return -1;
            };
            if (tc_mode) {
                // tensor cores: gather + split each child instance once into K-major planes
                const int NP = tc_planes(net.opt.precision), eb = tc_elem_bytes(net.opt.precision);
                const int64_t kblk = tc_k_block(net.opt.precision), T = tc_tile();
                const int64_t Mv = dimprod(fM), Nv = dimprod(fN);
                // instance blocks: group the instances into full products of M-side
                // and N-side child instances when every block has the same shape and
                // (nearly) no child instance is split twice; else one block per instance
                GemmGroups G = gemm_groups_of(v, true);
                const bool grouped = !G.itab.empty();
                const int64_t m_rows = G.nA * Mv, n_rows = G.nB * Nv;
                const int64_t m_pad = (m_rows + T - 1) / T * T, n_pad = (n_rows + T - 1) / T * T;
                const int64_t k_pad = (nK + kblk - 1) / kblk * kblk;
                const bool scaled = net.opt.precision == JET_PREC_FP16X3;
                auto split_child = [&](int32_t id, const View &V, const std::vector<int64_t> &f, int64_t rows_pad,
                                       const std::vector<std::vector<int32_t>> &groups, size_t &scale_off) {
                    const int64_t n_groups = (int64_t)groups.size(), per = (int64_t)groups[0].size();
                    const int64_t ninst = n_groups * per;
                    const size_t nbytes_p = (size_t)n_groups * NP * rows_pad * k_pad * eb;
                    size_t off = arena.alloc(nbytes_p);
                    scratch.push_back(off);
                    scratch_bytes.push_back(nbytes_p);
                    scale_off = 0;
                    if (scaled) {   // one float per (group, 64-wide K chunk, row)
                        const size_t sb = (size_t)n_groups * ((k_pad + 63) / 64) * rows_pad * 4;
                        scale_off = arena.alloc(sb);
                        scratch.push_back(scale_off);
                        scratch_bytes.push_back(sb);
                    }
                    TcSplitArgs sa;
                    std::memset(&sa, 0, sizeof sa);
                    sa.rows = dimprod(f);
                    sa.k = nK;
                    sa.rows_group = rows_pad;
                    sa.k_pad = k_pad;
                    sa.n_inst = (int32_t)ninst;
                    sa.per_group = (int32_t)per;
                    sa.n_planes = NP;
                    sa.mode = net.opt.precision;
                    sa.rank_r = (int32_t)f.size();
                    sa.rank_k = (int32_t)kappa.size();
                    if (sa.rank_r > JET_MAXR || sa.rank_k > JET_MAXR) fail(JET_EINVAL, "operand rank too large");
                    // tile rows along the source's fastest row labels: the row labels in
                    // decreasing source stride (the split reads them in that order and
                    // writes each row to its plane row, p_s the labels' plane strides)
                    std::vector<int64_t> vf = f;
                    std::stable_sort(vf.begin(), vf.end(), [&](int64_t x, int64_t y) {
                        return V.strides[find_pos(V.labels, x)] > V.strides[find_pos(V.labels, y)];
                    });
                    sa.row_perm = vf != f ? 1 : 0;
                    for (int j = 0; j < sa.rank_r; ++j) {
                        const int64_t l = (sa.row_perm ? vf : f)[f.size() - 1 - j];
                        int p = find_pos(V.labels, l);
                        sa.r_dim[j] = V.dims[p];
                        sa.r_s[j] = V.strides[p];
                        int64_t ps = 1;
                        for (size_t q = (size_t)find_pos(f, l) + 1; q < f.size(); ++q) ps *= net.labels.at(f[q]).dim;
                        sa.p_s[j] = ps;
                    }
                    for (int j = 0; j < sa.rank_k; ++j) {
                        int p = find_pos(V.labels, kappa[kappa.size() - 1 - j]);
                        sa.k_dim[j] = V.dims[p];
                        sa.k_s[j] = V.strides[p];
                    }
                    {
                        int64_t best = -1, bl = -1;
                        for (size_t q = 0; q < V.labels.size(); ++q)
                            if (best < 0 || V.strides[q] < best) {
                                best = V.strides[q];
                                bl = V.labels[q];
                            }
                        sa.fast_k = find_pos(kappa, bl) >= 0 ? 1 : 0;
                    }
                    // 16-byte copies of entry pairs: the fastest summed label has stride 1
                    // and even dim, every summed dim a power of two (pairs never straddle
                    // a row's end, and even source offsets keep them 16-byte aligned)
                    {
                        bool p16 = sa.fast_k && sa.rank_k > 0 && sa.k_s[0] == 1 && sa.k_dim[0] % 2 == 0;
                        for (int j = 0; j < sa.rank_k && p16; ++j) p16 = (sa.k_dim[j] & (sa.k_dim[j] - 1)) == 0;
                        for (int j = 0; j < sa.rank_r && p16; ++j) p16 = sa.r_s[j] % 2 == 0;
                        for (int j = 1; j < sa.rank_k && p16; ++j) p16 = sa.k_s[j] % 2 == 0;
                        sa.pair16 = p16 ? 1 : 0;
                    }
                    // already [rows][K] in this order, dense, K unpadded: a pure format conversion
                    bool conv = nK == k_pad && nK % 4 == 0 && V.labels.size() == f.size() + kappa.size();
                    for (size_t q = 0; conv && q < V.labels.size(); ++q)
                        conv = V.labels[q] == (q < f.size() ? f[q] : kappa[q - f.size()]);
                    if (conv) {
                        int64_t st = 1;
                        for (int q = (int)V.labels.size() - 1; conv && q >= 0; --q) {
                            conv = V.strides[q] == st;
                            st *= V.dims[q];
                        }
                    }
                    std::vector<std::pair<int32_t, int64_t>> ps;
                    for (const auto &gr : groups)
                        for (int32_t j : gr) ps.push_back(base_ref(id, j));
                    // (16-byte copies also need every instance's base 16-byte aligned; the
                    // buffers themselves are, so the byte offsets decide)
                    for (const auto &r : ps)
                        if (r.second % 16 != 0) sa.pair16 = 0;
                    size_t o_ps = blob.put_ptrs(ps);
                    size_t so = blob.reserve(sizeof sa);
                    std::memcpy(blob.bytes.data() + so, &sa, sizeof sa);
                    blob.patch_field(so, offsetof(TcSplitArgs, ptrSrc), BASE_BLOB, (int64_t)o_ps);
                    blob.patch_field(so, offsetof(TcSplitArgs, planes), BASE_ARENA, (int64_t)off);
                    if (scaled) blob.patch_field(so, offsetof(TcSplitArgs, scales), BASE_ARENA, (int64_t)scale_off);
                    Op op;
                    op.kind = OpKind::TcSplit;
                    op.node = v;
                    op.n_inst = ninst;
                    op.args_off = so;
                    op.args_bytes = sizeof sa;
                    op.bytes = (double)ninst * (double)V.size * 8.0 + (double)n_groups * NP * rows_pad * k_pad * eb;
                    int64_t gy = std::min<int64_t>(ninst, 65535);
                    op.grid_y = (int32_t)gy;
                    const int64_t tiles = ((sa.rows + 63) / 64) * ((k_pad + 63) / 64);   // 64 x 64 tiles
                    op.grid_x = (int32_t)std::max<int64_t>(
                        1, std::min<int64_t>(tiles, std::max<int64_t>(1, 148 * 16 / gy)));
                    {
                        bool pow2 = true;
                        for (int j = 0; j < sa.rank_r; ++j) pow2 = pow2 && (sa.r_dim[j] & (sa.r_dim[j] - 1)) == 0;
                        for (int j = 0; j < sa.rank_k; ++j) pow2 = pow2 && (sa.k_dim[j] & (sa.k_dim[j] - 1)) == 0;
                        if (pow2) op.variant |= 2;
                    }
                    if (sa.pair16) op.variant |= 16;   // (for the launch records: 16-byte copies)
                    if (conv) {
                        op.variant |= 1;
                        op.grid_x = (int32_t)std::max<int64_t>(
                            1, std::min<int64_t>((sa.rows * k_pad / 4 + 255) / 256, std::max<int64_t>(1, 148 * 16 / gy)));
                    }
                    P.ops.push_back(op);
                    P.bytes_executed += op.bytes;
                    return off;
                };
                size_t sclA = 0, sclB = 0;
                // a fused child's epilogue has already written its side's planes and scales
                size_t offA = fzM ? (size_t)node[idM].buf_off : split_child(idM, VM, fM, m_pad, G.gM, sclA);
                size_t offB = fzN ? (size_t)node[idN].buf_off : split_child(idN, VN, fN, n_pad, G.gN, sclB);
                if (fzM) sclA = node[idM].fz_scales_off;
                if (fzN) sclB = node[idN].fz_scales_off;
                const int64_t n_blocks = (int64_t)G.bM.size();
                std::vector<int32_t> zA, zB;
                if ((int64_t)(G.gM.size() + G.gN.size()) * NP > INT32_MAX) fail(JET_EINVAL, "too many instances of one GEMM node");
                for (int64_t i = 0; i < n_blocks; ++i) {
                    zA.push_back(G.bM[i] * NP);
                    zB.push_back(G.bN[i] * NP);
                }
                TcGemmArgs g;
                std::memset(&g, 0, sizeof g);
                g.M = m_rows;
                g.N = n_rows;
                g.K = nK;
                g.Mi = Mv;
                g.Ni = Nv;
                g.nA = G.nA;
                g.nB = G.nB;
                auto log2_or = [](int64_t x) {
                    if (x < 1 || (x & (x - 1))) return -1;
                    int sh = 0;
                    while ((int64_t)1 << sh < x) ++sh;
                    return sh;
                };
                g.mi_shift = log2_or(Mv);
                g.ni_shift = log2_or(Nv);
                // one product per instance into one contiguous buffer, an even row
                // length (16-byte strides): C leaves through bulk tensor stores
                // C leaves through bulk tensor stores when a warp's 32 rows and a
                // 16-column group lie in one instance: every product of a block
                // (or an instance) is an (Mi x Ni) matrix in the node's buffer
                g.c_tma = ((!grouped && Nv % 2 == 0) || (grouped && Mv % 32 == 0 && Nv % 16 == 0)) &&
                                  2 * Nv <= INT32_MAX && Mv <= INT32_MAX && N.n_inst <= INT32_MAX
                              ? 1
                              : 0;
                g.c_inst = N.n_inst;
                if (N.dot_ok) {
                    g.c_tma = 0;
                    g.dot_mbits = (int32_t)dot_sm.size();
                    for (size_t q = 0; q < dot_sm.size(); ++q) g.dot_sm[q] = dot_sm[q];
                    g.dot_tiles = N.dot_tiles;
                    g.dot_lcol = dot_lcol;
                    g.dot_nblk = (int32_t)(dot_pr.size() / 8);
                }
                if (N.fz_ok) {
                    int lmk = 0, lnk = 0;
                    while (((int64_t)1 << lmk) < dimprod(N.fz_mk)) ++lmk;
                    while (((int64_t)1 << lnk) < dimprod(N.fz_nk)) ++lnk;
                    g.c_tma = 0;
                    g.fz_plane_elems = fz_plane_elems;
                    g.fz_kpad = fz_kpad;
                    g.fz_rows_pad = fz_rows_pad;
                    g.fz_lmk = lmk;
                    g.fz_lnk = lnk;
                }
                g.m_pad = m_pad;
                g.n_pad = n_pad;
                g.k_pad = k_pad;
                g.planesA_total = (int64_t)G.gM.size() * NP;
                g.planesB_total = (int64_t)G.gN.size() * NP;
                g.n_inst = (int32_t)n_blocks;
                g.mode = net.opt.precision;
                g.n_kb = (int32_t)(k_pad / kblk);
                size_t o_za = blob.put_i32(zA), o_zb = blob.put_i32(zB), o_c = blob.put_ptrs(pc);
                size_t o_it = grouped ? blob.put_i32(G.itab) : 0;
                size_t so = blob.reserve(sizeof g, 128);
                std::memcpy(blob.bytes.data() + so, &g, sizeof g);
                blob.patch_field(so, offsetof(TcGemmArgs, planesA), BASE_ARENA, (int64_t)offA);
                blob.patch_field(so, offsetof(TcGemmArgs, planesB), BASE_ARENA, (int64_t)offB);
                blob.patch_field(so, offsetof(TcGemmArgs, zA), BASE_BLOB, (int64_t)o_za);
                blob.patch_field(so, offsetof(TcGemmArgs, zB), BASE_BLOB, (int64_t)o_zb);
                blob.patch_field(so, offsetof(TcGemmArgs, ptrC), BASE_BLOB, (int64_t)o_c);
                if (grouped) blob.patch_field(so, offsetof(TcGemmArgs, itab), BASE_BLOB, (int64_t)o_it);
                if (g.c_tma) blob.patch_field(so, offsetof(TcGemmArgs, baseC), N.base, N.buf_off);
                blob.patch_field(so, offsetof(TcGemmArgs, status), BASE_STATUS, 0);
                if (scaled) {
                    blob.patch_field(so, offsetof(TcGemmArgs, scaleA), BASE_ARENA, (int64_t)sclA);
                    blob.patch_field(so, offsetof(TcGemmArgs, scaleB), BASE_ARENA, (int64_t)sclB);
                }
                if (N.dot_ok) {   // dot epilogue: this epilogue forms the parent's products
                    // each instance's place in the launch: its block and its (j, l) there
                    std::vector<int32_t> cpos((size_t)N.n_inst * 3, -1);
                    if (grouped) {
                        for (int64_t b = 0; b < n_blocks; ++b)
                            for (int32_t j = 0; j < G.nA; ++j)
                                for (int32_t l = 0; l < G.nB; ++l) {
                                    const int32_t it = G.itab[((size_t)b * G.nA + j) * G.nB + l];
                                    if (it < 0) continue;
                                    cpos[3 * (size_t)it] = (int32_t)b;
                                    cpos[3 * (size_t)it + 1] = j;
                                    cpos[3 * (size_t)it + 2] = l;
                                }
                    } else {
                        for (int64_t i = 0; i < N.n_inst; ++i) {
                            cpos[3 * (size_t)i] = (int32_t)i;
                            cpos[3 * (size_t)i + 1] = cpos[3 * (size_t)i + 2] = 0;
                        }
                    }
                    for (size_t q = 0; q < dot_pr.size(); q += 8)
                        for (int k = 0; k < 2; ++k)
                            if (dot_pr[q + k] >= 0 && cpos[3 * (size_t)dot_pr[q + k]] < 0)
                                fail(JET_EINVAL, "dot epilogue: an instance outside the GEMM's blocks");
                    const size_t o_da = blob.put_ptrs(dot_a), o_dp = blob.put_i32(dot_pr), o_dx = blob.put_i32(dot_xn);
                    const size_t o_cp = blob.put_i32(cpos);
                    blob.patch_field(so, offsetof(TcGemmArgs, dot_cpos), BASE_BLOB, (int64_t)o_cp);
                    blob.patch_field(so, offsetof(TcGemmArgs, dot_parts), BASE_ARENA, N.buf_off);
                    blob.patch_field(so, offsetof(TcGemmArgs, dot_ptrA), BASE_BLOB, (int64_t)o_da);
                    blob.patch_field(so, offsetof(TcGemmArgs, dot_pair), BASE_BLOB, (int64_t)o_dp);
                    blob.patch_field(so, offsetof(TcGemmArgs, dot_xn), BASE_BLOB, (int64_t)o_dx);
                }
                if (N.fz_ok) {   // fused split: this epilogue writes the parent's planes
                    size_t o_ib = blob.reserve(fz_ibase.size() * 8, 8);
                    std::memcpy(blob.bytes.data() + o_ib, fz_ibase.data(), fz_ibase.size() * 8);
                    const size_t o_pm = blob.put_i32(fz_pm), o_pn = blob.put_i32(fz_pn);
                    blob.patch_field(so, offsetof(TcGemmArgs, fz_planes), BASE_ARENA, N.buf_off);
                    blob.patch_field(so, offsetof(TcGemmArgs, fz_scales), BASE_ARENA, (int64_t)N.fz_scales_off);
                    blob.patch_field(so, offsetof(TcGemmArgs, fz_ibase), BASE_BLOB, (int64_t)o_ib);
                    blob.patch_field(so, offsetof(TcGemmArgs, fz_pm), BASE_BLOB, (int64_t)o_pm);
                    blob.patch_field(so, offsetof(TcGemmArgs, fz_pn), BASE_BLOB, (int64_t)o_pn);
                }
                Op op;
                op.kind = OpKind::GemmTc;
                op.node = v;
                op.n_inst = N.n_inst;
                op.args_off = so;
                op.args_bytes = sizeof g;
                op.flop = flop;
                // grouped blocks read every operand instance once per launch: the
                // bytes to move are those of the distinct operand instances
                op.bytes = grouped ? (double)es * ((double)node[idM].n_inst * VM.size + (double)node[idN].n_inst * VN.size +
                                                   (double)N.n_inst * N.view.size)
                                   : bytes;
                op.grid_x = (int32_t)(n_pad / T);
                op.grid_y = (int32_t)(m_pad / T);
                op.grid_z = (int32_t)n_blocks;   // persistent launch: the tile count only
                // 4: writes its parent's planes; 8: forms its parent's dot products
                op.variant = (grouped ? 1 : 0) | (N.fz_ok ? 4 : 0) | (N.dot_ok ? 8 : 0);
                if (N.dot_ok)   // the operand instances, the sibling's instances once, the partials
                    op.bytes = (double)es * ((double)node[idM].n_inst * VM.size + (double)node[idN].n_inst * VN.size +
                                             (double)node[sibling[v]].n_inst * node[sibling[v]].view.size) +
                               (double)N.alloc_bytes;
                P.ops.push_back(op);
            } else {
            int formM = form(VM, fM), formN = form(VN, fN);
            // operands that are neither: gather each child instance into [free, K] once
            auto permute_child = [&](int32_t id, const View &V, const std::vector<int64_t> &f) {
                std::vector<int64_t> tgt = cat(f, kappa);
                const int64_t ninst = node[id].n_inst;
                const size_t bytes_p = (size_t)ninst * V.size * es;
                size_t off = arena.alloc(bytes_p);
                scratch.push_back(off);
                scratch_bytes.push_back(bytes_p);
                PermuteArgs pr;
                std::memset(&pr, 0, sizeof pr);
                pr.n = V.size;
                pr.rank = (int32_t)tgt.size();
                pr.n_inst = (int32_t)ninst;
                if (pr.rank > JET_MAXR) fail(JET_EINVAL, "permute rank too large");
                for (int j = 0; j < pr.rank; ++j) {
                    int64_t l = tgt[tgt.size() - 1 - j];
                    int p = find_pos(V.labels, l);
                    pr.dim[j] = V.dims[p];
                    pr.sstride[j] = V.strides[p];
                }
                std::vector<std::pair<int32_t, int64_t>> ps, pd;
                for (int64_t j = 0; j < ninst; ++j) {
                    ps.push_back(base_ref(id, (int32_t)j));
                    pd.push_back({BASE_ARENA, (int64_t)off + j * V.size * es});
                }
                size_t o_ps = blob.put_ptrs(ps), o_pd = blob.put_ptrs(pd);
                size_t so = blob.reserve(sizeof pr);
                std::memcpy(blob.bytes.data() + so, &pr, sizeof pr);
                blob.patch_field(so, offsetof(PermuteArgs, ptrSrc), BASE_BLOB, (int64_t)o_ps);
                blob.patch_field(so, offsetof(PermuteArgs, ptrDst), BASE_BLOB, (int64_t)o_pd);
                Op op;
                op.kind = OpKind::Permute;
                op.node = v;
                op.n_inst = ninst;
                op.args_off = so;
                op.args_bytes = sizeof pr;
                op.bytes = 2.0 * (double)es * (double)V.size * (double)ninst;
                op.variant = fp64 ? 1 : 0;
                int64_t gy = std::min<int64_t>(ninst, 65535);
                op.grid_y = (int32_t)gy;
                op.grid_x = (int32_t)std::max<int64_t>(
                    1, std::min<int64_t>((V.size + 255) / 256, std::max<int64_t>(1, 148 * 16 / gy)));
                P.ops.push_back(op);
                P.bytes_executed += op.bytes;
                return off;
            };
            std::vector<std::pair<int32_t, int64_t>> gA, gB;
            if (formM < 0) {
                size_t off = permute_child(idM, VM, fM);
                for (int64_t i = 0; i < N.n_inst; ++i) gA.push_back({BASE_ARENA, (int64_t)off + instM[i] * VM.size * es});
                formM = 1;
            } else {
                for (int64_t i = 0; i < N.n_inst; ++i) gA.push_back(base_ref(idM, instM[i]));
            }
            if (formN < 0) {
                size_t off = permute_child(idN, VN, fN);
                for (int64_t i = 0; i < N.n_inst; ++i) gB.push_back({BASE_ARENA, (int64_t)off + instN[i] * VN.size * es});
                formN = 1;
            } else {
                for (int64_t i = 0; i < N.n_inst; ++i) gB.push_back(base_ref(idN, instN[i]));
            }
            GemmArgs g;
            std::memset(&g, 0, sizeof g);
            g.M = dimprod(fM);
            g.N = dimprod(fN);
            g.K = nK;
            g.n_inst = (int32_t)N.n_inst;
            g.a_kmajor = formM == 1;
            g.b_kmajor = formN == 1;
            size_t o_a = blob.put_ptrs(gA), o_b = blob.put_ptrs(gB), o_c = blob.put_ptrs(pc);
            size_t so = blob.reserve(sizeof g);
            std::memcpy(blob.bytes.data() + so, &g, sizeof g);
            blob.patch_field(so, offsetof(GemmArgs, ptrA), BASE_BLOB, (int64_t)o_a);
            blob.patch_field(so, offsetof(GemmArgs, ptrB), BASE_BLOB, (int64_t)o_b);
            blob.patch_field(so, offsetof(GemmArgs, ptrC), BASE_BLOB, (int64_t)o_c);
            Op op;
            op.kind = OpKind::GemmSimt;
            op.node = v;
            op.n_inst = N.n_inst;
            op.args_off = so;
            op.args_bytes = sizeof g;
            op.flop = flop;
            op.bytes = bytes;
            op.variant = fp64 ? 1 : 0;
            if ((g.N + 63) / 64 > INT32_MAX) fail(JET_EINVAL, "GEMM N too large");
            op.grid_x = (int32_t)((g.N + 63) / 64);
            op.grid_y = (int32_t)std::min<int64_t>((g.M + 63) / 64, 65535);
            op.grid_z = (int32_t)std::min<int64_t>(N.n_inst, 65535);
            P.ops.push_back(op);
            }
        }
        // ------------------------------------------------ small operand applied to a large one
        else if (apply_ok(N, VA, VB)) {
            ++P.n_direct;
            emit_apply(v, VA, VB, N.view, K, a_big, N.n_inst, pa, pb, pc, flop, bytes);
        }
        // ------------------------------------------------ direct contraction
        else {
            ++P.n_direct;
            emit_direct(v, VA, VB, N.view, K, a_big, N.n_inst, pa, pb, pc, flop, bytes, scratch, scratch_bytes);
        }

        for (size_t s = 0; s < scratch.size(); ++s) arena.release(scratch[s], scratch_bytes[s]);
        // children are dead once this node's launches are issued
        release_children(v);
    }
    flush_batch();
    flush_chain();
    chain_on = false;   // (the adjoint sweep's batches run as plain level launches)

    // ---- adjoint sweep (environment contraction), reverse launch order.
    // For C = sum_K A B: env(A) = env(C) contracted with B over B's free labels,
    // laid out like A; env(B) likewise.  Several instances of C that read the
    // same child instance add their contributions in increasing instance order.
    if (grad) {
        const int32_t rootv = n_nodes - 1;
        if (rootv < n_leaves) fail(JET_EINVAL, "the adjoint needs at least two tensors");
        std::vector<char> need(n_nodes, 0);
        for (int32_t id : grad->leaves) need[id] = 1;
        for (int32_t k = 0; k < (int32_t)net.path.size(); ++k) {
            const int32_t v = n_leaves + k;
            need[v] = need[node[v].a] || need[node[v].b];
        }
        std::vector<std::pair<int32_t, int64_t>> env_base(n_nodes, {-1, 0});
        {   // seed: env(root instance) = sum of cot_b over the amplitudes mapped to it
            const NodeInfo &R = node[rootv];
            std::vector<double> seed(2 * R.n_inst, 0.0);
            for (int64_t x = 0; x < n_assign; ++x) {
                const int32_t i = inst_of[rootv][x];
                const int64_t b = x / n_sl;
                seed[2 * i] += grad->cot[2 * b];
                seed[2 * i + 1] += grad->cot[2 * b + 1];
            }
            const size_t off = blob.reserve((size_t)R.n_inst * es, 16);
            for (int64_t i = 0; i < R.n_inst; ++i) {
                if (fp64) {
                    std::memcpy(blob.bytes.data() + off + i * 16, &seed[2 * i], 16);
                } else {
                    const float f[2] = {(float)seed[2 * i], (float)seed[2 * i + 1]};
                    std::memcpy(blob.bytes.data() + off + i * 8, f, 8);
                }
            }
            env_base[rootv] = {BASE_BLOB, (int64_t)off};
            P.grad = true;
            P.grad_leaves = grad->leaves;
            P.grad_env_off = grad->env_off;
            P.seed_off = off;
            P.seed_n_inst = R.n_inst;
            P.seed_n_sl = n_sl;
            P.seed_inst.assign(inst_of[rootv].begin(), inst_of[rootv].begin() + n_assign);
        }
        auto emit_memset = [&](size_t off, size_t nbytes) {
            MemsetArgs m;
            m.ptr = 0;
            m.bytes = (int64_t)nbytes;
            const size_t so = blob.reserve(sizeof m);
            std::memcpy(blob.bytes.data() + so, &m, sizeof m);
            blob.patch_field(so, offsetof(MemsetArgs, ptr), BASE_ARENA, (int64_t)off);
            Op op;
            op.kind = OpKind::Memset;
            op.args_off = so;
            op.args_bytes = sizeof m;
            P.ops.push_back(op);
        };
        // every environment in one block of the arena, cleared by one memset
        {
            std::vector<size_t> local(n_nodes, 0);
            size_t total = 0;
            for (int32_t v : order)
                if (need[v] && v != rootv) {
                    local[v] = total;
                    total += ((size_t)node[v].n_inst * node[v].view.size * es + 255) / 256 * 256;
                }
            if (total) {
                const size_t blk = arena.alloc(total);
                for (int32_t v : order)
                    if (need[v] && v != rootv) env_base[v] = {BASE_ARENA, (int64_t)(blk + local[v])};
                emit_memset(blk, total);
            }
        }
        // sweep one tree level at a time, deepest first: a level's environment
        // contractions (the small ones batched into one launch), then all of its
        // accumulations into the children's environments in one launch
        std::vector<int32_t> rev(order.rbegin(), order.rend());
        for (size_t i0 = 0; i0 < rev.size();) {
            size_t i1 = i0;
            while (i1 < rev.size() && node[rev[i1]].depth == node[rev[i0]].depth) ++i1;
            std::vector<AccumTask> atasks;
            std::vector<Plan::Patch> apatches;   // offsets relative to the task array
            std::vector<std::pair<size_t, size_t>> tbufs;
            int32_t ablocks = 0;
            double abytes = 0;
            for (size_t ii = i0; ii < i1; ++ii) {
                const int32_t v = rev[ii];
                if (!need[v]) continue;
                const NodeInfo &N = node[v];
                for (int side = 0; side < 2; ++side) {
                    const int32_t c = side == 0 ? N.a : N.b, o = side == 0 ? N.b : N.a;
                    if (!need[c]) continue;
                    const std::vector<int32_t> &ic = side == 0 ? N.ia : N.ib, &io = side == 0 ? N.ib : N.ia;
                    const NodeInfo &NC = node[c], &NO = node[o];
                    const View Tv = dense_view(NC.view.labels, net);
                    std::vector<int64_t> Kb;   // summed: labels of C that come from the other child
                    for (int64_t l : N.view.labels)
                        if (find_pos(NO.view.labels, l) >= 0) Kb.push_back(l);
                    const bool leaf = c < n_leaves;
                    // an internal child whose every instance gets exactly one contribution
                    // takes it directly in its (zeroed, dense) environment: no accumulation
                    bool direct_env = !leaf && NC.n_inst == N.n_inst;
                    if (direct_env) {
                        std::vector<int32_t> cnt(NC.n_inst, 0);
                        for (int64_t i = 0; i < N.n_inst; ++i) direct_env = direct_env && ++cnt[ic[i]] == 1;
                    }
                    size_t toff = 0, tbytes = 0;
                    if (!direct_env) {
                        tbytes = (size_t)N.n_inst * Tv.size * es;
                        toff = arena.alloc(tbytes);
                        tbufs.push_back({toff, tbytes});
                    }
                    std::vector<std::pair<int32_t, int64_t>> pe, po, pt;
                    for (int64_t i = 0; i < N.n_inst; ++i) {
                        pe.push_back({env_base[v].first, env_base[v].second + i * N.view.size * es});
                        po.push_back(base_ref(o, io[i]));
                        if (direct_env)
                            pt.push_back({env_base[c].first, env_base[c].second + (int64_t)ic[i] * NC.view.size * es});
                        else
                            pt.push_back({BASE_ARENA, (int64_t)toff + i * Tv.size * es});
                    }
                    std::vector<int64_t> un = N.view.labels;
                    for (int64_t l : NO.view.labels)
                        if (find_pos(un, l) < 0) un.push_back(l);
                    const double flop = 8.0 * (double)dimprod(un) * (double)N.n_inst;
                    const double bytes = (double)es * (double)N.n_inst * (double)(N.view.size + NO.view.size + Tv.size);
                    const int64_t nKb = dimprod(Kb);
                    const bool small = Tv.size <= 4096 && nKb <= 2048 &&
                                       (double)N.n_inst * (double)Tv.size * (double)nKb <= (double)(1 << 24) &&
                                       N.view.size <= INT32_MAX && NO.view.size <= INT32_MAX;
                    if (small) {
                        add_small_task(N.view, NO.view, Tv, Kb, N.view.size >= NO.view.size, pe, po, pt, N.n_inst);
                        batch_flop += flop;
                        batch_bytes += bytes;
                    } else if (apply_ok_views(N.view, NO.view, Kb, N.view.size >= NO.view.size, N.n_inst)) {
                        emit_apply(v, N.view, NO.view, Tv, Kb, N.view.size >= NO.view.size, N.n_inst, pe, po, pt, flop,
                                   bytes, false);
                    } else {
                        std::vector<size_t> scr, scrb;
                        emit_direct(v, N.view, NO.view, Tv, Kb, N.view.size >= NO.view.size, N.n_inst, pe, po, pt,
                                    flop, bytes, scr, scrb, false);
                        for (size_t q = 0; q < scr.size(); ++q) arena.release(scr[q], scrb[q]);
                    }
                    P.flop_executed += flop;
                    if (direct_env) continue;
                    // the accumulation of these contributions into env(c)
                    AccumTask at;
                    std::memset(&at, 0, sizeof at);
                    AccumArgs &ac = at.a;
                    ac.n = Tv.size;
                    ac.n_tgt = (int32_t)NC.n_inst;
                    ac.rank = (int32_t)Tv.labels.size();
                    ac.src_fp64 = fp64 ? 1 : 0;
                    ac.tgt_fp64 = (leaf || fp64) ? 1 : 0;
                    if (ac.rank > JET_MAXR) fail(JET_EINVAL, "environment rank too large");
                    for (int j = 0; j < ac.rank; ++j) {
                        const size_t li = Tv.labels.size() - 1 - j;
                        ac.dim[j] = Tv.dims[li];
                        ac.tstride[j] = leaf ? NC.view.strides[li] : Tv.strides[li];
                    }
                    std::vector<int32_t> cptr(NC.n_inst + 1, 0), csrc(N.n_inst);
                    for (int64_t i = 0; i < N.n_inst; ++i) ++cptr[ic[i] + 1];
                    for (int64_t j = 0; j < NC.n_inst; ++j) cptr[j + 1] += cptr[j];
                    {
                        std::vector<int32_t> fill(cptr.begin(), cptr.end() - 1);
                        for (int64_t i = 0; i < N.n_inst; ++i) csrc[fill[ic[i]]++] = (int32_t)i;
                    }
                    std::vector<std::pair<int32_t, int64_t>> tg;
                    for (int64_t j = 0; j < NC.n_inst; ++j) {
                        if (leaf)
                            tg.push_back({BASE_ENV, (grad->env_off[c] + (NC.inst_off[j] - net.leaves[c].offset)) * 16});
                        else
                            tg.push_back({env_base[c].first, env_base[c].second + j * NC.view.size * es});
                    }
                    const size_t o_p = blob.put_i32(cptr), o_s = blob.put_i32(csrc), o_t = blob.put_ptrs(tg);
                    const size_t base = atasks.size() * sizeof(AccumTask) + offsetof(AccumTask, a);
                    apatches.push_back({base + offsetof(AccumArgs, src), BASE_ARENA, (int64_t)toff});
                    apatches.push_back({base + offsetof(AccumArgs, tgt), BASE_BLOB, (int64_t)o_t});
                    apatches.push_back({base + offsetof(AccumArgs, csr_ptr), BASE_BLOB, (int64_t)o_p});
                    apatches.push_back({base + offsetof(AccumArgs, csr_src), BASE_BLOB, (int64_t)o_s});
                    at.block0 = ablocks;
                    const int64_t items = (int64_t)NC.n_inst * Tv.size;
                    ablocks += (int32_t)std::max<int64_t>(1, std::min<int64_t>((items + 255) / 256, 1024));
                    abytes += (double)es * (double)N.n_inst * (double)Tv.size * 2.0;
                    atasks.push_back(at);
                }
            }
            flush_batch();
            if (!atasks.empty()) {
                const size_t o_tasks = blob.reserve(sizeof(AccumTask) * atasks.size(), 64);
                for (size_t k = 0; k < atasks.size(); ++k)
                    std::memcpy(blob.bytes.data() + o_tasks + k * sizeof(AccumTask), &atasks[k], sizeof(AccumTask));
                for (auto &pt : apatches) blob.patches.push_back({o_tasks + pt.at, pt.base, pt.byte_off});
                AccumBatchArgs ab;
                std::memset(&ab, 0, sizeof ab);
                ab.n_tasks = (int32_t)atasks.size();
                ab.n_blocks = ablocks;
                const size_t so = blob.reserve(sizeof ab);
                std::memcpy(blob.bytes.data() + so, &ab, sizeof ab);
                blob.patch_field(so, offsetof(AccumBatchArgs, tasks), BASE_BLOB, (int64_t)o_tasks);
                Op op;
                op.kind = OpKind::AccumBatch;
                op.node = rev[i0];
                op.n_inst = (int64_t)atasks.size();
                op.args_off = so;
                op.args_bytes = sizeof ab;
                op.bytes = abytes;
                op.grid_x = ablocks;
                P.ops.push_back(op);
            }
            for (auto &tb : tbufs) arena.release(tb.first, tb.second);
            i0 = i1;
        }
    }

    // ---- slice / amplitude reduction (Eq. sliced_sum), FP64, slices in increasing order
    // every root instance holds the free open legs (a scalar when there are none)
    const int32_t root = n_nodes - 1;
    const View &RV = node[root].view;
    if (RV.labels.size() != net.free_open.size()) fail(JET_EINVAL, "the network has undeclared open legs");
    {
        std::vector<std::pair<int32_t, int64_t>> roots;
        roots.reserve(n_assign);
        for (int64_t x = 0; x < n_assign; ++x) roots.push_back(base_ref(root, inst_of[root][x]));
        size_t off_roots = blob.put_ptrs(roots);
        // value e of the free legs (mixed radix, first free leg slowest) -> element offset
        std::vector<int64_t> eoff((size_t)P.n_elem, 0);
        for (int64_t e = 0; e < P.n_elem; ++e) {
            int64_t x = e;
            for (int j = (int)net.free_open.size() - 1; j >= 0; --j) {
                const int p = find_pos(RV.labels, net.free_open[j]);
                if (p < 0) fail(JET_EINVAL, "free open leg missing from the result");
                const int64_t dm = RV.dims[p];
                eoff[(size_t)e] += (x % dm) * RV.strides[p];
                x /= dm;
            }
        }
        size_t off_eoff = 0;
        if (P.n_elem > 1) {
            off_eoff = blob.reserve(eoff.size() * sizeof(int64_t));
            std::memcpy(blob.bytes.data() + off_eoff, eoff.data(), eoff.size() * sizeof(int64_t));
        }
        ReduceArgs r;
        std::memset(&r, 0, sizeof r);
        r.n_amps = n_amps;
        r.n_slices = (int32_t)n_sl;
        r.partials = P.partials ? 1 : 0;
        r.fp64_in = fp64 ? 1 : 0;
        r.n_elem = (int32_t)P.n_elem;
        size_t ro = blob.reserve(sizeof r);
        std::memcpy(blob.bytes.data() + ro, &r, sizeof r);
        blob.patch_field(ro, offsetof(ReduceArgs, roots), BASE_BLOB, (int64_t)off_roots);
        blob.patch_field(ro, offsetof(ReduceArgs, amps), BASE_AMPS, 0);
        if (P.n_elem > 1) blob.patch_field(ro, offsetof(ReduceArgs, eoff), BASE_BLOB, (int64_t)off_eoff);
        Op op;
        op.kind = OpKind::Reduce;
        op.node = root;
        op.n_inst = n_amps;
        op.args_off = ro;
        op.args_bytes = sizeof r;
        op.grid_x = (int32_t)(((P.partials ? n_assign : n_amps) * P.n_elem + 127) / 128);
        op.block = 128;
        P.ops.push_back(op);
    }

    P.arena_bytes = std::max<size_t>(arena.peak, 256);
    P.buffers = std::move(arena.log);
    P.parent.assign(parent.begin(), parent.end());
    P.host_args = std::move(blob.bytes);
    P.patches = std::move(blob.patches);
    P.max_intermediate = max_inter;
    return plan;
}

}  // namespace jet
