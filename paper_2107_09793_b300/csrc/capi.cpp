// C ABI entry points (declared in include/jet.h).  Each call validates its
// arguments, works on copies, and converts internal errors into JET_E* codes
// plus a thread-local message; nothing escapes the boundary as an exception.
#include <algorithm>
#include <array>
#include <cstdio>
#include <cstring>
#include <functional>
#include <exception>
#include <map>
#include <new>
#include <numeric>
#include <string>
#include <unordered_set>

#include "internal.h"

namespace jet {

static thread_local std::string g_last_error;

void set_last_error(const std::string &msg) { g_last_error = msg; }

[[noreturn]] void fail(int code, const std::string &msg) { throw Error{code, msg}; }

template <typename F>
static int guarded(F &&f)
{
    try {
        f();
        g_last_error.clear();
        return JET_OK;
    } catch (const Error &e) {
        g_last_error = e.msg;
        return e.code;
    } catch (const std::bad_alloc &) {
        g_last_error = "host allocation failed";
        return JET_ENOMEM;
    } catch (const std::exception &e) {
        g_last_error = e.what();
        return JET_EINVAL;
    } catch (...) {
        g_last_error = "unknown error";
        return JET_EINVAL;
    }
}

static void drop_ranges(Network &net)
{
    if (!net.ranges) return;
    for (auto &p : net.ranges->plans)
        if (p) {
            if (net.last_run == p.get()) net.last_run = nullptr;
            release_plan_device(*p);
        }
    net.ranges.reset();
}

static void invalidate_plan(Network &net)
{
    if (net.plan) {
        if (net.last_run == net.plan.get()) net.last_run = nullptr;
        release_plan_device(*net.plan);
        net.plan.reset();
    }
    drop_ranges(net);
}

// New cotangents into a cached adjoint plan: seed(root instance i) = sum of
// cot_b over the (amplitude b, slice) assignments mapped to i.
static void write_seed(Plan &P, const std::vector<double> &cot, bool fp64)
{
    std::vector<double> seed(2 * (size_t)P.seed_n_inst, 0.0);
    for (size_t x = 0; x < P.seed_inst.size(); ++x) {
        const int32_t i = P.seed_inst[x];
        const size_t b = x / (size_t)P.seed_n_sl;
        seed[2 * i] += cot[2 * b];
        seed[2 * i + 1] += cot[2 * b + 1];
    }
    uint8_t *dst = P.host_args.data() + P.seed_off;
    for (int64_t i = 0; i < P.seed_n_inst; ++i) {
        if (fp64) {
            std::memcpy(dst + i * 16, &seed[2 * i], 16);
        } else {
            const float f[2] = {(float)seed[2 * i], (float)seed[2 * i + 1]};
            std::memcpy(dst + i * 8, f, 8);
        }
    }
    P.seed_dirty = true;
}

// New tensor values: kept results are stale; a plan that reads them is dropped.
static void drop_kept(Network &net)
{
    ++net.tensors_version;
    if (net.kept.empty()) return;
    net.kept.clear();
    invalidate_plan(net);
}

// Kept results belong to one path, slicing, set of tensor values and of fixed
// legs: any change starts the pool afresh.
static void check_kept_key(Network &net)
{
    std::vector<int64_t> key{(int64_t)net.path_version, (int64_t)net.slice_version, (int64_t)net.tensors_version,
                             net.keep_min, (int64_t)net.open.size()};
    key.insert(key.end(), net.open.begin(), net.open.end());
    key.push_back(-1);
    key.insert(key.end(), net.free_open.begin(), net.free_open.end());
    if (key != net.kept_key) {
        net.kept.clear();
        net.kept_key = key;
    }
}

// After a run that computed kept results: they are ready, and the next call
// plans afresh to read them instead of their sub-trees (the stream is drained
// here, so the plan being replaced has finished running by then).
static void mark_kept(Network &net, Plan &P, void *stream)
{
    if (P.kept_fill.empty()) return;
    sync_stream(net, stream);
    for (int32_t v : P.kept_fill) net.kept.at(v).ready = true;
    P.superseded = true;
}

static Plan &get_plan(Network &net, int32_t n_amps, const int32_t *outputs,
                      const std::vector<int64_t> *slice_ids = nullptr)
{
    if (!outputs && !net.open.empty()) fail(JET_EINVAL, "outputs is NULL");
    const size_t n = (size_t)n_amps * net.open.size();
    Plan *P = net.plan.get();
    bool reuse = P && !P->superseded && P->n_amps == n_amps && P->path_version == net.path_version &&
                 P->slice_version == net.slice_version && P->precision == net.opt.precision &&
                 P->reuse == net.opt.reuse && P->outputs.size() == n &&
                 std::equal(P->outputs.begin(), P->outputs.end(), outputs) &&
                 P->partials == (slice_ids != nullptr) && (!slice_ids || P->slice_ids == *slice_ids);
    if (!reuse) {
        check_kept_key(net);
        auto fresh = build_plan(net, n_amps, outputs, slice_ids);
        invalidate_plan(net);
        net.plan = std::move(fresh);
    }
    return *net.plan;
}

}  // namespace jet

using namespace jet;

struct jet_network : public jet::Network {};

extern "C" {

void jet_options_default(jet_options *opt)
{
    if (!opt) return;
    std::memset(opt, 0, sizeof *opt);
    opt->precision = JET_PREC_FP32;
    opt->reuse = 1;
    opt->use_graph = 1;
    opt->device = 0;
    opt->gemm_min_k = 16;
    opt->workspace_limit = 0;
    opt->profile = 0;
    opt->apply_tc_min_kf = 1024;
    opt->gemm_group = 1;
    opt->fuse_split = 1;
}

int jet_network_create(const jet_tensor_desc *tensors, int32_t n, const jet_options *opt, jet_network **out)
{
    return guarded([&] {
        if (!out) fail(JET_EINVAL, "out is NULL");
        *out = nullptr;
        if (!tensors || n < 1) fail(JET_EINVAL, "need at least one tensor");
        auto net = std::make_unique<jet_network>();
        if (opt) net->opt = *opt;
        else jet_options_default(&net->opt);
        if (net->opt.precision < JET_PREC_FP32 || net->opt.precision > JET_PREC_FP16X3)
            fail(JET_EINVAL, "unknown precision mode");
        if (net->opt.gemm_min_k < 1) net->opt.gemm_min_k = 16;
        if (net->opt.apply_tc_min_kf < 1) net->opt.apply_tc_min_kf = 1024;
        int64_t off = 0;
        for (int32_t t = 0; t < n; ++t) {
            const jet_tensor_desc &d = tensors[t];
            if (d.rank < 0 || d.rank > 64) fail(JET_EINVAL, "tensor " + std::to_string(t) + ": bad rank");
            if (d.rank > 0 && (!d.labels || !d.dims)) fail(JET_EINVAL, "tensor " + std::to_string(t) + ": NULL labels/dims");
            if (!d.data) fail(JET_EINVAL, "tensor " + std::to_string(t) + ": NULL data");
            Leaf L;
            std::unordered_set<int64_t> seen;
            for (int32_t k = 0; k < d.rank; ++k) {
                int64_t l = d.labels[k];
                int32_t dim = d.dims[k];
                if (l < 0) fail(JET_EINVAL, "tensor " + std::to_string(t) + ": negative label");
                if (dim < 1 || dim > 65535) fail(JET_EINVAL, "tensor " + std::to_string(t) + ": dim out of range");
                if (!seen.insert(l).second)
                    fail(JET_EINVAL, "tensor " + std::to_string(t) + ": label " + std::to_string(l) + " repeated");
                LabelInfo &li = net->labels[l];
                if (li.n_owner == 2)
                    fail(JET_EINVAL, "label " + std::to_string(l) + " appears on more than two tensors");
                if (li.n_owner == 1 && li.dim != dim)
                    fail(JET_EINVAL, "label " + std::to_string(l) + ": dims differ between tensors");
                li.dim = dim;
                li.owner[li.n_owner++] = t;
                L.labels.push_back(l);
                L.dims.push_back(dim);
                L.size *= dim;
                if (L.size > ((int64_t)1 << 40)) fail(JET_EINVAL, "tensor too large");
            }
            L.offset = off;
            off += L.size;
            net->leaves.push_back(L);
        }
        net->n_values = off;
        net->host_values.resize(off);
        for (int32_t t = 0; t < n; ++t)
            std::memcpy(net->host_values.data() + net->leaves[t].offset, tensors[t].data,
                        (size_t)net->leaves[t].size * sizeof(jet_c64));
        // a single open leg set by default: none declared yet
        *out = net.release();
    });
}

int jet_network_set_open(jet_network *net, int32_t n_out, const int64_t *out_labels)
{
    return guarded([&] {
        if (!net) fail(JET_EINVAL, "net is NULL");
        if (n_out < 0 || (n_out > 0 && !out_labels)) fail(JET_EINVAL, "bad open-leg list");
        std::unordered_set<int64_t> seen;
        for (int32_t j = 0; j < n_out; ++j) {
            auto it = net->labels.find(out_labels[j]);
            if (it == net->labels.end() || it->second.n_owner != 1)
                fail(JET_EINVAL, "label " + std::to_string(out_labels[j]) + " is not an open leg");
            if (!seen.insert(out_labels[j]).second) fail(JET_EINVAL, "open leg listed twice");
        }
        size_t n_open = 0;
        for (auto &kv : net->labels) n_open += kv.second.n_owner == 1;
        if (n_open != (size_t)n_out)
            fail(JET_EINVAL, "every open leg must be listed (" + std::to_string(n_open) + " open legs)");
        net->open.assign(out_labels, out_labels + n_out);
        net->open_set = true;
        net->free_open.clear();
        for (int64_t l : net->open)
            if (std::find(net->sliced.begin(), net->sliced.end(), l) != net->sliced.end()) {
                net->sliced.clear();
                ++net->slice_version;
            }
        invalidate_plan(*net);
    });
}

int jet_network_set_free(jet_network *net, int32_t n_free, const int64_t *free_labels)
{
    return guarded([&] {
        if (!net) fail(JET_EINVAL, "net is NULL");
        if (n_free < 0 || (n_free > 0 && !free_labels)) fail(JET_EINVAL, "bad free-leg list");
        if (!net->open_set && n_free > 0) fail(JET_ESTATE, "declare the open legs first");
        std::vector<int64_t> fr(free_labels, free_labels + n_free);
        int64_t n_elem = 1;
        for (int32_t j = 0; j < n_free; ++j) {
            if (std::find(net->open.begin(), net->open.end(), fr[j]) == net->open.end())
                fail(JET_EINVAL, "label " + std::to_string(fr[j]) + " is not an open leg");
            if (std::find(fr.begin(), fr.begin() + j, fr[j]) != fr.begin() + j) fail(JET_EINVAL, "free leg listed twice");
            n_elem *= net->labels.at(fr[j]).dim;
            if (n_elem > ((int64_t)1 << 24)) fail(JET_EINVAL, "more than 2^24 values per row");
        }
        net->free_open = fr;
        invalidate_plan(*net);
    });
}

int jet_network_keep_shared(jet_network *net, int64_t min_elems)
{
    return guarded([&] {
        if (!net) fail(JET_EINVAL, "net is NULL");
        if (min_elems < 0) fail(JET_EINVAL, "min_elems must be >= 0");
        net->keep_min = min_elems;
        net->kept.clear();
        invalidate_plan(*net);
        if (min_elems == 0) {
            sync_stream(*net, nullptr);
            device_free(net->d_kept);
            net->d_kept = nullptr;
            net->d_kept_bytes = 0;
        }
    });
}

// What kept results depend on, by content (so that a file written by one
// process can be checked by another): precision, keep threshold, the path, the
// sliced labels, the open and free legs, and an FNV-1a hash of every tensor
// value as it sits on the device.
static std::vector<uint64_t> kept_content_key(Network &net)
{
    auto fnv = [](const void *p, size_t n, uint64_t h) {
        const uint8_t *b = (const uint8_t *)p;
        for (size_t i = 0; i < n; ++i) h = (h ^ b[i]) * 1099511628211ull;
        return h;
    };
    ensure_leaves_on_device(net);
    std::vector<jet_c64> vals((size_t)net.n_values);
    copy_d2h(vals.data(), net.d_leaves, vals.size() * sizeof(jet_c64), net.stream);
    std::vector<uint64_t> key{0x4A45544B45505431ull, (uint64_t)net.opt.precision, (uint64_t)net.keep_min,
                              (uint64_t)net.leaves.size(), (uint64_t)net.path.size()};
    for (auto &pr : net.path) key.push_back(((uint64_t)(uint32_t)pr.first << 32) | (uint32_t)pr.second);
    for (auto *ls : {&net.sliced, &net.open, &net.free_open}) {
        key.push_back(ls->size());
        for (int64_t l : *ls) key.push_back((uint64_t)l);
    }
    key.push_back(fnv(vals.data(), vals.size() * sizeof(jet_c64), 1469598103934665603ull));
    return key;
}

int jet_network_save_shared(jet_network *net, const char *file)
{
    return guarded([&] {
        if (!net || !file) fail(JET_EINVAL, "NULL argument");
        std::vector<std::pair<int32_t, Network::KeptEntry>> ready;
        for (auto &kv : net->kept)
            if (kv.second.ready) ready.push_back(kv);
        if (ready.empty()) fail(JET_ESTATE, "no kept shared work yet (jet_network_keep_shared, then contract)");
        std::sort(ready.begin(), ready.end(), [](auto &x, auto &y) { return x.first < y.first; });
        const auto key = kept_content_key(*net);
        std::vector<uint8_t> pool(net->d_kept_bytes);
        copy_d2h(pool.data(), net->d_kept, pool.size(), net->stream);
        FILE *f = std::fopen(file, "wb");
        if (!f) fail(JET_EINVAL, std::string("cannot open ") + file);
        bool ok = true;
        auto put = [&](const void *p, size_t n) { ok = ok && std::fwrite(p, 1, n, f) == n; };
        const uint64_t nk = key.size(), ne = ready.size(), np = pool.size();
        put(&nk, 8);
        put(key.data(), 8 * nk);
        put(&ne, 8);
        for (auto &e : ready) {
            const uint64_t rec[3] = {(uint64_t)e.first, e.second.off, e.second.bytes};
            put(rec, sizeof rec);
        }
        put(&np, 8);
        put(pool.data(), np);
        ok = (std::fclose(f) == 0) && ok;
        if (!ok) fail(JET_EINVAL, std::string("write failed: ") + file);
    });
}

int jet_network_load_shared(jet_network *net, const char *file)
{
    return guarded([&] {
        if (!net || !file) fail(JET_EINVAL, "NULL argument");
        if (net->keep_min <= 0) fail(JET_ESTATE, "keeping is off (jet_network_keep_shared)");
        FILE *f = std::fopen(file, "rb");
        if (!f) fail(JET_EINVAL, std::string("cannot open ") + file);
        bool ok = true;
        auto get = [&](void *p, size_t n) { ok = ok && std::fread(p, 1, n, f) == n; };
        uint64_t nk = 0;
        get(&nk, 8);
        std::vector<uint64_t> key(ok && nk < (1u << 24) ? nk : 0);
        get(key.data(), 8 * key.size());
        uint64_t ne = 0;
        get(&ne, 8);
        std::vector<std::array<uint64_t, 3>> recs(ok && ne < (1u << 24) ? ne : 0);
        for (auto &r : recs) get(r.data(), sizeof r);
        uint64_t np = 0;
        get(&np, 8);
        std::vector<uint8_t> pool(ok ? np : 0);
        get(pool.data(), pool.size());
        std::fclose(f);
        if (!ok || key.size() != nk || recs.size() != ne) fail(JET_EINVAL, std::string("not a kept-work file: ") + file);
        if (key != kept_content_key(*net))
            fail(JET_EINVAL, "the saved shared work belongs to another network, path, slicing, legs, precision, "
                             "threshold or tensor values");
        for (auto &r : recs)
            if (r[1] + r[2] > np) fail(JET_EINVAL, "corrupt kept-work file");
        invalidate_plan(*net);
        check_kept_key(*net);
        net->kept.clear();
        if (net->d_kept_bytes < np) {
            sync_stream(*net, nullptr);
            device_free(net->d_kept);
            net->d_kept = nullptr;
            net->d_kept_bytes = 0;
            net->d_kept = device_alloc(np);
            net->d_kept_bytes = np;
        }
        copy_h2d_sync(net->d_kept, pool.data(), np, net->stream);
        for (auto &r : recs) {
            Network::KeptEntry e;
            e.off = r[1];
            e.bytes = r[2];
            e.ready = true;
            net->kept[(int32_t)r[0]] = e;
        }
    });
}

int jet_tensor_update(jet_network *net, int32_t tensor_id, const jet_c64 *data)
{
    return guarded([&] {
        if (!net || !data) fail(JET_EINVAL, "NULL argument");
        if (tensor_id < 0 || tensor_id >= (int32_t)net->leaves.size()) fail(JET_EINVAL, "bad tensor id");
        const Leaf &L = net->leaves[tensor_id];
        std::memcpy(net->host_values.data() + L.offset, data, (size_t)L.size * sizeof(jet_c64));
        upload_leaf(*net, tensor_id, nullptr);
        drop_kept(*net);
    });
}

int jet_tensors_upload(jet_network *net, const jet_c64 *data, void *cuda_stream)
{
    return guarded([&] {
        if (!net || !data) fail(JET_EINVAL, "NULL argument");
        upload_all(*net, data, cuda_stream);
        drop_kept(*net);
    });
}

int64_t jet_network_n_values(const jet_network *net) { return net ? net->n_values : -1; }

int jet_path_set(jet_network *net, int32_t n_steps, const int32_t *pairs)
{
    return guarded([&] {
        if (!net) fail(JET_EINVAL, "net is NULL");
        if (n_steps < 0 || (n_steps > 0 && !pairs)) fail(JET_EINVAL, "bad path");
        std::vector<std::pair<int32_t, int32_t>> p;
        for (int32_t k = 0; k < n_steps; ++k) p.push_back({pairs[2 * k], pairs[2 * k + 1]});
        validate_path(*net, p);
        net->path = p;
        ++net->path_version;
        net->flop_planned = path_cost(*net, p, {}).flop;
        invalidate_plan(*net);
    });
}

int jet_path_get(const jet_network *net, int32_t *pairs_out)
{
    return guarded([&] {
        if (!net || !pairs_out) fail(JET_EINVAL, "NULL argument");
        if (net->path.size() + 1 != net->leaves.size()) fail(JET_ESTATE, "no path set");
        for (size_t k = 0; k < net->path.size(); ++k) {
            pairs_out[2 * k] = net->path[k].first;
            pairs_out[2 * k + 1] = net->path[k].second;
        }
    });
}

int jet_path_greedy(jet_network *net, uint64_t seed, int32_t n_trials, double *flop_out)
{
    return guarded([&] {
        if (!net) fail(JET_EINVAL, "net is NULL");
        double f = 0;
        auto p = greedy_path(*net, seed, std::max(n_trials, 1), &f);
        validate_path(*net, p);
        net->path = p;
        ++net->path_version;
        net->flop_planned = f;
        if (flop_out) *flop_out = f;
        invalidate_plan(*net);
    });
}

int jet_path_greedy_batch(jet_network *net, int32_t n_amps, const int32_t *outputs, int64_t max_elems,
                          uint64_t seed, int32_t n_trials, double *flop_out)
{
    return guarded([&] {
        if (!net) fail(JET_EINVAL, "net is NULL");
        if (!net->open_set) fail(JET_ESTATE, "open legs not declared (jet_network_set_open)");
        if (n_amps < 1 || !outputs) fail(JET_EINVAL, "need n_amps >= 1 and an outputs array");
        const int32_t n_open = (int32_t)net->open.size();
        for (int32_t b = 0; b < n_amps; ++b)
            for (int32_t j = 0; j < n_open; ++j) {
                const int32_t v = outputs[(int64_t)b * n_open + j];
                if (v < 0 || v >= net->labels.at(net->open[j]).dim)
                    fail(JET_EINVAL, "output digit out of range at amplitude " + std::to_string(b));
            }
        double f = 0;
        auto p = greedy_path(*net, seed, std::max(n_trials, 1), &f, n_amps, outputs, (double)max_elems);
        validate_path(*net, p);
        net->path = p;
        ++net->path_version;
        net->flop_planned = f;
        if (flop_out) *flop_out = f;
        invalidate_plan(*net);
    });
}

int jet_path_reconfigure(jet_network *net, int32_t passes, int32_t objective, int32_t n_amps, const int32_t *outputs,
                         double *cost_before, double *cost_after)
{
    return guarded([&] {
        if (!net) fail(JET_EINVAL, "net is NULL");
        if (net->path.size() + 1 != net->leaves.size()) fail(JET_ESTATE, "no contraction path set");
        if (passes < 1 || passes > 64) fail(JET_EINVAL, "passes must be in [1, 64]");
        if (objective != 0 && objective != 1) fail(JET_EINVAL, "objective must be 0 (FLOP) or 1 (time model)");
        if (outputs && n_amps > 1) {
            if (!net->open_set) fail(JET_ESTATE, "open legs not declared (jet_network_set_open)");
            const int32_t n_open = (int32_t)net->open.size();
            for (int32_t b = 0; b < n_amps; ++b)
                for (int32_t j = 0; j < n_open; ++j) {
                    const int32_t v = outputs[(int64_t)b * n_open + j];
                    if (v < 0 || v >= net->labels.at(net->open[j]).dim)
                        fail(JET_EINVAL, "output digit out of range at amplitude " + std::to_string(b));
                }
        }
        double f0 = 0, f1 = 0;
        auto p = reconfigure_sliced(*net, passes, n_amps, outputs, &f0, &f1, objective == 1);
        validate_path(*net, p);
        if (f1 < f0) {
            net->path = p;
            ++net->path_version;
            net->flop_planned = path_cost(*net, p, {}).flop;
            invalidate_plan(*net);
        }
        if (cost_before) *cost_before = f0;
        if (cost_after) *cost_after = f1;
    });
}

int jet_slice(jet_network *net, int32_t n, const int64_t *labels)
{
    return guarded([&] {
        if (!net) fail(JET_EINVAL, "net is NULL");
        if (n < 0 || (n > 0 && !labels)) fail(JET_EINVAL, "bad slice list");
        std::vector<int64_t> s;
        for (int32_t i = 0; i < n; ++i) {
            auto it = net->labels.find(labels[i]);
            if (it == net->labels.end()) fail(JET_EINVAL, "unknown label " + std::to_string(labels[i]));
            if (it->second.n_owner != 2) fail(JET_EINVAL, "label " + std::to_string(labels[i]) + " is an open leg");
            if (std::find(s.begin(), s.end(), labels[i]) != s.end()) fail(JET_EINVAL, "label sliced twice");
            s.push_back(labels[i]);
        }
        double nsl = 1;
        for (int64_t l : s) nsl *= net->labels.at(l).dim;
        if (nsl > (double)(1 << 30)) fail(JET_EINVAL, "too many slices");
        net->sliced = s;
        ++net->slice_version;
        invalidate_plan(*net);
    });
}

int jet_slice_auto(jet_network *net, int64_t max_elems, int32_t min_n, int32_t max_n, int32_t *n_out,
                   int64_t *labels_out)
{
    return guarded([&] {
        if (!net) fail(JET_EINVAL, "net is NULL");
        if (net->path.size() + 1 != net->leaves.size()) fail(JET_ESTATE, "no path set");
        if (max_elems < 1) fail(JET_EINVAL, "max_elems must be >= 1");
        auto s = slice_auto(*net, max_elems, std::max(min_n, 0), std::max(max_n, 0));
        if (n_out) *n_out = (int32_t)s.size();
        if (labels_out)
            for (size_t i = 0; i < s.size(); ++i) labels_out[i] = s[i];
        net->sliced = s;
        ++net->slice_version;
        invalidate_plan(*net);
    });
}

int jet_plan(jet_network *net, int32_t n_amps, const int32_t *outputs, size_t *bytes_out)
{
    return guarded([&] {
        if (!net) fail(JET_EINVAL, "net is NULL");
        Plan &P = get_plan(*net, n_amps, outputs);
        if (bytes_out) *bytes_out = P.arena_bytes;
    });
}

int jet_plan_slices(jet_network *net, int32_t n_amps, const int32_t *outputs, int32_t n_ids,
                    const int64_t *slice_ids, size_t *bytes_out)
{
    return guarded([&] {
        if (!net || !slice_ids || n_ids < 1) fail(JET_EINVAL, "bad arguments");
        std::vector<int64_t> ids(slice_ids, slice_ids + n_ids);
        Plan &P = get_plan(*net, n_amps, outputs, &ids);
        if (bytes_out) *bytes_out = P.arena_bytes;
    });
}

static RangeSet &get_ranges(Network &net, int32_t n_amps, const int32_t *outputs, size_t cap);

int jet_plan_ranges(jet_network *net, int32_t n_amps, const int32_t *outputs, size_t max_bytes,
                    int32_t *n_fixed_out, int64_t *fixed_labels_out, int64_t *n_ranges_out, double *flop_out,
                    size_t *bytes_out)
{
    return guarded([&] {
        if (!net) fail(JET_EINVAL, "net is NULL");
        if (max_bytes == 0) fail(JET_EINVAL, "max_bytes must be > 0");
        Plan &P = get_plan(*net, n_amps, outputs);
        int32_t nf = 0;
        int64_t nr = 1;
        double flop = P.flop_executed;
        size_t bytes = P.arena_bytes;
        if (P.arena_bytes > max_bytes) {
            if (P.n_slices <= 1) fail(JET_ENOMEM, "the plan needs more workspace than max_bytes and has no slices");
            RangeSet &RS = get_ranges(*net, n_amps, outputs, max_bytes);
            nf = (int32_t)RS.fixed_pos.size();
            for (int32_t j = 0; j < nf && fixed_labels_out; ++j) fixed_labels_out[j] = net->sliced[RS.fixed_pos[j]];
            nr = (int64_t)RS.ids.size();
            flop = RS.flop;
            bytes = RS.arena;
        }
        if (n_fixed_out) *n_fixed_out = nf;
        if (n_ranges_out) *n_ranges_out = nr;
        if (flop_out) *flop_out = flop;
        if (bytes_out) *bytes_out = bytes;
    });
}

int jet_sum_partials(int32_t n_amps, int64_t n_ids, int64_t n_elem, const jet_c128 *partials, jet_c128 *sums_out)
{
    return guarded([&] {
        if (n_amps < 0 || n_ids < 0 || n_elem < 1) fail(JET_EINVAL, "bad sizes");
        if ((n_amps > 0 && n_ids > 0 && !partials) || (n_amps > 0 && !sums_out)) fail(JET_EINVAL, "NULL argument");
        for (int64_t b = 0; b < n_amps; ++b)
            for (int64_t e = 0; e < n_elem; ++e) {
                double re = 0.0, im = 0.0;
                for (int64_t j = 0; j < n_ids; ++j) {
                    const jet_c128 &v = partials[(b * n_ids + j) * n_elem + e];
                    re += v.re;
                    im += v.im;
                }
                sums_out[b * n_elem + e] = jet_c128{re, im};
            }
    });
}

int jet_set_workspace(jet_network *net, void *dptr, size_t bytes)
{
    return guarded([&] {
        if (!net) fail(JET_EINVAL, "net is NULL");
        if (dptr && ((uintptr_t)dptr & 255)) fail(JET_EINVAL, "workspace must be 256-byte aligned");
        net->user_arena = dptr;
        net->user_arena_bytes = dptr ? bytes : 0;
    });
}

// Workspace the plan may use: jet_options.workspace_limit, and no more than a
// caller-provided workspace (0: no limit).
static size_t workspace_cap(const Network &net)
{
    size_t cap = net.opt.workspace_limit > 0 ? (size_t)net.opt.workspace_limit : 0;
    if (net.user_arena && (cap == 0 || net.user_arena_bytes < cap)) cap = net.user_arena_bytes;
    return cap;
}

// The cap a contraction runs under: workspace_cap, or, with no limit set and
// no caller workspace, 90% of the device memory that is free (plus the
// library's own arena, which a larger one replaces) once the plan would need
// more than that.
static size_t run_cap(Network &net, const Plan &P)
{
    size_t cap = workspace_cap(net);
    if (cap) return cap;
    if (P.n_slices <= 1 || P.arena_bytes <= net.own_arena_bytes) return 0;
    const size_t avail = (size_t)(0.9 * (double)device_free_bytes(net)) + net.own_arena_bytes;
    return P.arena_bytes > avail ? avail : 0;
}

// Section 4: when every slice's shared work does not fit at once, a subset of
// the slices is held in memory at a time, its size determined a priori.  A
// range fixes the digits of a set T of the sliced labels and holds every slice
// with those digits; an intermediate with a label of T under it is computed
// once in all (its instances split over the ranges), one without is computed
// again in every range.  Among the sets of the fewest labels whose range plan
// fits the cap, T minimises the FLOP of all ranges together (all subsets when
// there are at most 300 of that size, else the best smaller set extended by one
// label).  Every range has the same plan up to the fixed digits' values, so
// range 0's plan gives the size and the FLOP.
static RangeSet &get_ranges(Network &net, int32_t n_amps, const int32_t *outputs, size_t cap)
{
    const size_t n = (size_t)n_amps * net.open.size();
    RangeSet *R = net.ranges.get();
    if (R && R->n_amps == n_amps && R->path_version == net.path_version && R->slice_version == net.slice_version &&
        R->precision == net.opt.precision && R->reuse == net.opt.reuse && R->cap == cap && R->outputs.size() == n &&
        std::equal(R->outputs.begin(), R->outputs.end(), outputs))
        return *R;
    drop_ranges(net);
    const int ns = (int)net.sliced.size();
    std::vector<int64_t> dim(ns), w(ns, 1);
    for (int j = 0; j < ns; ++j) dim[j] = net.labels.at(net.sliced[j]).dim;
    for (int j = ns - 2; j >= 0; --j) w[j] = w[j + 1] * dim[j + 1];
    const int64_t n_sl = ns ? w[0] * dim[0] : 1;
    // slice ids of range `key` (mixed radix over T's digits, T's first label slowest)
    auto range_ids = [&](const std::vector<int32_t> &T, int64_t key) {
        std::vector<int64_t> want(T.size());
        for (int i = (int)T.size() - 1; i >= 0; --i) {
            want[i] = key % dim[T[i]];
            key /= dim[T[i]];
        }
        std::vector<int64_t> ids;
        for (int64_t s = 0; s < n_sl; ++s) {
            bool ok = true;
            for (size_t i = 0; i < T.size() && ok; ++i) ok = (s / w[T[i]]) % dim[T[i]] == want[i];
            if (ok) ids.push_back(s);
        }
        return ids;
    };
    struct Cand {
        std::vector<int32_t> T;
        double flop;
        size_t arena;
    };
    auto evaluate = [&](const std::vector<int32_t> &T) -> Cand {
        int64_t n_ranges = 1;
        for (int32_t j : T) n_ranges *= dim[j];
        auto ids = range_ids(T, 0);
        auto P = build_plan(net, n_amps, outputs, &ids);
        return {T, P->flop_executed * (double)n_ranges, P->arena_bytes};
    };
    auto binom = [](int nn, int k) {
        double c = 1;
        for (int i = 0; i < k; ++i) c = c * (nn - i) / (i + 1);
        return c;
    };
    Cand best{{}, 0, 0};
    bool found = false;
    std::vector<int32_t> prev_best;   // best set of the previous size, fitting or not
    for (int nt = 1; nt <= ns && !found; ++nt) {
        std::vector<std::vector<int32_t>> cands;
        if (binom(ns, nt) <= 300) {
            std::vector<int32_t> c(nt);
            std::function<void(int, int)> rec = [&](int at, int from) {
                if (at == nt) {
                    cands.push_back(c);
                    return;
                }
                for (int j = from; j < ns; ++j) {
                    c[at] = j;
                    rec(at + 1, j + 1);
                }
            };
            rec(0, 0);
        } else {
            for (int j = 0; j < ns; ++j)
                if (std::find(prev_best.begin(), prev_best.end(), j) == prev_best.end()) {
                    auto c = prev_best;
                    c.push_back(j);
                    std::sort(c.begin(), c.end());
                    cands.push_back(c);
                }
        }
        Cand size_best{{}, 0, 0};
        bool any = false;
        for (auto &T : cands) {
            Cand c = evaluate(T);
            if (!any || c.flop < size_best.flop) {
                size_best = c;
                any = true;
            }
            if (c.arena <= cap && (!found || c.flop < best.flop || (c.flop == best.flop && c.arena < best.arena))) {
                best = c;
                found = true;
            }
        }
        prev_best = size_best.T;
    }
    if (!found) fail(JET_ENOMEM, "one slice needs more workspace than the limit");
    auto RS = std::make_unique<RangeSet>();
    RS->outputs.assign(outputs, outputs + n);
    RS->n_amps = n_amps;
    RS->path_version = net.path_version;
    RS->slice_version = net.slice_version;
    RS->precision = net.opt.precision;
    RS->reuse = net.opt.reuse;
    RS->cap = cap;
    RS->fixed_pos = best.T;
    RS->flop = best.flop;
    RS->arena = best.arena;
    int64_t n_ranges = 1;
    for (int32_t j : best.T) n_ranges *= dim[j];
    for (int64_t k = 0; k < n_ranges; ++k) RS->ids.push_back(range_ids(best.T, k));
    RS->plans.resize((size_t)n_ranges);
    net.ranges = std::move(RS);
    return *net.ranges;
}

// Runs every range (its plan kept across calls, except while shared work is
// being kept: a range after the first reads what the first kept) and sums the
// per-slice partials in increasing slice id in FP64 -- the order of the single
// plan's reduction (a range's plan may route a node with fewer instances to
// another kernel form, so the values agree to the arithmetic's rounding).
// Writes n_amps * n_elem sums to `sums` (host).
static void contract_in_ranges(Network &net, int32_t n_amps, const int32_t *outputs, size_t cap, void *stream,
                               std::vector<jet_c128> &sums)
{
    const int64_t n_sl = net.plan->n_slices, n_elem = net.plan->n_elem;
    RangeSet &RS = get_ranges(net, n_amps, outputs, cap);
    ensure_workspace(net, RS.arena, stream);
    std::vector<jet_c128> all((size_t)n_amps * n_sl * n_elem, jet_c128{0.0, 0.0}), part;
    void *s = stream ? stream : net.stream;
    for (size_t r = 0; r < RS.plans.size(); ++r) {
        const std::vector<int64_t> &ids = RS.ids[r];
        const int64_t n_ids = (int64_t)ids.size();
        if (net.keep_min > 0) check_kept_key(net);
        if (!RS.plans[r] || RS.plans[r]->superseded || net.keep_min > 0) {
            if (RS.plans[r]) {
                if (net.last_run == RS.plans[r].get()) net.last_run = nullptr;
                release_plan_device(*RS.plans[r]);
            }
            RS.plans[r] = build_plan(net, n_amps, outputs, &ids);
        }
        Plan &P = *RS.plans[r];
        bind_and_run(net, P, nullptr, stream);
        part.resize((size_t)n_amps * n_ids * n_elem);
        copy_d2h(part.data(), net.d_amps, part.size() * sizeof(jet_c128), s);
        if (read_clear_status(net, stream))
            fail(JET_ETIMEOUT, "a bounded device-side wait ran out (status bits: 1 GEMM, 2 application, 8 chain barrier)");
        mark_kept(net, P, stream);
        for (int32_t b = 0; b < n_amps; ++b)
            for (int64_t j = 0; j < n_ids; ++j)
                std::memcpy(&all[((size_t)b * n_sl + ids[j]) * n_elem], &part[((size_t)b * n_ids + j) * n_elem],
                            (size_t)n_elem * sizeof(jet_c128));
    }
    sums.assign((size_t)n_amps * n_elem, jet_c128{0.0, 0.0});
    for (int32_t b = 0; b < n_amps; ++b)
        for (int64_t sid = 0; sid < n_sl; ++sid)
            for (int64_t e = 0; e < n_elem; ++e) {
                const jet_c128 &v = all[((size_t)b * n_sl + sid) * n_elem + e];
                jet_c128 &acc = sums[(size_t)b * n_elem + e];
                acc.re += v.re;
                acc.im += v.im;
            }
}

int jet_contract_async(jet_network *net, int32_t n_amps, const int32_t *outputs, jet_c128 *amps_dev,
                       void *cuda_stream)
{
    return guarded([&] {
        if (!net || !amps_dev) fail(JET_EINVAL, "NULL argument");
        Plan &P = get_plan(*net, n_amps, outputs);
        const size_t cap = run_cap(*net, P);
        if (cap && P.arena_bytes > cap && P.n_slices > 1) {   // slice ranges: synchronous
            std::vector<jet_c128> sums;
            contract_in_ranges(*net, n_amps, outputs, cap, cuda_stream, sums);
            copy_h2d_sync(amps_dev, sums.data(), sums.size() * sizeof(jet_c128), cuda_stream ? cuda_stream : net->stream);
            return;
        }
        bind_and_run(*net, P, nullptr, cuda_stream);
        copy_d2d_async(amps_dev, net->d_amps, (size_t)n_amps * P.n_elem * sizeof(jet_c128),
                       cuda_stream ? cuda_stream : net->stream);
        mark_kept(*net, P, cuda_stream);
    });
}

int jet_contract(jet_network *net, int32_t n_amps, const int32_t *outputs, jet_c128 *amps_out, void *cuda_stream)
{
    return guarded([&] {
        if (!net || !amps_out) fail(JET_EINVAL, "NULL argument");
        Plan &P = get_plan(*net, n_amps, outputs);
        const size_t cap = run_cap(*net, P);
        if (cap && P.arena_bytes > cap && P.n_slices > 1) {
            std::vector<jet_c128> sums;
            contract_in_ranges(*net, n_amps, outputs, cap, cuda_stream, sums);
            std::memcpy(amps_out, sums.data(), sums.size() * sizeof(jet_c128));
            return;
        }
        bind_and_run(*net, P, nullptr, cuda_stream);
        copy_d2h(amps_out, net->d_amps, (size_t)n_amps * P.n_elem * sizeof(jet_c128),
                 cuda_stream ? cuda_stream : net->stream);
        if (read_clear_status(*net, cuda_stream))
            fail(JET_ETIMEOUT, "a bounded device-side wait ran out (status bits: 1 GEMM, 2 application, 8 chain barrier)");
        mark_kept(*net, P, cuda_stream);
    });
}

int jet_contract_slices(jet_network *net, int32_t n_amps, const int32_t *outputs, int32_t n_ids,
                        const int64_t *slice_ids, jet_c128 *partials_out, void *cuda_stream)
{
    return guarded([&] {
        if (!net || !partials_out || !slice_ids || n_ids < 1) fail(JET_EINVAL, "bad arguments");
        std::vector<int64_t> ids(slice_ids, slice_ids + n_ids);
        Plan &P = get_plan(*net, n_amps, outputs, &ids);
        bind_and_run(*net, P, nullptr, cuda_stream);
        copy_d2h(partials_out, net->d_amps, (size_t)n_amps * n_ids * P.n_elem * sizeof(jet_c128),
                 cuda_stream ? cuda_stream : net->stream);
        if (read_clear_status(*net, cuda_stream))
            fail(JET_ETIMEOUT, "a bounded device-side wait ran out (status bits: 1 GEMM, 2 application, 8 chain barrier)");
        mark_kept(*net, P, cuda_stream);
    });
}

int jet_contract_grad(jet_network *net, int32_t n_amps, const int32_t *outputs, const jet_c128 *cot,
                      int32_t n_req, const int32_t *tensor_ids, jet_c64 *const *env_out, jet_c128 *amps_out,
                      void *cuda_stream)
{
    return guarded([&] {
        if (net && !net->free_open.empty()) fail(JET_EINVAL, "gradients need every open leg fixed (no free legs)");
        if (!net || !cot || n_amps < 1 || n_req < 0 || (n_req > 0 && (!tensor_ids || !env_out)))
            fail(JET_EINVAL, "bad arguments");
        if (net->path.size() + 1 != net->leaves.size()) fail(JET_ESTATE, "no contraction path set");
        GradRequest g;
        g.cot.resize(2 * (size_t)n_amps);
        for (int32_t b = 0; b < n_amps; ++b) {
            g.cot[2 * b] = cot[b].re;
            g.cot[2 * b + 1] = cot[b].im;
        }
        g.env_off.assign(net->leaves.size(), -1);
        int64_t total = 0;
        for (int32_t i = 0; i < n_req; ++i) {
            const int32_t id = tensor_ids[i];
            if (id < 0 || id >= (int32_t)net->leaves.size()) fail(JET_EINVAL, "bad tensor id " + std::to_string(id));
            if (g.env_off[id] >= 0) fail(JET_EINVAL, "tensor id requested twice");
            if (!env_out[i]) fail(JET_EINVAL, "NULL environment buffer");
            g.env_off[id] = total;
            total += net->leaves[id].size;
            g.leaves.push_back(id);
        }
        int64_t n_sl = 1;
        for (int64_t l : net->sliced) n_sl *= net->labels.at(l).dim;
        const bool fp64 = net->opt.precision == JET_PREC_FP64;
        // an unsliced network keeps its adjoint plan: later calls with the same
        // outputs and tensor ids only rewrite the cotangent seed
        const bool cacheable = n_sl == 1;
        Plan *GP = net->grad_plan.get();
        const bool hit = cacheable && GP && GP->n_amps == n_amps && GP->path_version == net->path_version &&
                         GP->slice_version == net->slice_version && GP->precision == net->opt.precision &&
                         GP->reuse == net->opt.reuse && GP->outputs.size() == (size_t)n_amps * net->open.size() &&
                         std::equal(GP->outputs.begin(), GP->outputs.end(), outputs) && GP->grad_leaves == g.leaves;
        std::unique_ptr<Plan> first;
        if (hit) {
            write_seed(*GP, g.cot, fp64);
        } else {   // plan the first slice on the host before any device work (argument errors surface here)
            std::vector<int64_t> ids0{0};
            first = build_plan(*net, n_amps, outputs, &ids0, &g);
            if (cacheable) {
                if (net->grad_plan) {
                    if (net->last_run == net->grad_plan.get()) net->last_run = nullptr;
                    release_plan_device(*net->grad_plan);
                }
                net->grad_plan = std::move(first);
                GP = net->grad_plan.get();
            }
        }
        ensure_leaves_on_device(*net);
        void *s = cuda_stream ? cuda_stream : net->stream;
        if (net->d_env_cap < std::max<int64_t>(total, 1)) {
            device_free(net->d_env);
            net->d_env = nullptr;
            net->d_env = device_alloc((size_t)std::max<int64_t>(total, 1) * sizeof(jet_c128));
            net->d_env_cap = std::max<int64_t>(total, 1);
        }
        device_memset_async(net->d_env, (size_t)std::max<int64_t>(total, 1) * sizeof(jet_c128), s);
        // per slice: recompute the forward tree (shared work reused across the
        // amplitudes, not across slices), sweep it backwards, accumulate in FP64
        std::vector<double> amps(2 * (size_t)n_amps, 0.0);
        std::vector<jet_c128> part(n_amps);
        for (int64_t sl = 0; sl < n_sl; ++sl) {
            if (cacheable) {   // one plan, kept (and its graph) for the next call
                bind_and_run(*net, *GP, nullptr, cuda_stream, true);
                copy_d2h(part.data(), net->d_amps, (size_t)n_amps * sizeof(jet_c128), s);
            } else {
                std::unique_ptr<Plan> P;
                if (sl == 0 && first) {
                    P = std::move(first);
                } else {
                    std::vector<int64_t> ids{sl};
                    P = build_plan(*net, n_amps, outputs, &ids, &g);
                }
                try {
                    bind_and_run(*net, *P, nullptr, cuda_stream, false);
                    copy_d2h(part.data(), net->d_amps, (size_t)n_amps * sizeof(jet_c128), s);
                } catch (...) {
                    net->last_run = nullptr;
                    release_plan_device(*P);
                    throw;
                }
                net->last_run = nullptr;
                release_plan_device(*P);
            }
            for (int32_t b = 0; b < n_amps; ++b) {
                amps[2 * b] += part[b].re;
                amps[2 * b + 1] += part[b].im;
            }
            if (read_clear_status(*net, cuda_stream))
                fail(JET_ETIMEOUT, "a bounded device-side wait ran out (status bits: 1 GEMM, 2 application, 8 chain barrier)");
        }
        std::vector<jet_c128> env((size_t)std::max<int64_t>(total, 1));
        copy_d2h(env.data(), net->d_env, (size_t)std::max<int64_t>(total, 1) * sizeof(jet_c128), s);
        for (int32_t i = 0; i < n_req; ++i) {
            const int64_t off = g.env_off[tensor_ids[i]], n = net->leaves[tensor_ids[i]].size;
            for (int64_t e = 0; e < n; ++e) env_out[i][e] = {(float)env[off + e].re, (float)env[off + e].im};
        }
        if (amps_out)
            for (int32_t b = 0; b < n_amps; ++b) amps_out[b] = {amps[2 * b], amps[2 * b + 1]};
    });
}

int jet_profile(const jet_network *net, jet_op_record *out, int32_t cap, int32_t *n_out)
{
    return guarded([&] {
        if (!net) fail(JET_EINVAL, "net is NULL");
        const Plan *PP = net->last_run ? net->last_run : net->plan.get();
        if (!PP) fail(JET_ESTATE, "no plan yet");
        const Plan &P = *PP;
        if (n_out) *n_out = (int32_t)P.ops.size();
        for (size_t i = 0; out && i < P.ops.size() && (int32_t)i < cap; ++i) {
            const Op &op = P.ops[i];
            out[i].kind = (int32_t)op.kind;
            out[i].node = op.node;
            out[i].n_inst = op.n_inst;
            out[i].flop = op.flop;
            out[i].bytes = op.bytes;
            out[i].ms = op_elapsed_ms(P, i);
            out[i].block = op.block;
            out[i].grid[0] = op.grid_x;
            out[i].grid[1] = op.grid_y;
            out[i].grid[2] = op.grid_z;
            out[i].smem = op.smem;
            out[i].variant = op.variant;
            out[i].pad_ = 0;
        }
    });
}

int jet_plan_buffers(const jet_network *net, jet_buffer_record *out, int32_t cap, int32_t *n_out)
{
    return guarded([&] {
        if (!net) fail(JET_EINVAL, "net is NULL");
        const Plan *PP = net->last_run ? net->last_run : net->plan.get();
        if (!PP) fail(JET_ESTATE, "no plan yet");
        const Plan &P = *PP;
        // launches of each tree node (a batched launch counts for every node it
        // holds); the slice reduction reads only the root's own result, so it
        // does not count as a read of the root's children
        std::vector<int32_t> first(P.parent.size(), -1), last(P.parent.size(), -1), last_contract(P.parent.size(), -1);
        auto touch = [&](int32_t v, int32_t i, bool reduce) {
            if (v < 0 || (size_t)v >= first.size()) return;
            if (first[v] < 0) first[v] = i;
            last[v] = i;
            if (!reduce) last_contract[v] = i;
        };
        for (size_t i = 0; i < P.ops.size(); ++i) {
            const Op &op = P.ops[i];
            if (op.batch_count > 0)
                for (int32_t j = 0; j < op.batch_count; ++j) touch(P.batch_nodes[op.batch_first + j], (int32_t)i, false);
            else
                touch(op.node, (int32_t)i, op.kind == OpKind::Reduce);
        }
        if (n_out) *n_out = (int32_t)P.buffers.size();
        for (size_t i = 0; out && i < P.buffers.size() && (int32_t)i < cap; ++i) {
            const Plan::BufferRec &b = P.buffers[i];
            jet_buffer_record &r = out[i];
            std::memset(&r, 0, sizeof r);
            r.node = b.node;
            r.offset = b.offset;
            r.bytes = b.bytes;
            r.t_alloc = b.t_alloc;
            r.t_release = b.t_release;
            r.first_use = r.last_use = -1;
            if (b.node >= 0) {
                r.first_use = first[b.node];
                const int32_t pa = P.parent[b.node];
                r.last_use = std::max(last[b.node], pa >= 0 ? last_contract[pa] : -1);
            }
        }
    });
}

int jet_stats(const jet_network *net, jet_stats_t *out)
{
    return guarded([&] {
        if (!net || !out) fail(JET_EINVAL, "NULL argument");
        std::memset(out, 0, sizeof *out);
        out->flop_planned = net->flop_planned;
        double nsl = 1;
        for (int64_t l : net->sliced) nsl *= net->labels.at(l).dim;
        out->n_slices = (int32_t)nsl;
        out->n_sliced_labels = (int32_t)net->sliced.size();
        if (net->path.size() + 1 == net->leaves.size()) {
            PathCost c = path_cost(*net, net->path, net->sliced);
            out->flop_sliced = nsl * c.flop;
            out->max_intermediate = (int64_t)c.max_size;
        }
        if (net->plan) {
            const Plan &P = *net->plan;
            out->flop_executed = P.flop_executed;
            out->bytes_executed = P.bytes_executed;
            out->workspace_bytes = (int64_t)P.arena_bytes;
            out->n_instances = P.n_instances;
            out->n_launches = (int64_t)P.ops.size();
            out->n_gemm_nodes = P.n_gemm;
            out->n_direct_nodes = P.n_direct;
            double per_assign = out->flop_sliced / std::max(nsl, 1.0);   // FLOP_sl
            double n_assign = (double)P.n_amps * nsl;
            double noreuse = n_assign * per_assign;
            if (n_assign > 1 && per_assign > 0)
                out->reuse_fraction = (noreuse - P.flop_executed) / ((n_assign - 1) * per_assign);
        }
    });
}

int jet_autotune(jet_network *net, int32_t n_amps, const int32_t *outputs, const char *cache_file,
                 void *cuda_stream, double *default_ms, double *tuned_ms, int32_t *n_changed)
{
    return guarded([&] {
        if (!net) fail(JET_EINVAL, "net is NULL");
        Network &N = *net;
        // the slices a tuning run contracts: every slice, or the first range of the
        // partition the workspace cap asks for (every range has the same launches)
        Plan &Pfull = get_plan(N, n_amps, outputs);
        const size_t cap = run_cap(N, Pfull);
        std::vector<int64_t> ids;
        const std::vector<int64_t> *idp = nullptr;
        if (cap && Pfull.arena_bytes > cap && Pfull.n_slices > 1) {
            RangeSet &RS = get_ranges(N, n_amps, outputs, cap);
            ids = RS.ids[0];
            idp = &ids;
        }
        N.tune.clear();
        N.tune_path_version = N.path_version;
        N.tune_slice_version = N.slice_version;
        invalidate_plan(N);
        // cache: one "signature choice" line per tunable shape
        std::map<std::string, int> cache;
        if (cache_file && *cache_file) {
            if (FILE *f = std::fopen(cache_file, "r")) {
                char key[512];
                int val;
                while (std::fscanf(f, "%511s %d", key, &val) == 2) cache[key] = val;
                std::fclose(f);
            }
        }
        // one timed run (the second of two) with every tunable node in its default
        // form (flip 0) or its other one (flip 1): per-node and total device time
        auto run = [&](int flip, std::map<int32_t, double> &node_ms, std::vector<Plan::Tunable> &tun) {
            N.tune_flip = flip;
            std::unique_ptr<Plan> P;
            try {
                P = build_plan(N, n_amps, outputs, idp);
            } catch (...) {
                N.tune_flip = 0;
                throw;
            }
            N.tune_flip = 0;
            const int32_t saved = N.opt.profile;
            N.opt.profile = 2;
            double total = 0;
            try {
                for (int rep = 0; rep < 2; ++rep) {
                    bind_and_run(N, *P, nullptr, cuda_stream);
                    sync_stream(N, cuda_stream);
                }
                if (read_clear_status(N, cuda_stream)) fail(JET_ETIMEOUT, "a bounded device-side wait ran out");
                for (size_t i = 0; i < P->ops.size(); ++i) {
                    const float ms = op_elapsed_ms(*P, i);
                    if (ms <= 0) continue;
                    total += ms;
                    if (P->ops[i].batch_count == 0) node_ms[P->ops[i].node] += ms;
                }
            } catch (...) {
                N.opt.profile = saved;
                if (N.last_run == P.get()) N.last_run = nullptr;
                release_plan_device(*P);
                throw;
            }
            N.opt.profile = saved;
            tun = P->tunables;
            if (N.last_run == P.get()) N.last_run = nullptr;
            release_plan_device(*P);
            return total;
        };
        std::map<int32_t, double> ms0, ms1, msx;
        std::vector<Plan::Tunable> tun0, tun1, tunx;
        const double t_default = run(0, ms0, tun0);
        int changed = 0;
        bool all_cached = !tun0.empty();
        for (const auto &t : tun0) all_cached = all_cached && cache.count(t.sig);
        auto set_choice = [&](const Plan::Tunable &t, int taken) {
            TuneChoice &c = N.tune[t.node];
            (t.kind == 0 ? c.group : t.kind == 1 ? c.apply_tc : c.dot) = (int8_t)taken;
            if (taken != t.taken) ++changed;
        };
        if (all_cached) {
            for (const auto &t : tun0) set_choice(t, cache[t.sig]);
        } else if (!tun0.empty()) {
            run(1, ms1, tun1);
            std::map<std::pair<int32_t, int32_t>, int32_t> other;
            for (const auto &t : tun1) other[{t.node, t.kind}] = t.taken;
            for (const auto &t : tun0) {
                auto it = other.find({t.node, t.kind});
                auto both = [&](std::map<int32_t, double> &ms) { return ms[t.node] + (t.node2 >= 0 ? ms[t.node2] : 0.0); };
                const bool flip = it != other.end() && it->second != t.taken && both(ms1) < 0.97 * both(ms0);
                set_choice(t, flip ? it->second : t.taken);
                cache[t.sig] = flip ? it->second : t.taken;
            }
        }
        double t_tuned = t_default;
        if (changed) {
            t_tuned = run(0, msx, tunx);
            if (t_tuned > 1.02 * t_default) {   // the choices did not combine well: keep the defaults
                N.tune.clear();
                for (const auto &t : tun0) cache[t.sig] = t.taken;
                changed = 0;
                t_tuned = t_default;
            }
        }
        if (cache_file && *cache_file && !all_cached && !tun0.empty()) {
            if (FILE *f = std::fopen(cache_file, "w")) {
                for (const auto &kv : cache) std::fprintf(f, "%s %d\n", kv.first.c_str(), kv.second);
                std::fclose(f);
            }
        }
        invalidate_plan(N);   // the next contraction plans with the choices
        if (default_ms) *default_ms = t_default;
        if (tuned_ms) *tuned_ms = t_tuned;
        if (n_changed) *n_changed = changed;
    });
}

int jet_selftest_wait(jet_network *net, int64_t limit_us, void *cuda_stream)
{
    return guarded([&] {
        if (!net) fail(JET_EINVAL, "net is NULL");
        if (limit_us < 1 || limit_us > 10000000) fail(JET_EINVAL, "limit_us must be in [1, 10^7]");
        const int st = selftest_wait(*net, limit_us, cuda_stream);
        if ((st & 12) == 12) fail(JET_ETIMEOUT, "the bounded device-side waits ran out (self-test)");
        fail(JET_ECUDA, "a self-test wait completed although nothing arrives on its barrier");
    });
}

int jet_pair_contract_noalloc(int32_t rank_a, const int64_t *labels_a, const int32_t *dims_a, const jet_c64 *a_dev,
                              int32_t rank_b, const int64_t *labels_b, const int32_t *dims_b, const jet_c64 *b_dev,
                              jet_c64 *c_dev, int32_t device, void *cuda_stream)
{
    return guarded([&] {
        pair_contract_noalloc(rank_a, labels_a, dims_a, a_dev, rank_b, labels_b, dims_b, b_dev, c_dev, device,
                              cuda_stream);
    });
}

void jet_network_destroy(jet_network *net)
{
    if (!net) return;
    try {
        free_network_device(*net);
    } catch (...) {
    }
    delete net;
}

const char *jet_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
