// Host-side planner: contraction tree, FLOP/size model, greedy path, slice finder.
//
// Section 2.3: a pairwise path is a binary contraction tree; each step sums the
// labels its two operands share.  Section 2.4 (Eq. sliced_flops): slicing
// fixes labels, shrinking every intermediate that carries them and multiplying
// the work by the number of slices.  Section 3.2 (Eq. task_based_amplitude_flops):
// with shared work reused, a tree node is computed once per distinct assignment
// of the sliced labels that occur under it, not once per slice.
#include <algorithm>
#include <array>
#include <cmath>
#include <functional>
#include <iterator>
#include <map>
#include <set>
#include <unordered_set>

#include "internal.h"

namespace jet {

static double label_size(const Network &net, const std::vector<int64_t> &ls,
                         const std::unordered_set<int64_t> &fixed)
{
    double s = 1;
    for (int64_t l : ls)
        if (!fixed.count(l)) s *= (double)net.labels.at(l).dim;
    return s;
}

// labels of a contraction result: symmetric difference, a's order then b's
static std::vector<int64_t> sym_diff(const std::vector<int64_t> &a, const std::vector<int64_t> &b)
{
    std::vector<int64_t> out;
    out.reserve(a.size() + b.size());
    for (int64_t x : a)
        if (std::find(b.begin(), b.end(), x) == b.end()) out.push_back(x);
    for (int64_t x : b)
        if (std::find(a.begin(), a.end(), x) == a.end()) out.push_back(x);
    return out;
}

static std::vector<int64_t> set_union(const std::vector<int64_t> &a, const std::vector<int64_t> &b)
{
    std::vector<int64_t> out = a;
    for (int64_t x : b)
        if (std::find(a.begin(), a.end(), x) == a.end()) out.push_back(x);
    return out;
}

void validate_path(const Network &net, const std::vector<std::pair<int32_t, int32_t>> &path)
{
    int32_t n = (int32_t)net.leaves.size();
    if ((int32_t)path.size() != n - 1)
        fail(JET_EINVAL, "path must have n_tensors - 1 = " + std::to_string(n - 1) + " steps, got " +
                             std::to_string(path.size()));
    std::vector<char> used(2 * n, 0);
    for (int32_t k = 0; k < (int32_t)path.size(); ++k) {
        int32_t a = path[k].first, b = path[k].second;
        int32_t limit = n + k;  // ids < n + k exist before step k
        if (a < 0 || b < 0 || a >= limit || b >= limit || a == b)
            fail(JET_EINVAL, "path step " + std::to_string(k) + ": invalid ids (" + std::to_string(a) +
                                 ", " + std::to_string(b) + ")");
        if (used[a] || used[b])
            fail(JET_EINVAL, "path step " + std::to_string(k) + ": an id is consumed twice");
        used[a] = used[b] = 1;
    }
}

Tree build_tree(const Network &net, const std::vector<std::pair<int32_t, int32_t>> &path)
{
    Tree t;
    t.n_leaves = (int32_t)net.leaves.size();
    t.children = path;
    t.labels.resize(t.n_leaves + path.size());
    for (int32_t i = 0; i < t.n_leaves; ++i) t.labels[i] = net.leaves[i].labels;
    for (size_t k = 0; k < path.size(); ++k)
        t.labels[t.n_leaves + k] = sym_diff(t.labels[path[k].first], t.labels[path[k].second]);
    return t;
}

static std::unordered_set<int64_t> fixed_set(const Network &net, const std::vector<int64_t> &extra)
{
    std::unordered_set<int64_t> f(extra.begin(), extra.end());
    for (auto &kv : net.labels)   // open legs: fixed by every amplitude, unless left free
        if (kv.second.n_owner == 1 &&
            std::find(net.free_open.begin(), net.free_open.end(), kv.first) == net.free_open.end())
            f.insert(kv.first);
    return f;
}

PathCost path_cost(const Network &net, const std::vector<std::pair<int32_t, int32_t>> &path,
                   const std::vector<int64_t> &fixed_extra)
{
    auto fixed = fixed_set(net, fixed_extra);
    Tree t = build_tree(net, path);
    PathCost c;
    c.node_size.resize(t.labels.size());
    for (size_t i = 0; i < t.labels.size(); ++i) c.node_size[i] = label_size(net, t.labels[i], fixed);
    for (size_t k = 0; k < path.size(); ++k) {
        auto u = set_union(t.labels[path[k].first], t.labels[path[k].second]);
        double f = 8.0 * label_size(net, u, fixed);
        c.step_flop.push_back(f);
        c.flop += f;
        c.max_size = std::max(c.max_size, c.node_size[t.n_leaves + k]);
    }
    return c;
}

// Sum over tree nodes of (number of distinct sliced-label assignments under the
// node) x (node FLOP with the sliced labels fixed): Eq. task_based_amplitude_flops
// counted exactly, node by node.
double reuse_aware_flop(const Network &net, const std::vector<std::pair<int32_t, int32_t>> &path,
                        const std::vector<int64_t> &sliced)
{
    auto fixed = fixed_set(net, sliced);
    std::unordered_set<int64_t> sl(sliced.begin(), sliced.end());
    Tree t = build_tree(net, path);
    int32_t n = t.n_leaves;
    std::vector<std::vector<int64_t>> under(t.labels.size());  // sliced labels under each node
    for (int32_t i = 0; i < n; ++i)
        for (int64_t l : net.leaves[i].labels)
            if (sl.count(l)) under[i].push_back(l);
    double total = 0;
    for (size_t k = 0; k < path.size(); ++k) {
        int32_t a = path[k].first, b = path[k].second;
        auto u = set_union(under[a], under[b]);
        double inst = 1;
        for (int64_t l : u) inst *= net.labels.at(l).dim;
        under[n + k] = u;
        auto un = set_union(t.labels[a], t.labels[b]);
        total += inst * 8.0 * label_size(net, un, fixed);
    }
    return total;
}

// ------------------------------------------------------------ greedy path
namespace {
struct Cand {
    int over;              // result above the memory cap: taken only when nothing else is left
    double score, flop;
    int32_t a, b;
    bool operator<(const Cand &o) const
    {
        if (over != o.over) return over < o.over;
        if (score != o.score) return score < o.score;
        if (flop != o.flop) return flop < o.flop;
        if (a != o.a) return a < o.a;
        return b < o.b;
    }
};

struct SplitMix {
    uint64_t s;
    uint64_t next()
    {
        s += 0x9E3779B97F4A7C15ull;
        uint64_t z = s;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    }
    double uniform() { return (next() >> 11) * (1.0 / 9007199254740992.0); }
};
}  // namespace

// Number of distinct restrictions of a batch of output patterns to a set of
// open legs: how many instances a tree node holding those legs has when the
// batch is contracted with shared work reused (Section 3.2; the legs are fixed
// by the amplitudes' bras).  Memoised per leg set.
struct BatchInstances {
    int32_t n_amps = 0, n_out = 0;
    const int32_t *outputs = nullptr;                 // n_amps x n_out digits
    std::unordered_map<int64_t, int32_t> digit;       // open label -> digit position
    std::map<std::vector<int32_t>, double> memo;

    double count(const std::vector<int32_t> &pos)
    {
        if (pos.empty() || n_amps <= 1) return 1;
        auto it = memo.find(pos);
        if (it != memo.end()) return it->second;
        std::vector<int32_t> rows(n_amps);
        for (int32_t i = 0; i < n_amps; ++i) rows[i] = i;
        auto less = [&](int32_t x, int32_t y) {
            for (int32_t p : pos) {
                const int32_t dx = outputs[(size_t)x * n_out + p], dy = outputs[(size_t)y * n_out + p];
                if (dx != dy) return dx < dy;
            }
            return false;
        };
        std::sort(rows.begin(), rows.end(), less);
        double distinct = 1;
        for (int32_t i = 1; i < n_amps; ++i)
            if (less(rows[i - 1], rows[i])) distinct += 1;
        memo[pos] = distinct;
        return distinct;
    }
};

static std::vector<int32_t> merge_pos(const std::vector<int32_t> &a, const std::vector<int32_t> &b)
{
    std::vector<int32_t> out;
    std::set_union(a.begin(), a.end(), b.begin(), b.end(), std::back_inserter(out));
    return out;
}

// One greedy pass.  Score of a candidate pair = (elements written) - (elements
// freed), each tensor counted once per instance it has under the batch `bt`
// (one instance each when bt is null: a single amplitude).
static std::vector<std::pair<int32_t, int32_t>> greedy_once(const Network &net, SplitMix *rng,
                                                            double temperature, double *flop_out,
                                                            BatchInstances *bt, double cap, double *peak_out)
{
    auto fixed = fixed_set(net, {});
    int32_t n = (int32_t)net.leaves.size();
    std::vector<std::vector<int64_t>> lab(2 * n);
    std::vector<double> size(2 * n, 0), inst(2 * n, 1);
    std::vector<std::vector<int32_t>> opos(2 * n);    // open-leg digit positions under each node
    std::vector<char> alive(2 * n, 0);
    std::unordered_map<int64_t, std::vector<int32_t>> owner;
    for (int32_t i = 0; i < n; ++i) {
        lab[i] = net.leaves[i].labels;
        size[i] = label_size(net, lab[i], fixed);
        alive[i] = 1;
        for (int64_t l : lab[i]) owner[l].push_back(i);
        if (bt) {
            for (int64_t l : lab[i]) {
                auto it = bt->digit.find(l);
                if (it != bt->digit.end()) opos[i].push_back(it->second);
            }
            std::sort(opos[i].begin(), opos[i].end());
            inst[i] = bt->count(opos[i]);
        }
    }
    std::set<Cand> cands;
    std::map<std::pair<int32_t, int32_t>, Cand> by_pair;
    auto add_pair = [&](int32_t a, int32_t b) {
        if (a > b) std::swap(a, b);
        if (by_pair.count({a, b})) return;
        auto out = sym_diff(lab[a], lab[b]);
        auto un = set_union(lab[a], lab[b]);
        const double io = bt ? bt->count(merge_pos(opos[a], opos[b])) : 1.0;
        double so = label_size(net, out, fixed);
        double score = io * so - inst[a] * size[a] - inst[b] * size[b];
        if (rng) {
            double g = -std::log(-std::log(std::max(rng->uniform(), 1e-300)));
            double ls = (score >= 0 ? 1 : -1) * std::log2(1 + std::fabs(score));
            score = ls - temperature * g;
        }
        Cand c{io * so > cap ? 1 : 0, score, io * 8.0 * label_size(net, un, fixed), a, b};
        cands.insert(c);
        by_pair[{a, b}] = c;
    };
    auto drop_node = [&](int32_t x) {
        for (int64_t l : lab[x])
            for (int32_t y : owner[l]) {
                if (y == x) continue;
                auto key = std::make_pair(std::min(x, y), std::max(x, y));
                auto it = by_pair.find(key);
                if (it != by_pair.end()) {
                    cands.erase(it->second);
                    by_pair.erase(it);
                }
            }
    };
    for (auto &kv : owner)
        if (kv.second.size() == 2) add_pair(kv.second[0], kv.second[1]);

    std::vector<std::pair<int32_t, int32_t>> path;
    double total = 0, peak = 0;
    int32_t next = n;
    int32_t n_alive = n;
    while (n_alive > 1) {
        int32_t a, b;
        if (!cands.empty()) {
            Cand c = *cands.begin();
            a = c.a;
            b = c.b;
        } else {  // disconnected: join the two smallest
            std::vector<int32_t> ids;
            for (int32_t i = 0; i < next; ++i)
                if (alive[i]) ids.push_back(i);
            std::sort(ids.begin(), ids.end(), [&](int32_t x, int32_t y) {
                return size[x] != size[y] ? size[x] < size[y] : x < y;
            });
            a = std::min(ids[0], ids[1]);
            b = std::max(ids[0], ids[1]);
        }
        drop_node(a);
        drop_node(b);
        int32_t c = next++;
        lab[c] = sym_diff(lab[a], lab[b]);
        size[c] = label_size(net, lab[c], fixed);
        opos[c] = merge_pos(opos[a], opos[b]);
        inst[c] = bt ? bt->count(opos[c]) : 1.0;
        total += inst[c] * 8.0 * label_size(net, set_union(lab[a], lab[b]), fixed);
        peak = std::max(peak, inst[c] * size[c]);
        alive[a] = alive[b] = 0;
        alive[c] = 1;
        --n_alive;
        for (int64_t l : lab[a]) {
            auto &o = owner[l];
            o.erase(std::remove(o.begin(), o.end(), a), o.end());
        }
        for (int64_t l : lab[b]) {
            auto &o = owner[l];
            o.erase(std::remove(o.begin(), o.end(), b), o.end());
        }
        for (int64_t l : lab[c]) owner[l].push_back(c);
        for (int64_t l : lab[c])
            for (int32_t y : owner[l])
                if (y != c) add_pair(c, y);
        path.push_back({a, b});
    }
    if (flop_out) *flop_out = total;
    if (peak_out) *peak_out = peak;
    return path;
}

// One linear (sequential) greedy pass: a single tensor grows from leaf
// `start`, each step absorbing the leaf that shares a label with it and leaves
// the smallest instance-weighted result (ties: smaller step FLOP, smaller id).
// For a circuit this includes the state-vector (Schroedinger) order and its
// light-cone variants, which pairwise greedy rarely finds.
static std::vector<std::pair<int32_t, int32_t>> greedy_linear(const Network &net, int32_t start, SplitMix *rng,
                                                              double temperature, double *flop_out,
                                                              BatchInstances *bt, double cap, double *peak_out)
{
    auto fixed = fixed_set(net, {});
    const int32_t n = (int32_t)net.leaves.size();
    std::vector<std::vector<int32_t>> lpos(n);
    if (bt)
        for (int32_t i = 0; i < n; ++i) {
            for (int64_t l : net.leaves[i].labels) {
                auto it = bt->digit.find(l);
                if (it != bt->digit.end()) lpos[i].push_back(it->second);
            }
            std::sort(lpos[i].begin(), lpos[i].end());
        }
    std::vector<char> used(n, 0);
    std::vector<int64_t> T = net.leaves[start].labels;
    std::vector<int32_t> tpos = lpos[start];
    used[start] = 1;
    int32_t tid = start;
    std::vector<std::pair<int32_t, int32_t>> path;
    double total = 0, peak = 0;
    for (int32_t k = 0; k + 1 < n; ++k) {
        std::set<int32_t> nb;
        for (int64_t l : T) {
            const LabelInfo &li = net.labels.at(l);
            for (int q = 0; q < li.n_owner; ++q)
                if (li.owner[q] >= 0 && !used[li.owner[q]]) nb.insert(li.owner[q]);
        }
        if (nb.empty())   // disconnected remainder: take the smallest leaf
            for (int32_t i = 0; i < n; ++i)
                if (!used[i]) {
                    if (nb.empty() || net.leaves[i].size < net.leaves[*nb.begin()].size) nb = {i};
                }
        double best_s = 0, best_f = 0, best_w = 0;
        int best_over = 0;
        int32_t best = -1;
        for (int32_t x : nb) {
            auto out = sym_diff(T, net.leaves[x].labels);
            const double io = bt ? bt->count(merge_pos(tpos, lpos[x])) : 1.0;
            const double w = io * label_size(net, out, fixed);
            const int over = w > cap ? 1 : 0;
            double sc = w;
            const double f = io * 8.0 * label_size(net, set_union(T, net.leaves[x].labels), fixed);
            if (rng) {
                const double g = -std::log(-std::log(std::max(rng->uniform(), 1e-300)));
                sc = std::log2(1 + sc) - temperature * g;
            }
            if (best < 0 || over < best_over || (over == best_over && (sc < best_s || (sc == best_s && f < best_f)))) {
                best = x;
                best_s = sc;
                best_f = f;
                best_w = w;
                best_over = over;
            }
        }
        total += best_f;
        peak = std::max(peak, best_w);
        T = sym_diff(T, net.leaves[best].labels);
        tpos = merge_pos(tpos, lpos[best]);
        used[best] = 1;
        path.push_back({std::min(tid, best), std::max(tid, best)});
        tid = n + k;
    }
    if (flop_out) *flop_out = total;
    if (peak_out) *peak_out = peak;
    return path;
}

// Linear path in leaf order.  strict: absorb leaves 1, 2, ... in turn (for a
// circuit whose leaves are listed in time order with the initial states first,
// the state-vector order); else: absorb the lowest-index leaf x that shares a
// label with the growing tensor, each unused lower-index leaf that shares a
// label with x (and none with the tensor) joining just before x as an outer
// factor (initial states join when their qudit is first touched).
// Weighted FLOP and peak as in the greedy passes.
static std::vector<std::pair<int32_t, int32_t>> leaf_order_linear(const Network &net, bool strict, double *flop_out,
                                                                  BatchInstances *bt, double *peak_out)
{
    auto fixed = fixed_set(net, {});
    const int32_t n = (int32_t)net.leaves.size();
    auto pos_of = [&](int32_t i) {
        std::vector<int32_t> p;
        if (bt)
            for (int64_t l : net.leaves[i].labels) {
                auto it = bt->digit.find(l);
                if (it != bt->digit.end()) p.push_back(it->second);
            }
        std::sort(p.begin(), p.end());
        return p;
    };
    std::vector<char> used(n, 0);
    std::vector<int64_t> T = net.leaves[0].labels;
    std::vector<int32_t> tpos = pos_of(0);
    used[0] = 1;
    int32_t tid = 0;
    std::vector<std::pair<int32_t, int32_t>> path;
    double total = 0, peak = 0;
    auto shares = [&](const std::vector<int64_t> &L, int32_t i) {
        for (int64_t l : net.leaves[i].labels)
            if (std::find(L.begin(), L.end(), l) != L.end()) return true;
        return false;
    };
    std::vector<int32_t> pending;   // outer factors queued before the next connected leaf
    for (int32_t k = 0; k + 1 < n; ++k) {
        int32_t x = -1;
        if (!pending.empty()) {
            x = pending.front();
            pending.erase(pending.begin());
        } else if (!strict) {
            for (int32_t i = 1; i < n && x < 0; ++i)
                if (!used[i] && shares(T, i)) x = i;
            if (x >= 0) {
                for (int32_t y = 1; y < x; ++y)
                    if (!used[y] && !shares(T, y) && shares(net.leaves[x].labels, y)) pending.push_back(y);
                if (!pending.empty()) {
                    pending.push_back(x);
                    x = pending.front();
                    pending.erase(pending.begin());
                }
            }
        }
        if (x < 0)
            for (int32_t i = 1; i < n; ++i)
                if (!used[i]) {
                    x = i;
                    break;
                }
        tpos = merge_pos(tpos, pos_of(x));
        const double io = bt ? bt->count(tpos) : 1.0;
        total += io * 8.0 * label_size(net, set_union(T, net.leaves[x].labels), fixed);
        T = sym_diff(T, net.leaves[x].labels);
        peak = std::max(peak, io * label_size(net, T, fixed));
        used[x] = 1;
        path.push_back({std::min(tid, x), std::max(tid, x)});
        tid = n + k;
    }
    if (flop_out) *flop_out = total;
    if (peak_out) *peak_out = peak;
    return path;
}

// Subtree reconfiguration: for every internal node, take the sub-tree below it
// down to a frontier of at most k tensors (k = 10 below) (splitting the largest intermediate
// first), find the cheapest order of contracting that frontier exactly by
// dynamic programming over its subsets, and substitute it when it lowers the
// (instance-weighted) FLOP without creating an intermediate above max_size.
// Repeated for a few passes over the tree.  Returns the new path.
// sliced (optional): labels fixed per slice.  A node's cost is then counted
// once per distinct assignment of the sliced labels under it (Eq.
// task_based_amplitude_flops) and its size is that of one slice; max_size caps
// the size of one slice's intermediate (times its batch instances).
// time_model: a node costs max(FLOP / 100 TFLOP/s, bytes / 4 TB/s) per
// instance instead of its FLOP, bytes = 8 B x (|A| + |B| + |C|): a contraction
// that only streams operands through HBM weighs by its traffic.
static std::vector<std::pair<int32_t, int32_t>> reconfigure(const Network &net,
                                                            const std::vector<std::pair<int32_t, int32_t>> &path,
                                                            BatchInstances *bt, int passes, int k, double max_size,
                                                            const std::vector<int64_t> &sliced = {},
                                                            bool time_model = false)
{
    auto fixed = fixed_set(net, sliced);
    std::unordered_set<int64_t> slset(sliced.begin(), sliced.end());
    const int32_t n = (int32_t)net.leaves.size();
    if (path.size() < 2) return path;
    const int32_t n_nodes = n + (int32_t)path.size();
    std::vector<std::array<int32_t, 2>> ch(n_nodes, {-1, -1});
    std::vector<std::vector<int64_t>> lab(n_nodes);
    std::vector<std::vector<int32_t>> opos(n_nodes);
    std::vector<std::vector<int64_t>> slu(n_nodes);   // sliced labels under each node (sorted)
    for (int32_t i = 0; i < n; ++i) {
        lab[i] = net.leaves[i].labels;
        std::sort(lab[i].begin(), lab[i].end());
        for (int64_t l : lab[i])
            if (slset.count(l)) slu[i].push_back(l);
        if (bt)
            for (int64_t l : lab[i]) {
                auto it = bt->digit.find(l);
                if (it != bt->digit.end()) opos[i].push_back(it->second);
            }
        std::sort(opos[i].begin(), opos[i].end());
    }
    auto xor_sorted = [](const std::vector<int64_t> &a, const std::vector<int64_t> &b) {
        std::vector<int64_t> out;
        std::set_symmetric_difference(a.begin(), a.end(), b.begin(), b.end(), std::back_inserter(out));
        return out;
    };
    auto union_sorted = [](const std::vector<int64_t> &a, const std::vector<int64_t> &b) {
        std::vector<int64_t> out;
        std::set_union(a.begin(), a.end(), b.begin(), b.end(), std::back_inserter(out));
        return out;
    };
    auto set_node = [&](int32_t v, int32_t a, int32_t b) {
        ch[v] = {a, b};
        lab[v] = xor_sorted(lab[a], lab[b]);
        opos[v] = merge_pos(opos[a], opos[b]);
        slu[v] = union_sorted(slu[a], slu[b]);
    };
    for (size_t s = 0; s < path.size(); ++s) set_node(n + (int32_t)s, path[s].first, path[s].second);
    const int32_t root = n_nodes - 1;
    auto weight = [&](const std::vector<int32_t> &pos) { return bt ? bt->count(pos) : 1.0; };
    auto sl_inst = [&](const std::vector<int64_t> &ls) {
        double p = 1;
        for (int64_t l : ls) p *= net.labels.at(l).dim;
        return p;
    };
    // cost of one instance of a pairwise step with operand sizes sa, sb, result sc, index union su
    auto step_cost = [&](double sa, double sb, double sc, double su) {
        if (!time_model) return 8.0 * su;
        return std::max(8.0 * su / 100e12, 8.0 * (sa + sb + sc) / 4e12);
    };

    for (int pass = 0; pass < passes; ++pass) {
        // internal nodes, parents before children
        std::vector<int32_t> order, st{root};
        while (!st.empty()) {
            const int32_t v = st.back();
            st.pop_back();
            if (v < n) continue;
            order.push_back(v);
            st.push_back(ch[v][0]);
            st.push_back(ch[v][1]);
        }
        int changed = 0;
        for (int32_t v : order) {
            if (v < n || ch[v][0] < 0) continue;
            // frontier: split the largest internal frontier tensor until k tensors
            std::vector<int32_t> front{v}, internal;
            while ((int)front.size() < k) {
                int best_i = -1;
                double best_s = -1;
                for (int i = 0; i < (int)front.size(); ++i)
                    if (front[i] >= n) {
                        const double sz =
                            label_size(net, lab[front[i]], fixed) * weight(opos[front[i]]) * sl_inst(slu[front[i]]);
                        if (sz > best_s) {
                            best_s = sz;
                            best_i = i;
                        }
                    }
                if (best_i < 0) break;
                const int32_t x = front[best_i];
                front.erase(front.begin() + best_i);
                internal.push_back(x);
                front.push_back(ch[x][0]);
                front.push_back(ch[x][1]);
            }
            const int m = (int)front.size();
            if (m < 3) continue;
            double cur = 0;
            for (int32_t x : internal)
                cur += weight(opos[x]) * sl_inst(slu[x]) *
                       step_cost(label_size(net, lab[ch[x][0]], fixed), label_size(net, lab[ch[x][1]], fixed),
                                 label_size(net, lab[x], fixed),
                                 label_size(net, union_sorted(lab[ch[x][0]], lab[ch[x][1]]), fixed));
            // subset outputs and weights
            const int full = (1 << m) - 1;
            std::vector<std::vector<int64_t>> outs(full + 1);
            std::vector<double> wts(full + 1, 1.0), osz(full + 1, 1.0), swt(full + 1, 1.0);
            std::vector<std::vector<int64_t>> sls(full + 1);
            for (int S = 1; S <= full; ++S) {
                const int low = __builtin_ctz(S);
                const int rest = S & (S - 1);
                outs[S] = rest ? xor_sorted(outs[rest], lab[front[low]]) : lab[front[low]];
                sls[S] = rest ? union_sorted(sls[rest], slu[front[low]]) : slu[front[low]];
                swt[S] = sl_inst(sls[S]);
                if (bt) {
                    std::vector<int32_t> pos;
                    for (int i = 0; i < m; ++i)
                        if (S >> i & 1) pos = merge_pos(pos, opos[front[i]]);
                    wts[S] = bt->count(pos);
                }
                osz[S] = label_size(net, outs[S], fixed);
            }
            std::vector<double> best(full + 1, 0.0);
            std::vector<int> split(full + 1, 0);
            for (int S = 1; S <= full; ++S) {
                if ((S & (S - 1)) == 0) continue;
                double bc = -1;
                int bs = 0;
                for (int s1 = (S - 1) & S; s1; s1 = (s1 - 1) & S) {
                    const int s2 = S ^ s1;
                    if (s1 > s2) continue;
                    if (S != full && osz[S] * wts[S] > max_size) continue;   // intermediate above the cap
                    const double c = best[s1] + best[s2] +
                                     wts[S] * swt[S] *
                                         step_cost(osz[s1], osz[s2], osz[S],
                                                   label_size(net, union_sorted(outs[s1], outs[s2]), fixed));
                    if (bc < 0 || c < bc) {
                        bc = c;
                        bs = s1;
                    }
                }
                best[S] = bc < 0 ? INFINITY : bc;
                split[S] = bs;
            }
            if (!(best[full] < cur * (1.0 - 1e-12))) continue;
            // rebuild: the removed internal ids carry the new internal nodes (v stays the sub-root)
            std::vector<int32_t> ids(internal.begin(), internal.end());
            std::vector<int32_t> spare;
            for (int32_t x : ids)
                if (x != v) spare.push_back(x);
            std::function<int32_t(int)> build = [&](int S) -> int32_t {
                if ((S & (S - 1)) == 0) return front[__builtin_ctz(S)];
                const int s1 = split[S], s2 = S ^ s1;
                const int32_t a = build(s1), b = build(s2);
                int32_t node;
                if (S == full) {
                    node = v;
                } else {
                    node = spare.back();
                    spare.pop_back();
                }
                set_node(node, a, b);
                return node;
            };
            build(full);
            ++changed;
        }
        if (!changed) break;
    }
    // SSA path, children before parents
    std::vector<std::pair<int32_t, int32_t>> out;
    std::vector<int32_t> ssa(n_nodes, -1);
    for (int32_t i = 0; i < n; ++i) ssa[i] = i;
    int32_t next = n;
    std::vector<std::pair<int32_t, int>> st{{root, 0}};
    while (!st.empty()) {
        auto &top = st.back();
        const int32_t v = top.first;
        if (v < n) {
            st.pop_back();
            continue;
        }
        if (top.second == 0) {
            top.second = 1;
            st.push_back({ch[v][0], 0});
            st.push_back({ch[v][1], 0});
        } else {
            const int32_t a = ssa[ch[v][0]], b = ssa[ch[v][1]];
            out.push_back({std::min(a, b), std::max(a, b)});
            ssa[v] = next++;
            st.pop_back();
        }
    }
    return out;
}

// Weighted FLOP and largest weighted intermediate of a path (the greedy's model).
// FLOP of a path, every node counted once per batch instance (bt) and per
// distinct assignment of the sliced labels under it; peak_out: the largest
// intermediate of one slice times its batch instances.
static double weighted_flop(const Network &net, const std::vector<std::pair<int32_t, int32_t>> &path,
                            BatchInstances *bt, double *peak_out, const std::vector<int64_t> &sliced = {},
                            bool time_model = false)
{
    auto fixed = fixed_set(net, sliced);
    std::unordered_set<int64_t> slset(sliced.begin(), sliced.end());
    const int32_t n = (int32_t)net.leaves.size();
    std::vector<std::vector<int64_t>> lab(n + path.size()), slu(n + path.size());
    std::vector<std::vector<int32_t>> opos(n + path.size());
    for (int32_t i = 0; i < n; ++i) {
        lab[i] = net.leaves[i].labels;
        for (int64_t l : lab[i])
            if (slset.count(l)) slu[i].push_back(l);
        std::sort(slu[i].begin(), slu[i].end());
        if (bt)
            for (int64_t l : lab[i]) {
                auto it = bt->digit.find(l);
                if (it != bt->digit.end()) opos[i].push_back(it->second);
            }
        std::sort(opos[i].begin(), opos[i].end());
    }
    double total = 0, peak = 0;
    for (size_t s = 0; s < path.size(); ++s) {
        const int32_t a = path[s].first, b = path[s].second, c = n + (int32_t)s;
        lab[c] = sym_diff(lab[a], lab[b]);
        opos[c] = merge_pos(opos[a], opos[b]);
        std::set_union(slu[a].begin(), slu[a].end(), slu[b].begin(), slu[b].end(), std::back_inserter(slu[c]));
        double si = 1;
        for (int64_t l : slu[c]) si *= net.labels.at(l).dim;
        const double w = bt ? bt->count(opos[c]) : 1.0;
        const double su = label_size(net, set_union(lab[a], lab[b]), fixed);
        const double bytes = 8.0 * (label_size(net, lab[a], fixed) + label_size(net, lab[b], fixed) +
                                    label_size(net, lab[c], fixed));
        total += w * si * (time_model ? std::max(8.0 * su / 100e12, bytes / 4e12) : 8.0 * su);
        peak = std::max(peak, w * label_size(net, lab[c], fixed));
    }
    if (peak_out) *peak_out = peak;
    return total;
}

std::vector<std::pair<int32_t, int32_t>> greedy_path(const Network &net, uint64_t seed, int32_t n_trials,
                                                     double *flop_out, int32_t n_amps, const int32_t *outputs,
                                                     double max_elems)
{
    if (net.leaves.size() == 1) {
        if (flop_out) *flop_out = 0;
        return {};
    }
    const bool batch_mode = outputs != nullptr;
    BatchInstances batch, *bt = nullptr;
    if (batch_mode && n_amps > 1) {
        batch.n_amps = n_amps;
        batch.n_out = (int32_t)net.open.size();
        batch.outputs = outputs;
        for (int32_t j = 0; j < batch.n_out; ++j)   // free open legs are not restricted by the rows
            if (std::find(net.free_open.begin(), net.free_open.end(), net.open[j]) == net.free_open.end())
                batch.digit[net.open[j]] = j;
        bt = &batch;
    }
    const double cap = max_elems > 0 ? max_elems : INFINITY;
    // keep the path of lowest FLOP among those whose largest (instance-weighted)
    // intermediate fits the cap; above the cap, the smaller peak wins
    double best_flop = 0, best_peak = 0;
    auto better = [&](double f, double pk) {
        const bool in = pk <= cap, best_in = best_peak <= cap;
        if (in != best_in) return in;
        return in ? f < best_flop : (pk < best_peak || (pk == best_peak && f < best_flop));
    };
    auto best = greedy_once(net, nullptr, 0, &best_flop, bt, cap, &best_peak);
    if (batch_mode) {   // the batch planner adds linear passes: leaf order, then greedy ones
        for (int v = 0; v < 3; ++v) {
            double f, pk;
            auto p = v < 2 ? leaf_order_linear(net, v == 0, &f, bt, &pk)
                           : greedy_linear(net, 0, nullptr, 0, &f, bt, cap, &pk);
            if (better(f, pk)) {
                best_flop = f;
                best_peak = pk;
                best = p;
            }
        }
    }
    SplitMix rng{seed};
    for (int32_t t = 1; t < n_trials; ++t) {
        double f, pk;
        double temp = 0.25 + 1.75 * rng.uniform();
        std::vector<std::pair<int32_t, int32_t>> p;
        if (batch_mode && (t & 1)) {
            const int32_t start = (int32_t)(rng.next() % net.leaves.size());
            p = greedy_linear(net, start, &rng, temp, &f, bt, cap, &pk);
        } else {
            p = greedy_once(net, &rng, temp, &f, bt, cap, &pk);
        }
        if (better(f, pk)) {
            best_flop = f;
            best_peak = pk;
            best = p;
        }
    }
    // local improvement of the kept path; intermediates stay within the larger of
    // the cap and the path's own largest one
    {
        double pk = 0;
        weighted_flop(net, best, bt, &pk);
        const double limit = std::isfinite(cap) ? std::max(cap, pk) : pk;
        auto better_path = reconfigure(net, best, bt, 8, 10, limit);
        double pk2 = 0;
        const double f2 = weighted_flop(net, better_path, bt, &pk2);
        if (f2 < best_flop && pk2 <= limit) {
            best = better_path;
            best_flop = f2;
        }
    }
    if (flop_out) *flop_out = best_flop;
    return best;
}

// ------------------------------------------------------------ slice finder
std::vector<int64_t> slice_auto(const Network &net, int64_t max_elems, int32_t min_n, int32_t max_n)
{
    std::vector<int64_t> sliced;
    while (true) {
        PathCost c = path_cost(net, net.path, sliced);
        if (c.max_size <= (double)max_elems && (int32_t)sliced.size() >= min_n) return sliced;
        if ((int32_t)sliced.size() >= max_n)
            fail(JET_EINVAL, "slice_auto: cap " + std::to_string(max_elems) + " not reachable with " +
                                 std::to_string(max_n) + " sliced labels");
        // candidates: closed, unsliced labels of the largest intermediates
        Tree t = build_tree(net, net.path);
        std::set<int64_t> cand;
        for (size_t i = t.n_leaves; i < t.labels.size(); ++i)
            if (c.node_size[i] >= c.max_size)
                for (int64_t l : t.labels[i]) {
                    const LabelInfo &li = net.labels.at(l);
                    if (li.n_owner == 2 && li.dim > 1 && c.node_size[i] > 1 &&
                        std::find(sliced.begin(), sliced.end(), l) == sliced.end())
                        cand.insert(l);
                }
        if (cand.empty()) fail(JET_EINVAL, "slice_auto: no sliceable label in the largest intermediate");
        int64_t best = -1;
        double best_cost = 0, best_total = 0;
        for (int64_t l : cand) {
            auto s2 = sliced;
            s2.push_back(l);
            double cost = reuse_aware_flop(net, net.path, s2);
            PathCost c2 = path_cost(net, net.path, s2);
            double nsl = 1;
            for (int64_t x : s2) nsl *= net.labels.at(x).dim;
            double total = nsl * c2.flop;
            if (best < 0 || cost < best_cost || (cost == best_cost && total < best_total)) {
                best = l;
                best_cost = cost;
                best_total = total;
            }
        }
        sliced.push_back(best);
    }
}

// Sub-tree reconfiguration of the current path under its slicing (Section 3.2:
// minimise Eq. task_based_amplitude_flops itself): every node's FLOP counts
// once per distinct assignment of the sliced labels under it (and per batch
// instance when outputs lists a batch), every sub-tree of up to 10 tensors is
// re-ordered optimally, and no intermediate of one slice grows above the
// current path's largest.  Returns the current path when nothing improves.
std::vector<std::pair<int32_t, int32_t>> reconfigure_sliced(const Network &net, int32_t passes, int32_t n_amps,
                                                            const int32_t *outputs, double *before, double *after,
                                                            bool time_model)
{
    BatchInstances batch, *bt = nullptr;
    if (outputs && n_amps > 1) {
        batch.n_amps = n_amps;
        batch.n_out = (int32_t)net.open.size();
        batch.outputs = outputs;
        for (int32_t j = 0; j < batch.n_out; ++j)
            if (std::find(net.free_open.begin(), net.free_open.end(), net.open[j]) == net.free_open.end())
                batch.digit[net.open[j]] = j;
        bt = &batch;
    }
    double pk = 0, pk2 = 0;
    const double f0 = weighted_flop(net, net.path, bt, &pk, net.sliced, time_model);
    auto p = reconfigure(net, net.path, bt, passes, 10, pk, net.sliced, time_model);
    double f1 = weighted_flop(net, p, bt, &pk2, net.sliced, time_model);
    if (!(f1 < f0 && pk2 <= pk)) {
        p = net.path;
        f1 = f0;
    }
    if (before) *before = f0;
    if (after) *after = f1;
    return p;
}

}  // namespace jet

