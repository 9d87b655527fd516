"""Host-side tests of the C ABI: the library loads and exports every declared
symbol, and the planner's path/slice/reuse bookkeeping matches brute-force
counts.  No call here touches a GPU (device work is lazy until a contraction)."""
import os
import re
from itertools import product

import numpy as np
import pytest

from paper_2107_09793_b300 import jet
from circuits import configs, random_grid_circuit, circuit_to_network
import oracle
from oracle.einsum import network_flops

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "jet.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(jet_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    L = jet.lib()
    names = _declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(L, n), n


def _net(name="grid12", **kw):
    w = configs.build(name)
    return w, jet.from_network(w.network, **kw)


def test_greedy_path_is_valid_and_flop_model_matches():
    w, net = _net()
    f = net.path_greedy(seed=3, n_trials=8)
    path = net.path_get()
    tn = w.network
    n = len(tn.labels)
    assert len(path) == n - 1
    seen = set()
    for k, (a, b) in enumerate(path):
        assert a < n + k and b < n + k and a != b and a not in seen and b not in seen
        seen |= {a, b}
    # the library's FLOP model equals the oracle's independent count with open legs at dim 1
    dims = {}
    for l, t in zip(tn.labels, tn.data):
        for x, s in zip(l, t.shape):
            dims[x] = 1 if x in tn.open_labels else s
    assert f == network_flops(tn.labels, dims, path)
    assert net.stats()["flop_planned"] == f


def test_path_set_validation_errors():
    w, net = _net()
    n = len(w.network.labels)
    with pytest.raises(jet.JetError) as e:
        net.path_set([(0, 1)])
    assert e.value.code == jet.JET_EINVAL
    bad = [(0, 1)] + [(0, k) for k in range(2, n)]
    with pytest.raises(jet.JetError) as e:
        net.path_set(bad)
    assert e.value.code == jet.JET_EINVAL


def test_contract_before_path_is_state_error():
    w, net = _net()
    with pytest.raises(jet.JetError) as e:
        net.plan(w.outputs)
    assert e.value.code == jet.JET_ESTATE


def test_create_rejects_bad_networks():
    a = np.ones((2, 2), np.complex64)
    with pytest.raises(jet.JetError) as e:
        jet.Network([[0, 0]], [a])             # label repeated in a tensor
    assert e.value.code == jet.JET_EINVAL
    with pytest.raises(jet.JetError):
        jet.Network([[0, 1], [1, 2], [1, 3]], [a, a, a])   # label on three tensors
    with pytest.raises(jet.JetError):
        jet.Network([[0, 1], [1, 2]], [a, np.ones((3, 2), np.complex64)])  # dims differ
    net = jet.Network([[0, 1], [1, 2]], [a, a])
    with pytest.raises(jet.JetError):
        net.set_open([0])                      # must list every open leg
    with pytest.raises(jet.JetError):
        net.set_open([0, 1])                   # 1 is closed
    net.set_open([2, 0])
    net.path_set([(0, 1)])
    with pytest.raises(jet.JetError) as e:
        net.plan([[2, 0]])                     # digit out of range
    assert e.value.code == jet.JET_EINVAL
    with pytest.raises(jet.JetError):
        net.slice([0])                         # open legs cannot be sliced


def _instances_brute(tn, path, sliced, outputs):
    """Distinct (node, values of the fixed labels under it) pairs, by enumeration."""
    fixed = set(sliced) | set(tn.open_labels)
    dims = {}
    for l, t in zip(tn.labels, tn.data):
        for x, s in zip(l, t.shape):
            dims[x] = s
    n = len(tn.labels)
    under = [sorted(set(l) & fixed) for l in tn.labels]
    labels = [list(l) for l in tn.labels]
    total_inst, total_flop = 0, 0
    for k, (a, b) in enumerate(path):
        u = sorted(set(under[a]) | set(under[b]))
        under.append(u)
        keys = set()
        for o in outputs:
            for sv in product(*[range(dims[x]) for x in sliced]):
                val = dict(zip(sliced, sv))
                val.update(zip(tn.open_labels, o))
                keys.add(tuple(val[x] for x in u))
        un = list(dict.fromkeys(labels[a] + labels[b]))
        labels.append([x for x in labels[a] if x not in labels[b]] + [x for x in labels[b] if x not in labels[a]])
        f = 8 * int(np.prod([dims[x] for x in un if x not in fixed]))
        total_inst += len(keys)
        total_flop += len(keys) * f
    return total_inst, total_flop


def test_reuse_dag_counts_match_brute_force():
    """Section 3.2: each (node, fixed-label values) instance is computed once."""
    circ = random_grid_circuit(2, 3, 5, seed=12)
    tn = circuit_to_network(circ)
    net = jet.from_network(tn)
    net.path_greedy(seed=1, n_trials=4)
    sliced = net.slice_auto(1 << 4, min_n=3, max_n=10)
    assert len(sliced) >= 3
    outputs = np.array([[0, 1, 0, 1, 1, 0], [0, 1, 0, 0, 0, 1], [1, 1, 1, 1, 1, 1]], np.int32)
    net.plan(outputs)
    st = net.stats()
    inst, flop = _instances_brute(tn, net.path_get(), sliced, outputs)
    assert st["n_instances"] == inst
    assert st["flop_executed"] == flop
    # no reuse: every (amplitude, slice) recomputes every node
    net2 = jet.from_network(tn, reuse=False)
    net2.path_set(net.path_get())
    net2.slice(sliced)
    net2.plan(outputs)
    nsl = 2 ** len(sliced)
    assert net2.stats()["n_instances"] == (len(tn.labels) - 1) * nsl * len(outputs)
    assert net2.stats()["flop_executed"] > st["flop_executed"]


def test_slice_auto_reaches_cap_and_min_count():
    w, net = _net("grid30")
    net.path_greedy(seed=1, n_trials=16)
    sl = net.slice_auto(1 << 24, min_n=6, max_n=30)
    st = net.stats()
    assert st["max_intermediate"] <= 1 << 24
    assert len(sl) >= 6 and st["n_slices"] == 2 ** len(sl)
    assert len(set(sl)) == len(sl) and not set(sl) & set(w.network.open_labels)


def test_workspace_plan_is_host_only():
    w, net = _net()
    net.path_greedy(seed=1, n_trials=2)
    nbytes = net.plan(w.outputs)
    assert nbytes >= 256 and nbytes % 256 == 0


def test_contract_slices_rejects_bad_ids_before_any_device_work():
    w, net = _net()
    net.path_greedy(seed=1, n_trials=2)
    net.slice_auto(1 << 8, min_n=2, max_n=12)
    nsl = net.stats()["n_slices"]
    for bad in ([nsl], [-1], []):
        with pytest.raises(jet.JetError) as e:
            net.contract_slices(w.outputs, bad)
        assert e.value.code == jet.JET_EINVAL


def test_contract_grad_argument_errors_before_device_work():
    w, net = _net()
    net.path_greedy(seed=1, n_trials=2)
    cot = np.ones(1, np.complex128)
    for ids in ([-1], [len(w.network.data)], [3, 3]):
        with pytest.raises(jet.JetError) as e:
            net.contract_grad(w.outputs, cot, ids)
        assert e.value.code == jet.JET_EINVAL
    one = jet.Network([[7]], [np.array([1, 2], np.complex64)])
    one.set_open([7])
    one.path_set([])
    with pytest.raises(jet.JetError) as e:
        one.contract_grad([[0]], cot, [0])
    assert e.value.code == jet.JET_EINVAL


def test_batch_greedy_flop_matches_reuse_dag_brute_force():
    """The batch planner's FLOP = sum over nodes of (distinct bra restrictions
    under the node) x (node FLOP), the same count the reuse DAG executes."""
    from circuits import gbs_lattice_circuit, random_patterns
    for circ, outs in [(gbs_lattice_circuit(2, 3, 4, 2, seed=17), random_patterns(6, 24, 5, 4)),
                       (random_grid_circuit(2, 3, 5, seed=12), np.array(list(product([0, 1], repeat=6))[::5], np.int32))]:
        tn = circuit_to_network(circ)
        net = jet.from_network(tn)
        f = net.path_greedy_batch(outs, seed=2, n_trials=8)
        net.plan(outs)
        inst, flop = _instances_brute(tn, net.path_get(), [], outs)
        assert net.stats()["flop_executed"] == flop == f
        assert net.stats()["n_instances"] == inst
        # a single-amplitude batch is costed like the plain greedy's open-legs-fixed model
        net1 = jet.from_network(tn)
        f1 = net1.path_greedy_batch(outs[:1], seed=2, n_trials=1)
        net1.plan(outs[:1])
        assert net1.stats()["flop_executed"] == f1


def test_batch_greedy_keeps_bras_late_on_the_bosonic_lattice():
    """16 modes, d = 4, 256 patterns: with the weighted cap at 2^32 the planner
    keeps a state-vector-like order (every tensor shared by the batch until the
    last layer), at or below the strict state-vector order and far below the
    per-amplitude greedy path run for the batch."""
    w = configs.build("gbs16")
    tn = w.network
    n = len(tn.labels)
    net = jet.from_network(tn)
    f = net.path_greedy_batch(w.outputs, seed=1, n_trials=8, max_elems=1 << 32)
    net.plan(w.outputs)
    st = net.stats()
    assert st["flop_executed"] == f and st["max_intermediate"] == 1 << 32
    sv = jet.from_network(tn)
    sv.path_set([(0, 1)] + [(k + 2, n + k) for k in range(n - 2)])
    sv.plan(w.outputs)
    assert f <= sv.stats()["flop_executed"]
    per_amp = jet.from_network(tn)
    per_amp.path_greedy(seed=1, n_trials=8)
    per_amp.plan(w.outputs)
    assert per_amp.stats()["flop_executed"] > 100 * f


def test_batch_greedy_argument_errors():
    w, net = _net("param20")
    with pytest.raises(jet.JetError) as e:
        net.path_greedy_batch(np.full((2, 20), 2, np.int32))
    assert e.value.code == jet.JET_EINVAL
    with pytest.raises(jet.JetError) as e:
        net.path_greedy_batch(np.zeros((0, 20), np.int32))
    assert e.value.code == jet.JET_EINVAL


def _optimal_flop_brute(labels, dims, cap):
    """Cheapest pairwise order of a few tensors, exhaustively (every binary tree), in the
    library's model: a step costs 8 * prod(dims of the union of its operands' labels);
    intermediates (not the final result) hold at most `cap` elements."""
    from functools import lru_cache
    sets = [frozenset(l) for l in labels]
    n = len(sets)

    def out(S):
        o = frozenset()
        for i in range(n):
            if S >> i & 1:
                o = o ^ sets[i]
        return o

    def size(S):
        return int(np.prod([dims[x] for x in out(S)] or [1]))

    @lru_cache(maxsize=None)
    def best(S):
        if S & (S - 1) == 0:
            return 0
        if S != (1 << n) - 1 and size(S) > cap:
            return float("inf")
        b = None
        s1 = (S - 1) & S
        while s1:
            s2 = S ^ s1
            if s1 < s2:
                c = best(s1) + best(s2) + 8 * int(np.prod([dims[x] for x in (out(s1) | out(s2))] or [1]))
                b = c if b is None or c < b else b
            s1 = (s1 - 1) & S
        return b
    return best((1 << n) - 1)


def test_planner_is_flop_optimal_on_networks_of_ten_tensors():
    """Up to ten tensors the subtree reconfiguration covers the whole tree, so the
    kept path must cost exactly the exhaustive optimum among the paths whose
    intermediates stay within the kept path's largest one."""
    rng = np.random.default_rng(5)
    for trial in range(12):
        n = int(rng.integers(4, 11))
        labels = [[] for _ in range(n)]
        nxt = 0
        for i in range(1, n):                      # a random spanning tree keeps it connected
            j = int(rng.integers(0, i))
            labels[i].append(nxt); labels[j].append(nxt); nxt += 1
        for _ in range(int(rng.integers(1, n + 2))):  # extra bonds
            i, j = rng.choice(n, 2, replace=False)
            labels[int(i)].append(nxt); labels[int(j)].append(nxt); nxt += 1
        dims = {l: int(rng.choice([2, 3, 4])) for l in range(nxt)}
        data = [np.ones([dims[l] for l in ls], np.complex64) for ls in labels]
        net = jet.Network(labels, data)
        net.set_open([])
        f = net.path_greedy(seed=trial, n_trials=2)
        cap = net.stats()["max_intermediate"]
        assert f == _optimal_flop_brute(labels, dims, cap), trial


def test_free_open_legs_arguments_and_planning():
    """jet_network_set_free: argument errors, and the planners count a free leg
    with its dim (a fixed open leg counts as 1), so freeing legs raises the
    planned FLOP; the plan of a free-leg network builds without a GPU."""
    from circuits import configs
    w = configs.build("grid12")
    net = jet.from_network(w.network)
    opens = w.network.open_labels
    with pytest.raises(jet.JetError):
        net.set_free([12345])                      # not an open leg
    with pytest.raises(jet.JetError):
        net.set_free([opens[0], opens[0]])         # listed twice
    f_fixed = net.path_greedy(seed=1, n_trials=4)
    net.set_free(opens[:6])
    assert net.n_elem == 64
    f_free = net.path_greedy(seed=1, n_trials=4)
    assert f_free > f_fixed
    net.plan(np.zeros((2, 12), np.int32))
    net.set_free([])
    assert net.n_elem == 1
    closed = jet.Network([[0, 1], [1, 0]], [np.eye(2, dtype=np.complex64)] * 2)
    with pytest.raises(jet.JetError):
        closed.set_free([0])                       # open legs not declared (none exist)
    net.close()
    closed.close()


def test_path_reconfigure_for_slicing():
    """jet_path_reconfigure: the cost it reports is Eq. task_based_amplitude_flops
    of the path under its slicing (equal to the FLOP the plan executes, reuse
    on), it never increases, the largest intermediate of one slice does not
    grow, and a batch-weighted call and argument errors behave."""
    w = configs.build("grid30")
    net = jet.from_network(w.network)
    net.path_greedy(seed=1, n_trials=16)
    net.slice_auto(1 << 24, min_n=6, max_n=24)
    net.plan(w.outputs)
    st0 = net.stats()
    before, after = net.path_reconfigure(4)
    assert before == pytest.approx(st0["flop_executed"], rel=1e-12)
    assert after <= before
    net.plan(w.outputs)
    st1 = net.stats()
    assert st1["flop_executed"] == pytest.approx(after, rel=1e-12)
    assert st1["max_intermediate"] <= st0["max_intermediate"]
    b2, a2 = net.path_reconfigure(2)          # a second call starts from the improved path
    assert b2 == pytest.approx(after, rel=1e-12) and a2 <= b2
    with pytest.raises(jet.JetError):
        net.path_reconfigure(0)
    rows = np.array([[0] * 30, [1] * 30], np.int32)
    bb, ab = net.path_reconfigure(2, outputs=rows)
    assert ab <= bb
    tb, ta = net.path_reconfigure(2, objective="time")   # estimated seconds
    assert 0 < ta <= tb < 1
    fresh = jet.from_network(w.network)
    with pytest.raises(jet.JetError):
        fresh.path_reconfigure(2)             # no path yet
    net.close()
    fresh.close()


def _check_liveness(net):
    """Intermediate deletion (Section 4): a node's buffer is released only after
    every launch that reads it was issued, and no two allocations whose launch
    windows meet share a byte of the workspace."""
    bufs = net.plan_buffers()
    ws = net.stats()["workspace_bytes"]
    assert bufs
    for b in bufs:
        assert 0 <= b["offset"] and b["offset"] + b["bytes"] <= ws, b
        assert b["t_release"] < 0 or b["t_alloc"] <= b["t_release"], b
        if b["node"] >= 0:
            assert b["first_use"] >= b["t_alloc"], b           # allocated before its node writes it
            assert b["t_release"] < 0 or b["last_use"] < b["t_release"], b   # released after its last reader
    INF = 1 << 40
    ev = sorted(bufs, key=lambda b: b["t_alloc"])
    live = []   # sweep over launch time: windows [t_alloc, t_release)
    n_pairs = 0
    for b in ev:
        live = [x for x in live if (x["t_release"] if x["t_release"] >= 0 else INF) > b["t_alloc"]]
        for x in live:
            n_pairs += 1
            assert x["offset"] + x["bytes"] <= b["offset"] or b["offset"] + b["bytes"] <= x["offset"], (x, b)
        live.append(b)
    return len(bufs), n_pairs


@pytest.mark.parametrize("name,prec", [("grid12", "fp32"), ("grid30", "fp32"), ("grid30", "tf32x3"),
                                       ("param20", "fp32"), ("gbs16", "fp32")])
def test_arena_liveness_no_overlap_among_live_buffers(name, prec):
    w = configs.build(name)
    net = jet.from_network(w.network, precision=prec)
    if len(w.outputs) > 1:
        net.path_greedy_batch(w.outputs, seed=1, n_trials=2, max_elems=1 << 32)
    else:
        net.path_greedy(seed=1, n_trials=4)
        net.slice_auto(1 << (8 if name == "grid12" else 24), min_n=2, max_n=24)
    net.plan(w.outputs)
    n, pairs = _check_liveness(net)
    assert n >= 3 and pairs >= 1
    net.close()


def test_small_levels_run_as_chained_launches():
    """Consecutive small tree levels (Section 3.1: the many tiny contractions of
    the first levels) are issued as one cooperative launch each run of them,
    at most one block per SM; grid30's first launch is such a chain."""
    w = configs.build("grid30")
    net = jet.from_network(w.network, precision="fp16x3")
    try:
        net.path_greedy(seed=1, n_trials=4)
        net.slice_auto(1 << 24, min_n=2, max_n=24)
        net.plan(w.outputs)
        recs = net.profile()
        chains = [r for r in recs if r["kind"] == "small_batch" and r["variant"] & 2]
        assert chains and recs[0] in chains
        assert all(1 <= r["grid"][0] <= 148 and r["block"] == 256 for r in chains)
        plain = [r for r in recs if r["kind"] in ("small_batch", "direct") and not r["variant"] & 2]
        assert len(chains) + len(plain) < 12, [(r["kind"], r["node"]) for r in chains + plain]
    finally:
        net.close()


@pytest.mark.parametrize("prec,fuse,form,dot", [("fp16x3", True, "pairs", True), ("tf32x3", True, "pairs", True),
                                                 ("bf16x6", True, "pairs", False), ("fp16x3", False, "pairs", False),
                                                 ("fp16x3", True, "single", True), ("fp16x3", True, "unpaired", True),
                                                 ("fp16x3", True, "four", False)])
def test_dot_epilogue_plan_and_arena_liveness(prec, fuse, form, dot):
    """A GEMM whose parent is a full dot product with its sibling: the plan takes
    the dot-epilogue form (the GEMM marked, the parent only a reduce of the tile
    parts) in the modes that have room for its staging, with the epilogue
    fusions on and at most two sibling instances per instance; the plain output
    and the parent's dot-product kernel otherwise; the tile parts' buffer obeys
    the liveness rule."""
    from test_gpu_dot_epilogue import network
    labels, data, path, sl = network("cols", form)
    net = jet.Network(labels, data, precision=prec, fuse_split=fuse)
    try:
        net.set_open([])
        net.path_set(path)
        net.slice(sl)
        net.plan_slices(np.zeros((1, 0), np.int32), list(range(2 ** len(sl))))
        recs = net.profile()
        gemm = [r for r in recs if r["kind"] == "gemm_tc" and r["node"] == 4]
        parent = {r["kind"] for r in recs if r["node"] == 5}
        assert gemm and bool(gemm[0]["variant"] & 8) == dot, recs
        assert (parent == {"splitk_reduce"}) if dot else ("direct" in parent), recs
        _check_liveness(net)
    finally:
        net.close()


def test_arena_liveness_with_fused_splits_on_the_53_qubit_range_plan():
    """The benchmark's FP16x3 range plan (GEMMs that write their parent's planes
    in place of their complex64 output): no two live buffers overlap, and the
    fused GEMMs' parents split only their other operand."""
    import json
    w = configs.build("grid53")
    plan = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "grid53_plan.json")))
    net = jet.from_network(w.network, precision="fp16x3")
    try:
        net.path_set([tuple(p) for p in plan["path"]])
        net.slice(plan["sliced_labels"])
        r = net.plan_ranges(w.outputs, int(216e9))
        sl = plan["sliced_labels"]
        T = [sl.index(x) for x in r["fixed_labels"]]
        n = len(sl)
        ids = [s_ for s_ in range(2 ** n) if all(((s_ >> (n - 1 - j)) & 1) == 0 for j in T)]
        net.plan_slices(w.outputs, ids)
        recs = net.profile()
        fused = {x["node"] for x in recs if x["kind"] == "gemm_tc" and x["variant"] & 4}
        assert len(fused) >= 3, recs
        _check_liveness(net)
    finally:
        net.close()


def test_arena_liveness_catches_a_planted_overlap():
    """The check itself: moving one live buffer onto another is caught."""
    w = configs.build("grid12")
    net = jet.from_network(w.network)
    net.path_greedy(seed=1, n_trials=4)
    net.plan(w.outputs)
    bufs = net.plan_buffers()
    orig = jet.Network.plan_buffers
    # find two buffers with meeting windows and put the second on the first
    for i, a in enumerate(bufs):
        for b in bufs[i + 1:]:
            ra = a["t_release"] if a["t_release"] >= 0 else 1 << 40
            if b["t_alloc"] < ra:
                bad = [dict(x) for x in bufs]
                bad[bufs.index(b)]["offset"] = a["offset"]
                try:
                    jet.Network.plan_buffers = lambda self: bad
                    with pytest.raises(AssertionError):
                        _check_liveness(net)
                finally:
                    jet.Network.plan_buffers = orig
                net.close()
                return
    pytest.fail("no two buffers live at once")


def test_selftest_wait_rejects_bad_limits_before_any_device_work():
    w, net = _net()
    for bad in (0, -5, 10 ** 8):
        with pytest.raises(jet.JetError) as e:
            net.selftest_wait(bad)
        assert e.value.code == jet.JET_EINVAL


def test_sum_partials_adds_in_increasing_slice_order():
    rng = np.random.default_rng(3)
    p = rng.standard_normal((3, 7, 2)) + 1j * rng.standard_normal((3, 7, 2))
    got = jet.sum_partials(p)
    ref = np.zeros((3, 2), np.complex128)
    for j in range(7):
        ref += p[:, j, :]
    assert got.tobytes() == ref.tobytes()   # the same FP64 order, bit for bit
    assert np.array_equal(jet.sum_partials(p[:, :0, :]), np.zeros((3, 2)))
