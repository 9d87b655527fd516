"""ctypes binding of libjet.so (the C ABI in include/jet.h).

Argument marshalling only: every step of the contraction runs in the library's
CUDA kernels.  There is no fallback: if the shared library is missing or a call
fails, a JetError is raised.
"""
import ctypes
import os
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libjet.so")

JET_OK, JET_EINVAL, JET_ENOMEM, JET_ECUDA, JET_ETIMEOUT, JET_ESTATE = 0, -1, -2, -3, -4, -5
PREC = {"fp32": 0, "tf32": 1, "tf32x3": 2, "bf16x3": 3, "bf16x6": 4, "fp64": 5, "fp16x3": 6}

EXPORTS = ["jet_options_default", "jet_network_create", "jet_network_set_open", "jet_tensor_update",
           "jet_tensors_upload", "jet_network_n_values", "jet_path_set", "jet_path_get",
           "jet_path_greedy", "jet_path_greedy_batch", "jet_slice", "jet_slice_auto", "jet_contract", "jet_contract_async",
           "jet_plan", "jet_set_workspace", "jet_contract_grad", "jet_stats",
           "jet_network_destroy", "jet_last_error", "jet_profile", "jet_pair_contract_noalloc",
           "jet_contract_slices", "jet_network_set_free", "jet_path_reconfigure", "jet_plan_slices",
           "jet_network_keep_shared", "jet_network_save_shared", "jet_network_load_shared", "jet_plan_buffers",
           "jet_plan_ranges", "jet_sum_partials", "jet_selftest_wait", "jet_autotune"]


class JetError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"jet error {code}: {msg}")
        self.code = code


class Options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("reuse", ctypes.c_int32), ("use_graph", ctypes.c_int32),
                ("device", ctypes.c_int32), ("gemm_min_k", ctypes.c_int64), ("workspace_limit", ctypes.c_int64),
                ("profile", ctypes.c_int32), ("apply_tc_min_kf", ctypes.c_int32), ("gemm_group", ctypes.c_int32),
                ("fuse_split", ctypes.c_int32)]


class OpRecord(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("node", ctypes.c_int32), ("n_inst", ctypes.c_int64),
                ("flop", ctypes.c_double), ("bytes", ctypes.c_double), ("ms", ctypes.c_float),
                ("block", ctypes.c_int32), ("grid", ctypes.c_int32 * 3), ("smem", ctypes.c_int32),
                ("variant", ctypes.c_int32), ("pad_", ctypes.c_int32)]


OP_KINDS = {0: "direct", 1: "permute", 2: "gemm_simt", 3: "gemm_tc", 4: "slice_reduce", 5: "splitk_reduce",
            6: "tc_split", 7: "small_batch", 8: "accum", 9: "memset", 10: "apply", 11: "accum_batch"}


class BufferRecord(ctypes.Structure):
    _fields_ = [("node", ctypes.c_int32), ("t_alloc", ctypes.c_int32), ("t_release", ctypes.c_int32),
                ("first_use", ctypes.c_int32), ("last_use", ctypes.c_int32), ("pad_", ctypes.c_int32),
                ("offset", ctypes.c_int64), ("bytes", ctypes.c_int64)]


class TensorDesc(ctypes.Structure):
    _fields_ = [("rank", ctypes.c_int32), ("labels", ctypes.POINTER(ctypes.c_int64)),
                ("dims", ctypes.POINTER(ctypes.c_int32)), ("data", ctypes.c_void_p)]


class Stats(ctypes.Structure):
    _fields_ = [("flop_planned", ctypes.c_double), ("flop_sliced", ctypes.c_double),
                ("flop_executed", ctypes.c_double), ("reuse_fraction", ctypes.c_double),
                ("bytes_executed", ctypes.c_double), ("max_intermediate", ctypes.c_int64),
                ("workspace_bytes", ctypes.c_int64), ("n_instances", ctypes.c_int64),
                ("n_launches", ctypes.c_int64), ("n_slices", ctypes.c_int32),
                ("n_sliced_labels", ctypes.c_int32), ("n_gemm_nodes", ctypes.c_int32),
                ("n_direct_nodes", ctypes.c_int32)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise JetError(JET_ESTATE, f"{LIB_PATH} not built (run __graft_entry__.build())")
        L = ctypes.CDLL(LIB_PATH)
        P, I32, I64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
        sig = {
            "jet_options_default": (None, [P]),
            "jet_network_create": (I32, [P, I32, P, P]),
            "jet_network_set_open": (I32, [P, I32, P]),
            "jet_network_set_free": (I32, [P, I32, P]),
            "jet_path_reconfigure": (I32, [P, I32, I32, I32, P, P, P]),
            "jet_plan_slices": (I32, [P, I32, P, I32, P, P]),
            "jet_network_keep_shared": (I32, [P, I64]),
            "jet_network_save_shared": (I32, [P, ctypes.c_char_p]),
            "jet_network_load_shared": (I32, [P, ctypes.c_char_p]),
            "jet_tensor_update": (I32, [P, I32, P]),
            "jet_tensors_upload": (I32, [P, P, P]),
            "jet_network_n_values": (I64, [P]),
            "jet_path_set": (I32, [P, I32, P]),
            "jet_path_get": (I32, [P, P]),
            "jet_path_greedy": (I32, [P, ctypes.c_uint64, I32, P]),
            "jet_path_greedy_batch": (I32, [P, I32, P, ctypes.c_int64, ctypes.c_uint64, I32, P]),
            "jet_slice": (I32, [P, I32, P]),
            "jet_slice_auto": (I32, [P, I64, I32, I32, P, P]),
            "jet_contract": (I32, [P, I32, P, P, P]),
            "jet_contract_async": (I32, [P, I32, P, P, P]),
            "jet_contract_slices": (I32, [P, I32, P, I32, P, P, P]),
            "jet_plan": (I32, [P, I32, P, P]),
            "jet_set_workspace": (I32, [P, P, ctypes.c_size_t]),
            "jet_contract_grad": (I32, [P, I32, P, P, I32, P, P, P, P]),
            "jet_stats": (I32, [P, P]),
            "jet_profile": (I32, [P, P, I32, P]),
            "jet_plan_buffers": (I32, [P, P, I32, P]),
            "jet_plan_ranges": (I32, [P, I32, P, ctypes.c_size_t, P, P, P, P, P]),
            "jet_sum_partials": (I32, [I32, I64, I64, P, P]),
            "jet_selftest_wait": (I32, [P, I64, P]),
            "jet_autotune": (I32, [P, I32, P, ctypes.c_char_p, P, P, P, P]),
            "jet_pair_contract_noalloc": (I32, [I32, P, P, P, I32, P, P, P, P, I32, P]),
            "jet_network_destroy": (None, [P]),
            "jet_last_error": (ctypes.c_char_p, []),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(rc: int):
    if rc != JET_OK:
        raise JetError(rc, lib().jet_last_error().decode())


def default_options(precision="fp32", reuse=True, use_graph=True, device=0, gemm_min_k=16, profile=0,
                    apply_tc_min_kf=1024, workspace_limit=0, gemm_group=True, fuse_split=True) -> Options:
    o = Options()
    lib().jet_options_default(ctypes.byref(o))
    o.precision = PREC[precision] if isinstance(precision, str) else int(precision)
    o.reuse = int(bool(reuse))
    o.use_graph = int(bool(use_graph))
    o.device = int(device)
    o.gemm_min_k = int(gemm_min_k)
    o.profile = int(profile)
    o.apply_tc_min_kf = int(apply_tc_min_kf)
    o.workspace_limit = int(workspace_limit)
    o.gemm_group = int(bool(gemm_group))
    o.fuse_split = int(bool(fuse_split))
    return o


class Network:
    """A tensor network handle (jet_network_create)."""

    def __init__(self, labels: Sequence[Sequence[int]], data: Sequence[np.ndarray], options: Options = None,
                 **opt_kwargs):
        L = lib()
        self._keep = []
        self._dims = {}
        n = len(data)
        descs = (TensorDesc * n)()
        self.shapes = []
        for i, (lab, t) in enumerate(zip(labels, data)):
            t = np.array(t, dtype=np.complex64, order="C")
            la = np.ascontiguousarray(np.asarray(lab, dtype=np.int64))
            di = np.ascontiguousarray(np.asarray(t.shape, dtype=np.int32))
            if la.size != t.ndim:
                raise JetError(JET_EINVAL, f"tensor {i}: {la.size} labels for rank {t.ndim}")
            self._keep += [t, la, di]
            descs[i].rank = t.ndim
            descs[i].labels = la.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
            descs[i].dims = di.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
            descs[i].data = t.ctypes.data
            self.shapes.append(t.shape)
            for l, d in zip(la.tolist(), t.shape):
                self._dims[l] = d
        opts = options if options is not None else default_options(**opt_kwargs)
        h = ctypes.c_void_p()
        _check(L.jet_network_create(descs, n, ctypes.byref(opts), ctypes.byref(h)))
        self._h = h
        self._keep = []
        self.n_tensors = n
        self.n_out = 0
        self.n_elem = 1   # values per amplitude row (product of the free open legs' dims)

    def close(self):
        if getattr(self, "_h", None):
            lib().jet_network_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    def set_open(self, out_labels: Sequence[int]):
        a = np.ascontiguousarray(np.asarray(out_labels, dtype=np.int64))
        _check(lib().jet_network_set_open(self._h, a.size, a.ctypes.data))
        self.n_out = a.size
        self.n_elem = 1

    def keep_shared(self, min_elems: int):
        """jet_network_keep_shared: keep results of sub-trees without fixed labels
        (at least min_elems elements) for later contractions; 0 switches it off."""
        _check(lib().jet_network_keep_shared(self._h, int(min_elems)))

    def save_shared(self, path: str):
        """jet_network_save_shared: the kept shared work to a file."""
        _check(lib().jet_network_save_shared(self._h, os.fsencode(path)))

    def load_shared(self, path: str):
        """jet_network_load_shared: kept shared work from a file written for this network."""
        _check(lib().jet_network_load_shared(self._h, os.fsencode(path)))

    def set_free(self, free_labels: Sequence[int]):
        """jet_network_set_free: these open legs stay unfixed; every contraction
        returns all their values per row (last axis, first free leg slowest)."""
        a = np.ascontiguousarray(np.asarray(free_labels, dtype=np.int64))
        _check(lib().jet_network_set_free(self._h, a.size, a.ctypes.data))
        self.n_elem = int(np.prod([self._dims[int(l)] for l in a])) if a.size else 1

    def update(self, tensor_id: int, data: np.ndarray):
        t = np.ascontiguousarray(data, dtype=np.complex64)
        _check(lib().jet_tensor_update(self._h, int(tensor_id), t.ctypes.data))

    def n_values(self) -> int:
        return int(lib().jet_network_n_values(self._h))

    def upload(self, host_ptr: int, stream: int = 0):
        _check(lib().jet_tensors_upload(self._h, ctypes.c_void_p(host_ptr), ctypes.c_void_p(stream)))

    def path_set(self, pairs: Sequence[Tuple[int, int]]):
        a = np.ascontiguousarray(np.asarray(pairs, dtype=np.int32).reshape(-1, 2))
        _check(lib().jet_path_set(self._h, a.shape[0], a.ctypes.data))

    def path_get(self) -> List[Tuple[int, int]]:
        a = np.zeros((max(self.n_tensors - 1, 0), 2), dtype=np.int32)
        _check(lib().jet_path_get(self._h, a.ctypes.data))
        return [tuple(map(int, r)) for r in a]

    def path_greedy(self, seed: int = 0, n_trials: int = 1) -> float:
        f = ctypes.c_double()
        _check(lib().jet_path_greedy(self._h, ctypes.c_uint64(seed), int(n_trials), ctypes.byref(f)))
        return f.value

    def path_greedy_batch(self, outputs, seed: int = 0, n_trials: int = 1, max_elems: int = 0) -> float:
        """Greedy path for contracting the batch `outputs` together (every node
        weighted by its number of distinct bra restrictions; pairwise and linear
        passes; intermediates capped at max_elems weighted elements when > 0).
        Returns the batch FLOP of the kept path."""
        o = self._outputs(outputs)
        f = ctypes.c_double()
        _check(lib().jet_path_greedy_batch(self._h, o.shape[0], o.ctypes.data, ctypes.c_int64(int(max_elems)),
                                           ctypes.c_uint64(seed), int(n_trials), ctypes.byref(f)))
        return f.value

    def path_reconfigure(self, passes: int = 8, outputs=None, objective: str = "flop") -> Tuple[float, float]:
        """jet_path_reconfigure: (cost before, after) for the current slicing;
        objective "flop" (Eq. task_based_amplitude_flops) or "time" (estimated seconds)."""
        b, a = ctypes.c_double(), ctypes.c_double()
        obj = {"flop": 0, "time": 1}[objective]
        if outputs is None:
            _check(lib().jet_path_reconfigure(self._h, int(passes), obj, 1, None, ctypes.byref(b), ctypes.byref(a)))
        else:
            o = self._outputs(outputs)
            _check(lib().jet_path_reconfigure(self._h, int(passes), obj, o.shape[0], o.ctypes.data, ctypes.byref(b),
                                              ctypes.byref(a)))
        return b.value, a.value

    def slice(self, labels: Sequence[int]):
        a = np.ascontiguousarray(np.asarray(labels, dtype=np.int64))
        _check(lib().jet_slice(self._h, a.size, a.ctypes.data))

    def slice_auto(self, max_elems: int, min_n: int = 0, max_n: int = 64) -> List[int]:
        n = ctypes.c_int32()
        out = np.zeros(max(max_n, 1), dtype=np.int64)
        _check(lib().jet_slice_auto(self._h, int(max_elems), int(min_n), int(max_n), ctypes.byref(n),
                                    out.ctypes.data))
        return [int(x) for x in out[:n.value]]

    def _outputs(self, outputs) -> np.ndarray:
        o = np.asarray(outputs, dtype=np.int32)
        if self.n_out == 0:   # closed network: one (empty) pattern per amplitude row
            return np.zeros((o.shape[0] if o.ndim == 2 else 1, 0), np.int32)
        return np.ascontiguousarray(o.reshape(-1, self.n_out))

    def plan(self, outputs) -> int:
        o = self._outputs(outputs)
        b = ctypes.c_size_t()
        _check(lib().jet_plan(self._h, o.shape[0], o.ctypes.data, ctypes.byref(b)))
        return b.value

    def plan_slices(self, outputs, slice_ids) -> int:
        """jet_plan_slices: build (and keep) contract_slices' plan; workspace bytes."""
        o = self._outputs(outputs)
        ids = np.ascontiguousarray(np.asarray(slice_ids, dtype=np.int64))
        b = ctypes.c_size_t()
        _check(lib().jet_plan_slices(self._h, o.shape[0], o.ctypes.data, ids.size, ids.ctypes.data, ctypes.byref(b)))
        return b.value

    def plan_ranges(self, outputs, max_bytes: int) -> Dict[str, object]:
        """jet_plan_ranges: the slice ranges a contraction runs under a workspace cap."""
        o = self._outputs(outputs)
        nf, nr = ctypes.c_int32(), ctypes.c_int64()
        flop, nb = ctypes.c_double(), ctypes.c_size_t()
        labels = (ctypes.c_int64 * max(int(self.stats()["n_sliced_labels"]), 1))()
        _check(lib().jet_plan_ranges(self._h, o.shape[0], o.ctypes.data, ctypes.c_size_t(int(max_bytes)),
                                     ctypes.byref(nf), labels, ctypes.byref(nr), ctypes.byref(flop), ctypes.byref(nb)))
        return {"fixed_labels": [int(labels[i]) for i in range(nf.value)], "n_ranges": nr.value,
                "flop": flop.value, "bytes": nb.value}

    def set_workspace(self, dptr: int, nbytes: int):
        _check(lib().jet_set_workspace(self._h, ctypes.c_void_p(dptr), ctypes.c_size_t(nbytes)))

    def contract(self, outputs, stream: int = 0) -> np.ndarray:
        o = self._outputs(outputs)
        amps = np.zeros(o.shape[0] * self.n_elem, dtype=np.complex128)
        _check(lib().jet_contract(self._h, o.shape[0], o.ctypes.data, amps.ctypes.data, ctypes.c_void_p(stream)))
        return amps if self.n_elem == 1 else amps.reshape(o.shape[0], self.n_elem)

    def contract_slices(self, outputs, slice_ids, stream: int = 0) -> np.ndarray:
        """Per-slice partials, shape (n_amps, len(slice_ids)) (with free legs: a
        last axis of their values)."""
        o = self._outputs(outputs)
        ids = np.ascontiguousarray(np.asarray(slice_ids, dtype=np.int64))
        out = np.zeros((o.shape[0], ids.size) + ((self.n_elem,) if self.n_elem > 1 else ()), dtype=np.complex128)
        _check(lib().jet_contract_slices(self._h, o.shape[0], o.ctypes.data, ids.size, ids.ctypes.data,
                                         out.ctypes.data, ctypes.c_void_p(stream)))
        return out

    def contract_async(self, outputs, amps_dev_ptr: int, stream: int = 0):
        o = self._outputs(outputs)
        _check(lib().jet_contract_async(self._h, o.shape[0], o.ctypes.data, ctypes.c_void_p(amps_dev_ptr),
                                        ctypes.c_void_p(stream)))

    def contract_grad(self, outputs, cot, tensor_ids: Sequence[int], stream: int = 0):
        o = self._outputs(outputs)
        c = np.ascontiguousarray(np.asarray(cot, dtype=np.complex128).reshape(o.shape[0]))
        ids = np.ascontiguousarray(np.asarray(tensor_ids, dtype=np.int32))
        # out-of-range ids get a placeholder buffer; the library rejects them
        envs = [np.zeros(self.shapes[i] if 0 <= i < len(self.shapes) else (1,), dtype=np.complex64) for i in ids]
        ptrs = (ctypes.c_void_p * max(len(envs), 1))(*[e.ctypes.data for e in envs])
        amps = np.zeros(o.shape[0], dtype=np.complex128)
        _check(lib().jet_contract_grad(self._h, o.shape[0], o.ctypes.data, c.ctypes.data, ids.size,
                                       ids.ctypes.data, ptrs, amps.ctypes.data, ctypes.c_void_p(stream)))
        return amps, envs

    def profile(self) -> List[Dict[str, float]]:
        n = ctypes.c_int32()
        _check(lib().jet_profile(self._h, None, 0, ctypes.byref(n)))
        recs = (OpRecord * max(n.value, 1))()
        _check(lib().jet_profile(self._h, recs, n.value, ctypes.byref(n)))
        return [{"kind": OP_KINDS.get(r.kind, str(r.kind)), "node": r.node, "n_inst": r.n_inst, "flop": r.flop,
                 "bytes": r.bytes, "ms": r.ms, "block": r.block, "grid": tuple(r.grid), "smem": r.smem,
                 "variant": r.variant}
                for r in recs[:n.value]]

    def plan_buffers(self) -> List[Dict[str, int]]:
        """jet_plan_buffers: the workspace allocations of the last plan with their
        launch-time windows (the intermediate-deletion record)."""
        n = ctypes.c_int32()
        _check(lib().jet_plan_buffers(self._h, None, 0, ctypes.byref(n)))
        recs = (BufferRecord * max(n.value, 1))()
        _check(lib().jet_plan_buffers(self._h, recs, n.value, ctypes.byref(n)))
        return [{name: getattr(r, name) for name, _ in BufferRecord._fields_ if name != "pad_"}
                for r in recs[:n.value]]

    def autotune(self, outputs, cache_file: Optional[str] = None, stream: int = 0) -> Dict[str, float]:
        """jet_autotune: per-node kernel-form choices timed on the device."""
        o = self._outputs(outputs)
        d, t = ctypes.c_double(), ctypes.c_double()
        n = ctypes.c_int32()
        _check(lib().jet_autotune(self._h, o.shape[0], o.ctypes.data, cache_file.encode() if cache_file else None,
                                  ctypes.c_void_p(stream), ctypes.byref(d), ctypes.byref(t), ctypes.byref(n)))
        return {"default_ms": d.value, "tuned_ms": t.value, "n_changed": n.value}

    def selftest_wait(self, limit_us: int, stream: int = 0):
        """jet_selftest_wait: raises JetError(JET_ETIMEOUT) when the bounded wait
        ran out and was reported (the expected outcome)."""
        _check(lib().jet_selftest_wait(self._h, int(limit_us), ctypes.c_void_p(stream)))

    def stats(self) -> Dict[str, float]:
        s = Stats()
        _check(lib().jet_stats(self._h, ctypes.byref(s)))
        return {name: getattr(s, name) for name, _ in Stats._fields_}


def pair_contract_noalloc(labels_a, shape_a, a_dev_ptr: int, labels_b, shape_b, b_dev_ptr: int, c_dev_ptr: int,
                          device: int = 0, stream: int = 0):
    """jet_pair_contract_noalloc: contract two complex64 device tensors into a
    caller-allocated device output without any device allocation."""
    la = np.ascontiguousarray(np.asarray(labels_a, dtype=np.int64))
    lb = np.ascontiguousarray(np.asarray(labels_b, dtype=np.int64))
    da = np.ascontiguousarray(np.asarray(shape_a, dtype=np.int32))
    db = np.ascontiguousarray(np.asarray(shape_b, dtype=np.int32))
    if la.size != da.size or lb.size != db.size:
        raise ValueError("each operand needs one dim per label")
    _check(lib().jet_pair_contract_noalloc(la.size, la.ctypes.data, da.ctypes.data, ctypes.c_void_p(a_dev_ptr),
                                           lb.size, lb.ctypes.data, db.ctypes.data, ctypes.c_void_p(b_dev_ptr),
                                           ctypes.c_void_p(c_dev_ptr), int(device), ctypes.c_void_p(stream)))


def sum_partials(partials: np.ndarray) -> np.ndarray:
    """jet_sum_partials: partials[b, j(, e)] summed over j in increasing order, FP64."""
    p = np.ascontiguousarray(np.asarray(partials, dtype=np.complex128))
    if p.ndim == 2:
        p = p[:, :, None]
    n_amps, n_ids, n_elem = p.shape
    out = np.zeros((n_amps, n_elem), dtype=np.complex128)
    _check(lib().jet_sum_partials(n_amps, n_ids, max(n_elem, 1), p.ctypes.data if p.size else None,
                                  out.ctypes.data))
    return out[:, 0] if np.ndim(partials) == 2 else out


def from_network(tn, **opt_kwargs) -> Network:
    """Build a handle from a circuits.TensorNetwork and declare its open legs."""
    net = Network(tn.labels, tn.data, **opt_kwargs)
    net.set_open(tn.open_labels)
    return net
