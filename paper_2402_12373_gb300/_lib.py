"""ctypes binding of libltl_gb300.so (argument marshalling only).

Every step of learning and evaluation runs in the library's CUDA kernels;
this module only converts Python / numpy / torch objects into the C ABI of
include/ltl.h.  PyTorch supplies device memory (the workspace tensor) and the
CUDA stream.  There is no fallback: if the shared library cannot be loaded the
import fails loudly.
"""
from __future__ import annotations

import ctypes
import os
from typing import Dict, List, Optional, Sequence

import numpy as np

from . import build as _build

LTL_OK, LTL_NOT_FOUND, LTL_CAP_REACHED = 0, 1, 2
LTL_ERR_INVALID, LTL_ERR_CUDA, LTL_ERR_OOM, LTL_ERR_TIMEOUT, LTL_ERR_BUFSIZE = -1, -2, -3, -4, -5
STATUS = {0: "found", 1: "not_found", 2: "cap", -1: "invalid", -2: "cuda", -3: "oom", -4: "timeout",
          -5: "bufsize"}
NOT, AND, OR, X, F, G, U, ALL = 1, 2, 4, 8, 16, 32, 64, 127
NNF = 256   # negation on atoms only (flag in the ops mask)
RUC_EXACT, RUC_HASH, RUC_FKP = 0, 1, 2   # cache admission policies
DC_DETERMINISTIC, DC_RANDOM = 0, 1       # divide-and-conquer split modes
KERNEL_AUTO, KERNEL_FUSED, KERNEL_WS = 0, 1, 2   # size-level kernel choice
PLAN_AUTO, PLAN_HOST = 0, 1                       # where size levels are planned
PROP_CARRY, PROP_LOGSTEP = 0, 1                   # how the level kernels compute F, G and U
STOP_NONE, STOP_FIRST, STOP_LEVEL = 0, 1, 2
MAX_LEVELS = 64

# Every symbol include/ltl.h declares.
EXPORTS = ["ltl_learn", "ltl_eval", "ltl_ctx_create", "ltl_ctx_destroy", "ltl_ctx_learn",
           "ltl_ctx_learn_device", "ltl_ctx_level_range", "ltl_ctx_entry", "ltl_last_error",
           "ltl_version", "ltl_eval_noalloc", "ltl_learn_batch", "ltl_server_create", "ltl_ctx_set_mem_budget",
           "ltl_server_submit", "ltl_server_poll", "ltl_server_pending", "ltl_server_destroy", "ltl_learn_dc",
           "ltl_ctx_autotune_dump", "ltl_int32_peak"]
FORMULA_MAX = 512
# level kernel used when a call does not choose one (tests switch it to run
# every entry point on both kernels)
DEFAULT_LEVEL_KERNEL = KERNEL_AUTO
# ltl_stats.op_kernel values (LTL_LAUNCH_*)
LAUNCH_KINDS = {0: None, 1: "fused_level_kernel", 2: "ws_level_kernel", 3: "stream_level_kernel",
                4: "cluster_level_kernel"}
# level planning used when a call does not choose one
DEFAULT_PLANNING = PLAN_AUTO
# F/G/U evaluation used when a call does not choose one (tests switch it to
# run the parity suite on both)
DEFAULT_PROPAGATION = PROP_CARRY


class LtlError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("%s: %s" % (STATUS.get(status, status), msg))
        self.status = status


class Traces(ctypes.Structure):
    _fields_ = [("letters", ctypes.c_void_p), ("offsets", ctypes.c_void_p), ("n_traces", ctypes.c_uint64)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)


class Opts(ctypes.Structure):
    _fields_ = [("mem_budget_bytes", ctypes.c_uint64), ("stop_on_solution", ctypes.c_int),
                ("spin_limit", ctypes.c_uint64), ("alloc", ALLOC_FN), ("free", FREE_FN),
                ("user", ctypes.c_void_p), ("stream", ctypes.c_void_p), ("workspace", ctypes.c_void_p),
                ("workspace_bytes", ctypes.c_uint64), ("autotune_path", ctypes.c_char_p),
                ("max_chunks", ctypes.c_uint32), ("costs", ctypes.c_uint32 * 8),
                ("max_errors", ctypes.c_uint32), ("ruc", ctypes.c_uint32), ("ruc_mask_bits", ctypes.c_uint32),
                ("level_kernel", ctypes.c_uint32), ("level_planning", ctypes.c_uint32),
                ("propagation", ctypes.c_uint32)]


class Stats(ctypes.Structure):
    _fields_ = [("levels_done", ctypes.c_int), ("found_size", ctypes.c_int),
                ("unique", ctypes.c_uint64 * MAX_LEVELS), ("candidates", ctypes.c_uint64 * MAX_LEVELS),
                ("ms", ctypes.c_double * MAX_LEVELS), ("entries", ctypes.c_uint64),
                ("n_traces", ctypes.c_uint64), ("words_per_trace", ctypes.c_uint32),
                ("threads_per_cta", ctypes.c_uint32), ("traces_per_thread", ctypes.c_uint32),
                ("chunk_groups", ctypes.c_uint32), ("batch", ctypes.c_uint32),
                ("traces_per_word", ctypes.c_uint32),
                ("ctas_per_sm", ctypes.c_uint32), ("launches", ctypes.c_uint64),
                ("h2d_bytes", ctypes.c_uint64), ("d2h_bytes", ctypes.c_uint64),
                ("max_entries", ctypes.c_uint64), ("total_ms", ctypes.c_double),
                ("op_ms", (ctypes.c_float * 8) * MAX_LEVELS),
                ("device_planned_levels", ctypes.c_uint32), ("graph_levels", ctypes.c_uint32),
                ("compares", ctypes.c_uint64), ("collisions", ctypes.c_uint64),
                ("op_staged", (ctypes.c_uint64 * 8) * MAX_LEVELS),
                ("op_kernel", (ctypes.c_uint8 * 8) * MAX_LEVELS),
                ("op_alone", (ctypes.c_uint8 * 8) * MAX_LEVELS)]

    def to_dict(self, max_size: int) -> Dict:
        # ctypes scalar fields read as Python numbers, array slices as lists
        K = max_size
        return {
            "levels_done": self.levels_done, "found_size": self.found_size,
            "unique": self.unique[:K + 1], "candidates": self.candidates[:K + 1], "ms": self.ms[:K + 1],
            "entries": self.entries, "n_traces": self.n_traces,
            "words_per_trace": self.words_per_trace, "threads_per_cta": self.threads_per_cta,
            "traces_per_thread": self.traces_per_thread, "chunk_groups": self.chunk_groups,
            "batch": self.batch, "ctas_per_sm": self.ctas_per_sm, "traces_per_word": self.traces_per_word,
            "launches": self.launches, "h2d_bytes": self.h2d_bytes,
            "d2h_bytes": self.d2h_bytes, "max_entries": self.max_entries,
            "total_ms": self.total_ms,
            "op_ms": [self.op_ms[c][:] for c in range(K + 1)],
            "device_planned_levels": self.device_planned_levels, "graph_levels": self.graph_levels,
            "compares": self.compares, "collisions": self.collisions,
            "op_staged": [self.op_staged[c][:] for c in range(K + 1)],
            "op_kernel": [[LAUNCH_KINDS[x] for x in self.op_kernel[c][:]] for c in range(K + 1)],
            "op_alone": [[x != 0 for x in self.op_alone[c][:]] for c in range(K + 1)],
        }


class ProblemDesc(ctypes.Structure):
    _fields_ = [("P", Traces), ("N", Traces), ("n_props", ctypes.c_int), ("ops", ctypes.c_uint32),
                ("max_size", ctypes.c_int), ("mem_budget_bytes", ctypes.c_uint64)]


class Result(ctypes.Structure):
    _fields_ = [("id", ctypes.c_uint64), ("status", ctypes.c_int), ("found_size", ctypes.c_int),
                ("levels_done", ctypes.c_int), ("formula", ctypes.c_char * FORMULA_MAX),
                ("unique", ctypes.c_uint64 * MAX_LEVELS), ("candidates", ctypes.c_uint64 * MAX_LEVELS),
                ("n_traces", ctypes.c_uint64), ("rounds", ctypes.c_uint32), ("queue_ms", ctypes.c_double),
                ("latency_ms", ctypes.c_double)]

    def to_dict(self) -> Dict:
        # ctypes scalar fields read as Python numbers, array slices as lists
        st = self.status
        return {"id": self.id, "status": STATUS.get(st, st), "size": self.found_size if st == 0 else None,
                "formula": self.formula.decode() if st == 0 else None, "levels_done": self.levels_done,
                "unique": self.unique[:], "candidates": self.candidates[:],
                "n_traces": self.n_traces, "rounds": self.rounds, "queue_ms": self.queue_ms,
                "latency_ms": self.latency_ms}


_lib = None


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Loads (building first if needed) the CUDA library; raises if impossible."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing and not _build.up_to_date():
        _build.build()
    if not os.path.exists(path):
        raise ImportError("libltl_gb300.so is missing; run paper_2402_12373_gb300.build.build()")
    L = ctypes.CDLL(path)
    vp, u64, i32, u32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int, ctypes.c_uint32
    TP = ctypes.POINTER(Traces)
    L.ltl_learn.argtypes = [TP, TP, i32, u32, i32, ctypes.POINTER(Opts), ctypes.c_char_p, ctypes.c_size_t,
                            ctypes.POINTER(Stats)]
    L.ltl_eval.argtypes = [ctypes.c_char_p, TP, i32, vp, i32]
    L.ltl_ctx_create.argtypes = [ctypes.POINTER(Opts), ctypes.POINTER(vp)]
    L.ltl_ctx_destroy.argtypes = [vp]
    L.ltl_ctx_destroy.restype = None
    L.ltl_ctx_learn.argtypes = [vp, TP, TP, i32, u32, i32, ctypes.c_char_p, ctypes.c_size_t,
                                ctypes.POINTER(Stats)]
    L.ltl_ctx_learn_device.argtypes = [vp, vp, vp, u64, u64, u32, i32, u32, i32, ctypes.c_char_p,
                                       ctypes.c_size_t, ctypes.POINTER(Stats)]
    L.ltl_ctx_level_range.argtypes = [vp, i32, ctypes.POINTER(u64), ctypes.POINTER(u64)]
    L.ltl_ctx_entry.argtypes = [vp, u64, ctypes.c_char_p, ctypes.c_size_t, vp, i32]
    L.ltl_eval_noalloc.argtypes = [ctypes.c_char_p, vp, vp, u64, u32, i32, vp, i32, vp]
    L.ltl_eval_noalloc.restype = ctypes.c_int
    L.ltl_ctx_set_mem_budget.argtypes = [vp, u64]
    L.ltl_ctx_set_mem_budget.restype = ctypes.c_int
    L.ltl_learn_batch.argtypes = [i32, ctypes.POINTER(ProblemDesc), ctypes.POINTER(Opts), ctypes.POINTER(Result)]
    L.ltl_learn_batch.restype = ctypes.c_int
    L.ltl_server_create.argtypes = [ctypes.POINTER(Opts), i32, ctypes.POINTER(vp)]
    L.ltl_server_create.restype = ctypes.c_int
    L.ltl_server_submit.argtypes = [vp, ctypes.POINTER(ProblemDesc), ctypes.POINTER(u64)]
    L.ltl_server_submit.restype = ctypes.c_int
    L.ltl_server_poll.argtypes = [vp, ctypes.POINTER(Result), i32, ctypes.POINTER(i32), i32]
    L.ltl_server_poll.restype = ctypes.c_int
    L.ltl_server_pending.argtypes = [vp, ctypes.POINTER(u64), ctypes.POINTER(u64)]
    L.ltl_server_pending.restype = ctypes.c_int
    L.ltl_server_destroy.argtypes = [vp]
    L.ltl_server_destroy.restype = None
    L.ltl_learn_dc.argtypes = [TP, TP, i32, u32, i32, ctypes.POINTER(Opts), ctypes.POINTER(DcOpts), ctypes.c_char_p,
                               ctypes.c_size_t, ctypes.POINTER(DcStats)]
    L.ltl_learn_dc.restype = ctypes.c_int
    L.ltl_ctx_autotune_dump.argtypes = [vp, ctypes.c_char_p, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)]
    L.ltl_ctx_autotune_dump.restype = ctypes.c_int
    L.ltl_int32_peak.argtypes = [i32, i32, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
    L.ltl_int32_peak.restype = ctypes.c_int
    L.ltl_last_error.restype = ctypes.c_char_p
    L.ltl_version.restype = ctypes.c_char_p
    for f in ("ltl_learn", "ltl_eval", "ltl_ctx_create", "ltl_ctx_learn", "ltl_ctx_learn_device",
              "ltl_ctx_level_range", "ltl_ctx_entry"):
        getattr(L, f).restype = ctypes.c_int
    _lib = L
    return L


def last_error() -> str:
    return load().ltl_last_error().decode(errors="replace")


def _check(rc: int, ok=(LTL_OK, LTL_NOT_FOUND, LTL_CAP_REACHED)) -> int:
    if rc not in ok:
        raise LtlError(rc, last_error())
    return rc


class _HostTraces:
    """Keeps numpy arrays alive while a ctypes Traces struct points at them."""

    def __init__(self, ts):
        self.letters = np.ascontiguousarray(np.asarray(ts.letters, dtype=np.uint32))
        self.offsets = np.ascontiguousarray(np.asarray(ts.offsets, dtype=np.uint64))
        if self.letters.size == 0:
            self.letters = np.zeros(1, dtype=np.uint32)
        self.struct = Traces(self.letters.ctypes.data, self.offsets.ctypes.data, self.offsets.shape[0] - 1)


def _opts(stop: int = STOP_FIRST, workspace=None, stream=None, mem_budget: int = 0,
          spin_limit: int = 0, max_chunks: int = 0, costs=None, max_errors: int = 0, ruc: int = RUC_EXACT,
          ruc_mask_bits: int = 0, level_kernel: Optional[int] = None, autotune: Optional[str] = None,
          planning: Optional[int] = None, propagation: Optional[int] = None) -> Opts:
    """costs: 8 connective costs (atoms, !, &, |, X, F, G, U), None = all 1;
    max_errors: misclassified traces a separator may have; ruc, ruc_mask_bits:
    cache admission policy and masked admission-key bits."""
    o = Opts()
    o.mem_budget_bytes = int(mem_budget)
    o.stop_on_solution = int(stop)
    o.spin_limit = int(spin_limit)
    o.alloc = ALLOC_FN()
    o.free = FREE_FN()
    o.user = None
    o.stream = stream
    o.workspace = None
    o.workspace_bytes = 0
    # None: fixed heuristics; "": tune in memory; a path: tune and keep the results there
    o.autotune_path = None if autotune is None else autotune.encode()
    o.max_chunks = int(max_chunks)
    if costs is not None:
        if len(costs) != 8 or min(costs) < 1:
            raise ValueError("costs: eight positive integers (atoms, !, &, |, X, F, G, U)")
        for i, c in enumerate(costs):
            o.costs[i] = int(c)
    o.max_errors = int(max_errors)
    o.ruc = int(ruc)
    o.ruc_mask_bits = int(ruc_mask_bits)
    o.level_kernel = int(DEFAULT_LEVEL_KERNEL if level_kernel is None else level_kernel)
    o.level_planning = int(DEFAULT_PLANNING if planning is None else planning)
    o.propagation = int(DEFAULT_PROPAGATION if propagation is None else propagation)
    if workspace is not None:
        o.workspace = workspace.data_ptr()
        o.workspace_bytes = workspace.numel() * workspace.element_size()
    return o


def default_workspace(nbytes: Optional[int] = None, device: int = 0):
    """A torch-allocated device workspace (uint8 tensor, 256-byte aligned)."""
    import torch
    if nbytes is None:
        free, _ = torch.cuda.mem_get_info(device)
        nbytes = int(free * 0.4)
    return torch.empty(int(nbytes), dtype=torch.uint8, device="cuda:%d" % device)


def _current_stream():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


class Context:
    """A reusable learner context: stream + torch workspace + last cache."""

    def __init__(self, workspace=None, stop: int = STOP_FIRST, stream=None, mem_budget: int = 0,
                 spin_limit: int = 0, workspace_bytes: Optional[int] = None, max_chunks: int = 0,
                 costs=None, max_errors: int = 0, ruc: int = RUC_EXACT, ruc_mask_bits: int = 0,
                 level_kernel: Optional[int] = None, autotune: Optional[str] = None,
                 planning: Optional[int] = None, propagation: Optional[int] = None):
        self._L = load()
        if workspace is None:
            workspace = default_workspace(workspace_bytes)
        self.workspace = workspace
        if stream is None:
            stream = _current_stream()
        self._opts = _opts(stop, workspace, stream, mem_budget, spin_limit, max_chunks, costs, max_errors, ruc,
                           ruc_mask_bits, level_kernel, autotune, planning, propagation)
        h = ctypes.c_void_p()
        _check(self._L.ltl_ctx_create(ctypes.byref(self._opts), ctypes.byref(h)), ok=(LTL_OK,))
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            self._L.ltl_ctx_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def autotune_dump(self) -> str:
        """The autotuner's measurements (ltl_ctx_autotune_dump)."""
        need = ctypes.c_size_t(0)
        self._L.ltl_ctx_autotune_dump(self._h, None, 0, ctypes.byref(need))
        buf = ctypes.create_string_buffer(max(int(need.value), 1))
        _check(self._L.ltl_ctx_autotune_dump(self._h, buf, len(buf), ctypes.byref(need)), ok=(LTL_OK,))
        return buf.value.decode()

    def set_mem_budget(self, nbytes: int) -> None:
        _check(self._L.ltl_ctx_set_mem_budget(self._h, int(nbytes)), ok=(LTL_OK,))

    def learn(self, P, N, n_props: int, ops: int = ALL, max_size: int = 7) -> Dict:
        hp, hn = _HostTraces(P), _HostTraces(N)
        buf = ctypes.create_string_buffer(8 * max_size + 64)
        st = Stats()
        rc = self._L.ltl_ctx_learn(self._h, ctypes.byref(hp.struct), ctypes.byref(hn.struct), n_props, ops,
                                   max_size, buf, len(buf), ctypes.byref(st))
        return _result(_check(rc), buf, st, max_size)

    def learn_device(self, letters, offsets, n_pos: int, n_neg: int, max_len: int, n_props: int,
                     ops: int = ALL, max_size: int = 7) -> Dict:
        """Traces already on the device: torch uint32/int32 letters, int64 offsets."""
        buf = ctypes.create_string_buffer(8 * max_size + 64)
        st = Stats()
        rc = self._L.ltl_ctx_learn_device(self._h, ctypes.c_void_p(letters.data_ptr()),
                                          ctypes.c_void_p(offsets.data_ptr()), n_pos, n_neg, max_len, n_props,
                                          ops, max_size, buf, len(buf), ctypes.byref(st))
        return _result(_check(rc), buf, st, max_size)

    def level_range(self, level: int):
        b, c = ctypes.c_uint64(), ctypes.c_uint64()
        _check(self._L.ltl_ctx_level_range(self._h, level, ctypes.byref(b), ctypes.byref(c)), ok=(LTL_OK,))
        return int(b.value), int(c.value)

    def entry(self, idx: int, n_traces: int, words_per_trace: int):
        buf = ctypes.create_string_buffer(1024)
        cs = np.zeros((max(n_traces, 1), words_per_trace), dtype=np.uint64)
        _check(self._L.ltl_ctx_entry(self._h, idx, buf, len(buf), cs.ctypes.data, words_per_trace),
               ok=(LTL_OK,))
        return buf.value.decode(), cs[:n_traces]


def _result(rc: int, buf, st: Stats, max_size: int) -> Dict:
    d = st.to_dict(max_size)
    d["status"] = STATUS[rc]
    d["formula"] = buf.value.decode() if rc == LTL_OK else None
    d["size"] = d["found_size"] if rc == LTL_OK else None
    return d


def learn(P, N, n_props: int, ops: int = ALL, max_size: int = 7, stop: int = STOP_FIRST,
          workspace=None, mem_budget: int = 0, costs=None, max_errors: int = 0, ruc: int = RUC_EXACT,
          ruc_mask_bits: int = 0) -> Dict:
    """One-shot ltl_learn with host traces (TraceSet-like P and N)."""
    L = load()
    hp, hn = _HostTraces(P), _HostTraces(N)
    o = _opts(stop, workspace, _current_stream() if workspace is not None else None, mem_budget, 0, 0, costs,
              max_errors, ruc, ruc_mask_bits)
    buf = ctypes.create_string_buffer(8 * max_size + 64)
    st = Stats()
    rc = L.ltl_learn(ctypes.byref(hp.struct), ctypes.byref(hn.struct), n_props, ops, max_size,
                     ctypes.byref(o), buf, len(buf), ctypes.byref(st))
    return _result(_check(rc), buf, st, max_size)


def evaluate(formula: str, traces, n_props: int, words_per_trace: Optional[int] = None) -> np.ndarray:
    """ltl_eval: uint64 [n_traces, words_per_trace] characteristic sequences."""
    L = load()
    ht = _HostTraces(traces)
    n = ht.offsets.shape[0] - 1
    lens = np.diff(ht.offsets.astype(np.int64)) if n else np.zeros(0, np.int64)
    W = max(1, (int(max(lens.max(), 0)) + 63) // 64) if n else 1
    if words_per_trace is None:
        words_per_trace = W
    out = np.zeros((max(n, 1), words_per_trace), dtype=np.uint64)
    rc = L.ltl_eval(formula.encode(), ctypes.byref(ht.struct), n_props, out.ctypes.data, words_per_trace)
    _check(rc, ok=(LTL_OK,))
    return out[:n]


def evaluate_noalloc(formula: str, letters, offsets, n_traces: int, max_len: int, n_props: int, out,
                     words_per_trace: int, stream=None) -> None:
    """ltl_eval_noalloc on device tensors (letters int32/uint32, offsets int64,
    out int64 [n_traces, words_per_trace]); allocates no device memory."""
    L = load()
    if stream is None:
        stream = _current_stream()
    rc = L.ltl_eval_noalloc(formula.encode(), ctypes.c_void_p(letters.data_ptr()),
                            ctypes.c_void_p(offsets.data_ptr()), n_traces, max_len, n_props,
                            ctypes.c_void_p(out.data_ptr()), words_per_trace, stream)
    _check(rc, ok=(LTL_OK,))


def _problem_desc(P, N, n_props: int, ops: int, max_size: int, budget: int = 0):
    hp, hn = _HostTraces(P), _HostTraces(N)
    d = ProblemDesc(hp.struct, hn.struct, n_props, ops, max_size, int(budget))
    return d, (hp, hn)


def learn_batch(problems: Sequence, stop: int = STOP_FIRST, workspace=None, mem_budget: int = 0,
                max_chunks: int = 0, costs=None, max_errors: int = 0, ruc: int = RUC_EXACT,
                ruc_mask_bits: int = 0) -> List[Dict]:
    """ltl_learn_batch.  problems: sequence of (P, N, n_props, ops, max_size[, budget])."""
    L = load()
    n = len(problems)
    descs = (ProblemDesc * max(n, 1))()
    keep = []
    for i, pr in enumerate(problems):
        P, N, n_props, ops, max_size = pr[:5]
        budget = pr[5] if len(pr) > 5 else 0
        d, k = _problem_desc(P, N, n_props, ops, max_size, budget)
        descs[i] = d
        keep.append(k)
    out = (Result * max(n, 1))()
    o = _opts(stop, workspace, _current_stream() if workspace is not None else None, mem_budget, 0, max_chunks,
              costs, max_errors, ruc, ruc_mask_bits)
    _check(L.ltl_learn_batch(n, descs, ctypes.byref(o), out), ok=(LTL_OK,))
    return [out[i].to_dict() for i in range(n)]


class Server:
    """ltl_server_*: continuous batching of submitted learning problems."""

    def __init__(self, workspace=None, stop: int = STOP_FIRST, max_resident: int = 64, mem_budget: int = 0,
                 workspace_bytes: Optional[int] = None, max_chunks: int = 0, costs=None,
                 max_errors: int = 0, ruc: int = RUC_EXACT, ruc_mask_bits: int = 0):
        self._L = load()
        if workspace is None:
            workspace = default_workspace(workspace_bytes)
        self.workspace = workspace
        self._opts = _opts(stop, workspace, None, mem_budget, 0, max_chunks, costs, max_errors, ruc, ruc_mask_bits)
        h = ctypes.c_void_p()
        _check(self._L.ltl_server_create(ctypes.byref(self._opts), max_resident, ctypes.byref(h)), ok=(LTL_OK,))
        self._h = h

    def submit(self, P, N, n_props: int, ops: int = ALL, max_size: int = 7, budget: int = 0) -> int:
        d, _keep = _problem_desc(P, N, n_props, ops, max_size, budget)
        i = ctypes.c_uint64()
        _check(self._L.ltl_server_submit(self._h, ctypes.byref(d), ctypes.byref(i)), ok=(LTL_OK,))
        return int(i.value)

    def poll(self, max_results: int = 64, wait_ms: int = 0) -> List[Dict]:
        out = (Result * max_results)()
        n = ctypes.c_int()
        _check(self._L.ltl_server_poll(self._h, out, max_results, ctypes.byref(n), wait_ms), ok=(LTL_OK,))
        return [out[i].to_dict() for i in range(n.value)]

    def pending(self):
        q, r = ctypes.c_uint64(), ctypes.c_uint64()
        _check(self._L.ltl_server_pending(self._h, ctypes.byref(q), ctypes.byref(r)), ok=(LTL_OK,))
        return int(q.value), int(r.value)

    def close(self):
        if getattr(self, "_h", None):
            self._L.ltl_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class DcOpts(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int), ("window", ctypes.c_uint64), ("seed", ctypes.c_uint64),
                ("max_resident", ctypes.c_int)]


class DcStats(ctypes.Structure):
    _fields_ = [("enum_calls", ctypes.c_uint64), ("enum_failed", ctypes.c_uint64), ("fallbacks", ctypes.c_uint64),
                ("evals", ctypes.c_uint64), ("rounds", ctypes.c_uint64), ("min_window", ctypes.c_uint64),
                ("max_depth", ctypes.c_int), ("formula_size", ctypes.c_uint64), ("formula_len", ctypes.c_uint64),
                ("total_ms", ctypes.c_double)]

    def to_dict(self) -> Dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


def learn_dc(P, N, n_props: int, ops: int = ALL, max_size: int = 7, mode: int = DC_RANDOM, window: int = 64,
             seed: int = 0, max_resident: int = 0, workspace=None, mem_budget: int = 0, costs=None,
             ruc: int = RUC_EXACT, ruc_mask_bits: int = 0) -> Dict:
    """ltl_learn_dc: divide and conquer over the enumerator (host traces).
    Returns the formula, the status and the split statistics."""
    L = load()
    hp, hn = _HostTraces(P), _HostTraces(N)
    o = _opts(STOP_FIRST, workspace, _current_stream() if workspace is not None else None, mem_budget, 0, 0, costs,
              0, ruc, ruc_mask_bits)
    dc = DcOpts(int(mode), int(window), int(seed), int(max_resident))
    st = DcStats()
    cap = 1 << 16
    for _ in range(2):
        buf = ctypes.create_string_buffer(cap)
        rc = L.ltl_learn_dc(ctypes.byref(hp.struct), ctypes.byref(hn.struct), n_props, ops, max_size,
                            ctypes.byref(o), ctypes.byref(dc), buf, len(buf), ctypes.byref(st))
        if rc != LTL_ERR_BUFSIZE:
            break
        cap = int(st.formula_len) + 1
    _check(rc)
    d = st.to_dict()
    d["status"] = STATUS[rc]
    d["formula"] = buf.value.decode() if rc == LTL_OK else None
    return d


def version() -> str:
    return load().ltl_version().decode()


def int32_peak(iters: int = 1 << 16, repeats: int = 3) -> Dict:
    """Measured 32-bit shift + logic throughput of the current device (ltl_int32_peak)."""
    ops, ms = ctypes.c_double(), ctypes.c_double()
    _check(load().ltl_int32_peak(iters, repeats, ctypes.byref(ops), ctypes.byref(ms)), ok=(LTL_OK,))
    return {"ops_per_s": ops.value, "ms": ms.value}
