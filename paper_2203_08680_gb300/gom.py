"""Thin Python binding of libgom.so (include/gom.h): same names, argument
marshalling only.  Every step of the method runs in the library's CUDA
kernels; there is no Python or CPU fallback, and a missing library is an
error.

Device buffers are passed as torch CUDA tensors (or raw integer device
addresses); PyTorch only provides device memory and streams.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

GOM_OK = 0
GOM_FOS_NEIGHBOURHOOD = 0
GOM_FOS_SINGLETON = 1
GOM_FOS_BFLT = 2
GOM_MAX_POPULATION = 1024
GOM_MAX_ELEMENT = 128
GOM_OPT_PERSISTENT = 1
GOM_OPT_PHASE_TRACE = 2
GOM_OPT_DYNAMIC = 3
GOM_OPT_BITSLICED = 4
GOM_OPT_FORCED_IMPROVEMENT = 5
GOM_OPT_FI_NIS = 6
GOM_OPT_FILTER_LABEL = 7
INT64_MAX = 2 ** 63 - 1

ERRORS = {-1: "GOM_E_ARG", -2: "GOM_E_GRAPH", -3: "GOM_E_NOT_COLORED", -4: "GOM_E_WORKSPACE",
          -5: "GOM_E_CUDA", -6: "GOM_E_TIMEOUT", -7: "GOM_E_STATE", -8: "GOM_E_LIMIT",
          -9: "GOM_E_FOS"}


class GomError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__(f"{what}: {ERRORS.get(code, code)} ({gom_strerror(code)})")


class GraphT(C.Structure):
    _fields_ = [("num_vertices", C.c_int32), ("num_adj", C.c_int64), ("row_ptr", C.c_void_p),
                ("col", C.c_void_p), ("weight", C.c_void_p)]


class GenStats(C.Structure):
    _fields_ = [(name, C.c_int64) for name in
                ("generation", "best_fitness", "elite_fitness", "trials", "donorless", "accepted",
                 "improving", "reached_target", "fi_individuals", "fi_trials", "fi_accepted", "fi_improving",
                 "fi_replaced")]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


_lib = None

# (name, restype, argtypes) of every entry point declared in include/gom.h
_P, _I32, _I64, _U64, _SZ = C.c_void_p, C.c_int32, C.c_int64, C.c_uint64, C.c_size_t
SIGNATURES = [
    ("gom_build_fos", C.c_int, [_P, _I32, _I32, _P]),
    ("gom_fos_create", C.c_int, [_I32, _I64, _P, _P, _P]),
    ("gom_color_fos", C.c_int, [_P, _P, _P]),
    ("gom_fos_sizes", C.c_int, [_P, _P, _P, _P]),
    ("gom_fos_export", C.c_int, [_P, _P, _P, _P, _P, _P]),
    ("gom_fos_destroy", None, [_P]),
    ("gom_workspace_bytes", _SZ, [_P, _P, _I32]),
    ("gom_init_population", C.c_int, [_P, _P, _I32, _U64, _P, _SZ, _P, _P]),
    ("gom_generation", C.c_int, [_P, _I32, _I64, _P, _P]),
    ("gom_fitness", C.c_int, [_P, _P]),
    ("gom_get_population", C.c_int, [_P, _P, _P, _P]),
    ("gom_get_elite", C.c_int, [_P, _P, _P]),
    ("gom_set_population", C.c_int, [_P, _P, _P, _I64, _I64]),
    ("gom_get_generation", C.c_int, [_P, _P]),
    ("gom_set_timing", C.c_int, [_P, _I32]),
    ("gom_read_timing", C.c_int, [_P, _P, _P]),
    ("gom_launches_per_generation", C.c_int, [_P, _P]),
    ("gom_set_option", C.c_int, [_P, _I32, _I64]),
    ("gom_get_option", C.c_int, [_P, _I32, _P]),
    ("gom_read_phase_trace", C.c_int, [_P, _P, _I32, _P]),
    ("gom_selftest_barrier", C.c_int, [_P, _I32, _I32, _I64, _P, _P]),
    ("gom_fitness_noalloc", C.c_int, [_P, _P, _P, _I32, _P, _I32, _P, _P]),
    ("gom_last_cuda_error", C.c_int, [_P]),
    ("gom_batch_workspace_bytes", _SZ, [_I32]),
    ("gom_batch_create", C.c_int, [_P, _I32, _P, _P, _SZ, _P, _P]),
    ("gom_batch_generation", C.c_int, [_P, _I32, _P, _P]),
    ("gom_batch_generation_each", C.c_int, [_P, _P, _P, _P]),
    ("gom_batch_stats", C.c_int, [_P, _I32, _P, _I32, _P]),
    ("gom_batch_layout", C.c_int, [_P, _I32, _P, _P, _P]),
    ("gom_batch_destroy", None, [_P]),
    ("gom_filter_workspace_bytes", _SZ, [_P, _I64]),
    ("gom_filter_attach", C.c_int, [_P, _P, _SZ, _I64]),
    ("gom_filter_set_mode", C.c_int, [_P, _I32]),
    ("gom_filter_configure", C.c_int, [_P, C.c_float, C.c_float, C.c_float]),
    ("gom_filter_train", C.c_int, [_P, _I32, C.c_float, C.c_float, C.c_float, _U64, _P]),
    ("gom_filter_stats", C.c_int, [_P, _P]),
    ("gom_filter_skipped", C.c_int, [_P, _P]),
    ("gom_filter_get_params", C.c_int, [_P, _P, _P, _P, _P]),
    ("gom_filter_set_params", C.c_int, [_P, _P, _P, _P]),
    ("gom_filter_epoch", C.c_int, [_P, C.c_float, C.c_float, _I32, _P]),
    ("gom_filter_log", C.c_int, [_P, _I64, _P, _P, _P]),
    ("gom_filter_logits", C.c_int, [_P, _I64, _P]),
    ("gom_ims_workspace_bytes", _SZ, [_P, _P, _I32, _I32]),
    ("gom_ims_create", C.c_int, [_P, _P, _I32, _I32, _I32, _U64, _P, _SZ, _P, _P]),
    ("gom_ims_run", C.c_int, [_P, _I32, _I64, _P]),
    ("gom_ims_population", C.c_int, [_P, _I32, _P]),
    ("gom_ims_num_populations", _I32, [_P]),
    ("gom_ims_destroy", None, [_P]),
    ("gom_batch_scratch_bytes", _SZ, [_P, _I32]),
    ("gom_batch_autotune", C.c_int, [_P, _I32, _P, _I32, _I32, _P, _SZ, _P, _P, _P]),
    ("gom_destroy", None, [_P]),
    ("gom_strerror", C.c_char_p, [C.c_int]),
]


def library_path() -> str:
    return _build.LIB


def load():
    """Loads libgom.so, building it first if its sources are newer."""
    global _lib
    if _lib is None:
        path = _build.build()
        if not os.path.exists(path):
            raise ImportError(f"libgom.so not found at {path}; run __graft_entry__.build()")
        L = C.CDLL(path)
        for name, res, args in SIGNATURES:
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(rc: int, what: str, ctx=None):
    if rc != GOM_OK:
        if rc == -5 and ctx is not None and getattr(ctx, "h", None):
            what = f"{what} (cudaError {load().gom_last_cuda_error(ctx.h)})"
        raise GomError(rc, what)


def _ptr(x):
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    return int(x)


def _stream(s):
    if s is None:
        return None
    if hasattr(s, "cuda_stream"):
        return s.cuda_stream
    return int(s)


class Graph:
    """Keeps the CSR arrays alive for a gom_graph_t."""

    def __init__(self, g):
        self.n = int(g.n)
        self.row_ptr = np.ascontiguousarray(g.row_ptr, dtype=np.int64)
        self.col = np.ascontiguousarray(g.col, dtype=np.int32)
        self.weight = np.ascontiguousarray(g.weight, dtype=np.int32)
        self.c = GraphT(self.n, int(self.row_ptr[-1]), self.row_ptr.ctypes.data,
                        self.col.ctypes.data if len(self.col) else None,
                        self.weight.ctypes.data if len(self.weight) else None)

    def ref(self):
        return C.byref(self.c)


def _graph(g):
    return g if isinstance(g, Graph) else Graph(g)


class FilterTrain(C.Structure):
    _fields_ = [("samples", C.c_int64), ("useful", C.c_int64), ("loss", C.c_double), ("threshold", C.c_float),
                ("skip_fraction", C.c_double), ("recall", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class FilterStats(C.Structure):
    _fields_ = [("mode", C.c_int32), ("enabled", C.c_int32), ("disabled_at", C.c_int32), ("threshold", C.c_float),
                ("log_count", C.c_int64), ("last", C.c_int64 * 5), ("total", C.c_int64 * 5)]

    def as_dict(self):
        names = ("run", "run_useful", "skipped", "audited", "audited_useful")
        return {"mode": self.mode, "enabled": self.enabled, "disabled_at": self.disabled_at,
                "threshold": self.threshold, "log_count": self.log_count,
                "last": dict(zip(names, list(self.last))), "total": dict(zip(names, list(self.total)))}


class ImsResult(C.Structure):
    _fields_ = [("steps", C.c_int64), ("best_fitness", C.c_int64), ("reached", C.c_int32),
                ("reached_population", C.c_int32), ("reached_step", C.c_int64), ("reached_generation", C.c_int64)]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


class BatchConfig(C.Structure):
    _fields_ = [("warps_per_block", C.c_int32), ("min_blocks", C.c_int32), ("max_blocks", C.c_int32),
                ("item_cost", C.c_int32)]


class Fos:
    """Owning wrapper of a gom_fos_t handle."""

    def __init__(self, handle):
        self.h = handle

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.gom_fos_destroy(self.h)
            self.h = None


class Ctx:
    """Wrapper of a gom_ctx_t handle; keeps its workspace alive.  A non-owning
    view (owner = the object that owns the handle) does not destroy it."""

    def __init__(self, handle, workspace, n: int, p: int, owner=None):
        self.h = handle
        self.workspace = workspace
        self.n, self.p = n, p
        self.owner = owner

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None and getattr(self, "owner", None) is None:
            _lib.gom_destroy(self.h)
        self.h = None


# ---------------------------------------------------------------------------
# entry points (same names as the C ABI)

def gom_strerror(code: int) -> str:
    return load().gom_strerror(code).decode()


def gom_build_fos(g, kind: int = GOM_FOS_NEIGHBOURHOOD, param: int = 0) -> Fos:
    G = _graph(g)
    h = C.c_void_p()
    _check(load().gom_build_fos(G.ref(), kind, param, C.byref(h)), "gom_build_fos")
    return Fos(h)


def gom_fos_create(num_vars: int, elem_ptr, elem_vars) -> Fos:
    ep = np.ascontiguousarray(elem_ptr, dtype=np.int64)
    ev = np.ascontiguousarray(elem_vars, dtype=np.int32)
    h = C.c_void_p()
    _check(load().gom_fos_create(num_vars, len(ep) - 1, ep.ctypes.data,
                                 ev.ctypes.data if len(ev) else None, C.byref(h)), "gom_fos_create")
    return Fos(h)


def gom_color_fos(g, fos: Fos) -> int:
    G = _graph(g)
    k = C.c_int32()
    _check(load().gom_color_fos(G.ref(), fos.h, C.byref(k)), "gom_color_fos")
    return int(k.value)


def gom_fos_sizes(fos: Fos):
    m, t, k = C.c_int64(), C.c_int64(), C.c_int32()
    _check(load().gom_fos_sizes(fos.h, C.byref(m), C.byref(t), C.byref(k)), "gom_fos_sizes")
    return int(m.value), int(t.value), int(k.value)


def gom_fos_export(fos: Fos) -> dict:
    m, total, k = gom_fos_sizes(fos)
    ep = np.zeros(m + 1, dtype=np.int64)
    ev = np.zeros(max(total, 1), dtype=np.int32)
    out = {"elem_ptr": ep, "elem_vars": ev[:total], "k": k}
    if k >= 0:
        co = np.zeros(max(m, 1), dtype=np.int32)
        cp = np.zeros(k + 1, dtype=np.int64)
        ce = np.zeros(max(m, 1), dtype=np.int32)
        _check(load().gom_fos_export(fos.h, ep.ctypes.data, ev.ctypes.data, co.ctypes.data, cp.ctypes.data,
                                     ce.ctypes.data), "gom_fos_export")
        out.update(color_of_elem=co[:m], color_ptr=cp, color_elems=ce[:m])
    else:
        _check(load().gom_fos_export(fos.h, ep.ctypes.data, ev.ctypes.data, None, None, None),
               "gom_fos_export")
    return out


def gom_fos_destroy(fos: Fos):
    if fos.h:
        load().gom_fos_destroy(fos.h)
        fos.h = None


def gom_workspace_bytes(g, fos: Fos, pop: int) -> int:
    G = _graph(g)
    return int(load().gom_workspace_bytes(G.ref(), fos.h, pop))


def gom_init_population(g, fos: Fos, pop: int, seed: int, workspace, ws_bytes: int = None,
                        stream=None) -> Ctx:
    """workspace: a CUDA tensor (kept alive by the handle) or a device address."""
    G = _graph(g)
    if ws_bytes is None:
        ws_bytes = workspace.numel() * workspace.element_size()
    h = C.c_void_p()
    _check(load().gom_init_population(G.ref(), fos.h, pop, seed & 0xFFFFFFFFFFFFFFFF, _ptr(workspace),
                                      ws_bytes, _stream(stream), C.byref(h)), "gom_init_population")
    return Ctx(h, workspace, G.n, pop)


def gom_generation(ctx: Ctx, num_generations: int, target_fitness: int = INT64_MAX,
                   want_stats: bool = True):
    """Returns (list of per-generation stats dicts, generations run); with
    want_stats=False only enqueues and returns (None, None)."""
    if not want_stats:
        _check(load().gom_generation(ctx.h, num_generations, target_fitness, None, None), "gom_generation", ctx)
        return None, None
    arr = (GenStats * max(num_generations, 1))()
    run = C.c_int32()
    _check(load().gom_generation(ctx.h, num_generations, target_fitness, arr, C.byref(run)), "gom_generation", ctx)
    return [arr[q].as_dict() for q in range(run.value)], int(run.value)


def gom_fitness(ctx: Ctx, d_fitness_out):
    _check(load().gom_fitness(ctx.h, _ptr(d_fitness_out)), "gom_fitness")


def gom_get_population(ctx: Ctx, d_pop=None, d_fit=None, want_elite: bool = True):
    fe = C.c_int64()
    _check(load().gom_get_population(ctx.h, _ptr(d_pop), _ptr(d_fit), C.byref(fe) if want_elite else None),
           "gom_get_population")
    return int(fe.value) if want_elite else None


def gom_get_elite(ctx: Ctx, d_elite=None, want_elite: bool = True):
    fe = C.c_int64()
    _check(load().gom_get_elite(ctx.h, _ptr(d_elite), C.byref(fe) if want_elite else None), "gom_get_elite")
    return int(fe.value) if want_elite else None


def gom_set_population(ctx: Ctx, d_pop, d_elite, elite_f: int, generation: int):
    _check(load().gom_set_population(ctx.h, _ptr(d_pop), _ptr(d_elite), elite_f, generation),
           "gom_set_population")


def gom_get_generation(ctx: Ctx) -> int:
    g = C.c_int64()
    _check(load().gom_get_generation(ctx.h, C.byref(g)), "gom_get_generation")
    return int(g.value)


def gom_set_timing(ctx: Ctx, enable: bool):
    _check(load().gom_set_timing(ctx.h, 1 if enable else 0), "gom_set_timing")


def gom_read_timing(ctx: Ctx):
    ms, n = C.c_double(), C.c_int64()
    _check(load().gom_read_timing(ctx.h, C.byref(ms), C.byref(n)), "gom_read_timing")
    return float(ms.value), int(n.value)


def gom_launches_per_generation(ctx: Ctx) -> int:
    n = C.c_int64()
    _check(load().gom_launches_per_generation(ctx.h, C.byref(n)), "gom_launches_per_generation")
    return int(n.value)


def gom_set_option(ctx: Ctx, option: int, value: int):
    _check(load().gom_set_option(ctx.h, option, value), "gom_set_option")


def gom_get_option(ctx: Ctx, option: int) -> int:
    v = C.c_int64()
    _check(load().gom_get_option(ctx.h, option, C.byref(v)), "gom_get_option")
    return int(v.value)


def gom_read_phase_trace(ctx: Ctx):
    """Phase stamps (ns) of the last persistent-path generation (see include/gom.h)."""
    cnt = C.c_int32()
    load().gom_read_phase_trace(ctx.h, None, 0, C.byref(cnt))
    buf = (C.c_int64 * cnt.value)()
    _check(load().gom_read_phase_trace(ctx.h, buf, cnt.value, C.byref(cnt)), "gom_read_phase_trace", ctx)
    return [int(x) for x in buf]


def gom_selftest_barrier(d_scratch, blocks: int, extra: int, limit_ns: int, stream=None) -> bool:
    """True if the barrier's bounded wait gave up (expected when extra > 0)."""
    out = C.c_int32()
    _check(load().gom_selftest_barrier(_ptr(d_scratch), blocks, extra, limit_ns, _stream(stream), C.byref(out)),
           "gom_selftest_barrier")
    return bool(out.value)


def gom_fitness_noalloc(d_row_ptr, d_col, d_weight, num_vertices: int, d_pop, pop: int, d_fitness_out,
                        stream=None):
    """Full fitness of a device uint8 population without any device
    allocation (the library's fixed scratch array; see include/gom.h)."""
    _check(load().gom_fitness_noalloc(_ptr(d_row_ptr), _ptr(d_col), _ptr(d_weight), num_vertices, _ptr(d_pop),
                                      pop, _ptr(d_fitness_out), _stream(stream)), "gom_fitness_noalloc")


def gom_last_cuda_error(ctx: Ctx) -> int:
    return int(load().gom_last_cuda_error(ctx.h))


def gom_destroy(ctx: Ctx):
    if ctx.h:
        load().gom_destroy(ctx.h)
        ctx.h = None


class Batch:
    """Owning wrapper of a gom_batch_t handle; keeps its contexts and workspace alive."""

    def __init__(self, handle, ctxs, workspace):
        self.h = handle
        self.ctxs = list(ctxs)
        self.workspace = workspace

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.gom_batch_destroy(self.h)
            self.h = None


def _ctx_array(ctxs):
    arr = (C.c_void_p * len(ctxs))()
    for b, c in enumerate(ctxs):
        arr[b] = c.h.value if isinstance(c.h, C.c_void_p) else c.h
    return arr


def gom_batch_workspace_bytes(num: int) -> int:
    return int(load().gom_batch_workspace_bytes(num))


def gom_batch_create(ctxs, config=None, workspace=None, stream=None) -> Batch:
    """ctxs: Ctx handles made on `stream`; config: (warps_per_block, min_blocks[,
    max_blocks[, item_cost]]) or None; workspace: a CUDA tensor of at least gom_batch_workspace_bytes(len(ctxs))
    bytes, 256-byte aligned."""
    arr = _ctx_array(ctxs)
    cfg = BatchConfig(*config) if config is not None else None
    nbytes = workspace.numel() * workspace.element_size()
    h = C.c_void_p()
    _check(load().gom_batch_create(arr, len(ctxs), C.byref(cfg) if cfg is not None else None, _ptr(workspace),
                                   nbytes, _stream(stream), C.byref(h)), "gom_batch_create")
    return Batch(h, ctxs, workspace)


def gom_batch_generation(batch: Batch, num_generations: int, targets=None, want_counts: bool = True):
    """Returns the generations each instance ran (numpy int32), or None when
    want_counts is False (asynchronous)."""
    B = len(batch.ctxs)
    t = None
    if targets is not None:
        t = np.ascontiguousarray(targets, dtype=np.int64)
        assert len(t) == B
    runs = np.zeros(B, dtype=np.int32) if want_counts else None
    _check(load().gom_batch_generation(batch.h, num_generations, t.ctypes.data if t is not None else None,
                                       runs.ctypes.data if runs is not None else None), "gom_batch_generation")
    return runs


def gom_batch_generation_each(batch: Batch, num_generations, targets=None, want_counts: bool = True):
    """Generation counts per instance (sequence of len(batch.ctxs) ints)."""
    B = len(batch.ctxs)
    gens = np.ascontiguousarray(num_generations, dtype=np.int32)
    assert len(gens) == B
    t = None
    if targets is not None:
        t = np.ascontiguousarray(targets, dtype=np.int64)
        assert len(t) == B
    runs = np.zeros(B, dtype=np.int32) if want_counts else None
    _check(load().gom_batch_generation_each(batch.h, gens.ctypes.data, t.ctypes.data if t is not None else None,
                                            runs.ctypes.data if runs is not None else None),
           "gom_batch_generation_each")
    return runs


def gom_batch_stats(batch: Batch, b: int, capacity: int):
    arr = (GenStats * max(capacity, 1))()
    cnt = C.c_int32()
    _check(load().gom_batch_stats(batch.h, b, arr, capacity, C.byref(cnt)), "gom_batch_stats")
    return [arr[q].as_dict() for q in range(cnt.value)]


def gom_batch_layout(batch: Batch, b: int):
    b0, nb, grid = C.c_int32(), C.c_int32(), C.c_int32()
    _check(load().gom_batch_layout(batch.h, b, C.byref(b0), C.byref(nb), C.byref(grid)), "gom_batch_layout")
    return int(b0.value), int(nb.value), int(grid.value)


def gom_batch_destroy(batch: Batch):
    if batch.h:
        load().gom_batch_destroy(batch.h)
        batch.h = None


def gom_filter_workspace_bytes(ctx: Ctx, log_capacity: int) -> int:
    return int(load().gom_filter_workspace_bytes(ctx.h, log_capacity))


def gom_filter_attach(ctx: Ctx, workspace, log_capacity: int):
    """workspace: a CUDA tensor (kept alive by the handle), 256-byte aligned."""
    nbytes = workspace.numel() * workspace.element_size()
    _check(load().gom_filter_attach(ctx.h, _ptr(workspace), nbytes, log_capacity), "gom_filter_attach", ctx)
    ctx.filter_workspace = workspace


def gom_filter_set_mode(ctx: Ctx, mode: int):
    _check(load().gom_filter_set_mode(ctx.h, mode), "gom_filter_set_mode", ctx)


def gom_filter_configure(ctx: Ctx, threshold: float, target_recall: float = 0.9, min_recall: float = 0.5):
    _check(load().gom_filter_configure(ctx.h, threshold, target_recall, min_recall), "gom_filter_configure", ctx)


def gom_filter_train(ctx: Ctx, epochs: int = 200, learning_rate: float = 0.01, pos_weight: float = 1.0,
                     target_recall: float = 0.95, seed: int = 1) -> dict:
    out = FilterTrain()
    _check(load().gom_filter_train(ctx.h, epochs, learning_rate, pos_weight, target_recall, seed, C.byref(out)),
           "gom_filter_train", ctx)
    return out.as_dict()


def gom_filter_stats(ctx: Ctx) -> dict:
    out = FilterStats()
    _check(load().gom_filter_stats(ctx.h, C.byref(out)), "gom_filter_stats", ctx)
    return out.as_dict()


GOM_FILTER_PARAMS = 1153


def gom_filter_get_params(ctx: Ctx) -> dict:
    """theta, Adam moments and the last gradient (numpy float32 [1153] each)."""
    out = {k: np.zeros(GOM_FILTER_PARAMS, dtype=np.float32) for k in ("theta", "adam_m", "adam_v", "grad")}
    _check(load().gom_filter_get_params(ctx.h, *(out[k].ctypes.data for k in ("theta", "adam_m", "adam_v", "grad"))),
           "gom_filter_get_params", ctx)
    return out


def gom_filter_set_params(ctx: Ctx, theta, adam_m=None, adam_v=None):
    arrs = [np.ascontiguousarray(a, dtype=np.float32) if a is not None else None for a in (theta, adam_m, adam_v)]
    _check(load().gom_filter_set_params(ctx.h, *(a.ctypes.data if a is not None else None for a in arrs)),
           "gom_filter_set_params", ctx)


def gom_filter_epoch(ctx: Ctx, learning_rate: float, pos_weight: float, step: int) -> float:
    loss = C.c_double()
    _check(load().gom_filter_epoch(ctx.h, learning_rate, pos_weight, step, C.byref(loss)), "gom_filter_epoch", ctx)
    return loss.value


def gom_filter_log(ctx: Ctx, max_samples: int = 1 << 30):
    """The training log: (features as bf16 bits uint16 [n][16], labels uint8 [n])."""
    n = C.c_int64()
    _check(load().gom_filter_log(ctx.h, 0, None, None, C.byref(n)), "gom_filter_log", ctx)
    c = min(n.value, max_samples)
    x = np.zeros((c, 16), dtype=np.uint16)
    y = np.zeros(c, dtype=np.uint8)
    _check(load().gom_filter_log(ctx.h, c, x.ctypes.data, y.ctypes.data, C.byref(n)), "gom_filter_log", ctx)
    return x, y


def gom_filter_logits(ctx: Ctx, n: int):
    out = np.zeros(n, dtype=np.float32)
    _check(load().gom_filter_logits(ctx.h, n, out.ctypes.data), "gom_filter_logits", ctx)
    return out


def gom_filter_skipped(ctx: Ctx, m: int):
    mask = np.zeros(m, dtype=np.uint8)
    _check(load().gom_filter_skipped(ctx.h, mask.ctypes.data), "gom_filter_skipped", ctx)
    return mask


class Ims:
    """Owning wrapper of a gom_ims_t handle; keeps its workspace alive."""

    def __init__(self, handle, workspace, graph, fos):
        self.h = handle
        self.workspace = workspace
        self.graph, self.fos = graph, fos

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.gom_ims_destroy(self.h)
            self.h = None


def gom_ims_workspace_bytes(g, fos: Fos, base_pop: int, max_pop: int) -> int:
    return int(load().gom_ims_workspace_bytes(_graph(g).ref(), fos.h, base_pop, max_pop))


def gom_ims_create(g, fos: Fos, base_pop: int, c: int, max_pop: int, seed: int, workspace, stream=None) -> Ims:
    """workspace: a CUDA tensor of at least gom_ims_workspace_bytes(...) bytes, 256-byte aligned."""
    G = _graph(g)
    h = C.c_void_p()
    nbytes = workspace.numel() * workspace.element_size()
    _check(load().gom_ims_create(G.ref(), fos.h, base_pop, c, max_pop, seed & 0xFFFFFFFFFFFFFFFF, _ptr(workspace),
                                 nbytes, _stream(stream), C.byref(h)), "gom_ims_create")
    return Ims(h, workspace, G, fos)


def gom_ims_run(ims: Ims, steps: int, target: int = INT64_MAX) -> dict:
    res = ImsResult()
    _check(load().gom_ims_run(ims.h, steps, target, C.byref(res)), "gom_ims_run")
    return res.as_dict()


def gom_ims_population(ims: Ims, i: int) -> Ctx:
    """Population i as a non-owning Ctx view (the scheme owns it)."""
    h = C.c_void_p()
    _check(load().gom_ims_population(ims.h, i, C.byref(h)), "gom_ims_population")
    return Ctx(h, None, ims.graph.n, 0, owner=ims)


def gom_ims_num_populations(ims: Ims) -> int:
    return int(load().gom_ims_num_populations(ims.h))


def gom_batch_scratch_bytes(ctxs) -> int:
    return int(load().gom_batch_scratch_bytes(_ctx_array(ctxs), len(ctxs)))


def gom_batch_autotune(ctxs, configs, generations: int, scratch, stream=None):
    """Returns (index of the fastest configuration, ms per generation of each)."""
    cfgs = (BatchConfig * len(configs))(*[BatchConfig(*c) for c in configs])
    ms = (C.c_double * len(configs))()
    best = C.c_int32()
    nbytes = scratch.numel() * scratch.element_size()
    _check(load().gom_batch_autotune(_ctx_array(ctxs), len(ctxs), cfgs, len(configs), generations, _ptr(scratch),
                                     nbytes, _stream(stream), C.byref(best), ms), "gom_batch_autotune")
    return int(best.value), [float(x) for x in ms]


# ---------------------------------------------------------------------------
# convenience: a population with a torch-allocated workspace

class Population:
    """One GOM population on the current CUDA device.  Allocates the device
    workspace with torch and drives the C ABI above."""

    def __init__(self, graph, pop: int, seed: int, kind: int = GOM_FOS_NEIGHBOURHOOD, fos: Fos = None,
                 stream=None, device=None, persistent: bool = None, dynamic: bool = None,
                 bitsliced: bool = None, forced_improvement: bool = None, fi_nis: int = None):
        import torch
        self.torch = torch
        self.graph = _graph(graph)
        if fos is None:
            fos = gom_build_fos(self.graph, kind)
            self.k = gom_color_fos(self.graph, fos)
        else:
            self.k = gom_fos_sizes(fos)[2]
            if self.k < 0:
                self.k = gom_color_fos(self.graph, fos)
        self.fos = fos
        self.n, self.p = self.graph.n, pop
        self.m = gom_fos_sizes(fos)[0]
        self.device = torch.device(device or "cuda")
        nbytes = gom_workspace_bytes(self.graph, fos, pop)
        if nbytes == 0:
            raise GomError(-1, "gom_workspace_bytes")
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        off = (-self.workspace.data_ptr()) % 256
        self.stream = stream
        self.ctx = gom_init_population(self.graph, fos, pop, seed, self.workspace.data_ptr() + off, nbytes,
                                       stream)
        self.ctx.workspace = self.workspace
        if persistent is not None:
            gom_set_option(self.ctx, GOM_OPT_PERSISTENT, 1 if persistent else 0)
        if dynamic is not None:
            gom_set_option(self.ctx, GOM_OPT_DYNAMIC, 1 if dynamic else 0)
        if bitsliced is not None:
            gom_set_option(self.ctx, GOM_OPT_BITSLICED, 1 if bitsliced else 0)
        if fi_nis is not None:
            gom_set_option(self.ctx, GOM_OPT_FI_NIS, fi_nis)
        if forced_improvement is not None:
            gom_set_option(self.ctx, GOM_OPT_FORCED_IMPROVEMENT, 1 if forced_improvement else 0)

    def generation(self, num: int = 1, target: int = INT64_MAX, want_stats: bool = True):
        return gom_generation(self.ctx, num, target, want_stats)

    def population(self):
        t = self.torch
        pop = t.empty((self.p, self.n), dtype=t.uint8, device=self.device)
        fit = t.empty(self.p, dtype=t.int64, device=self.device)
        fe = gom_get_population(self.ctx, pop, fit, True)
        return pop, fit, fe

    def elite(self):
        t = self.torch
        xe = t.empty(self.n, dtype=t.uint8, device=self.device)
        fe = gom_get_elite(self.ctx, xe, True)
        return xe, fe

    def fitness(self):
        t = self.torch
        out = t.empty(self.p, dtype=t.int64, device=self.device)
        gom_fitness(self.ctx, out)
        return out

    def set_population(self, pop, elite, elite_f: int, generation: int):
        gom_set_population(self.ctx, pop, elite, elite_f, generation)

    def generation_counter(self) -> int:
        return gom_get_generation(self.ctx)
