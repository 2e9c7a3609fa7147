"""ctypes wrapper of the CPU oracle (gom_oracle.c) -- TEST INFRASTRUCTURE ONLY.

Only the test suite, the smoke check and the benchmark's CPU-baseline /
reference arm may import this module.  It imports nothing from the CUDA
package: graphs are passed as any object with ``n``, ``row_ptr`` (int64),
``col`` (int32) and ``weight`` (int32) attributes.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gom_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")

NEIGHBOURHOOD = 0
SINGLETON = 1


def build(force: bool = False) -> str:
    """Compile the oracle with gcc into oracle/_build/liboracle.so."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        os.makedirs(os.path.dirname(_LIB), exist_ok=True)
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-Wall", "-shared", "-fPIC", "-o", tmp, _SRC]
        try:  # with OpenMP where the compiler has it (orc_generation_par), else serial
            subprocess.check_call(cmd[:1] + ["-fopenmp"] + cmd[1:], stderr=subprocess.DEVNULL)
        except subprocess.CalledProcessError:
            subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        P = C.c_void_p
        i32, i64, u32, u64 = C.c_int32, C.c_int64, C.c_uint32, C.c_uint64
        L.orc_philox4x32_10.argtypes = [P, P, P]
        L.orc_check_graph.argtypes = [i32, P, P, P]
        L.orc_check_graph.restype = C.c_int
        L.orc_cut_value.argtypes = [i32, P, P, P, P]
        L.orc_cut_value.restype = i64
        L.orc_brute_force_maxcut.argtypes = [i32, P, P, P, P]
        L.orc_brute_force_maxcut.restype = i64
        L.orc_fos_total.argtypes = [i32, P, i32]
        L.orc_fos_total.restype = i64
        L.orc_build_fos.argtypes = [i32, P, P, i32, P, P]
        L.orc_build_bflt.argtypes = [i32, P, P, P, i32, P, P]
        L.orc_build_bflt.restype = i64
        L.orc_lmig_edges.argtypes = [i32, P, P, i64, P, P, P, i64]
        L.orc_lmig_edges.restype = i64
        L.orc_color.argtypes = [i32, P, P, i64, P, P, P]
        L.orc_color.restype = i32
        L.orc_partial_delta.argtypes = [i32, P, P, P, P, P, i32, P]
        L.orc_partial_delta.restype = i64
        L.orc_group_order.argtypes = [u64, i32, u32, P]
        L.orc_new.argtypes = [i32, P, P, P, i64, P, P, P, i32, i32, u64]
        L.orc_new.restype = P
        L.orc_new_ex.argtypes = [i32, P, P, P, i64, P, P, P, i32, i32, u64, i32]
        L.orc_new_ex.restype = P
        L.orc_init_individual.argtypes = [u64, i32, i32, P]
        L.orc_free.argtypes = [P]
        L.orc_load.argtypes = [P, P, P, P, i64, u32]
        L.orc_get.argtypes = [P, P, P, P, P, P]
        L.orc_generation_ex.argtypes = [P, i64, u64, P, i32, P]
        L.orc_generation_ex.restype = i32
        L.orc_generation_skip.argtypes = [P, i64, P, P]
        L.orc_generation_skip.restype = i32
        L.orc_generation_par.argtypes = [P, i64, i32, P]
        L.orc_generation_par.restype = i32
        L.orc_generation_par_ex.argtypes = [P, i64, i32, P, i32, P]
        L.orc_generation_par_ex.restype = i32
        L.orc_set_fi.argtypes = [P, i32, i32]
        L.orc_keep_element_counts.argtypes = [P, i32]
        L.orc_element_counts.argtypes = [P, P, P, P]
        L.orc_max_threads.argtypes = []
        L.orc_max_threads.restype = i32
        _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _csr(g):
    rp = np.ascontiguousarray(g.row_ptr, dtype=np.int64)
    col = np.ascontiguousarray(g.col, dtype=np.int32)
    w = np.ascontiguousarray(g.weight, dtype=np.int32)
    if len(col) == 0:  # keep valid pointers for empty graphs
        col = np.zeros(1, dtype=np.int32)
        w = np.zeros(1, dtype=np.int32)
    return rp, col, w


class Stats(C.Structure):
    _fields_ = [(name, C.c_int64) for name in
                ("generation", "best", "elite", "trials", "donorless", "accepted", "improving",
                 "reached", "fi_individuals", "fi_trials", "fi_accepted", "fi_improving", "fi_replaced")]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


def philox(ctr, key):
    c = np.asarray(ctr, dtype=np.uint32)
    k = np.asarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def check_graph(g) -> bool:
    rp, col, w = _csr(g)
    return lib().orc_check_graph(g.n, _p(rp), _p(col), _p(w)) == 0


def cut_value(g, x) -> int:
    rp, col, w = _csr(g)
    x = np.ascontiguousarray(x, dtype=np.uint8)
    return int(lib().orc_cut_value(g.n, _p(rp), _p(col), _p(w), _p(x)))


def brute_force_maxcut(g):
    rp, col, w = _csr(g)
    x = np.zeros(max(g.n, 1), dtype=np.uint8)
    best = int(lib().orc_brute_force_maxcut(g.n, _p(rp), _p(col), _p(w), _p(x)))
    return best, x[: g.n]


def build_fos(g, kind: int = NEIGHBOURHOOD):
    rp, col, _ = _csr(g)
    total = int(lib().orc_fos_total(g.n, _p(rp), kind))
    eptr = np.zeros(g.n + 1, dtype=np.int64)
    evars = np.zeros(max(total, 1), dtype=np.int32)
    lib().orc_build_fos(g.n, _p(rp), _p(col), kind, _p(eptr), _p(evars))
    return eptr, evars[:total]


def build_bflt(g, bound: int):
    """Bounded fixed linkage tree: UPGMA on the edge weights (reading R11)."""
    rp, col, w = _csr(g)
    n = g.n
    eptr = np.zeros(2 * n + 2, dtype=np.int64)
    evars = np.zeros(max(n * max(bound, 1), 1), dtype=np.int32)
    m = int(lib().orc_build_bflt(n, _p(rp), _p(col), _p(w), bound, _p(eptr), _p(evars)))
    return eptr[: m + 1].copy(), evars[: eptr[m]].copy()


def _fos_arrays(eptr, evars):
    eptr = np.ascontiguousarray(eptr, dtype=np.int64)
    evars = np.ascontiguousarray(evars, dtype=np.int32)
    if len(evars) == 0:
        evars = np.zeros(1, dtype=np.int32)
    return eptr, evars


def lmig_edges(g, eptr, evars):
    rp, col, _ = _csr(g)
    eptr, evars = _fos_arrays(eptr, evars)
    m = len(eptr) - 1
    cnt = int(lib().orc_lmig_edges(g.n, _p(rp), _p(col), m, _p(eptr), _p(evars), None, 0))
    pairs = np.zeros(2 * max(cnt, 1), dtype=np.int32)
    lib().orc_lmig_edges(g.n, _p(rp), _p(col), m, _p(eptr), _p(evars), _p(pairs), cnt)
    return pairs[: 2 * cnt].reshape(-1, 2)


def color(g, eptr, evars):
    rp, col, _ = _csr(g)
    eptr, evars = _fos_arrays(eptr, evars)
    m = len(eptr) - 1
    colors = np.zeros(max(m, 1), dtype=np.int32)
    k = int(lib().orc_color(g.n, _p(rp), _p(col), m, _p(eptr), _p(evars), _p(colors)))
    return k, colors[:m]


def partial_delta(g, x, F, y_on_f) -> int:
    rp, col, w = _csr(g)
    x = np.ascontiguousarray(x, dtype=np.uint8)
    F = np.ascontiguousarray(F, dtype=np.int32)
    y = np.ascontiguousarray(y_on_f, dtype=np.uint8)
    return int(lib().orc_partial_delta(g.n, _p(rp), _p(col), _p(w), _p(x), _p(F), len(F), _p(y)))


def group_order(seed: int, k: int, g: int):
    out = np.zeros(max(k, 1), dtype=np.int32)
    lib().orc_group_order(seed, k, g, _p(out))
    return out[:k]


def max_threads() -> int:
    """Threads available to Run.generation(threads=...): 1 without OpenMP."""
    return int(lib().orc_max_threads())


def init_individual(seed: int, i: int, n: int):
    """Initial bits of individual i (InitializePopulation, Alg. 3)."""
    x = np.zeros(max(n, 1), dtype=np.uint8)
    lib().orc_init_individual(seed, i, n, _p(x))
    return x[:n]


class Run:
    """One parallel-GOMEA run of the oracle (population, fitness, elitist).
    With init=False the population starts empty, to be set with load()."""

    def __init__(self, g, eptr, evars, colors, k: int, p: int, seed: int, init: bool = True):
        rp, col, w = _csr(g)
        eptr, evars = _fos_arrays(eptr, evars)
        colors = np.ascontiguousarray(colors, dtype=np.int32)
        self.n, self.p, self.m, self.k = g.n, p, len(eptr) - 1, k
        self._h = lib().orc_new_ex(g.n, _p(rp), _p(col), _p(w), self.m, _p(eptr), _p(evars),
                                   _p(colors), k, p, seed, 1 if init else 0)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_free(h)
            self._h = None

    def generation(self, target: int = 2 ** 63 - 1, shuffle: int = 0, only=None, threads: int = 1) -> dict:
        """One generation; threads > 1 splits each group's individuals over
        that many threads (same result)."""
        st = Stats()
        if threads > 1 and only is not None:
            assert not shuffle
            o = np.ascontiguousarray(only, dtype=np.int32)
            lib().orc_generation_par_ex(self._h, target, threads, _p(o), len(o), C.byref(st))
        elif threads > 1:
            assert not shuffle
            lib().orc_generation_par(self._h, target, threads, C.byref(st))
        elif only is None:
            lib().orc_generation_ex(self._h, target, shuffle, None, 0, C.byref(st))
        else:
            o = np.ascontiguousarray(only, dtype=np.int32)
            lib().orc_generation_ex(self._h, target, shuffle, _p(o), len(o), C.byref(st))
        return st.as_dict()

    def keep_element_counts(self, on: bool = True):
        """Per-element counters of each generation (single-threaded generations only)."""
        lib().orc_keep_element_counts(self._h, 1 if on else 0)

    def element_counts(self):
        """Accepted, donor-less and improving trials per element of the last generation."""
        out = [np.zeros(max(self.m, 1), dtype=np.int32) for _ in range(3)]
        lib().orc_element_counts(self._h, *(_p(a) for a in out))
        return tuple(a[: self.m] for a in out)

    def set_fi(self, on: bool, nis: int = 0):
        """Forced Improvement after each generation's mixing (reading R12)."""
        lib().orc_set_fi(self._h, 1 if on else 0, nis)

    def generation_skip(self, skip_elem, target: int = 2 ** 63 - 1) -> dict:
        """One generation without the trials of the elements marked in skip_elem[j]."""
        sk = np.ascontiguousarray(skip_elem, dtype=np.uint8)
        assert len(sk) == self.m
        st = Stats()
        lib().orc_generation_skip(self._h, target, _p(sk), C.byref(st))
        return st.as_dict()

    def run(self, generations: int, target: int = 2 ** 63 - 1):
        """Up to `generations` generations, stopping after the first that reaches target."""
        out = []
        for _ in range(generations):
            st = self.generation(target)
            out.append(st)
            if st["reached"]:
                break
        return out

    def get(self):
        pop = np.zeros((self.p, self.n), dtype=np.uint8)
        f = np.zeros(self.p, dtype=np.int64)
        xe = np.zeros(max(self.n, 1), dtype=np.uint8)
        fe = C.c_int64()
        g = C.c_uint32()
        lib().orc_get(self._h, _p(pop), _p(f), _p(xe), C.byref(fe), C.byref(g))
        return {"pop": pop, "f": f, "xe": xe[: self.n], "fe": int(fe.value), "g": int(g.value)}

    def load(self, pop, f, xe, fe: int, g: int):
        pop = np.ascontiguousarray(pop, dtype=np.uint8)
        f = np.ascontiguousarray(f, dtype=np.int64)
        xe = np.ascontiguousarray(xe, dtype=np.uint8)
        lib().orc_load(self._h, _p(pop), _p(f), _p(xe), fe, g)
