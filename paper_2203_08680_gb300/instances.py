"""Seeded synthetic Max-Cut instances (inputs only).

This module builds the weighted graphs that both the CUDA library and the CPU
oracle take as input.  It holds none of the method's arithmetic: no objective,
no FOS, no colouring, no Philox.  Its random numbers come from SplitMix64
(Steele, Lea & Flood, OOPSLA 2014) applied as a counter-based hash, so every
instance is a pure function of its parameters on any machine.

The shapes follow the paper's benchmark sets (Sec. 6.2), which are not
available here: Set B's 4-regular torus becomes the 2D L x L torus, and the
sparse Set C graphs become random d-regular graphs.  Weights are int32,
uniform in [wmin, wmax] per undirected edge, or all 1 for the unit-weight
variant.

A graph is returned in symmetric CSR form: ``row_ptr`` int64[n+1], ``col``
int32[2|E|] (each row sorted ascending) and ``weight`` int32[2|E|], with the
two directions of every edge carrying the same weight.
"""
from __future__ import annotations

import dataclasses

import numpy as np

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)


@dataclasses.dataclass
class Graph:
    """Symmetric CSR of an undirected weighted graph (the Max-Cut instance)."""

    n: int
    row_ptr: np.ndarray  # int64 [n+1]
    col: np.ndarray  # int32 [2|E|]
    weight: np.ndarray  # int32 [2|E|]
    name: str = ""

    @property
    def num_edges(self) -> int:
        return int(self.row_ptr[-1]) // 2

    def total_weight(self) -> int:
        return int(self.weight.astype(np.int64).sum()) // 2

    def degrees(self) -> np.ndarray:
        return np.diff(self.row_ptr)

    def edges(self):
        """(u, v, w) arrays of the undirected edges with u < v."""
        u = np.repeat(np.arange(self.n, dtype=np.int64), self.degrees())
        v = self.col.astype(np.int64)
        keep = u < v
        return u[keep], v[keep], self.weight[keep]


def _mix64(x: np.ndarray) -> np.ndarray:
    """SplitMix64 output function on a uint64 array (wrapping arithmetic)."""
    x = np.asarray(x, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = x + np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def _hash(seed: int, stream: int, idx: np.ndarray) -> np.ndarray:
    base = _mix64(np.array([(seed * 0x100000001B3 + stream) & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64))[0]
    with np.errstate(over="ignore"):
        return _mix64(np.asarray(idx, dtype=np.uint64) ^ base)


def edge_weights(u: np.ndarray, v: np.ndarray, seed: int, wmin: int = 1, wmax: int = 100,
                 unit: bool = False) -> np.ndarray:
    """Weight of each undirected edge, uniform in [wmin, wmax] from (seed, min, max)."""
    if unit:
        return np.ones(len(u), dtype=np.int32)
    a = np.minimum(u, v).astype(np.uint64)
    b = np.maximum(u, v).astype(np.uint64)
    h = _hash(seed, 0x57, (a << np.uint64(32)) | b)
    span = np.uint64(wmax - wmin + 1)
    with np.errstate(over="ignore"):
        r = ((h >> np.uint64(32)) * span) >> np.uint64(32)
    return (r.astype(np.int64) + wmin).astype(np.int32)


def from_edges(n: int, u, v, w, name: str = "") -> Graph:
    """Symmetric CSR from undirected edges (u_e, v_e, w_e); no validation here."""
    u = np.asarray(u, dtype=np.int64)
    v = np.asarray(v, dtype=np.int64)
    w = np.asarray(w, dtype=np.int32)
    src = np.concatenate([u, v])
    dst = np.concatenate([v, u])
    ww = np.concatenate([w, w])
    order = np.lexsort((dst, src))
    src, dst, ww = src[order], dst[order], ww[order]
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(src, minlength=n), out=row_ptr[1:])
    return Graph(n, row_ptr, dst.astype(np.int32), ww.astype(np.int32), name)


def torus2d(L: int, seed: int = 1, wmin: int = 1, wmax: int = 100, unit: bool = False) -> Graph:
    """L x L torus (4-regular, 2L^2 edges); vertex v = y*L + x."""
    if L < 3:
        raise ValueError("torus side must be >= 3")
    v = np.arange(L * L, dtype=np.int64)
    x, y = v % L, v // L
    right = y * L + (x + 1) % L
    down = ((y + 1) % L) * L + x
    u = np.concatenate([v, v])
    t = np.concatenate([right, down])
    w = edge_weights(u, t, seed, wmin, wmax, unit)
    return from_edges(L * L, u, t, w, f"torus2d_{L}x{L}")


def torus3d(L: int, seed: int = 1, wmin: int = 1, wmax: int = 100, unit: bool = False) -> Graph:
    """L x L x L torus (6-regular, 3L^3 edges); vertex v = (z*L + y)*L + x."""
    if L < 3:
        raise ValueError("torus side must be >= 3")
    v = np.arange(L ** 3, dtype=np.int64)
    x, y, z = v % L, (v // L) % L, v // (L * L)
    px = (z * L + y) * L + (x + 1) % L
    py = (z * L + (y + 1) % L) * L + x
    pz = (((z + 1) % L) * L + y) * L + x
    u = np.concatenate([v, v, v])
    t = np.concatenate([px, py, pz])
    w = edge_weights(u, t, seed, wmin, wmax, unit)
    return from_edges(L ** 3, u, t, w, f"torus3d_{L}^3")


def random_regular(n: int, d: int, seed: int = 1, wmin: int = 1, wmax: int = 100,
                   unit: bool = False, max_rounds: int = 100000) -> Graph:
    """Simple random d-regular graph: configuration model, then random
    double-edge swaps applied to self-loops and repeated edges until none remain."""
    if n * d % 2 or d >= n or d < 1:
        raise ValueError("need n*d even and 1 <= d < n")
    ne = n * d // 2
    stubs = np.repeat(np.arange(n, dtype=np.int64), d)
    perm = np.argsort(_hash(seed, 0x11, np.arange(n * d)), kind="stable")
    s = stubs[perm]
    u, v = s[0::2].copy(), s[1::2].copy()
    for rnd in range(max_rounds):
        a, b = np.minimum(u, v), np.maximum(u, v)
        key = a * n + b
        order = np.argsort(key, kind="stable")
        dup = np.zeros(ne, dtype=bool)
        ks = key[order]
        dup[order[1:]] = ks[1:] == ks[:-1]
        bad = np.nonzero((a == b) | dup)[0]
        if len(bad) == 0:
            break
        h = _hash(seed, 0x1000 + rnd, bad)
        partner = (h % np.uint64(ne)).astype(np.int64)
        flip = ((h >> np.uint64(40)) & np.uint64(1)).astype(bool)
        # use each edge in at most one swap this round
        used = np.zeros(ne, dtype=bool)
        for e, f, fl in zip(bad.tolist(), partner.tolist(), flip.tolist()):
            if e == f or used[e] or used[f]:
                continue
            used[e] = used[f] = True
            ue, ve, uf, vf = u[e], v[e], u[f], v[f]
            if fl:
                u[e], v[e], u[f], v[f] = ue, uf, ve, vf
            else:
                u[e], v[e], u[f], v[f] = ue, vf, ve, uf
    else:
        raise RuntimeError("random_regular: did not converge")
    w = edge_weights(u, v, seed, wmin, wmax, unit)
    return from_edges(n, u, v, w, f"rreg_n{n}_d{d}")


def empty_graph(n: int) -> Graph:
    """n isolated vertices (no edges)."""
    return Graph(n, np.zeros(n + 1, dtype=np.int64), np.zeros(0, dtype=np.int32),
                 np.zeros(0, dtype=np.int32), f"empty_{n}")


def batch_mix(count: int = 256, seed: int = 1, nmin: int = 1000, nmax: int = 65536, dmin: int = 3,
              dmax: int = 8, pops=(32, 64, 128, 256)):
    """Shapes of a batch of independent random d-regular Max-Cut instances:
    n log-uniform in [nmin, nmax] (rounded up to even), d uniform in
    {dmin..dmax}, population uniform over `pops`, graph and Philox seeds
    1..count.  Returns a list of (n, d, p, seed); graphs are built with
    random_regular(n, d, seed)."""
    idx = np.arange(count, dtype=np.uint64)
    u = (_hash(seed, 0x2001, idx) >> np.uint64(11)).astype(np.float64) / float(1 << 53)
    n = np.ceil(np.exp(np.log(nmin) + u * (np.log(nmax) - np.log(nmin)))).astype(np.int64)
    n = np.minimum(n + (n & 1), nmax)
    d = dmin + (_hash(seed, 0x2002, idx) % np.uint64(dmax - dmin + 1)).astype(np.int64)
    p = np.asarray(pops, dtype=np.int64)[(_hash(seed, 0x2003, idx) % np.uint64(len(pops))).astype(np.int64)]
    return [(int(n[b]), int(d[b]), int(p[b]), b + 1) for b in range(count)]


# The workload shapes of the benchmark configurations, by name.
def workload(name: str) -> Graph:
    """Named synthetic workloads: 'torus10' (10x10), 'torus100' (100x100),
    'torus3d50' (50^3), 'rreg1m_d3/6/12' (n=10^6), 'torus1000' (1000x1000)."""
    if name == "torus10":
        return torus2d(10)
    if name == "torus100":
        return torus2d(100)
    if name == "torus100_unit":
        return torus2d(100, unit=True)
    if name == "torus3d50":
        return torus3d(50)
    if name.startswith("rreg1m_d"):
        return random_regular(1_000_000, int(name[len("rreg1m_d"):]))
    if name == "torus1000":
        return torus2d(1000)
    raise KeyError(name)
