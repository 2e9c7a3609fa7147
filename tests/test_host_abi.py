"""CPU-only checks of the C ABI: the library loads and exports every entry
point declared in include/gom.h, the host set-up (FOS, Welsh-Powell colouring)
equals the oracle's, and invalid input maps to error codes before any GPU
work.  No call here touches a GPU."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_2203_08680_gb300 import gom
from paper_2203_08680_gb300 import instances as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(gom_\w+)\s*\(", src))
    return names


def test_library_exports_every_declared_symbol():
    L = gom.load()
    declared = _declared_functions()
    assert len(declared) >= 20
    for name in declared:
        assert hasattr(L, name), name
    assert declared == {s[0] for s in gom.SIGNATURES}


def test_strerror_names_every_code():
    for code in range(-9, 1):
        assert gom.gom_strerror(code) != "unknown error"
    assert gom.gom_strerror(-99) == "unknown error"


GRAPHS = {
    "torus10": lambda: I.torus2d(10),
    "torus7": lambda: I.torus2d(7, seed=3),
    "torus3d4": lambda: I.torus3d(4),
    "rreg3": lambda: I.random_regular(300, 3, seed=2),
    "rreg6": lambda: I.random_regular(200, 6, seed=5),
    "rreg12": lambda: I.random_regular(150, 12, seed=7),
    "neg": lambda: I.random_regular(100, 5, seed=9, wmin=-100, wmax=100),
    "empty": lambda: I.empty_graph(20),
}

# larger FOS (4,096 to 20,000 elements), colouring only: the oracle's plain
# UPGMA of the linkage-tree test would take too long on them
LARGE = {
    "torus100": lambda: I.torus2d(100),
    "torus3d20": lambda: I.torus3d(20, seed=4),
    "rreg20k_d6": lambda: I.random_regular(20000, 6, seed=11),
    "rreg5k_d12": lambda: I.random_regular(5000, 12, seed=13),
}


@pytest.mark.parametrize("name", sorted(LARGE))
def test_large_coloring_equals_oracle(oracle, name):
    """The library's Welsh-Powell colouring equals the oracle's on larger graphs."""
    g = LARGE[name]()
    fos = gom.gom_build_fos(g)
    k = gom.gom_color_fos(g, fos)
    ep, ev = oracle.build_fos(g)
    ko, co = oracle.color(g, ep, ev)
    assert k == ko and np.array_equal(gom.gom_fos_export(fos)["color_of_elem"], co)


@pytest.mark.parametrize("name", sorted(GRAPHS))
@pytest.mark.parametrize("kind", [gom.GOM_FOS_NEIGHBOURHOOD, gom.GOM_FOS_SINGLETON])
def test_host_fos_and_coloring_equal_oracle(oracle, name, kind):
    g = GRAPHS[name]()
    assert oracle.check_graph(g)
    fos = gom.gom_build_fos(g, kind)
    k = gom.gom_color_fos(g, fos)
    ex = gom.gom_fos_export(fos)
    ep, ev = oracle.build_fos(g, kind)
    ko, co = oracle.color(g, ep, ev)
    assert np.array_equal(ex["elem_ptr"], ep)
    assert np.array_equal(ex["elem_vars"], ev)
    assert k == ko
    assert np.array_equal(ex["color_of_elem"], co)
    # groups list their elements ascending
    for c in range(k):
        grp = ex["color_elems"][ex["color_ptr"][c]:ex["color_ptr"][c + 1]]
        assert np.array_equal(grp, np.nonzero(co == c)[0])


@pytest.mark.parametrize("name", sorted(GRAPHS))
@pytest.mark.parametrize("bound", [1, 2, 5, 10, 64])
def test_host_bflt_equal_oracle(oracle, name, bound):
    """The bounded fixed linkage tree (UPGMA on the weights) and its colouring
    equal the oracle's."""
    g = GRAPHS[name]()
    fos = gom.gom_build_fos(g, gom.GOM_FOS_BFLT, bound)
    k = gom.gom_color_fos(g, fos)
    ex = gom.gom_fos_export(fos)
    ep, ev = oracle.build_bflt(g, bound)
    assert np.array_equal(ex["elem_ptr"], ep)
    assert np.array_equal(ex["elem_vars"], ev)
    ko, co = oracle.color(g, ep, ev)
    assert k == ko and np.array_equal(ex["color_of_elem"], co)


def test_bflt_arguments():
    g = I.torus2d(5)
    with pytest.raises(gom.GomError):
        gom.gom_build_fos(g, gom.GOM_FOS_BFLT, 0)
    with pytest.raises(gom.GomError):
        gom.gom_build_fos(g, gom.GOM_FOS_NEIGHBOURHOOD, 3)


def test_custom_fos_figure2_coloring(oracle):
    # the linkage tree of the paper's Figure 2 over the VIG of Figure 1
    g = I.from_edges(5, [0, 0, 1, 2, 2, 3], [1, 2, 2, 3, 4, 4], np.ones(6, dtype=np.int32))
    sets = [[0], [1], [2], [3], [4], [0, 2], [3, 4], [0, 1, 2]]
    ep = np.cumsum([0] + [len(s) for s in sets]).astype(np.int64)
    ev = np.concatenate([np.array(s, dtype=np.int32) for s in sets])
    fos = gom.gom_fos_create(5, ep, ev)
    k = gom.gom_color_fos(g, fos)
    ko, co = oracle.color(g, ep, ev)
    assert k == ko == 6
    assert np.array_equal(gom.gom_fos_export(fos)["color_of_elem"], co)


def _bad_graph_cases():
    g = I.torus2d(4)
    out = {}
    col = g.col.copy()
    col[0], col[1] = col[1], col[0]  # unsorted row
    out["unsorted"] = I.Graph(g.n, g.row_ptr, col, g.weight)
    w = g.weight.copy()
    w[0] += 1  # asymmetric weight
    out["asym_weight"] = I.Graph(g.n, g.row_ptr, g.col, w)
    col = g.col.copy()
    col[0] = 0  # self-loop at vertex 0
    out["self_loop"] = I.Graph(g.n, g.row_ptr, np.sort(col[:4]).tolist() + col[4:].tolist(), g.weight)
    col = g.col.copy()
    col[1] = col[0]  # repeated neighbour
    out["duplicate"] = I.Graph(g.n, g.row_ptr, col, g.weight)
    col = g.col.copy()
    col[5] = g.n + 3  # out of range
    out["range"] = I.Graph(g.n, g.row_ptr, col, g.weight)
    return out


@pytest.mark.parametrize("case", sorted(_bad_graph_cases()))
def test_invalid_graph_is_rejected(oracle, case):
    g = _bad_graph_cases()[case]
    assert not oracle.check_graph(g)
    with pytest.raises(gom.GomError) as ei:
        gom.gom_build_fos(g)
    assert ei.value.code == -2


def test_argument_errors_before_any_device_work():
    g = I.torus2d(5)
    fos = gom.gom_build_fos(g)
    L = gom.load()
    G = gom.Graph(g)
    h = C.c_void_p()
    # FOS not coloured yet
    rc = L.gom_init_population(G.ref(), fos.h, 16, 1, 256, 1 << 30, None, C.byref(h))
    assert rc == -3
    gom.gom_color_fos(g, fos)
    assert L.gom_init_population(G.ref(), fos.h, 1, 1, 256, 1 << 30, None, C.byref(h)) == -1
    assert L.gom_init_population(G.ref(), fos.h, 2000, 1, 256, 1 << 30, None, C.byref(h)) == -8
    need = gom.gom_workspace_bytes(g, fos, 16)
    assert need > 0
    assert L.gom_init_population(G.ref(), fos.h, 16, 1, None, need, None, C.byref(h)) == -4
    assert L.gom_init_population(G.ref(), fos.h, 16, 1, 256, need - 1, None, C.byref(h)) == -4
    assert L.gom_init_population(G.ref(), fos.h, 16, 1, 256 + 8, need, None, C.byref(h)) == -4
    assert gom.gom_workspace_bytes(g, fos, 1) == 0
    with pytest.raises(gom.GomError) as ei:
        gom.gom_build_fos(g, kind=7)
    assert ei.value.code == -1
    # FOS for another graph
    other = gom.gom_build_fos(I.torus2d(6))
    with pytest.raises(gom.GomError) as ei:
        gom.gom_color_fos(g, other)
    assert ei.value.code == -9
    assert L.gom_generation(None, 1, 0, None, None) == -1


def test_incomplete_or_bad_custom_fos():
    with pytest.raises(gom.GomError) as ei:
        gom.gom_fos_create(4, [0, 1, 2], [0, 1])  # variables 2, 3 uncovered
    assert ei.value.code == -9
    with pytest.raises(gom.GomError) as ei:
        gom.gom_fos_create(3, [0, 2, 3], [1, 0, 2])  # element not ascending
    assert ei.value.code == -9
    with pytest.raises(gom.GomError) as ei:
        gom.gom_fos_create(3, [0, 2, 3], [0, 5, 2])  # out of range
    assert ei.value.code == -9


def test_oversized_element_is_rejected_at_init():
    # a star: the centre's neighbourhood element has 129 variables, one above GOM_MAX_ELEMENT
    n = 129
    g = I.from_edges(n, np.zeros(n - 1, dtype=np.int64), np.arange(1, n), np.ones(n - 1, dtype=np.int32))
    fos = gom.gom_build_fos(g)
    gom.gom_color_fos(g, fos)
    L = gom.load()
    G = gom.Graph(g)
    h = C.c_void_p()
    need = gom.gom_workspace_bytes(g, fos, 8)
    assert L.gom_init_population(G.ref(), fos.h, 8, 1, 256, need, None, C.byref(h)) == -8
