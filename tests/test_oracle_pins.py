"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

None of these compares the oracle with itself: each checks a published value
(Philox known answers, the paper's worked LMIG example), a closed form (maximum
cuts of bipartite tori and complete graphs), brute force on tiny inputs, or an
invariant that a dropped term, a wrong sign or a wrong index would break.
"""
import itertools
import os

import numpy as np
import pytest

from paper_2203_08680_gb300 import instances as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


# ----------------------------------------------------------------------------
# Philox4x32-10 (the method's random numbers; Salmon et al., SC'11)

def test_philox_known_answers(oracle):
    for row in _read_golden("philox4x32_10_kat.txt"):
        vals = [int(v, 16) for v in row]
        out = oracle.philox(vals[0:4], vals[4:6])
        assert [int(x) for x in out] == vals[6:10]


def test_philox_bit_balance(oracle):
    ones = 0
    n = 4000
    for c in range(n):
        out = oracle.philox((c, 7, 0, 0x494E4954), (1, 0))
        ones += sum(bin(int(x)).count("1") for x in out)
    bits = n * 128
    # binomial(bits, 1/2): 6 standard deviations
    assert abs(ones - bits / 2) < 6 * np.sqrt(bits / 4)


# ----------------------------------------------------------------------------
# The Max-Cut objective (Sec. 6.2)

def _paper_formula(g, x01):
    """1/2 sum_{i<j} w_ij (1 - x_i x_j) with x in {-1, 1}, over a dense matrix."""
    W = np.zeros((g.n, g.n), dtype=np.int64)
    u = np.repeat(np.arange(g.n), g.degrees())
    W[u, g.col] = g.weight
    x = 2 * np.asarray(x01, dtype=np.int64) - 1
    iu = np.triu_indices(g.n, 1)
    return int((W[iu] * (1 - np.outer(x, x)[iu])).sum()) // 2


@pytest.mark.parametrize("gname", ["torus4", "rreg", "torus3d3"])
def test_objective_matches_paper_formula(oracle, gname):
    g = {"torus4": I.torus2d(4, seed=3), "rreg": I.random_regular(30, 5, seed=2),
         "torus3d3": I.torus3d(3, seed=4)}[gname]
    rng = np.random.default_rng(0)
    for _ in range(20):
        x = rng.integers(0, 2, g.n).astype(np.uint8)
        assert oracle.cut_value(g, x) == _paper_formula(g, x)


def test_negative_weights_objective(oracle):
    g = I.random_regular(20, 4, seed=5, wmin=-50, wmax=50)
    rng = np.random.default_rng(1)
    for _ in range(10):
        x = rng.integers(0, 2, g.n).astype(np.uint8)
        assert oracle.cut_value(g, x) == _paper_formula(g, x)


def test_even_torus_optimum_is_total_weight(oracle):
    # An even torus is bipartite: the checkerboard cuts every edge.
    for L, unit in [(4, False), (4, True)]:
        g = I.torus2d(L, seed=9, unit=unit)
        best, x = oracle.brute_force_maxcut(g)
        assert best == g.total_weight()
        if unit:
            assert best == 2 * L * L
        cb = np.array([(v % L + v // L) % 2 for v in range(g.n)], dtype=np.uint8)
        assert oracle.cut_value(g, cb) == g.total_weight()
    g3 = I.torus3d(4, seed=2, unit=True)
    cb = np.array([((v % 4) + (v // 4) % 4 + v // 16) % 2 for v in range(g3.n)], dtype=np.uint8)
    assert oracle.cut_value(g3, cb) == 3 * 4 ** 3 == g3.total_weight()


def test_odd_torus_and_complete_graph_closed_forms(oracle):
    # 3x3 unit torus: 6 odd 3-cycles, each cut at most twice -> 12, attained.
    g = I.torus2d(3, unit=True)
    assert oracle.brute_force_maxcut(g)[0] == 12
    # K_n with unit weights: floor(n/2) * ceil(n/2).
    for n in (5, 7, 8):
        u, v = zip(*itertools.combinations(range(n), 2))
        Kn = I.from_edges(n, u, v, np.ones(len(u), dtype=np.int32))
        assert oracle.brute_force_maxcut(Kn)[0] == (n // 2) * ((n + 1) // 2)


def test_brute_force_dominates_random_assignments(oracle):
    g = I.random_regular(16, 3, seed=11)
    best, bx = oracle.brute_force_maxcut(g)
    assert oracle.cut_value(g, bx) == best
    rng = np.random.default_rng(2)
    for _ in range(200):
        assert oracle.cut_value(g, rng.integers(0, 2, g.n).astype(np.uint8)) <= best


# ----------------------------------------------------------------------------
# Partial evaluation (Sec. 2.2, Alg. 4)

@pytest.mark.parametrize("kind", [0, 1])
def test_partial_delta_equals_full_difference(oracle, kind):
    g = I.random_regular(40, 6, seed=3, wmin=-20, wmax=100)
    eptr, evars = oracle.build_fos(g, kind)
    rng = np.random.default_rng(kind)
    for _ in range(300):
        j = int(rng.integers(0, g.n))
        F = evars[eptr[j]:eptr[j + 1]]
        x = rng.integers(0, 2, g.n).astype(np.uint8)
        y = rng.integers(0, 2, len(F)).astype(np.uint8)
        x2 = x.copy()
        x2[F] = y
        assert oracle.partial_delta(g, x, F, y) == oracle.cut_value(g, x2) - oracle.cut_value(g, x)


def test_partial_delta_random_subsets(oracle):
    g = I.torus2d(6, seed=8)
    rng = np.random.default_rng(5)
    for _ in range(300):
        sz = int(rng.integers(1, 12))
        F = np.sort(rng.choice(g.n, sz, replace=False)).astype(np.int32)
        x = rng.integers(0, 2, g.n).astype(np.uint8)
        y = rng.integers(0, 2, sz).astype(np.uint8)
        x2 = x.copy()
        x2[F] = y
        assert oracle.partial_delta(g, x, F, y) == oracle.cut_value(g, x2) - oracle.cut_value(g, x)


@pytest.mark.parametrize("sz", [65, 100, 128])
def test_partial_delta_large_elements(oracle, sz):
    """Elements of 65 to 128 variables (the largest linkage sets the library
    takes), with many edges inside them and across their border."""
    g = I.random_regular(200, 5, seed=9, wmin=-50, wmax=100)
    rng = np.random.default_rng(sz)
    for _ in range(40):
        F = np.sort(rng.choice(g.n, sz, replace=False)).astype(np.int32)
        x = rng.integers(0, 2, g.n).astype(np.uint8)
        y = rng.integers(0, 2, sz).astype(np.uint8)
        x2 = x.copy()
        x2[F] = y
        assert oracle.partial_delta(g, x, F, y) == oracle.cut_value(g, x2) - oracle.cut_value(g, x)


def test_singleton_delta_is_one_flip_gain(oracle):
    g = I.random_regular(30, 4, seed=6)
    rng = np.random.default_rng(3)
    x = rng.integers(0, 2, g.n).astype(np.uint8)
    for u in range(g.n):
        nb = g.col[g.row_ptr[u]:g.row_ptr[u + 1]]
        wt = g.weight[g.row_ptr[u]:g.row_ptr[u + 1]].astype(np.int64)
        # flipping u: uncut edges become cut (+w), cut edges become uncut (-w)
        gain = int((wt * np.where(x[nb] == x[u], 1, -1)).sum())
        assert oracle.partial_delta(g, x, [u], [1 - x[u]]) == gain


# ----------------------------------------------------------------------------
# FOS, LMIG and colouring (Sec. 4.1, Sec. 5.2)

def _golden_fig3():
    rows = _read_golden("fig3_lmig.txt")
    vig = [(int(a) - 1, int(b) - 1) for t, a, b in (r for r in rows if r[0] == "vig")]
    fos = [[int(v) - 1 for v in r[2:]] for r in rows if r[0] == "fos"]
    lmig = {tuple(sorted((int(a) - 1, int(b) - 1))) for t, a, b in (r for r in rows if r[0] == "lmig")}
    ncol = [int(r[1]) for r in rows if r[0] == "colors"][0]
    return vig, fos, lmig, ncol


def test_paper_figure3_lmig(oracle):
    vig, fos, lmig, _ = _golden_fig3()
    u, v = zip(*vig)
    g = I.from_edges(5, u, v, np.ones(len(u), dtype=np.int32))
    eptr = np.cumsum([0] + [len(F) for F in fos]).astype(np.int64)
    evars = np.concatenate([np.array(F, dtype=np.int32) for F in fos])
    got = {tuple(p) for p in oracle.lmig_edges(g, eptr, evars).tolist()}
    assert len(lmig) == 22
    assert got == lmig


def test_paper_figure3_coloring(oracle):
    vig, fos, lmig, ncol = _golden_fig3()
    u, v = zip(*vig)
    g = I.from_edges(5, u, v, np.ones(len(u), dtype=np.int32))
    eptr = np.cumsum([0] + [len(F) for F in fos]).astype(np.int64)
    evars = np.concatenate([np.array(F, dtype=np.int32) for F in fos])
    k, colors = oracle.color(g, eptr, evars)
    # {F3,F4,F5,F6,F7,F8} is a 6-clique of the figure, so 6 colours is optimal
    clique = [2, 3, 4, 5, 6, 7]
    assert all(tuple(sorted(p)) in lmig for p in itertools.combinations(clique, 2))
    assert k == ncol == 6
    for a, b in lmig:
        assert colors[a] != colors[b]
    groups = sorted(sorted(np.nonzero(colors == c)[0].tolist()) for c in range(k))
    # Welsh-Powell order by (degree desc, index asc): F3 F6 F8 F4 F5 F7 F1 F2
    assert groups == sorted([[2], [5], [7], [0, 3], [1, 4], [6]])


def _brute_lmig(g, eptr, evars):
    sets = [set(evars[eptr[j]:eptr[j + 1]].tolist()) for j in range(len(eptr) - 1)]
    adj = [set(g.col[g.row_ptr[v]:g.row_ptr[v + 1]].tolist()) for v in range(g.n)]
    out = set()
    for a, b in itertools.combinations(range(len(sets)), 2):
        if sets[a] & sets[b] or any(adj[x] & sets[b] for x in sets[a]):
            out.add((a, b))
    return out


@pytest.mark.parametrize("gname,kind", [("torus5", 0), ("torus5", 1), ("rreg", 0), ("t3d", 0)])
def test_lmig_brute_force_and_coloring_properties(oracle, gname, kind):
    g = {"torus5": I.torus2d(5, seed=1), "rreg": I.random_regular(24, 3, seed=4),
         "t3d": I.torus3d(3, seed=1)}[gname]
    eptr, evars = oracle.build_fos(g, kind)
    # FOS is complete and each element is {j} u adj(j) (or {j})
    assert set(evars.tolist()) == set(range(g.n))
    for j in range(g.n):
        F = evars[eptr[j]:eptr[j + 1]].tolist()
        want = [j] if kind == 1 else sorted([j] + g.col[g.row_ptr[j]:g.row_ptr[j + 1]].tolist())
        assert F == want
    edges = _brute_lmig(g, eptr, evars)
    got = {tuple(p) for p in oracle.lmig_edges(g, eptr, evars).tolist()}
    assert got == edges
    k, colors = oracle.color(g, eptr, evars)
    assert colors.min() == 0 and colors.max() == k - 1
    for a, b in edges:
        assert colors[a] != colors[b]
    # first-fit in (degree desc, index asc) order
    m = len(eptr) - 1
    nbrs = [set() for _ in range(m)]
    for a, b in edges:
        nbrs[a].add(b)
        nbrs[b].add(a)
    order = sorted(range(m), key=lambda j: (-len(nbrs[j]), j))
    rank = {j: t for t, j in enumerate(order)}
    for j in range(m):
        earlier = {colors[q] for q in nbrs[j] if rank[q] < rank[j]}
        assert colors[j] == min(set(range(k + 1)) - earlier)


def test_torus_neighbourhood_lmig_needs_eight_colours(oracle):
    # On Z^2 the neighbourhood elements of a 3x2 block of vertices plus the
    # vertex above and below its middle column are pairwise within graph
    # distance 3, so the LMIG holds an 8-clique.
    g = I.torus2d(8, seed=1)
    eptr, evars = oracle.build_fos(g, 0)
    k, colors = oracle.color(g, eptr, evars)
    pts = [(x, y) for y in (1, 2) for x in (0, 1, 2)] + [(1, 0), (1, 3)]
    block = [y * 8 + x for x, y in pts]
    edges = {tuple(p) for p in oracle.lmig_edges(g, eptr, evars).tolist()}
    assert all(tuple(sorted(q)) in edges for q in itertools.combinations(block, 2))
    assert k >= 8
    assert len(set(colors[block].tolist())) == 8


def test_group_order_is_uniform_permutation(oracle):
    k = 3
    counts = {}
    for g in range(3000):
        o = tuple(oracle.group_order(1, k, g).tolist())
        assert sorted(o) == list(range(k))
        counts[o] = counts.get(o, 0) + 1
    assert len(counts) == 6
    exp = 3000 / 6
    chi2 = sum((c - exp) ** 2 / exp for c in counts.values())
    assert chi2 < 25  # 5 dof, far above the 0.999 quantile (20.5)


# ----------------------------------------------------------------------------
# Parallel GOMEA (Alg. 2, Alg. 3)

def _setup(oracle, g, kind=0):
    eptr, evars = oracle.build_fos(g, kind)
    k, colors = oracle.color(g, eptr, evars)
    return eptr, evars, k, colors


@pytest.mark.parametrize("gname,p", [("torus10", 16), ("rreg", 40), ("t3d", 33), ("neg", 20)])
def test_gom_incremental_fitness_and_monotonicity(oracle, gname, p):
    g = {"torus10": I.torus2d(10), "rreg": I.random_regular(60, 5, seed=2),
         "t3d": I.torus3d(4, seed=3), "neg": I.random_regular(50, 4, seed=1, wmin=-30, wmax=60)}[gname]
    eptr, evars, k, colors = _setup(oracle, g)
    run = oracle.Run(g, eptr, evars, colors, k, p, seed=7)
    s0 = run.get()
    assert all(s0["f"][i] == oracle.cut_value(g, s0["pop"][i]) for i in range(p))
    assert s0["fe"] == s0["f"].max()
    assert np.array_equal(s0["xe"], s0["pop"][int(np.argmax(s0["f"]))])
    prev_f, prev_fe = s0["f"].copy(), s0["fe"]
    for gen in range(12):
        st = run.generation()
        s = run.get()
        assert st["trials"] == p * (len(eptr) - 1)
        assert st["improving"] <= st["accepted"] <= st["trials"] - st["donorless"]
        for i in range(p):
            assert s["f"][i] == oracle.cut_value(g, s["pop"][i])
        assert np.all(s["f"] >= prev_f)
        assert s["fe"] >= prev_fe and s["fe"] == max(prev_fe, s["f"].max())
        assert s["fe"] == oracle.cut_value(g, s["xe"])
        assert st["best"] == s["f"].max() and st["elite"] == s["fe"]
        assert s["g"] == gen + 1
        prev_f, prev_fe = s["f"].copy(), s["fe"]


@pytest.mark.parametrize("gname,p", [("torus10", 16), ("rreg", 24)])
def test_gom_group_order_invariance(oracle, gname, p):
    """Trials of one colour group give the same result in any order: the
    sequential run equals the parallel semantics of Alg. 3."""
    g = {"torus10": I.torus2d(10), "rreg": I.random_regular(60, 4, seed=5)}[gname]
    eptr, evars, k, colors = _setup(oracle, g)
    a = oracle.Run(g, eptr, evars, colors, k, p, seed=3)
    b = oracle.Run(g, eptr, evars, colors, k, p, seed=3)
    for gen in range(8):
        sa = a.generation()
        sb = b.generation(shuffle=1000 + gen)
        assert sa == sb
    ga, gb = a.get(), b.get()
    assert np.array_equal(ga["pop"], gb["pop"]) and np.array_equal(ga["f"], gb["f"])


def test_gom_linkage_tree_large_sets(oracle):
    """GOM over the bounded linkage tree at 128 variables (sets of 65 and more
    variables among the nested ones, Sec. 4.1): incremental fitness equals full
    evaluation after every generation, fitness never drops, and each colour
    group gives the same result in a shuffled trial order."""
    g = I.random_regular(300, 6, seed=53)
    eptr, evars = oracle.build_bflt(g, 128)
    assert np.diff(eptr).max() > 64
    k, colors = oracle.color(g, eptr, evars)
    a = oracle.Run(g, eptr, evars, colors, k, 40, seed=4)
    b = oracle.Run(g, eptr, evars, colors, k, 40, seed=4)
    prev = a.get()["f"].copy()
    for gen in range(5):
        sa = a.generation()
        assert sa == b.generation(shuffle=2000 + gen)
        s = a.get()
        assert all(s["f"][i] == oracle.cut_value(g, s["pop"][i]) for i in range(40))
        assert np.all(s["f"] >= prev)
        prev = s["f"].copy()
    assert np.array_equal(a.get()["pop"], b.get()["pop"])


def test_gom_wrong_coloring_breaks_invariance(oracle):
    """Putting all elements into one group violates the LMIG: the order of the
    trials then changes the result, which the invariance test would catch."""
    g = I.torus2d(6, seed=2)
    eptr, evars = oracle.build_fos(g, 0)
    one = np.zeros(g.n, dtype=np.int32)
    a = oracle.Run(g, eptr, evars, one, 1, 8, seed=3)
    b = oracle.Run(g, eptr, evars, one, 1, 8, seed=3)
    differ = False
    for gen in range(5):
        a.generation()
        b.generation(shuffle=77 + gen)
        if not np.array_equal(a.get()["pop"], b.get()["pop"]):
            differ = True
    assert differ


def test_gom_identical_population_is_all_donorless(oracle):
    g = I.torus2d(5, seed=1)
    eptr, evars, k, colors = _setup(oracle, g)
    p = 6
    run = oracle.Run(g, eptr, evars, colors, k, p, seed=1)
    x = run.get()["pop"][0]
    pop = np.tile(x, (p, 1))
    f = np.full(p, oracle.cut_value(g, x), dtype=np.int64)
    run.load(pop, f, x, int(f[0]), 0)
    st = run.generation()
    assert st["donorless"] == st["trials"] == p * g.n
    assert st["accepted"] == 0
    assert np.array_equal(run.get()["pop"], pop)


FI_OFF = {"fi_individuals": 0, "fi_trials": 0, "fi_accepted": 0, "fi_improving": 0, "fi_replaced": 0}


def test_gom_tie_rule_uses_generation_start_genotype(oracle):
    """Empty graph, singleton FOS: every move is neutral (delta = 0), so a
    move is accepted exactly when P[i] differs from the elitist (Alg. 2 with
    the flag of Sec. 5.3).  Individuals 0..2 equal the elitist, 3 does not."""
    g = I.empty_graph(9)
    eptr, evars, k, colors = _setup(oracle, g, kind=1)
    assert k == 1
    p = 4
    run = oracle.Run(g, eptr, evars, colors, k, p, seed=5)
    pop = np.zeros((p, g.n), dtype=np.uint8)
    pop[3] = 1
    run.load(pop, np.zeros(p, dtype=np.int64), pop[0], 0, 0)
    st = run.generation()
    assert st == {"generation": 0, "best": 0, "elite": 0, "trials": p * g.n, "donorless": 0,
                  "accepted": g.n, "improving": 0, "reached": 0, **FI_OFF}
    assert np.array_equal(run.get()["pop"], np.zeros((p, g.n), dtype=np.uint8))
    st = run.generation()
    assert st["donorless"] == st["trials"] and st["accepted"] == 0


def test_gom_two_individuals_neutral_copy(oracle):
    """p = 2 on an empty graph: the donor of each individual is the other.
    Individual 0 is the elitist (all f = 0, lowest index) and rejects its
    neutral moves; individual 1 takes every differing bit of individual 0."""
    g = I.empty_graph(40)
    eptr, evars, k, colors = _setup(oracle, g, kind=1)
    run = oracle.Run(g, eptr, evars, colors, k, 2, seed=9)
    s0 = run.get()
    ndiff = int((s0["pop"][0] != s0["pop"][1]).sum())
    assert ndiff > 0
    st = run.generation()
    assert st["accepted"] == ndiff and st["donorless"] == 2 * (g.n - ndiff)
    s1 = run.get()
    assert np.array_equal(s1["pop"][1], s0["pop"][0]) and np.array_equal(s1["pop"][0], s0["pop"][0])


def test_gom_split_runs_and_resume(oracle):
    g = I.torus2d(8, seed=4)
    eptr, evars, k, colors = _setup(oracle, g)
    a = oracle.Run(g, eptr, evars, colors, k, 12, seed=2)
    for _ in range(10):
        a.generation()
    b = oracle.Run(g, eptr, evars, colors, k, 12, seed=2)
    for _ in range(4):
        b.generation()
    snap = b.get()
    c = oracle.Run(g, eptr, evars, colors, k, 12, seed=2)
    c.load(snap["pop"], snap["f"], snap["xe"], snap["fe"], snap["g"])
    for _ in range(6):
        c.generation()
    ga, gc = a.get(), c.get()
    for key in ("pop", "f", "xe"):
        assert np.array_equal(ga[key], gc[key])
    assert ga["fe"] == gc["fe"] and ga["g"] == gc["g"] == 10


def test_gom_target_stop_and_optimum_bound(oracle):
    """A run that reaches the brute-force optimum after a few generations
    (random 3-regular graph on 20 vertices, singleton FOS, p = 8, seed 1:
    best 1463, 1540, 1540, then the optimum 1547 at the fourth generation)
    stops exactly there; fitness never exceeds the optimum; the stop does not
    change the trajectory (a run without target has the same state after
    four generations and goes past the optimum never)."""
    g = I.random_regular(20, 3, seed=2)
    best, xbest = oracle.brute_force_maxcut(g)
    assert best == 1547 and oracle.cut_value(g, xbest) == best
    eptr, evars = oracle.build_fos(g, oracle.SINGLETON)
    k, colors = oracle.color(g, eptr, evars)
    run = oracle.Run(g, eptr, evars, colors, k, 8, seed=1)
    stats = run.run(60, target=best)
    assert [s["best"] for s in stats] == [1463, 1540, 1540, 1547]
    assert stats[-1]["reached"] and not any(s["reached"] for s in stats[:-1])
    free = oracle.Run(g, eptr, evars, colors, k, 8, seed=1)
    fst = free.run(10)
    assert [s["best"] for s in fst[:4]] == [1463, 1540, 1540, 1547]
    assert all(s["best"] <= best for s in fst)
    a = run.get()
    b = oracle.Run(g, eptr, evars, colors, k, 8, seed=1)
    b.run(4)
    for key in ("pop", "f", "xe"):
        assert np.array_equal(a[key], b.get()[key])
    # a target above the optimum is never reached
    c = oracle.Run(g, eptr, evars, colors, k, 8, seed=1)
    cst = c.run(30, target=best + 1)
    assert len(cst) == 30 and not any(s["reached"] for s in cst)


def test_gom_subset_replay_matches_full_generation(oracle):
    """Individuals are independent within a generation (donors come from the
    frozen P), so replaying a generation for a subset reproduces those rows."""
    g = I.random_regular(80, 5, seed=3)
    eptr, evars, k, colors = _setup(oracle, g)
    a = oracle.Run(g, eptr, evars, colors, k, 20, seed=4)
    for _ in range(3):
        a.generation()
    snap = a.get()
    a.generation()
    full = a.get()
    b = oracle.Run(g, eptr, evars, colors, k, 20, seed=4)
    b.load(snap["pop"], snap["f"], snap["xe"], snap["fe"], snap["g"])
    only = [0, 7, 19]
    b.generation(only=only)
    part = b.get()
    for i in only:
        assert np.array_equal(part["pop"][i], full["pop"][i])
        assert part["f"][i] == full["f"][i]
    # the same subset on the multi-threaded generation (the reference arm's timing sample)
    c = oracle.Run(g, eptr, evars, colors, k, 20, seed=4)
    c.load(snap["pop"], snap["f"], snap["xe"], snap["fe"], snap["g"])
    sc = c.generation(only=only, threads=3)
    part2 = c.get()
    assert sc["trials"] == len(only) * (len(eptr) - 1)
    for i in only:
        assert np.array_equal(part2["pop"][i], full["pop"][i])
        assert part2["f"][i] == full["f"][i]


def test_multithreaded_generation_equals_single_threaded(oracle):
    """The oracle's multi-threaded generation (individuals of a group split
    over threads) gives the single-threaded state: trials of one colour group
    are independent of each other (LMIG colouring, donors from P, fixed
    elitist flags)."""
    g = I.torus2d(12, seed=4)
    ep, ev = oracle.build_fos(g)
    k, co = oracle.color(g, ep, ev)
    a = oracle.Run(g, ep, ev, co, k, 37, 9)
    b = oracle.Run(g, ep, ev, co, k, 37, 9)
    for _ in range(6):
        sa = a.generation()
        sb = b.generation(threads=4)
        assert sa == sb
    ra, rb = a.get(), b.get()
    for key in ("pop", "f", "xe"):
        assert np.array_equal(ra[key], rb[key])
    assert ra["fe"] == rb["fe"] and ra["g"] == rb["g"]


# ---------------------------------------------------------------------------
# Bounded fixed linkage tree (Sec. 4.1): UPGMA on the edge weights

def _bflt_sets(oracle, g, bound):
    ep, ev = oracle.build_bflt(g, bound)
    return [tuple(int(x) for x in ev[ep[j]:ep[j + 1]]) for j in range(len(ep) - 1)]


def test_bflt_hand_example(oracle):
    """Path 0-1-2-3-4 with weights 5, 1, 5, 2, worked by hand from the UPGMA
    definition: {0,1} (average 5, before the tied {2,3} by the smaller id),
    {2,3} (5), then {2,3,4} (2/2 = 1 beats {0,1}+{2,3} at 1/4); the last merge
    would hold all five variables and is left out."""
    g = I.from_edges(5, np.array([0, 1, 2, 3]), np.array([1, 2, 3, 4]), np.array([5, 1, 5, 2]))
    single = [(0,), (1,), (2,), (3,), (4,)]
    assert _bflt_sets(oracle, g, 1) == single
    assert _bflt_sets(oracle, g, 2) == single + [(0, 1), (2, 3)]
    assert _bflt_sets(oracle, g, 3) == single + [(0, 1), (2, 3), (2, 3, 4)]
    assert _bflt_sets(oracle, g, 4) == single + [(0, 1), (2, 3), (2, 3, 4)]
    assert _bflt_sets(oracle, g, 5) == single + [(0, 1), (2, 3), (2, 3, 4)]
    # one more vertex (edge 4-5 of weight 1): {4,5} and {4,{2,3}} tie at
    # average 1, the smaller second id (vertex 5) wins; then {2,3}+{4,5}
    # (2/4) beats {0,1}+{2,3} (1/4); the six-variable root is left out
    g6 = I.from_edges(6, np.array([0, 1, 2, 3, 4]), np.array([1, 2, 3, 4, 5]), np.array([5, 1, 5, 2, 1]))
    assert _bflt_sets(oracle, g6, 6) == [(i,) for i in range(6)] + [(0, 1), (2, 3), (4, 5), (2, 3, 4, 5)]


def test_bflt_average_not_single_linkage(oracle):
    """After {0,1} forms (weight 50), vertex 2 (one edge of 10 to 0) has
    average 10/2 = 5 to it and vertex 3 (edges of 6 to 0 and to 1) has 12/2 = 6:
    average linkage takes 3 first; single linkage would take 2."""
    u = np.array([0, 0, 0, 1])
    v = np.array([1, 2, 3, 3])
    w = np.array([50, 10, 6, 6])
    g = I.from_edges(5, np.append(u, 2), np.append(v, 4), np.append(w, 1))
    sets = _bflt_sets(oracle, g, 3)
    assert sets[5] == (0, 1) and sets[6] == (0, 1, 3)


def _upgma_replay(g, bound):
    """Independent replay with exact fractions: at every step the merged pair
    is the best linked pair under the rule (highest average, then smaller ids)."""
    from fractions import Fraction
    n = g.n
    W = {}
    for a in range(n):
        for e in range(g.row_ptr[a], g.row_ptr[a + 1]):
            W[(a, int(g.col[e]))] = int(g.weight[e])
    clusters = {i: (i,) for i in range(n)}
    out = [(i,) for i in range(n)]
    nxt = n
    while True:
        best = None
        ids = sorted(clusters)
        for i, a in enumerate(ids):
            for b in ids[i + 1:]:
                A, B = clusters[a], clusters[b]
                if len(A) + len(B) > bound:
                    continue
                pairs = [(x, y) for x in A for y in B if (x, y) in W]
                if not pairs:
                    continue
                avg = Fraction(sum(W[p] for p in pairs), len(A) * len(B))
                if best is None or avg > best[0]:
                    best = (avg, a, b)
        if best is None or len(clusters[best[1]]) + len(clusters[best[2]]) >= n:
            return out
        merged = tuple(sorted(clusters.pop(best[1]) + clusters.pop(best[2])))
        clusters[nxt] = merged
        out.append(merged)
        nxt += 1


@pytest.mark.parametrize("seed", [1, 2, 3])
@pytest.mark.parametrize("bound", [2, 4, 7, 40])
def test_bflt_replay_and_tree_properties(oracle, seed, bound):
    g = I.random_regular(24, 3, seed=seed, wmin=-5, wmax=9)
    sets = _bflt_sets(oracle, g, bound)
    assert sets == _upgma_replay(g, bound)
    n = g.n
    assert sets[:n] == [(i,) for i in range(n)]  # complete: every singleton
    for j, s in enumerate(sets[n:], start=n):
        assert 2 <= len(s) <= bound and len(s) < n
        # the union of exactly two disjoint earlier sets (Sec. 4.1)
        earlier = [set(x) for x in sets[:j]]
        splits = [(a, b) for ia, a in enumerate(earlier) for b in earlier[ia + 1:]
                  if not (a & b) and (a | b) == set(s)]
        assert len(splits) >= 1
    assert len(set(sets)) == len(sets)


def test_generation_skip_mask(oracle):
    """The replay of a filtered generation: an all-zero mask is the plain
    generation; an all-one mask runs no trial and changes nothing but the
    generation counter."""
    g = I.torus2d(8, seed=7)
    ep, ev = oracle.build_fos(g)
    k, co = oracle.color(g, ep, ev)
    a = oracle.Run(g, ep, ev, co, k, 12, 4)
    b = oracle.Run(g, ep, ev, co, k, 12, 4)
    m = len(ep) - 1
    assert a.generation() == b.generation_skip(np.zeros(m, dtype=np.uint8))
    ra, rb = a.get(), b.get()
    assert np.array_equal(ra["pop"], rb["pop"]) and np.array_equal(ra["f"], rb["f"])
    before = b.get()
    st = b.generation_skip(np.ones(m, dtype=np.uint8))
    after = b.get()
    assert st["trials"] == 0 and st["accepted"] == 0
    assert np.array_equal(before["pop"], after["pop"]) and after["g"] == before["g"] + 1


# ---------------------------------------------------------------------------
# Forced Improvement (Sec. 4, Alg. 1), in its parallel reading (R12 of the oracle)

def _fi_path_case(oracle):
    """Path 0-1-2-3-4-5 with weights 7, 5, 9, 9, 8, singleton FOS.  Welsh-Powell
    on the path-shaped LMIG gives the groups {1,3,5} (colour 0) and {0,2,4}."""
    g = I.from_edges(6, np.arange(5), np.arange(1, 6), np.array([7, 5, 9, 9, 8]))
    ep, ev = oracle.build_fos(g, oracle.SINGLETON)
    k, co = oracle.color(g, ep, ev)
    assert k == 2 and list(np.flatnonzero(co == 0)) == [1, 3, 5] and list(np.flatnonzero(co == 1)) == [0, 2, 4]
    return g, ep, ev, k, co


def test_fi_hand_example_stops_after_first_improving_group(oracle):
    """Both individuals are y = 111011 (cut 18) and the elitist is 010100
    (cut 30), not in the population.  Mixing has no donor (the two
    individuals are equal), so both enter FI with the elitist as donor.
    Worked by hand: with group {1,3,5} first, {1} needs no change, {3} would
    lose 18 (rejected), {5} gains 8 (accepted, f = 26) -- an improvement, so
    FI stops there: 111010, although group {0,2,4} would gain 7 more.  With
    group {0,2,4} first, {0} gains 7 (f = 25), {2} would lose 4 and {4}
    would lose 1 (rejected): FI stops with 011011."""
    g, ep, ev, k, co = _fi_path_case(oracle)
    y = np.array([1, 1, 1, 0, 1, 1], dtype=np.uint8)
    xe = np.array([0, 1, 0, 1, 0, 0], dtype=np.uint8)
    assert oracle.cut_value(g, y) == 18 and oracle.cut_value(g, xe) == 30
    seen = set()
    for seed in range(1, 40):
        order = list(oracle.group_order(seed, k, 0))
        run = oracle.Run(g, ep, ev, co, k, 2, seed)
        run.load(np.stack([y, y]), np.array([18, 18]), xe, 30, 0)
        run.set_fi(True)
        st = run.generation()
        s = run.get()
        want, fw = ([1, 1, 1, 0, 1, 0], 26) if order[0] == 0 else ([0, 1, 1, 0, 1, 1], 25)
        for i in range(2):
            assert list(s["pop"][i]) == want and s["f"][i] == fw, (seed, order)
        assert s["fe"] == 30 and list(s["xe"]) == list(xe)
        assert st["trials"] == 12 and st["donorless"] == 12 and st["accepted"] == 0
        assert (st["fi_individuals"], st["fi_trials"], st["fi_accepted"], st["fi_improving"], st["fi_replaced"]) \
            == (2, 6, 2, 2, 0)
        seen.add(order[0])
    assert seen == {0, 1}  # both group orders were exercised


def test_fi_replaces_with_elitist_when_nothing_improves(oracle):
    """An individual that no elitist step can improve becomes a copy of the
    elitist.  y = 100100 (cut 25) differs from the elitist 010100 (cut 30) on
    vertices 0 and 1 only; by hand, moving vertex 0 to the elitist's value
    uncuts edge (0,1) (-7) and moving vertex 1 uncuts (0,1) and cuts (1,2)
    (-7 + 5 = -2): FI improves nothing, and y is replaced (f 25 -> 30)."""
    g, ep, ev, k, co = _fi_path_case(oracle)
    xe = np.array([0, 1, 0, 1, 0, 0], dtype=np.uint8)
    y = np.array([1, 0, 0, 1, 0, 0], dtype=np.uint8)
    assert oracle.cut_value(g, y) == 25
    run = oracle.Run(g, ep, ev, co, k, 2, 3)
    run.load(np.stack([y, y]), np.array([25, 25]), xe, 30, 0)
    run.set_fi(True)
    st = run.generation()
    s = run.get()
    for i in range(2):
        assert np.array_equal(s["pop"][i], xe) and s["f"][i] == 30
    assert st["fi_individuals"] == 2 and st["fi_replaced"] == 2 and st["fi_improving"] == 0


def test_fi_identical_population_equal_to_elitist_is_unchanged(oracle):
    """Every individual equals the elitist: mixing has no donor, every
    individual enters FI, no step varies anything, each is 'replaced' by the
    elitist it already equals -- the state does not change."""
    g = I.torus2d(6, seed=3)
    eptr, evars, k, colors = _setup(oracle, g)
    run = oracle.Run(g, eptr, evars, colors, k, 5, 2)
    x = run.get()["xe"].copy()
    fx = oracle.cut_value(g, x)
    run.load(np.tile(x, (5, 1)), np.full(5, fx), x, fx, 0)
    run.set_fi(True)
    st = run.generation()
    s = run.get()
    assert np.array_equal(s["pop"], np.tile(x, (5, 1))) and (s["f"] == fx).all()
    assert st["fi_individuals"] == 5 and st["fi_replaced"] == 5 and st["fi_accepted"] == 0
    assert st["fi_trials"] == 5 * (len(eptr) - 1)  # no improvement: every group is visited


@pytest.mark.parametrize("nis", [0, 2])
def test_fi_against_the_same_generation_without_it(oracle, nis):
    """From the same state, one generation with FI and one without: mixing is
    identical (FI comes after it), so every individual FI left alone has the
    same row and fitness, and every one it touched either improved on its
    FI-less fitness or became a copy of the elitist.  FI never lowers a
    fitness; incremental fitness equals full evaluation; each individual that
    entered FI and was not replaced took at least one improving step."""
    g = I.random_regular(120, 4, seed=9)
    eptr, evars, k, colors = _setup(oracle, g)
    base = oracle.Run(g, eptr, evars, colors, k, 24, 5)
    for gen in range(12):
        snap = base.get()
        off = oracle.Run(g, eptr, evars, colors, k, 24, 5, init=False)
        off.load(snap["pop"], snap["f"], snap["xe"], snap["fe"], snap["g"])
        so = off.generation()
        base.set_fi(True, nis)
        sb = base.generation()
        a, b = base.get(), off.get()
        assert so["accepted"] == sb["accepted"] and so["donorless"] == sb["donorless"]
        assert (a["f"] >= b["f"]).all() and (a["f"] >= snap["f"]).all()
        assert a["fe"] >= b["fe"]
        for i in range(24):
            if not np.array_equal(a["pop"][i], b["pop"][i]):
                assert a["f"][i] > b["f"][i] or (np.array_equal(a["pop"][i], a["xe"]) and a["f"][i] == a["fe"])
            assert oracle.cut_value(g, a["pop"][i]) == a["f"][i]
        assert sb["fi_improving"] >= sb["fi_individuals"] - sb["fi_replaced"] >= 0
        assert sum(np.array_equal(a["pop"][i], a["xe"]) for i in range(24)) >= sb["fi_replaced"]


def test_element_counters_sum_to_the_generation_counters(oracle):
    """The per-element counters (accepted, donor-less, improving trials of
    each element in the last generation) add up to the generation's own
    counters, and an element's counts never exceed p."""
    g = I.random_regular(150, 4, seed=12)
    eptr, evars, k, colors = _setup(oracle, g)
    run = oracle.Run(g, eptr, evars, colors, k, 20, 3)
    run.keep_element_counts(True)
    for _ in range(5):
        st = run.generation()
        acc, dl, imp = run.element_counts()
        assert (acc.sum(), dl.sum(), imp.sum()) == (st["accepted"], st["donorless"], st["improving"])
        assert (acc + dl <= 20).all() and (imp <= acc).all()
