"""GPU parity at the benchmark configurations' full sizes.

The oracle cannot run whole generations of 10^6-vertex graphs with 512
individuals in test time, but individuals are independent within a
generation (donors come from the frozen generation-start population P), so
it can replay one generation for a sample of individuals: the GPU runs a
generation, its state is exported, the GPU runs the next generation, and the
oracle replays that generation from the exported state for a few individuals,
which must match bit for bit.  Around the sample, properties that hold at any
size are checked on every individual: incremental fitness equals full
re-evaluation, the elitist's bits evaluate to its fitness, the elitist never
gets worse.  The oracle computes its own FOS and colouring, which must equal
the library's.

The 2D torus 100x100 run is checked in full: every generation's counters, and
the whole state every 50 generations, up to the target or 500 generations.
"""
import numpy as np
import pytest

from paper_2203_08680_gb300 import gom
from paper_2203_08680_gb300 import instances as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

_GRAPHS = {}


def _graph(name):
    if name not in _GRAPHS:
        _GRAPHS[name] = {"torus3d50": lambda: I.torus3d(50), "rreg1m_d3": lambda: I.random_regular(1_000_000, 3),
                         "rreg1m_d6": lambda: I.random_regular(1_000_000, 6),
                         "rreg1m_d12": lambda: I.random_regular(1_000_000, 12),
                         "torus1000": lambda: I.torus2d(1000)}[name]()
    return _GRAPHS[name]


_FOS = {}


def _oracle_fos(oracle, name, g):
    if name not in _FOS:
        ep, ev = oracle.build_fos(g)
        k, co = oracle.color(g, ep, ev)
        _FOS[name] = (ep, ev, k, co)
    return _FOS[name]


def _sample(p, seed):
    """Individuals 0 and p - 1 and one random individual of every population
    word of 32, so every word's lanes and bits are checked."""
    rng = np.random.default_rng(seed)
    words = (p + 31) // 32
    return sorted({0, p - 1, *[min(p - 1, 32 * w + int(rng.integers(32))) for w in range(words)]})


def _threads():
    import os
    return max(1, min(16, os.cpu_count() or 1))


def _state(P):
    pop, fit, fe = P.population()
    xe, _ = P.elite()
    return pop.cpu().numpy(), fit.cpu().numpy(), xe.cpu().numpy(), fe


@pytest.mark.parametrize("name,p", [("torus3d50", 128), ("torus3d50", 512), ("rreg1m_d3", 128), ("rreg1m_d3", 512),
                                    ("rreg1m_d6", 128), ("rreg1m_d6", 512), ("rreg1m_d12", 128),
                                    ("rreg1m_d12", 512), ("torus1000", 256)])
def test_full_size_sampled_generation(oracle, name, p):
    g = _graph(name)
    seed = 1
    P = gom.Population(g, p, seed)
    ep, ev, k, co = _oracle_fos(oracle, name, g)
    ex = gom.gom_fos_export(P.fos)
    assert P.k == k and np.array_equal(ex["color_of_elem"], co)
    assert np.array_equal(ex["elem_ptr"], ep) and np.array_equal(ex["elem_vars"], ev)

    sample = _sample(p, p + len(name))

    pop0, f0, xe0, fe0 = _state(P)
    for i in sample:  # InitializePopulation, sampled
        assert np.array_equal(pop0[i], oracle.init_individual(seed, i, g.n))
        assert f0[i] == oracle.cut_value(g, pop0[i])
    st1, _ = P.generation(1)
    pop1, f1, xe1, fe1 = _state(P)
    st2, _ = P.generation(1)
    pop2, f2, xe2, fe2 = _state(P)
    assert st2[0]["generation"] == 1 and st2[0]["trials"] == p * g.n

    run = oracle.Run(g, ep, ev, co, k, p, seed, init=False)
    run.load(pop1, f1, xe1, fe1, 1)
    run.generation(only=sample, threads=_threads())
    ref = run.get()
    for i in sample:
        assert np.array_equal(pop2[i], ref["pop"][i]), (name, p, i)
        assert f2[i] == ref["f"][i], (name, p, i)
        assert f2[i] == oracle.cut_value(g, pop2[i])

    # any-size properties over the whole population
    assert np.array_equal(P.fitness().cpu().numpy(), f2)
    assert np.all(f2 >= f1) and np.all(f1 >= f0)
    assert fe2 == max(fe1, int(f2.max())) and fe1 == max(fe0, int(f1.max()))
    assert oracle.cut_value(g, xe2) == fe2
    assert st2[0]["best_fitness"] == f2.max() and st2[0]["elite_fitness"] == fe2


@pytest.mark.parametrize("bitsliced", [False, True])
@pytest.mark.parametrize("name,p,late", [("rreg1m_d12", 512, 100), ("torus1000", 256, 100), ("torus3d50", 512, 150),
                                         ("rreg1m_d6", 128, 100)])
def test_full_size_late_generation(oracle, name, p, late, bitsliced):
    """A late generation (after `late` generations, the population partly
    converged): the oracle replays it from the GPU's exported state for one
    individual of every population word (and the first and last), bit for
    bit, on either mixing path."""
    g = _graph(name)
    P = gom.Population(g, p, 1)
    try:
        gom.gom_set_option(P.ctx, gom.GOM_OPT_BITSLICED, 1 if bitsliced else 0)
    except gom.GomError:
        pytest.skip("bit-sliced mixing unavailable")
    ep, ev, k, co = _oracle_fos(oracle, name, g)
    P.generation(late, want_stats=False)
    popA, fA, xeA, feA = _state(P)
    st, _ = P.generation(1)
    popB, fB, xeB, feB = _state(P)
    assert st[0]["generation"] == late
    sample = _sample(p, 7 * p + late)
    run = oracle.Run(g, ep, ev, co, k, p, 1, init=False)
    run.load(popA, fA, xeA, feA, late)
    run.generation(only=sample, threads=_threads())
    ref = run.get()
    for i in sample:
        assert np.array_equal(popB[i], ref["pop"][i]), (name, p, i)
        assert fB[i] == ref["f"][i], (name, p, i)
    assert np.array_equal(P.fitness().cpu().numpy(), fB)
    assert np.all(fB >= fA) and feB == max(feA, int(fB.max()))


def test_torus100_full_run(oracle):
    """2D torus 100x100, weights U[1,100], p = 64: to the closed-form optimum
    (every edge cut; bipartite torus) or 500 generations, bit for bit."""
    g = I.torus2d(100)
    target = g.total_weight()
    ep, ev = oracle.build_fos(g)
    k, co = oracle.color(g, ep, ev)
    run = oracle.Run(g, ep, ev, co, k, 64, 1)
    P = gom.Population(g, 64, 1)
    done = 0
    while done < 500:
        gst, nrun = P.generation(50, target)
        ost = run.run(50, target)
        assert nrun == len(ost)
        for a, b in zip(gst, ost):
            assert (a["generation"], a["best_fitness"], a["elite_fitness"], a["donorless"], a["accepted"],
                    a["improving"], a["reached_target"]) == (b["generation"], b["best"], b["elite"], b["donorless"],
                                                             b["accepted"], b["improving"], b["reached"])
        pop, fit, xe, fe = _state(P)
        ref = run.get()
        assert np.array_equal(pop, ref["pop"]) and np.array_equal(fit, ref["f"])
        assert np.array_equal(xe, ref["xe"]) and fe == ref["fe"]
        done += nrun
        if nrun < 50:
            break
