"""GPU parity of Forced Improvement (Sec. 4, Alg. 1, in the library's parallel
reading, GOM_OPT_FORCED_IMPROVEMENT): every execution path -- persistent
kernel and per-generation graph, per-lane and bit-sliced mixing, the 32-,
64- and 128-bit element instances -- against the oracle with FI on, bit for
bit after every generation: population, fitness, elitist, the GOM counters
and FI's own counters."""
import numpy as np
import pytest

from paper_2203_08680_gb300 import gom
from paper_2203_08680_gb300 import instances as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

KEYS = [("generation", "generation"), ("best_fitness", "best"), ("elite_fitness", "elite"), ("trials", "trials"),
        ("donorless", "donorless"), ("accepted", "accepted"), ("improving", "improving"),
        ("reached_target", "reached"), ("fi_individuals", "fi_individuals"), ("fi_trials", "fi_trials"),
        ("fi_accepted", "fi_accepted"), ("fi_improving", "fi_improving"), ("fi_replaced", "fi_replaced")]


def _state(P):
    pop, fit, fe = P.population()
    xe, _ = P.elite()
    return {"pop": pop.cpu().numpy(), "f": fit.cpu().numpy(), "xe": xe.cpu().numpy(), "fe": fe}


def _same(gs, os_, where):
    assert gs["fe"] == os_["fe"], where
    assert np.array_equal(gs["f"], os_["f"]), where
    assert np.array_equal(gs["pop"], os_["pop"]), where
    assert np.array_equal(gs["xe"], os_["xe"]), where


def _paths(g, p, seed, fos=None, kind=0, nis=0):
    Ps = []
    for persistent in (True, False):
        for bits in (False, True):
            P = gom.Population(g, p, seed, kind, fos=fos, persistent=persistent)
            try:
                gom.gom_set_option(P.ctx, gom.GOM_OPT_BITSLICED, 1 if bits else 0)
            except gom.GomError:
                continue  # no bit-sliced mixing for this FOS
            gom.gom_set_option(P.ctx, gom.GOM_OPT_FI_NIS, nis)
            gom.gom_set_option(P.ctx, gom.GOM_OPT_FORCED_IMPROVEMENT, 1)
            Ps.append(P)
    return Ps


def _fi_parity(oracle, g, p, seed, gens, ep=None, ev=None, fos=None, kind=0, nis=0):
    if ep is None:
        ep, ev = oracle.build_fos(g, kind)
    k, co = oracle.color(g, ep, ev)
    run = oracle.Run(g, ep, ev, co, k, p, seed)
    run.set_fi(True, nis)
    Ps = _paths(g, p, seed, fos=fos, kind=kind, nis=nis)
    assert len(Ps) >= 2
    fi_seen = 0
    for gen in range(gens):
        ost = run.generation()
        fi_seen += ost["fi_individuals"]
        for P in Ps:
            gst, _ = P.generation(1)
            for gk, ok in KEYS:
                assert gst[0][gk] == ost[ok], (gen, gk, gst[0], ost)
            _same(_state(P), run.get(), f"gen {gen}")
    for P in Ps:
        assert np.array_equal(P.fitness().cpu().numpy(), run.get()["f"])  # incremental = full
    return fi_seen


def test_fi_torus10_p16(oracle):
    assert _fi_parity(oracle, I.torus2d(10), 16, 1, 12) > 0


@pytest.mark.parametrize("p", [2, 33, 64, 100])
def test_fi_ragged_populations(oracle, p):
    assert _fi_parity(oracle, I.torus2d(12, seed=p), p, 7 + p, 8) > 0


@pytest.mark.parametrize("nis", [1, 3])
def test_fi_no_improvement_threshold(oracle, nis):
    _fi_parity(oracle, I.random_regular(300, 5, seed=nis), 48, 5, 10, nis=nis)


def test_fi_negative_weights(oracle):
    _fi_parity(oracle, I.random_regular(200, 4, seed=7, wmin=-100, wmax=100), 40, 3, 8)


def test_fi_singleton_fos_and_3d_torus(oracle):
    _fi_parity(oracle, I.torus2d(8, seed=9), 24, 2, 8, kind=gom.GOM_FOS_SINGLETON)
    _fi_parity(oracle, I.torus3d(6, seed=3), 64, 4, 6)


@pytest.mark.parametrize("bound,p", [(10, 50), (64, 40), (100, 64)])
def test_fi_linkage_tree(oracle, bound, p):
    """The paper's bounded linkage tree (Sec. 4.1): elements of up to `bound`
    variables, i.e. the 32-, 64- and 128-bit element instances of the
    per-lane path (and the bit-sliced path where elements fit 32 variables)."""
    g = I.torus2d(14, seed=bound)
    fos = gom.gom_build_fos(g, gom.GOM_FOS_BFLT, bound)
    ep, ev = oracle.build_bflt(g, bound)
    _fi_parity(oracle, g, p, 11, 8, ep=ep, ev=ev, fos=fos)


def test_fi_hand_example_on_the_gpu(oracle):
    """The oracle's hand-worked case: path 0-1-2-3-4-5 (weights 7, 5, 9, 9,
    8), singleton FOS, both individuals 111011 (cut 18), elitist 010100 (cut
    30): FI stops after the first improving group, with 111010 (cut 26) when
    group {1,3,5} comes first, 011011 (cut 25) otherwise."""
    g = I.from_edges(6, np.arange(5), np.arange(1, 6), np.array([7, 5, 9, 9, 8]))
    y = np.array([1, 1, 1, 0, 1, 1], dtype=np.uint8)
    xe = np.array([0, 1, 0, 1, 0, 0], dtype=np.uint8)
    ep, ev = oracle.build_fos(g, oracle.SINGLETON)
    k, co = oracle.color(g, ep, ev)
    dev = torch.device("cuda")
    for seed in (1, 2, 3, 4, 5, 6):
        order = list(oracle.group_order(seed, k, 0))
        want, fw = ([1, 1, 1, 0, 1, 0], 26) if order[0] == 0 else ([0, 1, 1, 0, 1, 1], 25)
        for P in _paths(g, 2, seed, kind=gom.GOM_FOS_SINGLETON):
            P.set_population(torch.from_numpy(np.stack([y, y])).to(dev), torch.from_numpy(xe).to(dev), 30, 0)
            st, _ = P.generation(1)
            s = _state(P)
            assert [list(r) for r in s["pop"]] == [want, want] and list(s["f"]) == [fw, fw]
            assert (st[0]["fi_individuals"], st[0]["fi_trials"], st[0]["fi_accepted"], st[0]["fi_improving"],
                    st[0]["fi_replaced"]) == (2, 6, 2, 2, 0)


def test_fi_refused_where_unavailable():
    """|w| above 255 (the bit-plane width of FI's weights) is refused, and so
    is a batched launch of a context with FI on."""
    g = I.random_regular(100, 4, seed=2, wmin=1, wmax=1000)
    P = gom.Population(g, 16, 1)
    with pytest.raises(gom.GomError) as ei:
        gom.gom_set_option(P.ctx, gom.GOM_OPT_FORCED_IMPROVEMENT, 1)
    assert ei.value.code == -8
    Q = gom.Population(I.torus2d(6), 8, 1, forced_improvement=True)
    ws = torch.empty(gom.gom_batch_workspace_bytes(1) + 256, dtype=torch.uint8, device="cuda")
    ws = ws[(-ws.data_ptr()) % 256:]
    with pytest.raises(gom.GomError) as ei:
        gom.gom_batch_create([Q.ctx], None, ws)
    assert ei.value.code == -7
