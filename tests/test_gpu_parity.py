"""GPU parity: the CUDA path through the C ABI against the CPU oracle, bit for
bit (population, int64 fitness, elitist and counters), on seeded synthetic
instances small enough for the oracle, spanning several tiles and ragged
population words, plus the method's degenerate cases."""
import numpy as np
import pytest

from paper_2203_08680_gb300 import gom
from paper_2203_08680_gb300 import instances as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

STAT_KEYS = [("generation", "generation"), ("best_fitness", "best"), ("elite_fitness", "elite"),
             ("trials", "trials"), ("donorless", "donorless"), ("accepted", "accepted"),
             ("improving", "improving"), ("reached_target", "reached")]


def _oracle_run(oracle, g, p, seed, kind=0):
    ep, ev = oracle.build_fos(g, kind)
    k, co = oracle.color(g, ep, ev)
    return oracle.Run(g, ep, ev, co, k, p, seed), k


def _gpu_state(P):
    pop, fit, fe = P.population()
    xe, fe2 = P.elite()
    assert fe == fe2
    return {"pop": pop.cpu().numpy(), "f": fit.cpu().numpy(), "xe": xe.cpu().numpy(), "fe": fe}


def _assert_same_state(gs, os_, where=""):
    assert np.array_equal(gs["f"], os_["f"]), where
    assert gs["fe"] == os_["fe"], where
    assert np.array_equal(gs["pop"], os_["pop"]), where
    assert np.array_equal(gs["xe"], os_["xe"]), where


def _assert_same_stats(gst, ost):
    for gk, ok in STAT_KEYS:
        assert gst[gk] == ost[ok], (gk, gst, ost)


def _bitsliced_available(P) -> bool:
    try:
        gom.gom_set_option(P.ctx, gom.GOM_OPT_BITSLICED, 1)
        return True
    except gom.GomError:
        return False


def _populations(g, p, seed, kind=0):
    """Every execution path: the per-lane mixing and, where the FOS and the
    weights allow it, the bit-sliced mixing, each on the persistent kernel and
    on the per-generation graph (the graph with the other item schedule,
    static stride / dynamic claims, than the persistent default)."""
    A = gom.Population(g, p, seed, kind, persistent=True, bitsliced=False)
    dyn = gom.gom_get_option(A.ctx, gom.GOM_OPT_DYNAMIC)
    Ps = [A, gom.Population(g, p, seed, kind, persistent=False, dynamic=not dyn, bitsliced=False)]
    B = gom.Population(g, p, seed, kind, persistent=True)
    if _bitsliced_available(B):
        Ps += [B, gom.Population(g, p, seed, kind, persistent=False, dynamic=not dyn, bitsliced=True)]
    return Ps


def _parity(oracle, g, p, seed, gens, kind=0, check_every=1, target=gom.INT64_MAX):
    """Every execution path (_populations) against the oracle after every
    generation."""
    Ps = _populations(g, p, seed, kind)
    run, k = _oracle_run(oracle, g, p, seed, kind)
    for P in Ps:
        assert P.k == k
        _assert_same_state(_gpu_state(P), run.get(), "init")
    for gen in range(gens):
        ost = run.generation(target)
        for P in Ps:
            gst, nrun = P.generation(1, target)
            assert nrun == 1
            _assert_same_stats(gst[0], ost)
        if (gen + 1) % check_every == 0 or gen == gens - 1:
            for P in Ps:
                _assert_same_state(_gpu_state(P), run.get(), f"gen {gen}")
                # incremental fitness equals full re-evaluation on the device
                assert np.array_equal(P.fitness().cpu().numpy(), run.get()["f"])
    return Ps[0], run


def test_torus10_p16_every_generation(oracle):
    """2D torus 10x10, int32 weights U[1,100], p = 16, 20 generations, seed 1."""
    _parity(oracle, I.torus2d(10), 16, 1, 20)


def test_torus100_p64(oracle):
    """2D torus 100x100, weights U[1,100], p = 64 (oracle-sized run length)."""
    _parity(oracle, I.torus2d(100), 64, 1, 30, check_every=5)


@pytest.mark.parametrize("p", [2, 3, 31, 33, 100, 257])
def test_ragged_population_sizes(oracle, p):
    _parity(oracle, I.torus2d(9, seed=p), p, 11 + p, 6)


def test_torus3d_ragged(oracle):
    _parity(oracle, I.torus3d(8, seed=2), 100, 5, 8, check_every=2)


@pytest.mark.parametrize("d,p", [(3, 128), (6, 40), (12, 96)])
def test_random_regular(oracle, d, p):
    _parity(oracle, I.random_regular(2000, d, seed=d), p, 3, 5)


def test_singleton_fos(oracle):
    _parity(oracle, I.random_regular(500, 4, seed=1), 64, 2, 8, kind=gom.GOM_FOS_SINGLETON)


def test_negative_weights(oracle):
    _parity(oracle, I.random_regular(400, 5, seed=3, wmin=-100, wmax=100), 48, 9, 8)


def test_max_population(oracle):
    _parity(oracle, I.torus2d(6, seed=4), 1024, 21, 3)


def test_empty_graph_all_neutral(oracle):
    _parity(oracle, I.empty_graph(70), 40, 5, 3, kind=gom.GOM_FOS_SINGLETON)


def _pop(g, p, seed, bitsliced, **kw):
    """A population on the per-lane (bitsliced=False) or the bit-sliced mixing
    path; skips the test where the bit-sliced path is unavailable."""
    P = gom.Population(g, p, seed, **kw)
    if bitsliced and not _bitsliced_available(P):
        pytest.skip("bit-sliced path unavailable for this FOS")
    if not bitsliced:
        gom.gom_set_option(P.ctx, gom.GOM_OPT_BITSLICED, 0)
    return P


@pytest.mark.parametrize("bitsliced", [False, True])
def test_unit_weight_torus_reaches_closed_form(oracle, bitsliced):
    """Even torus, unit weights: the optimum is every edge cut (2 L^2); the
    target stop must match the oracle generation by generation."""
    g = I.torus2d(8, unit=True)
    target = 2 * 8 * 8
    P = _pop(g, 32, 3, bitsliced)
    run, _ = _oracle_run(oracle, g, 32, 3)
    gst, nrun = P.generation(200, target)
    ost = run.run(200, target)
    assert nrun == len(ost)
    for a, b in zip(gst, ost):
        _assert_same_stats(a, b)
    _assert_same_state(_gpu_state(P), run.get())
    if ost[-1]["reached"]:
        assert gst[-1]["best_fitness"] == target


@pytest.mark.parametrize("bitsliced", [False, True])
def test_target_stop_midway(oracle, bitsliced):
    g = I.torus2d(20, seed=3)
    run, _ = _oracle_run(oracle, g, 24, 4)
    probe = run.run(6)
    target = probe[3]["best"]  # reached at or before generation 3
    P = _pop(g, 24, 4, bitsliced)
    run2, _ = _oracle_run(oracle, g, 24, 4)
    gst, nrun = P.generation(10, target)
    ost = run2.run(10, target)
    assert nrun == len(ost) <= 4
    for a, b in zip(gst, ost):
        _assert_same_stats(a, b)
    _assert_same_state(_gpu_state(P), run2.get())
    # the next call starts from where this one stopped
    gst2, nrun2 = P.generation(2)
    ost2 = run2.run(2)
    assert nrun2 == 2
    for a, b in zip(gst2, ost2):
        _assert_same_stats(a, b)


def test_split_calls_equal_one_call():
    g = I.random_regular(1000, 4, seed=8)
    A = gom.Population(g, 64, 5)
    A.generation(12)
    B = gom.Population(g, 64, 5)
    for n in (3, 4, 5):
        B.generation(n)
    sa, sb = _gpu_state(A), _gpu_state(B)
    for key in ("pop", "f", "xe"):
        assert np.array_equal(sa[key], sb[key])
    assert sa["fe"] == sb["fe"] and A.generation_counter() == B.generation_counter() == 12


def test_async_calls_equal_sync_calls():
    g = I.torus2d(30, seed=2)
    A = gom.Population(g, 48, 6)
    A.generation(7)
    B = gom.Population(g, 48, 6)
    B.generation(7, want_stats=False)
    torch.cuda.synchronize()
    sa, sb = _gpu_state(A), _gpu_state(B)
    assert np.array_equal(sa["pop"], sb["pop"]) and np.array_equal(sa["f"], sb["f"])


@pytest.mark.parametrize("bitsliced", [False, True])
def test_resume_from_oracle_state(oracle, bitsliced):
    """Checkpoint/resume: a state written into the GPU continues exactly as the
    oracle continues from the same state."""
    g = I.random_regular(600, 5, seed=4)
    run, _ = _oracle_run(oracle, g, 40, 7)
    for _ in range(3):
        run.generation()
    s = run.get()
    P = _pop(g, 40, 7, bitsliced)
    dev = torch.device("cuda")
    P.set_population(torch.from_numpy(s["pop"]).to(dev), torch.from_numpy(s["xe"]).to(dev), s["fe"], s["g"])
    assert np.array_equal(P.fitness().cpu().numpy(), s["f"])
    for _ in range(4):
        gst, _ = P.generation(1)
        _assert_same_stats(gst[0], run.generation())
    _assert_same_state(_gpu_state(P), run.get())


@pytest.mark.parametrize("bitsliced", [False, True])
def test_identical_population_is_all_donorless(oracle, bitsliced):
    g = I.torus2d(12, seed=6)
    run, _ = _oracle_run(oracle, g, 36, 2)
    x = run.get()["pop"][5]
    pop = np.tile(x, (36, 1))
    fx = oracle.cut_value(g, x)
    P = _pop(g, 36, 2, bitsliced)
    dev = torch.device("cuda")
    P.set_population(torch.from_numpy(pop).to(dev), torch.from_numpy(x).to(dev), fx, 0)
    gst, _ = P.generation(1)
    assert gst[0]["donorless"] == gst[0]["trials"] == 36 * g.n
    assert gst[0]["accepted"] == 0
    assert np.array_equal(_gpu_state(P)["pop"], pop)


def test_timing_mode_keeps_results_and_counts_launches(oracle):
    g = I.torus2d(16, seed=7)
    A = gom.Population(g, 64, 8, persistent=False)
    gom.gom_set_timing(A.ctx, True)
    A.generation(5)
    ms, launches = gom.gom_read_timing(A.ctx)
    assert launches == 5 * A.k and ms > 0
    B = gom.Population(g, 64, 8)
    B.generation(5)
    sa, sb = _gpu_state(A), _gpu_state(B)
    assert np.array_equal(sa["pop"], sb["pop"]) and np.array_equal(sa["f"], sb["f"])
    assert gom.gom_launches_per_generation(A.ctx) == A.k + 3
    assert gom.gom_launches_per_generation(B.ctx) == (1 if gom.gom_get_option(B.ctx, gom.GOM_OPT_PERSISTENT) else A.k + 3)


def test_user_stream(oracle):
    g = I.torus2d(10)
    s = torch.cuda.Stream()
    P = gom.Population(g, 16, 1, stream=s)
    run, _ = _oracle_run(oracle, g, 16, 1)
    for _ in range(5):
        gst, _ = P.generation(1)
        _assert_same_stats(gst[0], run.generation())
    with torch.cuda.stream(s):
        st = _gpu_state(P)
    torch.cuda.synchronize()
    _assert_same_state(st, run.get())


def test_wide_elements_64bit_masks(oracle):
    """Elements of 41 variables: the kernel instance with 64-bit masks."""
    _parity(oracle, I.random_regular(300, 40, seed=5), 70, 4, 4)


def test_large_weights_64bit_deltas(oracle):
    """Sums of |w| above 2^30 per element: the instance with int64 deltas."""
    g = I.random_regular(500, 6, seed=6, wmin=-(2 ** 29), wmax=2 ** 29)
    _parity(oracle, g, 40, 8, 5)


def _overlapping_fos(n, seed):
    """Singletons, consecutive pairs and consecutive quads: overlapping
    elements of mixed sizes, as in a linkage tree (Sec. 4.1)."""
    sets = [[v] for v in range(n)]
    sets += [[v, v + 1] for v in range(0, n - 1, 2)]
    sets += [list(range(v, v + 4)) for v in range(0, n - 3, 4)]
    ep = np.cumsum([0] + [len(s) for s in sets]).astype(np.int64)
    ev = np.concatenate([np.array(s, dtype=np.int32) for s in sets])
    return ep, ev


@pytest.mark.parametrize("bitsliced", [False, True])
@pytest.mark.parametrize("p", [16, 100])
def test_custom_overlapping_fos(oracle, p, bitsliced):
    g = I.torus2d(8, seed=12)
    ep, ev = _overlapping_fos(g.n, 1)
    fos = gom.gom_fos_create(g.n, ep, ev)
    P = _pop(g, p, 13, bitsliced, fos=fos)
    k, co = oracle.color(g, ep, ev)
    assert P.k == k
    run = oracle.Run(g, ep, ev, co, k, p, 13)
    _assert_same_state(_gpu_state(P), run.get(), "init")
    for _ in range(6):
        gst, _ = P.generation(1)
        _assert_same_stats(gst[0], run.generation())
    _assert_same_state(_gpu_state(P), run.get())


@pytest.mark.parametrize("persistent", [True, False])
def test_long_call_target_stop_both_paths(oracle, persistent):
    """One call of many generations (the persistent kernel runs them all in
    one launch) stops at the same generation as the oracle."""
    g = I.torus2d(12, seed=9)
    run, _ = _oracle_run(oracle, g, 48, 2)
    probe = run.run(40)
    target = probe[25]["best"]
    P = gom.Population(g, 48, 2, persistent=persistent)
    run2, _ = _oracle_run(oracle, g, 48, 2)
    gst, nrun = P.generation(40, target)
    ost = run2.run(40, target)
    assert nrun == len(ost)
    for a, b in zip(gst, ost):
        _assert_same_stats(a, b)
    _assert_same_state(_gpu_state(P), run2.get())


def test_grid_barrier_bounded_wait():
    """Failure detection without a hang: a barrier that expects one arrival
    too many gives up after its wall-clock limit and reports it; the context
    stays usable."""
    scratch = torch.zeros(64, dtype=torch.uint8, device="cuda")
    assert gom.gom_selftest_barrier(scratch, 8, 0, 200_000_000) is False
    assert gom.gom_selftest_barrier(scratch, 8, 1, 50_000_000) is True
    assert gom.gom_selftest_barrier(scratch, 8, 0, 200_000_000) is False
    P = gom.Population(I.torus2d(6), 8, 1)
    P.generation(2)


@pytest.mark.parametrize("bitsliced", [False, True])
@pytest.mark.parametrize("dynamic", [False, True])
def test_large_groups_one_warp_per_element(oracle, dynamic, bitsliced):
    """Colour groups of ~20,000 elements: several items per warp, with either
    item schedule on the persistent path; per-lane mixing (one warp per
    element walking all its word groups) and bit-sliced mixing (an item of 8
    elements, one (element, word) pair per lane)."""
    g = I.torus2d(400, seed=12)
    P = _pop(g, 96, 6, bitsliced, persistent=True, dynamic=dynamic)
    run, _ = _oracle_run(oracle, g, 96, 6)
    for gen in range(3):
        ost = run.generation()
        gst, _ = P.generation(1)
        _assert_same_stats(gst[0], ost)
    _assert_same_state(_gpu_state(P), run.get(), "gen 3")


@pytest.mark.parametrize("p", [64, 200])
def test_runs_of_identical_individuals(oracle, p):
    """A population made of long runs of equal individuals: donor search
    passes whole runs of candidates equal to the parent and skips the parent's
    own column, exactly as the sequential cyclic scan does."""
    g = I.torus2d(14, seed=5)
    run, _ = _oracle_run(oracle, g, p, 3)
    base = run.get()["pop"]
    idx = np.repeat(np.arange(5), (p + 4) // 5)[:p]  # 5 runs of individuals 0..4
    pop = base[idx].copy()
    f = np.array([oracle.cut_value(g, x) for x in pop], dtype=np.int64)
    xe = pop[int(np.argmax(f))].copy()
    dev = torch.device("cuda")
    run.load(pop, f, xe, int(f.max()), 0)
    Ps = []
    for persistent in (True, False):
        for bitsliced in (False, True):
            P = gom.Population(g, p, 3, persistent=persistent, bitsliced=bitsliced)
            P.set_population(torch.from_numpy(pop).to(dev), torch.from_numpy(xe).to(dev), int(f.max()), 0)
            Ps.append(P)
    for _ in range(6):
        ost = run.generation()
        for P in Ps:
            gst, _ = P.generation(1)
            _assert_same_stats(gst[0], ost)
    for P in Ps:
        _assert_same_state(_gpu_state(P), run.get())


def _fos_parity(oracle, g, fos, ep, ev, p, seed, gens):
    """A given FOS (library handle and the oracle's arrays of the same sets)
    on both execution paths, the persistent one with either item schedule,
    against the oracle, every generation."""
    k, co = oracle.color(g, ep, ev)
    run = oracle.Run(g, ep, ev, co, k, p, seed)
    Ps = [gom.Population(g, p, seed, fos=fos, persistent=True, bitsliced=False),
          gom.Population(g, p, seed, fos=fos, persistent=False, bitsliced=False),
          gom.Population(g, p, seed, fos=fos, persistent=True, dynamic=False, bitsliced=False)]
    B = gom.Population(g, p, seed, fos=fos, persistent=True, dynamic=False)
    if _bitsliced_available(B):  # sets of at most 32 variables
        Ps += [B, gom.Population(g, p, seed, fos=fos, persistent=False, bitsliced=True)]
    for P in Ps:
        assert P.k == k
        _assert_same_state(_gpu_state(P), run.get(), "init")
    for gen in range(gens):
        ost = run.generation()
        for P in Ps:
            gst, _ = P.generation(1)
            _assert_same_stats(gst[0], ost)
            _assert_same_state(_gpu_state(P), run.get(), f"gen {gen}")
    for P in Ps:
        assert np.array_equal(P.fitness().cpu().numpy(), run.get()["f"])


@pytest.mark.parametrize("name,bound,p", [("torus12", 10, 50), ("rreg300_d5", 20, 100), ("rreg200_d4", 64, 40)])
def test_bflt_fos(oracle, name, bound, p):
    """The paper's own linkage model (Sec. 4.1): a bounded fixed linkage tree
    learned by UPGMA on the edge weights -- nested sets of 1 to `bound`
    variables (64: 64-bit masks) -- on both execution paths, every generation."""
    g = {"torus12": lambda: I.torus2d(12, seed=21), "rreg300_d5": lambda: I.random_regular(300, 5, seed=22),
         "rreg200_d4": lambda: I.random_regular(200, 4, seed=23)}[name]()
    fos = gom.gom_build_fos(g, gom.GOM_FOS_BFLT, bound)
    ep, ev = oracle.build_bflt(g, bound)
    _fos_parity(oracle, g, fos, ep, ev, p, 31, 6)


@pytest.mark.parametrize("name,bound,p", [("torus20", 100, 50), ("rreg400_d4", 100, 100), ("rreg300_d6", 128, 200)])
def test_bflt_paper_bound_100_128bit_masks(oracle, name, bound, p):
    """The paper's larger linkage-tree bound (100, Sec. 6.1) and the library's
    maximum (128): sets of 65 to 128 variables take the kernel instance with
    128-bit masks (at most two population words per item; p = 50, 100, 200
    give 2, 4 and 8 words; p = 200 runs in block mode), on both execution
    paths, every generation."""
    g = {"torus20": lambda: I.torus2d(20, seed=51), "rreg400_d4": lambda: I.random_regular(400, 4, seed=52),
         "rreg300_d6": lambda: I.random_regular(300, 6, seed=53)}[name]()
    fos = gom.gom_build_fos(g, gom.GOM_FOS_BFLT, bound)
    ep, ev = oracle.build_bflt(g, bound)
    assert np.diff(ep).max() > 64
    _fos_parity(oracle, g, fos, ep, ev, p, 32, 6)


@pytest.mark.parametrize("p", [33, 96, 300, 1024])
def test_elements_of_128_variables(oracle, p):
    """Elements at the library's maximum of 128 variables, next to elements of
    65 and 100 variables that overlap them, and the singletons: variables
    0..127 of a random 5-regular graph in one element, so that lanes hold up
    to four variables each and edges run inside and out of every quarter.
    p = 300 and 1024 (5 and 16 two-word groups per element) run in block mode:
    the warps of a block stage each element once and share its word groups."""
    g = I.random_regular(400, 5, seed=61)
    sets = [[v] for v in range(g.n)]
    sets += [list(range(0, 128)), list(range(128, 228)), list(range(300, 365)), list(range(100, 165)),
             list(range(272, 400))]
    ep = np.cumsum([0] + [len(x) for x in sets]).astype(np.int64)
    ev = np.concatenate([np.array(x, dtype=np.int32) for x in sets])
    fos = gom.gom_fos_create(g.n, ep, ev)
    _fos_parity(oracle, g, fos, ep, ev, p, 62, 8)


def test_no_learned_filter_for_elements_above_64_variables():
    """The learned filter's kernel instances take elements of up to 64
    variables: switching it on for a larger FOS is refused, plain GOM goes on."""
    g = I.random_regular(300, 6, seed=53)
    P = gom.Population(g, 64, 3, fos=gom.gom_build_fos(g, gom.GOM_FOS_BFLT, 100))
    ws = torch.empty(gom.gom_filter_workspace_bytes(P.ctx, 1024) + 256, dtype=torch.uint8, device="cuda")
    ws = ws[(-ws.data_ptr()) % 256:]
    gom.gom_filter_attach(P.ctx, ws, 1024)
    with pytest.raises(gom.GomError) as ei:
        gom.gom_filter_set_mode(P.ctx, 1)
    assert ei.value.code == -8
    P.generation(2)
