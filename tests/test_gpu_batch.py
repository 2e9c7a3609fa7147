"""Batched GOM on the GPU: many instances in one persistent launch, each bit
for bit equal to the CPU oracle run of that instance alone (population,
int64 fitness, elitist and per-generation counters), whatever the batch
configuration, with per-instance targets, after autotuning, and when batched
calls and single-instance calls alternate."""
import numpy as np
import pytest

from paper_2203_08680_gb300 import gom
from paper_2203_08680_gb300 import instances as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from test_gpu_parity import _assert_same_state, _assert_same_stats, _gpu_state, _oracle_run  # noqa: E402

# (graph, population, seed): uneven sizes, degrees, ragged population words,
# p = 2, wide elements (a 40-variable star centre) and an empty graph
_MIX = [
    (lambda: I.torus2d(9, seed=3), 17, 5),
    (lambda: I.random_regular(300, 3, seed=4), 64, 6),
    (lambda: I.random_regular(500, 8, seed=5), 100, 7),
    (lambda: I.torus3d(6, seed=6), 2, 8),
    (lambda: I.random_regular(1200, 5, seed=7), 256, 9),
    (lambda: I.torus2d(20, seed=8), 33, 10),
    (lambda: I.empty_graph(40), 31, 11),
    (lambda: I.random_regular(64, 4, seed=9), 129, 12),
]


def _star(n_leaves, seed):
    u = np.zeros(n_leaves, dtype=np.int64)
    v = np.arange(1, n_leaves + 1, dtype=np.int64)
    w = I.edge_weights(u, v, seed)
    return I.from_edges(n_leaves + 1, u, v, w, f"star{n_leaves}")


def _instances(mix, extra_wide=False):
    items = [(f(), p, s) for f, p, s in mix]
    if extra_wide:
        items.append((_star(40, 3), 48, 13))
    return items


def _populations(items):
    return [gom.Population(g, p, s) for g, p, s in items]


def _batch(pops, config=None):
    ws = torch.empty(gom.gom_batch_workspace_bytes(len(pops)) + 256, dtype=torch.uint8, device="cuda")
    off = (-ws.data_ptr()) % 256
    ws = ws[off:]
    return gom.gom_batch_create([P.ctx for P in pops], config, ws)


def _check_against_oracle(oracle, items, pops, batch, gens, targets=None):
    """Runs the oracle of every instance for the generations its batched run
    did and compares counters and state."""
    if targets is None:
        targets = [gom.INT64_MAX] * len(items)
    for b, ((g, p, s), P) in enumerate(zip(items, pops)):
        run, k = _oracle_run(oracle, g, p, s)
        assert P.k == k
        ost = run.run(gens, targets[b])
        gst = gom.gom_batch_stats(batch, b, gens)
        assert len(gst) == len(ost), (b, len(gst), len(ost))
        for a, o in zip(gst, ost):
            _assert_same_stats(a, o)
        _assert_same_state(_gpu_state(P), run.get(), f"instance {b}")


@pytest.mark.parametrize("config", [None, (1, 2), (8, 3), (2, 3)])
def test_batch_equals_oracle_per_instance(oracle, config):
    items = _instances(_MIX, extra_wide=True)
    pops = _populations(items)
    batch = _batch(pops, config)
    runs = gom.gom_batch_generation(batch, 5)
    assert list(runs) == [5] * len(items)
    _check_against_oracle(oracle, items, pops, batch, 5)
    # every instance has its own blocks, and they tile the grid
    spans = [gom.gom_batch_layout(batch, b) for b in range(len(items))]
    assert spans[0][0] == 0
    for (b0, nb, grid), (b1, _, _) in zip(spans, spans[1:]):
        assert nb >= 1 and b0 + nb == b1
    assert spans[-1][0] + spans[-1][1] == spans[-1][2]


@pytest.mark.parametrize("config", [(4, 2), (8, 2), (1, 2)])
@pytest.mark.parametrize("share", ["all", "half"])
def test_batch_bitsliced_instances_equal_oracle(oracle, config, share):
    """Instances on the bit-sliced phase inside the batched launch (the
    kernel with the larger register budget): every instance where it is
    available ("all"), or every other one ("half", the rest per lane), each
    bit for bit equal to its own oracle run."""
    items = _instances(_MIX, extra_wide=True)
    pops = _populations(items)
    on = 0
    for b, P in enumerate(pops):
        want = 1 if share == "all" or b % 2 == 0 else 0
        try:
            gom.gom_set_option(P.ctx, gom.GOM_OPT_BITSLICED, want)
            on += want
        except gom.GomError:
            pass  # not available for this instance (the 40-variable star)
    assert on >= 3
    batch = _batch(pops, config)
    runs = gom.gom_batch_generation(batch, 6)
    assert list(runs) == [6] * len(items)
    _check_against_oracle(oracle, items, pops, batch, 6)


def test_batch_per_instance_targets(oracle):
    """Instance b stops after the first generation reaching targets[b];
    the others go on."""
    items = _instances(_MIX[:5])
    # targets: from an oracle run, the best fitness of generation 2 (reached
    # at generation <= 2), an unreachable one, and no target
    targets = []
    for b, (g, p, s) in enumerate(items):
        run, _ = _oracle_run(oracle, g, p, s)
        st = run.run(3)
        targets.append(st[1]["best"] if b % 2 == 0 else 2 ** 62)
    pops = _populations(items)
    batch = _batch(pops)
    runs = gom.gom_batch_generation(batch, 6, targets)
    for b, (g, p, s) in enumerate(items):
        run, _ = _oracle_run(oracle, g, p, s)
        ost = run.run(6, targets[b])
        assert runs[b] == len(ost)
        assert ost[-1]["reached"] == (b % 2 == 0)
        gst = gom.gom_batch_stats(batch, b, 6)
        for a, o in zip(gst, ost):
            _assert_same_stats(a, o)
        _assert_same_state(_gpu_state(pops[b]), run.get(), f"instance {b}")


def test_batch_and_single_calls_alternate(oracle):
    """Batched generations, then single-instance generations (both paths),
    then batched again: every instance follows its own oracle run."""
    items = _instances(_MIX[:4])
    pops = _populations(items)
    batch = _batch(pops, (2, 3))
    gom.gom_batch_generation(batch, 2)
    for P in pops[:2]:
        P.generation(1)
    for P in pops[2:]:
        gom.gom_set_option(P.ctx, gom.GOM_OPT_PERSISTENT, 0)
        P.generation(1)
    gom.gom_batch_generation(batch, 2)
    for b, ((g, p, s), P) in enumerate(zip(items, pops)):
        run, _ = _oracle_run(oracle, g, p, s)
        run.run(5)
        _assert_same_state(_gpu_state(P), run.get(), f"instance {b}")
        assert gom.gom_get_generation(P.ctx) == 5


def test_autotune_changes_no_result(oracle):
    items = _instances(_MIX[:6])
    pops = _populations(items)
    ctxs = [P.ctx for P in pops]
    scratch = torch.empty(gom.gom_batch_scratch_bytes(ctxs) + 256, dtype=torch.uint8, device="cuda")
    scratch = scratch[(-scratch.data_ptr()) % 256:]
    cfgs = [(1, 2), (2, 3), (4, 3), (8, 2)]
    best, ms = gom.gom_batch_autotune(ctxs, cfgs, 2, scratch)
    assert 0 <= best < len(cfgs) and ms[best] > 0 and all(m > 0 for m in ms)
    for P in pops:
        assert gom.gom_get_generation(P.ctx) == 0
    batch = _batch(pops, cfgs[best])
    gom.gom_batch_generation(batch, 3)
    _check_against_oracle(oracle, items, pops, batch, 3)


def test_batch_arguments():
    items = _instances(_MIX[:2])
    pops = _populations(items)
    with pytest.raises(gom.GomError):
        _batch([pops[0], pops[0]])  # the same context twice
    with pytest.raises(gom.GomError):
        _batch(pops, (3, 3))  # 3 warps per block
    with pytest.raises(gom.GomError):
        _batch(pops, (4, 5))
    batch = _batch(pops)
    assert list(gom.gom_batch_generation(batch, 0)) == [0, 0]


def test_batch_256_instances_full_size_sampled(oracle):
    """The 256-instance batch of random d-regular graphs (n log-uniform in
    [1000, 65536], d in 3..8, p in {32, 64, 128, 256}): one batched
    generation, then the oracle replays it for a sample of instances
    (including the largest), bit for bit; every instance's incremental
    fitness equals its full re-evaluation."""
    mix = I.batch_mix()
    graphs = [I.random_regular(n, d, s) for n, d, p, s in mix]
    pops = [gom.Population(g, p, s) for g, (n, d, p, s) in zip(graphs, mix)]
    batch = _batch(pops)
    runs = gom.gom_batch_generation(batch, 1)
    assert list(runs) == [1] * len(mix)
    big = int(np.argmax([n * p for n, d, p, s in mix]))
    for b in sorted({0, 101, 203, big}):
        n, d, p, s = mix[b]
        run, _ = _oracle_run(oracle, graphs[b], p, s)
        ost = run.run(1)
        _assert_same_stats(gom.gom_batch_stats(batch, b, 1)[0], ost[0])
        _assert_same_state(_gpu_state(pops[b]), run.get(), f"instance {b}")
    for b, P in enumerate(pops):
        pop, fit, fe = P.population()
        assert np.array_equal(P.fitness().cpu().numpy(), fit.cpu().numpy()), b


@pytest.mark.parametrize("config", [(2, 3), (4, 2)])
def test_batch_with_linkage_tree_instances(oracle, config):
    """Instances whose FOS is the paper's bounded linkage tree (nested sets of
    up to 32, 64, 100 and 128 variables: all three mask widths, the last with
    p = 300 in block mode) next to neighbourhood ones, in one launch."""
    specs = [(I.random_regular(200, 4, seed=41), 40, 3, 32), (I.torus2d(12, seed=42), 70, 4, 64),
             (I.random_regular(300, 3, seed=43), 33, 5, 0), (I.random_regular(400, 4, seed=52), 100, 6, 100),
             (I.torus2d(20, seed=51), 50, 7, 100), (I.random_regular(300, 6, seed=53), 300, 8, 128)]
    pops, runs = [], []
    for g, p, s, bound in specs:
        fos = gom.gom_build_fos(g, gom.GOM_FOS_BFLT, bound) if bound else None
        pops.append(gom.Population(g, p, s, fos=fos))
        if bound:
            ep, ev = oracle.build_bflt(g, bound)
        else:
            ep, ev = oracle.build_fos(g)
        k, co = oracle.color(g, ep, ev)
        runs.append(oracle.Run(g, ep, ev, co, k, p, s))
    batch = _batch(pops, config)
    assert list(gom.gom_batch_generation(batch, 4)) == [4] * len(specs)
    for b, (P, run) in enumerate(zip(pops, runs)):
        ost = run.run(4)
        for a, o in zip(gom.gom_batch_stats(batch, b, 4), ost):
            _assert_same_stats(a, o)
        _assert_same_state(_gpu_state(P), run.get(), f"instance {b}")
