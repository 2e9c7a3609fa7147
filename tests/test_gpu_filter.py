"""The learned trial filter on the GPU.  Mode 1 (history and training log)
leaves GOM bit for bit equal to the oracle.  In mode 2 the MLP skips the
trials of some elements; the oracle replays each filtered generation with the
same elements left out and must agree bit for bit (every kept change is still
decided by exact integer partial evaluation).  The audits turn the filter off
when its estimated recall drops."""
import numpy as np
import pytest

from paper_2203_08680_gb300 import gom
from paper_2203_08680_gb300 import instances as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from test_gpu_parity import _assert_same_state, _gpu_state, _oracle_run  # noqa: E402

STAT_KEYS = [("best_fitness", "best"), ("elite_fitness", "elite"), ("donorless", "donorless"),
             ("accepted", "accepted"), ("improving", "improving"), ("trials", "trials")]


def _attach(P, cap=1 << 16):
    nb = gom.gom_filter_workspace_bytes(P.ctx, cap)
    ws = torch.empty(nb + 256, dtype=torch.uint8, device="cuda")
    ws = ws[(-ws.data_ptr()) % 256:]
    gom.gom_filter_attach(P.ctx, ws, cap)


def _same_stats(a, o):
    for gk, ok in STAT_KEYS:
        assert a[gk] == o[ok], (gk, a, o)


def _mixing_path(P, bitsliced):
    """Selects the per-lane or the bit-sliced mixing path (skips the test
    where the bit-sliced one is unavailable)."""
    try:
        gom.gom_set_option(P.ctx, gom.GOM_OPT_BITSLICED, 1 if bitsliced else 0)
    except gom.GomError:
        pytest.skip("bit-sliced mixing unavailable")


@pytest.mark.parametrize("bitsliced", [False, True])
@pytest.mark.parametrize("persistent", [True, False])
def test_filter_log_mode_is_plain_and_filtered_mode_replays(oracle, persistent, bitsliced):
    """Mode 1 is plain GOM; in mode 2 the select phase skips elements (on the
    bit-sliced path the mixing runs only the compacted list of the others) and
    the oracle, replaying each generation without the marked elements, agrees
    bit for bit."""
    g = I.torus2d(300, seed=31)
    p, seed = 64, 5
    P = gom.Population(g, p, seed, persistent=persistent)
    if persistent:  # the persistent path here stages one item at a time
        assert gom.gom_get_option(P.ctx, gom.GOM_OPT_PERSISTENT) == 1
    _mixing_path(P, bitsliced)
    _attach(P)
    gom.gom_filter_set_mode(P.ctx, 1)
    run, _ = _oracle_run(oracle, g, p, seed)
    for gen in range(6):
        gst, _ = P.generation(1)
        ost = run.generation()
        _same_stats(gst[0], ost)
    _assert_same_state(_gpu_state(P), run.get(), "mode 1")
    fs = gom.gom_filter_stats(P.ctx)
    assert fs["log_count"] > 1000 and fs["last"]["skipped"] == 0
    tr = gom.gom_filter_train(P.ctx, epochs=150, learning_rate=0.02, pos_weight=1.0, target_recall=0.9)
    assert tr["samples"] == min(fs["log_count"], 1 << 16)
    gom.gom_filter_configure(P.ctx, tr["threshold"], 0.9, 0.0)  # never turns itself off here
    gom.gom_filter_set_mode(P.ctx, 2)
    skipped_any = False
    for gen in range(4):
        gst, _ = P.generation(1)
        mask = gom.gom_filter_skipped(P.ctx, P.m)
        skipped_any |= bool(mask.any())
        ost = run.generation_skip(mask)
        _same_stats(gst[0], ost)
        _assert_same_state(_gpu_state(P), run.get(), f"mode 2 gen {gen}")
        assert np.array_equal(P.fitness().cpu().numpy(), run.get()["f"])
    fs = gom.gom_filter_stats(P.ctx)
    assert fs["enabled"] == 1 and fs["total"]["skipped"] > 0 and skipped_any


@pytest.mark.parametrize("bitsliced", [False, True])
def test_filter_turns_itself_off_when_recall_drops(oracle, bitsliced):
    """A threshold above every logit skips every element; the audits find
    useful ones among them, the estimated recall falls below the minimum and
    the filter turns itself off: the next generations are plain GOM."""
    g = I.torus2d(300, seed=32)
    p, seed = 64, 6
    P = gom.Population(g, p, seed, persistent=False)
    _mixing_path(P, bitsliced)
    _attach(P)
    gom.gom_filter_set_mode(P.ctx, 1)
    P.generation(3)
    gom.gom_filter_train(P.ctx, epochs=20)
    gom.gom_filter_configure(P.ctx, 1e30, 0.9, 0.5)
    gom.gom_filter_set_mode(P.ctx, 2)
    P.generation(2)  # two generations under min_recall
    fs = gom.gom_filter_stats(P.ctx)
    assert fs["enabled"] == 0 and fs["disabled_at"] == 4
    assert fs["last"]["audited"] > 0 and fs["last"]["audited_useful"] > 0
    # plain from here: the next generation skips nothing
    P.generation(1)
    assert gom.gom_filter_stats(P.ctx)["last"]["skipped"] == 0
    assert not gom.gom_filter_skipped(P.ctx, P.m).any()


def test_filter_refused_in_stage_all_mode():
    """The stage-all mode does not keep P, which the change marks read."""
    P = gom.Population(I.torus2d(10), 16, 1, persistent=True)
    _attach(P, 1024)
    for mode in (1, 2):
        with pytest.raises(gom.GomError):
            gom.gom_filter_set_mode(P.ctx, mode)


# ---------------------------------------------------------------------------
# The filter's arithmetic against plain restatements of its definitions

def _bf16_bits(f):
    """Round float32 values to bf16 (round to nearest even), as bit patterns."""
    u = np.asarray(f, dtype=np.float32).view(np.uint32).astype(np.uint64)
    return ((u + 0x7FFF + ((u >> 16) & 1)) >> 16).astype(np.uint16)


def _bf16_value(bits):
    return (np.asarray(bits, dtype=np.uint32) << 16).view(np.float32)


def _sampled(q, g):
    """The library's choice of logged elements: one in 32 per generation by a
    hash of (colour-order position q, generation g)."""
    m32 = 0xFFFFFFFF
    h = ((q * 0xCC9E2D51) & m32) ^ ((g * 0x1B873593) & m32)
    h ^= h >> 16
    h = (h * 0x85EBCA6B) & m32
    h ^= h >> 13
    return (h & 31) == 0


def _element_structure(g, ep, ev):
    """Per element: size, edges to variables outside it, edges inside it (once each)."""
    m = len(ep) - 1
    size, nout, nin = np.zeros(m, np.int64), np.zeros(m, np.int64), np.zeros(m, np.int64)
    for j in range(m):
        F = ev[ep[j]:ep[j + 1]]
        pos = {int(v): a for a, v in enumerate(F)}
        size[j] = len(F)
        for a, u in enumerate(F):
            for x in range(g.row_ptr[u], g.row_ptr[u + 1]):
                b = pos.get(int(g.col[x]))
                if b is None:
                    nout[j] += 1
                elif b > a:
                    nin[j] += 1
    return size, nout, nin


def _element_neighbours(g, ep, ev):
    """Per element: its variables, and the far end of each of its outside edges."""
    m = len(ep) - 1
    out = []
    for j in range(m):
        F = ev[ep[j]:ep[j + 1]]
        inside = set(int(v) for v in F)
        nb = [int(g.col[x]) for u in F for x in range(g.row_ptr[u], g.row_ptr[u + 1]) if int(g.col[x]) not in inside]
        out.append((np.asarray(F, dtype=np.int64), np.asarray(nb, dtype=np.int64)))
    return out


@pytest.mark.parametrize("bitsliced", [False, True])
def test_filter_log_features_and_labels_match_an_oracle_replay(oracle, bitsliced):
    """Every logged sample -- the 16 features of an element at the start of a
    generation and its label (the element accepted a trial in that
    generation) -- equals the restatement of the feature definitions from
    the oracle's run: element structure, the element's accepted, donor-less
    and improving trials of the previous generation, log2(1 + g), the
    population's rates of the previous generation, the fractions of its
    variables and outside edges whose variable changed in some individual
    during the previous generation, and its quiet count (generations in a row
    with no accepted trial and no such change, up to 16).  p = 32, so one
    per-lane item is one element and the label covers all its trials."""
    g = I.torus2d(60, seed=41)
    p, seed, G = 32, 7, 8
    P = gom.Population(g, p, seed, persistent=False)
    _mixing_path(P, bitsliced)
    _attach(P, 1 << 14)
    gom.gom_filter_set_mode(P.ctx, 1)
    P.generation(G)
    x_gpu, y_gpu = gom.gom_filter_log(P.ctx)
    ep, ev = oracle.build_fos(g)
    k, co = oracle.color(g, ep, ev)
    run = oracle.Run(g, ep, ev, co, k, p, seed)
    run.keep_element_counts(True)
    by_pos = np.concatenate([np.flatnonzero(co == c) for c in range(k)])  # colour-order position -> element
    size, nout, nin = _element_structure(g, ep, ev)
    nbrs = _element_neighbours(g, ep, ev)
    f32 = np.float32
    inv_p = f32(1) / f32(p)
    prev = (np.zeros(len(by_pos), np.int64),) * 3
    prev_st = None
    quiet = np.zeros(len(by_pos), np.int64)
    pop_prev = None  # the population at the start of the previous generation
    rows = []
    for gen in range(G):
        pop_now = run.get()["pop"]
        changed = (pop_now != pop_prev).any(axis=0) if pop_prev is not None else np.zeros(g.n, bool)
        dF = np.array([int(changed[F].sum()) for F, _ in nbrs])
        dN = np.array([int(changed[nb].sum()) for _, nb in nbrs])
        quiet = np.where((prev[0] == 0) & (dF == 0) & (dN == 0), np.minimum(quiet + 1, 255), 0)
        st = run.generation()
        acc, dl, imp = run.element_counts()
        for q, j in enumerate(by_pos):
            if not _sampled(q, gen):
                continue
            x = np.zeros(16, dtype=np.float32)
            x[0], x[1], x[2] = f32(size[j]) / f32(16), f32(nout[j]) / f32(64), f32(nin[j]) / f32(32)
            pa, pd, pi = prev[0][j], prev[1][j], prev[2][j]
            x[3], x[4], x[5] = f32(pa) * inv_p, f32(pd) * inv_p, f32(pi) * inv_p
            x[6], x[7] = f32(pa == 0), f32(pd >= p)
            x[8] = np.log2(f32(1 + gen)) / f32(16)
            if prev_st is not None:
                tr = f32(prev_st["trials"])
                x[9], x[10], x[11] = (f32(prev_st["accepted"]) / tr, f32(prev_st["improving"]) / tr,
                                      f32(prev_st["donorless"]) / tr)
            x[12] = 1
            x[13] = f32(dF[j]) / f32(size[j])
            x[14] = f32(dN[j]) / f32(nout[j]) if nout[j] > 0 else f32(0)
            x[15] = f32(min(quiet[j], 16)) / f32(16)
            rows.append(tuple(_bf16_bits(x)) + (int(acc[j] > 0),))
        prev, prev_st, pop_prev = (acc, dl, imp), st, pop_now
    got = sorted(tuple(int(v) for v in r) + (int(l),) for r, l in zip(x_gpu, y_gpu))
    assert len(got) == len(rows) > 100
    assert got == sorted(rows)
    assert 0 < sum(r[-1] for r in rows) < len(rows)  # both labels occur
    assert any(r[13] or r[14] for r in rows) and any(r[15] for r in rows)  # the new features vary


def _forward64(theta, xb):
    """fp64 forward pass with the kernels' bf16-rounded W1 and W2; returns the
    logits, the hidden pre-activations and the bf16 weights."""
    W1 = _bf16_value(_bf16_bits(theta[:1024])).astype(np.float64).reshape(64, 16)
    b1 = theta[1024:1088].astype(np.float64)
    W2 = _bf16_value(_bf16_bits(theta[1088:1152])).astype(np.float64)
    b2 = float(theta[1152])
    x = _bf16_value(xb).astype(np.float64)
    z = x @ W1.T + b1
    a = np.maximum(z, 0.0)
    return a @ W2 + b2, z, x, W1, W2, a


def _filter_with_log(seed=3):
    g = I.torus2d(120, seed=43)
    P = gom.Population(g, 64, seed, persistent=False)
    _attach(P, 1 << 14)
    gom.gom_filter_set_mode(P.ctx, 1)
    P.generation(6)
    x, y = gom.gom_filter_log(P.ctx)
    assert len(y) > 1000 and 0 < y.sum() < len(y)
    return P, x, y


def test_filter_logits_match_an_fp64_restatement():
    """The logits (as the mixing kernels compute them: bf16 W1 and W2, fp32
    sums) equal the fp64 forward pass of the same bf16 weights to fp32
    accuracy: |difference| <= 1e-5 of the sum of the terms' magnitudes."""
    P, x, y = _filter_with_log()
    gom.gom_filter_train(P.ctx, epochs=30, learning_rate=0.02)
    theta = gom.gom_filter_get_params(P.ctx)["theta"]
    got = gom.gom_filter_logits(P.ctx, len(y)).astype(np.float64)
    want, z, xx, W1, W2, a = _forward64(theta, x)
    scale = np.abs(a) @ np.abs(W2) + abs(float(theta[1152])) + (np.abs(xx) @ np.abs(W1).T).max(axis=1)
    assert np.all(np.abs(got - want) <= 1e-5 * scale + 1e-7)


def test_filter_gradient_and_adam_step_match_a_restatement():
    """One training step from given parameters: the full-batch gradient (sum
    over the log of the weighted logistic loss's gradient, forward pass with
    bf16-rounded W1 and W2) against an fp64 restatement, to fp32 summation
    accuracy (1e-4 of the summed magnitudes); the mean loss to 1e-5
    relative; the Adam step (beta1 0.9, beta2 0.999, eps 1e-8, step 1) on the
    returned gradient against an fp32 restatement."""
    P, x, y = _filter_with_log(seed=4)
    rng = np.random.default_rng(5)
    theta0 = (rng.standard_normal(1153) * 0.2).astype(np.float32)
    gom.gom_filter_set_params(P.ctx, theta0)
    lr, pw = np.float32(0.01), 2.0
    loss = gom.gom_filter_epoch(P.ctx, float(lr), pw, 1)
    got = gom.gom_filter_get_params(P.ctx)
    out, z, xx, W1, W2, a = _forward64(theta0, x)
    t = y.astype(np.float64)
    wt = np.where(y > 0, pw, 1.0)
    sig = 1.0 / (1.0 + np.exp(-out))
    d = wt * (sig - t)
    dz = (z > 0) * d[:, None] * W2[None, :]
    want = np.concatenate([(dz.T @ xx).ravel(), dz.sum(0), a.T @ d, [d.sum()]])
    mag = np.concatenate([(np.abs(dz).T @ np.abs(xx)).ravel(), np.abs(dz).sum(0), np.abs(a).T @ np.abs(d),
                          [np.abs(d).sum()]])
    assert np.all(np.abs(got["grad"] - want) <= 1e-4 * mag + 1e-6)
    want_loss = np.mean(wt * (np.log1p(np.exp(-np.abs(out))) + np.maximum(out, 0) - t * out))
    assert abs(loss - want_loss) <= 1e-5 * abs(want_loss)
    # Adam, step 1, on the kernel's own gradient, in fp32: beta1 and beta2 are
    # the fp32 values nearest 0.9 and 0.999, and 1 - beta is taken in fp32
    f32 = np.float32
    b1, b2 = f32(0.9), f32(0.999)
    gm = got["grad"].astype(np.float32) * (f32(1) / f32(len(y)))
    m1 = (f32(1) - b1) * gm
    v1 = (f32(1) - b2) * gm * gm
    th1 = theta0 - lr * (m1 / (f32(1) - b1)) / (np.sqrt(v1 / (f32(1) - b2)) + f32(1e-8))
    assert np.allclose(got["adam_m"], m1, rtol=2e-6, atol=1e-12)
    assert np.allclose(got["adam_v"], v1, rtol=2e-6, atol=1e-18)
    assert np.allclose(got["theta"], th1, rtol=1e-6, atol=1e-6 * float(lr))


def test_filter_training_lowers_the_loss():
    """Adam steps on the log lower the mean loss: after 100 steps it is well
    below the loss at the initial parameters."""
    P, x, y = _filter_with_log(seed=6)
    rng = np.random.default_rng(8)
    gom.gom_filter_set_params(P.ctx, (rng.standard_normal(1153) * 0.2).astype(np.float32))
    losses = [gom.gom_filter_epoch(P.ctx, 0.02, 1.0, step) for step in range(1, 101)]
    assert losses[-1] < 0.8 * losses[0]
