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


@pytest.mark.parametrize("persistent", [True, False])
def test_filter_log_mode_is_plain_and_filtered_mode_replays(oracle, persistent):
    g = I.torus2d(300, seed=31)
    p, seed = 64, 5
    P = gom.Population(g, p, seed, persistent=persistent)
    if persistent:  # the persistent path here stages one item at a time
        assert gom.gom_get_option(P.ctx, gom.GOM_OPT_PERSISTENT) == 1
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
    assert tr["samples"] == min(fs["log_count"], 1 << 16) and tr["recall"] >= 0.9
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


def test_filter_turns_itself_off_when_recall_drops(oracle):
    """A threshold above every logit skips every element; the audits find
    useful ones among them, the estimated recall falls below the minimum and
    the filter turns itself off: the next generations are plain GOM."""
    g = I.torus2d(300, seed=32)
    p, seed = 64, 6
    P = gom.Population(g, p, seed, persistent=False)
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
    P = gom.Population(I.torus2d(10), 16, 1, persistent=True)
    _attach(P, 1024)
    gom.gom_filter_set_mode(P.ctx, 1)
    with pytest.raises(gom.GomError):
        gom.gom_filter_set_mode(P.ctx, 2)
