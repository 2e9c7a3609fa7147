"""Interleaved Multi-start Scheme (Sec. 6.3) on the GPU: every population of
the scheme follows its own oracle run for its share of generations (P_i makes
floor(T / c^i) generations when P_0 has made T), and the first reach of a
target is the one the scheme's sequential order gives, replayed with the
oracle."""
import numpy as np
import pytest

from paper_2203_08680_gb300 import gom
from paper_2203_08680_gb300 import instances as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)


def _ims(g, base, c, maxp, seed):
    fos = gom.gom_build_fos(g)
    gom.gom_color_fos(g, fos)
    nb = gom.gom_ims_workspace_bytes(g, fos, base, maxp)
    ws = torch.empty(nb + 256, dtype=torch.uint8, device="cuda")
    ws = ws[(-ws.data_ptr()) % 256:]
    return gom.gom_ims_create(g, fos, base, c, maxp, seed, ws)


def _ctx_state(ctx, n, p):
    pop = torch.empty((p, n), dtype=torch.uint8, device="cuda")
    fit = torch.empty(p, dtype=torch.int64, device="cuda")
    xe = torch.empty(n, dtype=torch.uint8, device="cuda")
    fe = gom.gom_get_population(ctx, pop, fit, True)
    gom.gom_get_elite(ctx, xe, False)
    return {"pop": pop.cpu().numpy(), "f": fit.cpu().numpy(), "xe": xe.cpu().numpy(), "fe": fe}


def _oracle(oracle, g, p, seed):
    ep, ev = oracle.build_fos(g)
    k, co = oracle.color(g, ep, ev)
    return oracle.Run(g, ep, ev, co, k, p, seed)


def test_ims_populations_follow_oracle(oracle):
    g = I.torus2d(10, seed=4)
    base, c, maxp, seed = 4, 4, 64, 3
    ims = _ims(g, base, c, maxp, seed)
    L = gom.gom_ims_num_populations(ims)
    assert L == 5
    r = gom.gom_ims_run(ims, 30)
    assert r["steps"] == 30 and not r["reached"]
    r = gom.gom_ims_run(ims, 41)
    assert r["steps"] == 71
    for i in range(L):
        p = base << i
        gens = 71 // c ** i
        run = _oracle(oracle, g, p, seed + i)
        run.run(gens)
        ctx = gom.gom_ims_population(ims, i)
        assert gom.gom_get_generation(ctx) == gens
        st = _ctx_state(ctx, g.n, p)
        ref = run.get()
        for key in ("pop", "f", "xe"):
            assert np.array_equal(st[key], ref[key]), (i, key)
        assert st["fe"] == ref["fe"]


def test_ims_first_reach_in_scheme_order(oracle):
    """The sequential scheme replayed with the oracle: after P_0's generation
    T, P_1 makes one if c divides T, then P_2 if c^2 does, ...; the first
    generation whose best reaches the target fixes (step, population)."""
    g = I.random_regular(120, 4, seed=6)
    base, c, maxp, seed = 4, 2, 32, 9
    L = 4
    runs = [_oracle(oracle, g, base << i, seed + i) for i in range(L)]
    events = []  # (step, population, best)
    for T in range(1, 41):
        for i in range(L):
            if T % c ** i:
                break
            st = runs[i].generation()
            events.append((T, i, st["best"]))
    target = max(b for _, _, b in events)
    first = next((T, i) for T, i, b in events if b >= target)
    ims = _ims(g, base, c, maxp, seed)
    r = gom.gom_ims_run(ims, 40, target)
    assert r["reached"] == 1
    assert (r["reached_step"], r["reached_population"]) == first
    assert r["best_fitness"] >= target


def test_ims_on_the_linkage_tree(oracle):
    """The scheme over the paper's bounded linkage tree FOS (Sec. 4.1 and 6.3 together)."""
    g = I.torus2d(9, seed=8)
    base, c, maxp, seed = 8, 2, 32, 4
    fos = gom.gom_build_fos(g, gom.GOM_FOS_BFLT, 16)
    gom.gom_color_fos(g, fos)
    nb = gom.gom_ims_workspace_bytes(g, fos, base, maxp)
    ws = torch.empty(nb + 256, dtype=torch.uint8, device="cuda")
    ws = ws[(-ws.data_ptr()) % 256:]
    ims = gom.gom_ims_create(g, fos, base, c, maxp, seed, ws)
    gom.gom_ims_run(ims, 12)
    ep, ev = oracle.build_bflt(g, 16)
    k, co = oracle.color(g, ep, ev)
    for i in range(gom.gom_ims_num_populations(ims)):
        p = base << i
        run = oracle.Run(g, ep, ev, co, k, p, seed + i)
        run.run(12 // c ** i)
        st = _ctx_state(gom.gom_ims_population(ims, i), g.n, p)
        ref = run.get()
        assert np.array_equal(st["pop"], ref["pop"]) and np.array_equal(st["f"], ref["f"]) and st["fe"] == ref["fe"]
