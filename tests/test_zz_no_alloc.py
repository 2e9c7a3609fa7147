"""The entry point that allocates no device memory (gom_fitness_noalloc).

It is for callers that must not allocate device memory: cudaMalloc can
synchronise the device and fail under memory pressure, and some host
programs hand out all device memory through their own allocator.  Its
scratch is a fixed array inside the library, shared by all calls.

Each individual's output must equal the oracle's full evaluation of its cut
weight (integer arithmetic: exact equality is the tolerance), on two calls in
a row whose populations differ; the population sizes cover one word of 32
individuals up to 32 words, and one graph has negative weights.  The same
populations also go through the handle-based gom_fitness.
"""
import numpy as np
import pytest

from paper_2203_08680_gb300 import gom
from paper_2203_08680_gb300 import instances as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)


def _device_csr(g):
    dev = torch.device("cuda")
    return (torch.from_numpy(g.row_ptr).to(dev), torch.from_numpy(g.col).to(dev),
            torch.from_numpy(g.weight).to(dev))


GRAPHS = {
    "rreg": lambda: I.random_regular(3000, 5, seed=4),
    "torus": lambda: I.torus2d(60, seed=2),
    "rreg_negative": lambda: I.random_regular(2000, 6, seed=7, wmin=-100, wmax=100),
}


@pytest.mark.parametrize("gname,p", [("torus", 20), ("torus", 64), ("rreg", 100), ("rreg", 300),
                                     ("rreg_negative", 257), ("torus", 1024)])
def test_fitness_noalloc_equals_oracle(oracle, gname, p):
    g = GRAPHS[gname]()
    P = gom.Population(g, p, 3)
    rp, col, w = _device_csr(g)
    for call in range(2):
        pop, _, _ = P.population()            # device uint8 rows
        out = torch.full((p,), -7, dtype=torch.int64, device="cuda")
        gom.gom_fitness_noalloc(rp, col, w, g.n, pop, p, out)
        torch.cuda.synchronize()
        hpop = pop.cpu().numpy()
        want = np.array([oracle.cut_value(g, hpop[i]) for i in range(p)], dtype=np.int64)
        got = out.cpu().numpy()
        assert np.array_equal(got, want), f"call {call}: first mismatch at {np.flatnonzero(got != want)[:5]}"
        assert torch.equal(out, P.fitness()), f"call {call}"
        P.generation(3)                       # the next call sees another population


GOM_E_ARG, GOM_E_LIMIT = -1, -8  # include/gom.h


def test_fitness_noalloc_rejects_bad_arguments():
    L = gom.load()
    dummy = torch.zeros(16, dtype=torch.int64, device="cuda")
    d = dummy.data_ptr()
    n_over = (4 * 1024 * 1024) // 2 + 1  # W = 2 words per variable for pop = 64
    assert L.gom_fitness_noalloc(d, d, d, n_over, d, 64, d, None) == GOM_E_LIMIT
    assert L.gom_fitness_noalloc(d, d, d, 10, d, 2000, d, None) == GOM_E_LIMIT
    for k in range(5):  # each pointer null in turn
        ptrs = [d] * 5
        ptrs[k] = None
        rp, col, wt, pp, out = ptrs
        assert L.gom_fitness_noalloc(rp, col, wt, 10, pp, 4, out, None) == GOM_E_ARG
    assert L.gom_fitness_noalloc(d, d, d, 0, d, 4, d, None) == GOM_E_ARG
