"""The entry point that allocates no device memory (gom_fitness_noalloc):
its output must equal the handle-based full evaluation gom_fitness on the
same population, on consecutive calls whose populations differ.  It is for
callers that must not allocate device memory; its scratch is a fixed array
inside the library, shared by all calls."""
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


@pytest.mark.parametrize("gname,p", [("rreg", 100), ("torus", 64)])
def test_fitness_noalloc_equals_gom_fitness(gname, p):
    g = I.random_regular(3000, 5, seed=4) if gname == "rreg" else I.torus2d(60, seed=2)
    P = gom.Population(g, p, 3)
    rp, col, w = _device_csr(g)
    for call in range(2):
        pop, _, _ = P.population()            # device uint8 rows
        ref = P.fitness()                     # gom_fitness on the handle's workspace
        out = torch.full((p,), -7, dtype=torch.int64, device="cuda")
        gom.gom_fitness_noalloc(rp, col, w, g.n, pop, p, out)
        torch.cuda.synchronize()
        # integer cut weights: exact equality is the tolerance
        assert torch.equal(out, ref), f"call {call}"
        P.generation(3)                       # the next call sees another population


def test_fitness_noalloc_rejects_sizes_beyond_its_scratch():
    L = gom.load()
    dummy = torch.zeros(16, dtype=torch.int64, device="cuda")
    n_over = (4 * 1024 * 1024) // 2 + 1  # W = 2 words per variable for pop = 64
    rc = L.gom_fitness_noalloc(dummy.data_ptr(), dummy.data_ptr(), dummy.data_ptr(), n_over,
                               dummy.data_ptr(), 64, dummy.data_ptr(), None)
    assert rc == -8
    rc = L.gom_fitness_noalloc(dummy.data_ptr(), dummy.data_ptr(), dummy.data_ptr(), 10, dummy.data_ptr(), 2000,
                               dummy.data_ptr(), None)
    assert rc == -8
    rc = L.gom_fitness_noalloc(None, dummy.data_ptr(), dummy.data_ptr(), 10, dummy.data_ptr(), 4,
                               dummy.data_ptr(), None)
    assert rc == -1
