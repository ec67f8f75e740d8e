"""The no-allocation local search (plse_local_search_noalloc) against the
regular entry point (plse_local_search), through the C ABI, two calls in a row.

The variant exists for callers that cannot allocate device memory at call time
(a fixed device-memory budget owned by their own allocator, or a loop that must
not stall on cudaMalloc/cudaFree); it keeps its scratch in a fixed array inside
the library.  Results are integers, so the comparison is exact, as in the other
local-search tests.  This file is collected last on purpose."""
import numpy as np
import pytest

from paper_2103_10453_gb300 import inputs
from _gpu import dev, empty, host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def plse():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2103_10453_gb300 import plse as P
    P.load()
    return P


def run(G, fn, P, ind0, gen, iters, seed, flags):
    import torch
    count = P.shape[0]
    S_out = empty(P.shape, torch.uint8)
    f = empty((count,), torch.int32)
    F = empty((count,), torch.int64)
    st = empty((count, 7), torch.int64)
    getattr(G, fn)(dev(P), S_out, count, ind0, gen, iters, seed, flags, f, F, st)
    G.sync()
    return host(S_out), host(f), host(F), host(st)


@pytest.mark.parametrize("grid_fn", [lambda: inputs.random_insertion(24, 0.6, 41),
                                     lambda: inputs.n70(0.7)])
def test_noalloc_matches_local_search_twice(plse, oracle_mod, grid_fn):
    grid = grid_fn()
    G = plse.Instance(grid)
    I = oracle_mod.Instance(grid)
    flags = plse.LS_PHASE1 | plse.LS_PHASE2 | plse.LS_REPAIR
    for call in range(2):                       # two calls in a row share the scratch array
        count = 300 + 37 * call
        P = I.init_population(count, 100 + call)
        iters = min(3 * I.nv, 4000)
        a = run(G, "local_search", P, 7 * call, call, iters, 5 + call, flags)
        b = run(G, "local_search_noalloc", P, 7 * call, call, iters, 5 + call, flags)
        for x, y in zip(a, b):
            assert np.array_equal(x, y), call
