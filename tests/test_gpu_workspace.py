"""Runs whose device memory is a caller-supplied range (plse_bind_workspace):
a torch tensor sized by plse_workspace_size gives the same results as the
library's pool, a range too small fails cleanly with PLSE_ENOMEM, and the
handle keeps working after unbinding."""
import numpy as np
import pytest

from paper_2103_10453_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def plse():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2103_10453_gb300 import plse as P
    P.load()
    return P


@pytest.mark.parametrize("grid_fn,pop,gens", [(lambda: inputs.random_insertion(30, 0.5, 77), 96, 4),
                                              (lambda: inputs.n70(0.7), 320, 2)])
def test_torch_workspace_equals_pool(plse, grid_fn, pop, gens):
    import torch
    grid = grid_fn()
    A, B = plse.Instance(grid), plse.Instance(grid)
    for G in (A, B):
        G.set_params(plse.default_params(stop_at_bound=0))
    iters = 3 * A.nv
    need = B.workspace_size(pop, gens)
    assert need > pop * B.nv
    buf = torch.empty(need, dtype=torch.uint8, device="cuda")
    B.bind_workspace(buf)
    ra = A.solve(pop, gens, iters, 5, with_stats=True)
    rb = B.solve(pop, gens, iters, 5, with_stats=True)
    assert rb["score"] == ra["score"] and rb["walks"] == ra["walks"]
    assert np.array_equal(rb["best_grid"], ra["best_grid"])
    # a second run reuses the same range
    rb2 = B.solve(pop, gens, iters, 6, with_stats=True)
    ra2 = A.solve(pop, gens, iters, 6, with_stats=True)
    assert rb2["score"] == ra2["score"] and np.array_equal(rb2["best_grid"], ra2["best_grid"])
    # unbound: buffers come from the pool again
    B.bind_workspace(None)
    rb3 = B.solve(pop, gens, iters, 5, with_stats=True)
    assert rb3["walks"] == ra["walks"]
    del buf
    A.close()
    B.close()


def test_small_workspace_fails_cleanly(plse):
    import torch
    grid = inputs.random_insertion(24, 0.6, 41)
    G = plse.Instance(grid)
    need = G.workspace_size(64, 3)
    small = torch.empty(need // 2, dtype=torch.uint8, device="cuda")
    G.bind_workspace(small)
    with pytest.raises(plse.PlseError) as e:
        G.solve(64, 3, 100, 1)
    assert e.value.code == plse.PLSE_ENOMEM
    G.bind_workspace(None)
    res = G.solve(64, 3, 100, 1)                    # the handle still works
    assert res["score"] > 0
    with pytest.raises(plse.PlseError) as e:      # misaligned ranges are refused
        G.bind_workspace(small[1:], 1024)
    assert e.value.code == plse.PLSE_EINVAL
    G.close()
