"""mpm_block_sort_noalloc: the block sort for callers that may not allocate
device memory (their host owns the GPU's memory through its own pool or a
fixed budget), keeping its scratch in a static device array instead.

Its result must equal the existing path's -- mpm_load_particles followed by
mpm_read_order -- on two calls in a row (the second call must not see the
first call's counters).  This file is collected last so that a failure here
does not stop the other GPU tests."""
import ctypes as ct

import numpy as np
import pytest

from paper_2402_01181_gb300 import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    import __graft_entry__ as ge
    ge.build()
    from paper_2402_01181_gb300 import mpm
    return mpm


def _existing_order(M, sc):
    sim = M.sim_from_scene(sc)
    ids, keys = sim.read_order()
    sim.close()
    return ids, keys


def _noalloc_order(M, x, n_grid):
    import torch
    xd = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).cuda()
    n = x.shape[0]
    ids = torch.empty(n, dtype=torch.int32, device="cuda")
    keys = torch.empty(n, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    st = M.mpm_block_sort_noalloc(ct.c_void_p(xd.data_ptr()), n, n_grid, ct.c_void_p(ids.data_ptr()),
                                  ct.c_void_p(keys.data_ptr()), ct.c_void_p(stream.cuda_stream))
    assert st == M.MPM_OK, M.mpm_last_error()
    return ids.cpu().numpy().view(np.uint32), keys.cpu().numpy().view(np.uint32)


def test_noalloc_sort_matches_the_load_sort_twice(M):
    first = scenes.slab30k(seed=4)
    second = scenes.block1m(seed=5)          # larger grid: stale counters would show
    for sc in (first, second):
        ids_ref, keys_ref = _existing_order(M, sc)
        ids, keys = _noalloc_order(M, sc.x, sc.n_grid)
        assert np.array_equal(ids, ids_ref)
        assert np.array_equal(keys, keys_ref)


def test_noalloc_sort_rejects_oversized_grids(M):
    x = np.zeros((4, 3), np.float32)
    st = M.mpm_block_sort_noalloc(ct.c_void_p(1), 4, 512, ct.c_void_p(1), ct.c_void_p(1), None)
    assert st == M.MPM_ERR_ARG and "256" in M.mpm_last_error()
