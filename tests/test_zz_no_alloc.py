"""mpm_block_sort_noalloc: the block sort for callers that may not allocate
device memory (their host owns the GPU's memory through its own pool or a
fixed budget), keeping its scratch in a static device array instead.

Its result must equal the stable counting sort of the oracle
(O.sorted_order of O.block_keys) and the existing path's -- mpm_load_particles
followed by mpm_read_order -- on calls in a row (a later call must not see an
earlier call's counters), at the largest grid it accepts (256^3, where the
block offsets reach the end of the static array), and after a call that
failed on a non-finite or out-of-grid position.  This file is collected last
so that a failure here does not stop the other GPU tests."""
import ctypes as ct

import numpy as np
import pytest

from oracle import oracle as O
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


def _noalloc_call(M, x, n_grid):
    import torch
    xd = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).cuda()
    n = x.shape[0]
    ids = torch.empty(n, dtype=torch.int32, device="cuda")
    keys = torch.empty(n, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    st = M.mpm_block_sort_noalloc(ct.c_void_p(xd.data_ptr()), n, n_grid, ct.c_void_p(ids.data_ptr()),
                                  ct.c_void_p(keys.data_ptr()), ct.c_void_p(stream.cuda_stream))
    return st, ids.cpu().numpy().view(np.uint32), keys.cpu().numpy().view(np.uint32)


def _noalloc_order(M, x, n_grid):
    st, ids, keys = _noalloc_call(M, x, n_grid)
    assert st == M.MPM_OK, M.mpm_last_error()
    return ids, keys


def _oracle_order(x, n_grid):
    k = O.block_keys(n_grid, x)
    ids = O.sorted_order(k)
    return ids.astype(np.uint32), k[ids]


def test_noalloc_sort_matches_the_load_sort_twice(M):
    first = scenes.slab30k(seed=4)
    second = scenes.block1m(seed=5)          # larger grid: stale counters would show
    for sc in (first, second):
        ids_ref, keys_ref = _existing_order(M, sc)
        ids, keys = _noalloc_order(M, sc.x, sc.n_grid)
        ids_o, keys_o = _oracle_order(sc.x, sc.n_grid)
        assert np.array_equal(ids, ids_o)
        assert np.array_equal(keys, keys_o)
        assert np.array_equal(ids, ids_ref)
        assert np.array_equal(keys, keys_ref)


def test_noalloc_sort_on_the_largest_grid(M):
    """n_grid = 256 (64^3 blocks, the capacity of the static array): particles
    spread over the whole interior plus a dense cluster of 5,000 in one block
    (a segment larger than the in-shared-memory sort takes), twice."""
    rng = np.random.default_rng(31)
    spread = rng.uniform(0.02, 0.98, size=(300_000, 3))
    cluster = 0.5 + rng.uniform(0.0, 4.0 / 256, size=(5_000, 3))
    x = np.concatenate([spread, cluster]).astype(np.float32)
    x = x[rng.permutation(x.shape[0])]
    ids_o, keys_o = _oracle_order(x, 256)
    assert keys_o.max() > 60 ** 3                     # the last blocks of the array are in use
    for _ in range(2):
        ids, keys = _noalloc_order(M, x, 256)
        assert np.array_equal(ids, ids_o)
        assert np.array_equal(keys, keys_o)


def test_noalloc_sort_reports_bad_positions_and_recovers(M):
    sc = scenes.slab30k(seed=6)
    ids_o, keys_o = _oracle_order(sc.x, sc.n_grid)
    bad = sc.x.copy()
    bad[123, 1] = np.nan
    st, _, _ = _noalloc_call(M, bad, sc.n_grid)
    assert st == M.MPM_ERR_NUMERIC, M.mpm_last_error()
    ids, keys = _noalloc_order(M, sc.x, sc.n_grid)     # the next call starts clean
    assert np.array_equal(ids, ids_o) and np.array_equal(keys, keys_o)
    out = sc.x.copy()
    out[7] = (1.5, 0.5, 0.5)                           # outside the grid: its stencil is clamped
    st, _, _ = _noalloc_call(M, out, sc.n_grid)
    assert st == M.MPM_ERR_DOMAIN, M.mpm_last_error()
    ids, keys = _noalloc_order(M, sc.x, sc.n_grid)
    assert np.array_equal(ids, ids_o) and np.array_equal(keys, keys_o)


def test_noalloc_sort_rejects_oversized_grids(M):
    st = M.mpm_block_sort_noalloc(ct.c_void_p(1), 4, 512, ct.c_void_p(1), ct.c_void_p(1), None)
    assert st == M.MPM_ERR_ARG and "256" in M.mpm_last_error()
