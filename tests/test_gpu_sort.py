"""The load-time stable block sort on dense scenes, where every 4^3-cell
block holds more particles than one shared-memory sort takes (2,048): the
segments are sorted in chunks and merged.  Its order must equal the oracle's
stable counting sort (O.sorted_order of O.block_keys) bit for bit, and its
time must grow with n, not with n times the number of blocks."""
import time

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


def _scene(cells, sub, seed, n_grid=128):
    lo = (n_grid - cells) // 2
    x = scenes.jittered_lattice((lo, 8, lo), (lo + cells, 8 + cells, lo + cells), n_grid, sub, seed)
    rng = np.random.default_rng(seed + 1)
    x = x[rng.permutation(x.shape[0])]          # ids in random spatial order
    return scenes.Scene("dense", n_grid=n_grid, dt=2e-5, E=1e4, nu=0.3, rho=1e3, x=x,
                        particle_volume=(1.0 / n_grid) ** 3 / float(np.prod(sub)))


def _load_time_and_order(M, sc):
    import torch
    sim = M.sim_from_scene(sc, load=False)
    xd = torch.tensor(sc.x, device="cuda")
    torch.cuda.synchronize()
    sim.load(xd, sc.particle_volume)            # warm: kernels loaded, buffers touched
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sim.load(xd, sc.particle_volume)
    sim.synchronize()
    dt = time.perf_counter() - t0
    ids, keys = sim.read_order()
    sim.close()
    return dt, ids, keys


def test_dense_load_sort_is_the_stable_counting_sort(M):
    """1M particles at 64 per cell (4,096 per block: two chunks and a merge)
    and a 128-per-cell block region (8,192 per block: two merge passes)."""
    for cells, sub in (((25, (4, 4, 4))), ((16, (8, 4, 4)))):
        sc = _scene(cells, sub, seed=cells)
        _, ids, keys = _load_time_and_order(M, sc)
        k = O.block_keys(sc.n_grid, sc.x)
        ref = O.sorted_order(k)
        assert np.array_equal(ids, ref.astype(np.uint32))
        assert np.array_equal(keys, k[ref])
        per_block = np.bincount(k)
        assert per_block.max() > 2048


def test_dense_load_time_is_linear(M):
    """Loading 1M particles at 64 per cell costs about 4x what 250K do, not
    the 16x of a scan of all particles per crowded block."""
    t_small, _, _ = _load_time_and_order(M, _scene(16, (4, 4, 4), seed=3))     # 262K particles
    t_big, _, _ = _load_time_and_order(M, _scene(25, (4, 4, 4), seed=4))       # 1M particles
    assert t_big < 8.0 * t_small + 0.02, (t_small, t_big)
