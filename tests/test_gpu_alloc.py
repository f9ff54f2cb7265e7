"""Allocation failure through the allocator callback of mpm_create.

The failure is made on the host: a callback that returns NULL on its k-th
call.  mpm_create must then return MPM_ERR_ALLOC, hand every buffer it had
already received back to the free callback (no leak, no double free), and
leave nothing behind that stops a later mpm_create with a working allocator
from succeeding and stepping a scene."""
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


class _CountingAllocator:
    """Torch caching-allocator callbacks that fail on call number fail_at
    (1-based; 0 = never) and record every pointer handed out and freed."""

    def __init__(self, M, fail_at=0):
        import torch
        self.calls = 0
        self.live = {}
        self.freed = []
        self.double_free = 0
        dev = torch.cuda.current_device()
        stream = torch.cuda.current_stream(dev)

        def _alloc(nbytes, s, ctx):
            self.calls += 1
            if self.calls == fail_at:
                return None
            p = torch.cuda.caching_allocator_alloc(int(nbytes), dev, stream)
            self.live[p] = int(nbytes)
            return p

        def _free(ptr, s, ctx):
            if ptr not in self.live:
                self.double_free += 1
                return
            del self.live[ptr]
            self.freed.append(ptr)
            torch.cuda.caching_allocator_delete(ptr)

        self.a = M.mpm_alloc_fn(_alloc)
        self.f = M.mpm_free_fn(_free)


def _create(M, cfg, alloc):
    import torch
    h = ct.c_void_p()
    st = M.mpm_create(ct.byref(cfg), ct.c_void_p(torch.cuda.current_stream().cuda_stream), alloc.a, alloc.f, None,
                      ct.byref(h))
    return st, h


@pytest.mark.parametrize("pipeline", ["fused", "split"])
def test_allocation_failure_releases_everything(M, pipeline):
    sc = scenes.cube8k()
    pl = M.MPM_PIPELINE_FUSED if pipeline == "fused" else M.MPM_PIPELINE_SPLIT
    cfg = M.make_config(sc.n_grid, sc.dt, sc.E, sc.nu, sc.rho, pipeline=pl, max_particles=sc.n)
    ok = _CountingAllocator(M)
    st, h = _create(M, cfg, ok)
    assert st == M.MPM_OK, M.mpm_last_error()
    total = ok.calls
    assert total >= 10 and len(ok.live) == total
    assert M.mpm_destroy(h) == M.MPM_OK
    assert not ok.live and ok.double_free == 0
    for k in sorted({1, 2, 3, total // 2, total - 1, total}):
        bad = _CountingAllocator(M, fail_at=k)
        st, h = _create(M, cfg, bad)
        assert st == M.MPM_ERR_ALLOC, (k, st, M.mpm_last_error())
        assert not h.value                                 # no handle is returned
        assert "NULL" in M.mpm_last_error()
        assert bad.calls == k                              # it stops at the first failure
        assert not bad.live, (k, len(bad.live))            # every earlier buffer was freed ...
        assert len(bad.freed) == k - 1 and bad.double_free == 0   # ... exactly once
    # a working allocator afterwards: the scene loads and steps
    good = _CountingAllocator(M)
    st, h = _create(M, cfg, good)
    assert st == M.MPM_OK, M.mpm_last_error()
    x = np.ascontiguousarray(sc.x, dtype=np.float32)
    assert M.mpm_load_particles(h, sc.n, x.ctypes.data_as(ct.c_void_p), None, None, None,
                                ct.c_float(sc.particle_volume), 0) == M.MPM_OK, M.mpm_last_error()
    assert M.mpm_step(h, 5) == M.MPM_OK, M.mpm_last_error()
    out = np.empty((sc.n, 3), np.float32)
    assert M.mpm_read_particles(h, out.ctypes.data_as(ct.c_void_p), None, None, None, 0) == M.MPM_OK
    assert np.isfinite(out).all() and (out[:, 1] < sc.x[:, 1]).all()     # it fell
    assert M.mpm_destroy(h) == M.MPM_OK
    assert not good.live and good.double_free == 0
