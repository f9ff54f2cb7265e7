"""Host-side checks of the C ABI that need no GPU: the library loads, it
exports every entry point include/mpm.h declares, and argument validation
rejects bad calls before touching CUDA."""
import ctypes as ct
import os
import re

import pytest

import __graft_entry__ as ge

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    ge.build()
    from paper_2402_01181_gb300 import mpm
    return mpm


def declared_functions():
    txt = open(os.path.join(ROOT, "include", "mpm.h")).read()
    return sorted(set(re.findall(r"^\s*(?:mpm_status|const char \*)\s*(mpm_\w+)\s*\(", txt, re.M)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for core in ("mpm_create", "mpm_load_particles", "mpm_set_tool_pose", "mpm_step", "mpm_read_particles",
                 "mpm_destroy", "mpm_last_error"):
        assert core in names


def test_library_exports_every_declared_symbol(lib):
    so = ct.CDLL(lib._build.library_path())
    for name in declared_functions():
        assert hasattr(so, name), name
    bound = {s[0] for s in lib.SIGNATURES}
    assert set(declared_functions()) == bound


def test_config_struct_matches_header(lib):
    # offsets follow the C layout of mpm_config (int64 at the end is 8-aligned)
    c = lib.mpm_config
    assert c.n_envs.offset == 48 and c.max_particles.offset == 56 and ct.sizeof(c) == 64


def test_argument_validation_without_gpu(lib):
    h = ct.c_void_p()
    st = lib.mpm_create(None, None, lib.mpm_alloc_fn(), lib.mpm_free_fn(), None, ct.byref(h))
    assert st == lib.MPM_ERR_ARG and "NULL" in lib.mpm_last_error()
    for bad in (dict(n_grid=30), dict(n_grid=4), dict(dt=0.0), dict(nu=0.5), dict(rho=-1.0),
                dict(pipeline=7), dict(max_particles=0), dict(bound=40)):
        kw = dict(n_grid=32, dt=1e-4, E=1e3, nu=0.3, rho=1e3, max_particles=10)
        kw.update(bad)
        cfg = lib.make_config(**kw)
        st = lib.mpm_create(ct.byref(cfg), None, lib.mpm_alloc_fn(), lib.mpm_free_fn(), None, ct.byref(h))
        assert st == lib.MPM_ERR_ARG, bad
    assert lib.mpm_step(None, 1) == lib.MPM_ERR_ARG
    fid = ct.c_int32(-1)
    o = (ct.c_double * 3)()
    assert lib.mpm_add_sampled_field(None, 4, o, 0.1, None, 0, ct.byref(fid)) == lib.MPM_ERR_ARG
    assert lib.mpm_set_kernel_config(None, 0) == lib.MPM_ERR_ARG
    assert lib.mpm_autotune(None, 1, None, None) == lib.MPM_ERR_ARG
    assert lib.mpm_tape_record(None, 1, None, 1) == lib.MPM_ERR_ARG
    assert lib.mpm_tape_backward(None, None, None, None, None, 0, None, None, None, None, None, None) == lib.MPM_ERR_ARG
    n_tri = ct.c_int64()
    assert lib.mpm_extract_surface(None, 0, 0.5, None, 0, ct.byref(n_tri), 0) == lib.MPM_ERR_ARG
    assert lib.mpm_read_particles_async(None, None, None, None, None) == lib.MPM_ERR_ARG
    assert lib.mpm_wait_read(None) == lib.MPM_ERR_ARG
    assert lib.mpm_get_kernel_config(None, None, None, None) == lib.MPM_ERR_ARG
    assert lib.mpm_destroy(None) == lib.MPM_ERR_ARG
    assert lib.mpm_read_particles(None, None, None, None, None, 0) == lib.MPM_ERR_ARG
