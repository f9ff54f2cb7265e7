"""Surface extraction on the GPU (mpm_extract_surface) against the oracle's
on the same FP32 density field: the same triangle count, and every triangle,
in order, within FP32 interpolation error.  The GPU surface of a ball of
particles is closed, consistently oriented and of Euler characteristic 2."""
import numpy as np
import pytest

import test_oracle_surface_pins as SP
from oracle import oracle as O
from paper_2402_01181_gb300 import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    import __graft_entry__ as ge
    ge.build()
    from paper_2402_01181_gb300 import mpm
    return mpm


def _oracle_triangles(sim, sc, iso):
    """The oracle's surface of the density the GPU computes: node mass times
    the FP32 scale 1 / (rho dx^3), rounded to FP32 as on the GPU."""
    g = sim.read_grid()                       # dense [i, j, k, (m, mv)]
    scale = np.float32(1.0 / (sc.rho * sc.dx ** 3))
    field = (g[..., 0].astype(np.float32) * scale).astype(np.float64)
    return O.surface(field, np.float32(iso), sc.dx)


@pytest.mark.parametrize("name,steps", [("block1m", 25), ("slab30k", 600)])
def test_surface_matches_oracle(M, name, steps):
    sc = scenes.SCENES[name]()
    sim = M.sim_from_scene(sc)
    tool = sc.tools[0]
    for s in range(0, steps, 25):
        sim.set_tool(0, tool.pose(s + 24), tool.shape)
        sim.step(25)
    got = sim.extract_surface(0.5)
    ref = _oracle_triangles(sim, sc, 0.5)
    sim.close()
    assert got.shape == ref.shape and got.shape[0] > 1000
    assert np.abs(got - ref).max() <= 4e-6


def test_gpu_surface_of_a_ball_is_closed(M):
    n = 64
    c, R = np.array([0.5013, 0.4487, 0.5209]), 0.2
    x = scenes.jittered_lattice((16, 14, 17), (48, 46, 49), n, (2, 2, 2), seed=5).astype(np.float64)
    x = x[np.linalg.norm(x - c, axis=1) < R]                # 8 particles per cell inside the ball
    sc = scenes.Scene("ball", n_grid=n, dt=1e-4, E=5e3, nu=0.3, rho=1e3, x=x.astype(np.float32),
                      particle_volume=(1.0 / n) ** 3 / 8)
    sim = M.sim_from_scene(sc)
    tri = sim.extract_surface(0.5).astype(np.float64)
    dev = sim.extract_surface(0.5, device=True).cpu().numpy().astype(np.float64)
    sim.close()
    assert np.array_equal(tri, dev)
    closed, chi = SP._closed_and_oriented(tri)
    assert closed and chi == 2
    r = np.linalg.norm(tri.reshape(-1, 3) - c, axis=1)
    assert abs(np.median(r) - R) < 2.0 / n                    # the density falls to 1/2 near the ball's edge
    nrm = SP._normals(tri)
    assert np.einsum("ij,ij->i", tri.mean(axis=1) - c, nrm).min() > 0


def test_surface_capacity_and_arguments(M):
    import ctypes as ct
    sc = scenes.cube8k()
    sim = M.sim_from_scene(sc)
    full = sim.extract_surface(0.5)
    part = np.zeros((10, 3, 3), np.float32)
    n_tri = ct.c_int64()
    M.check(M.mpm_extract_surface(sim.h, 0, 0.5, part.ctypes.data_as(ct.c_void_p), 10, ct.byref(n_tri), 0))
    assert n_tri.value == full.shape[0] and np.array_equal(part, full[:10])
    assert M.mpm_extract_surface(sim.h, 1, 0.5, None, 0, ct.byref(n_tri), 0) == M.MPM_ERR_ARG
    assert M.mpm_extract_surface(sim.h, 0, 0.5, None, 5, ct.byref(n_tri), 0) == M.MPM_ERR_ARG
    assert M.mpm_extract_surface(sim.h, 0, 0.5, None, 0, None, 0) == M.MPM_ERR_ARG
    sim.close()
