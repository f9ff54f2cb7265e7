"""Every configuration of the fused sub-step kernel (CTA size x passes per
shared-memory P2G flush) against the FP64 oracle and the bit-exact sort
order, and the autotuner: it picks one of them, reports a time for each, and
leaves the particle state as it found it."""
import numpy as np
import pytest

import helpers as H
from oracle import oracle as O
from paper_2402_01181_gb300 import scenes

pytestmark = pytest.mark.gpu

CONFIGS = [0, 1, 2, 3, 4]


@pytest.fixture(scope="module")
def M():
    import __graft_entry__ as ge
    ge.build()
    from paper_2402_01181_gb300 import mpm
    return mpm


def _tool_scene(seed=0):
    sc = H.perturbed_scene(scenes.cube8k(seed), seed=seed + 1)
    cap = scenes.capsule_shape(0.06, 0.08)
    p0 = np.array([0.47, 0.57, 0.51, 0.3, 0.1, 0.2])
    vel = np.array([0.2, -1.5, 0.1, 20.0, -10.0, 5.0])
    sc.tools = [scenes.Tool(cap, lambda s: p0 + vel * sc.dt * (s + 1))]
    sc.friction = 0.4
    return sc


@pytest.mark.parametrize("config", CONFIGS)
def test_each_kernel_config_single_substep_parity(M, config):
    sc = _tool_scene(seed=7)
    sim = M.sim_from_scene(sc)
    sim.set_kernel_config(config)
    assert sim.kernel_config()["config"] == config
    start = sim.read()
    sim.set_tool(0, sc.tools[0].pose(0), sc.tools[0].shape)
    sim.step(1)
    out = sim.read()
    sim.close()
    st = H.oracle_state(start)
    mask = H.contact_mask_nodes(sc, st, 0)
    skip = H.particles_touching(mask, st.x, sc.n_grid)
    H.oracle_steps(sc, st, 0, 1, call_len=1)
    assert mask.sum() <= 5
    ok, errs = H.compare_particles(out, st, sc.dx, skip)
    assert ok, (config, errs)


@pytest.mark.parametrize("config", CONFIGS)
def test_each_kernel_config_sort_order_and_crowded_block(M, config):
    """The per-sub-step stable sort is bit-exact for every CTA size, and a
    block holding far more particles than one CTA pass (the inbox overflow
    and run-table path) still steps like the oracle."""
    rng = np.random.default_rng(31)
    n = 32
    x = (0.40625 + 0.09375 * rng.random((6000, 3))).astype(np.float32)     # inside one 4^3-cell block
    v = (0.5 * (2 * rng.random((6000, 3)) - 1)).astype(np.float32)
    sc = scenes.Scene("crowd", n_grid=n, dt=1e-4, E=2e3, nu=0.3, rho=1e3, x=x, particle_volume=1e-8, v=v)
    sim = M.sim_from_scene(sc)
    sim.set_kernel_config(config)
    prev = None
    for _ in range(3):
        ids, keys = sim.read_order()
        k_ref = O.block_keys(n, sim.read()["x"])
        assert np.array_equal(ids, O.sorted_order(k_ref, prev)), config
        assert np.array_equal(keys, k_ref[ids])
        prev = ids.copy()
        sim.step(1)
    out = sim.read()
    sim.close()
    st = O.State(sc.x, sc.v)
    H.oracle_steps(sc, st, 0, 3)
    assert np.abs(out["x"] - st.x).max() <= 1e-4 * sc.dx


def test_batched_environments_under_every_config(M):
    envs = scenes.batch_envs(6, seed=3, n_min=1000, n_max=6000)
    outs = []
    for config in CONFIGS:
        cfg = M.make_config(64, envs[0].dt, 1e4, 0.3, 1e3, friction=0.3, n_envs=len(envs),
                            max_particles=sum(e.n for e in envs))
        sim = M.Sim(cfg)
        sim.set_kernel_config(config)
        for i, sc in enumerate(envs):
            sim.set_env_material(i, sc.E, sc.nu, sc.rho)
        sim.load_batch([sc.x for sc in envs], [sc.particle_volume for sc in envs])
        for i, sc in enumerate(envs):
            sim.set_env_tool(i, 0, sc.tools[0].pose(-1), sc.tools[0].shape)
            sim.set_env_tool(i, 0, sc.tools[0].pose(24), sc.tools[0].shape)
        sim.step(25)
        outs.append(sim.read())
        sim.close()
    for o in outs[1:]:      # contact branches may flip over 25 sub-steps: bound the bulk and the rest
        dxp = np.abs(o["x"] - outs[0]["x"]).max(axis=1)
        assert np.quantile(dxp, 0.99) <= 1e-4 / 64 and dxp.max() <= 1e-2 / 64


def test_autotune_picks_a_config_and_restores_the_state(M):
    sc = scenes.slab30k()
    sim = M.sim_from_scene(sc)
    tool = sc.tools[0]
    sim.set_tool(0, tool.pose(49), tool.shape)
    sim.step(50)
    before = sim.read()
    best, times = sim.autotune(10)
    after = sim.read()
    assert best in CONFIGS and sim.kernel_config()["config"] == best
    assert all(t > 0 for t in times) and times[best] == min(times)
    for k in ("x", "v", "F", "C"):
        assert np.array_equal(before[k], after[k]), k
    # stepping on with the chosen kernel matches the default one
    sim.set_tool(0, tool.pose(74), tool.shape)
    sim.step(25)
    tuned = sim.read()
    sim.close()
    ref = M.sim_from_scene(sc)
    ref.set_tool(0, tool.pose(49), tool.shape)
    ref.step(50)
    ref.set_tool(0, tool.pose(74), tool.shape)
    ref.step(25)
    base = ref.read()
    ref.close()
    dxp = np.abs(tuned["x"] - base["x"]).max(axis=1)
    assert np.quantile(dxp, 0.99) <= 1e-4 * sc.dx and dxp.max() <= 1e-2 * sc.dx


@pytest.mark.parametrize("config", CONFIGS)
def test_particles_moving_more_than_a_cell_scatter_directly(M, config):
    """A lattice block moving 1.8, 0.6 and -1.2 cells per sub-step along x,
    y, z: after one sub-step the particles near its +x and -z faces have base
    cells outside the 8^3 shared arena of their block, so their P2G goes
    straight into G_{k+1} with float atomics.  The grid the next sub-step
    starts from matches the oracle's P2G of the GPU's own new state, and so
    does the next sub-step."""
    n, dt = 32, 1e-4
    x = scenes.jittered_lattice((8, 8, 8), (16, 16, 16), n, (2, 2, 2), seed=9)
    cell_per_step = np.array([1.8, 0.6, -1.2]) / n / dt
    v = np.tile(cell_per_step, (x.shape[0], 1)).astype(np.float32)
    sc = scenes.Scene("fast", n_grid=n, dt=dt, E=50.0, nu=0.3, rho=1e3, x=x, particle_volume=(1.0 / n) ** 3 / 8, v=v)
    sim = M.sim_from_scene(sc)
    sim.set_kernel_config(config)
    sim.step(1)
    g = sim.read_grid().astype(np.float64)
    out = sim.read()
    st = H.oracle_state(out)
    # some particles did leave their block's arena: base cell more than one cell past the block
    base = np.floor(st.x * n - 0.5).astype(int)
    blk_before = np.floor(sc.x * n - 0.5).astype(int) // 4
    assert ((base[:, 0] - 4 * blk_before[:, 0] > 4) | (base[:, 2] - 4 * blk_before[:, 2] < -1)).sum() > 100
    gm, gmv = O.p2g(O.OracleParams.from_scene(sc), st.copy())
    assert H.rel_err(g[..., 0], gm) <= 1e-5
    assert H.rel_err(g[..., 1:], gmv) <= 1e-5
    sim.step(1)
    out2 = sim.read()
    assert sim.status() == M.MPM_OK
    sim.close()
    H.oracle_steps(sc, st, 1, 1)
    ok, errs = H.compare_particles(out2, st, sc.dx)
    assert ok, (config, errs)
