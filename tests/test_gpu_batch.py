"""Several independent environments stepped by one handle (one fused launch
per sub-step over all environments' blocks): each environment must match
the oracle and its own single-environment handle, and the batch's sort order
must be the stable counting sort by global block key."""
import numpy as np
import pytest

import helpers as H
from oracle import oracle as O
from paper_2402_01181_gb300 import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    import __graft_entry__ as ge
    ge.build()
    from paper_2402_01181_gb300 import mpm
    return mpm


def _envs():
    """Four small environments on 32^3 grids with different particle counts
    (one of them empty), materials, states and moving tools."""
    out = []
    specs = [(3000, 4e3, 0.25), (0, 5e3, 0.3), (1500, 9e3, 0.4), (4200, 2.5e3, 0.33)]
    for e, (N, E, nu) in enumerate(specs):
        rng = np.random.default_rng(100 + e)
        x = (0.35 + 0.3 * rng.random((N, 3))).astype(np.float32)
        v, C, F = scenes.random_state(x, 200 + e, v_scale=0.3, c_scale=1.0, f_dev=0.05)
        p0 = np.array([0.45 + 0.03 * e, 0.62, 0.5, 0.1 * e, 0.2, 0.0])
        vel = np.array([0.1, -1.0, 0.05 * e, 5.0, 0.0, -3.0 * e])
        sc = scenes.Scene("e%d" % e, n_grid=32, dt=1e-4, E=E, nu=nu, rho=1e3, x=x,
                          particle_volume=0.3 ** 3 / max(N, 1), friction=0.3, v=v, C=C, F=F,
                          tools=[scenes.Tool(scenes.capsule_shape(0.05, 0.06),
                                             (lambda p0, vel: (lambda s: p0 + vel * 1e-4 * (s + 1)))(p0, vel))])
        out.append(sc)
    return out


def _batch(M, envs):
    cfg = M.make_config(32, 1e-4, 5e3, 0.3, 1e3, friction=0.3, n_envs=len(envs),
                        max_particles=max(1, sum(e.n for e in envs)))
    sim = M.Sim(cfg)
    for i, sc in enumerate(envs):
        sim.set_env_material(i, sc.E, sc.nu, sc.rho)
    sim.load_batch([sc.x for sc in envs], [sc.particle_volume for sc in envs], [sc.v for sc in envs],
                   [sc.F for sc in envs], [sc.C for sc in envs])
    for i, sc in enumerate(envs):
        sim.set_env_tool(i, 0, sc.tools[0].pose(-1), sc.tools[0].shape)
    return sim


def _split(out, envs):
    res, o = [], 0
    for sc in envs:
        res.append({k: v[o:o + sc.n] for k, v in out.items()})
        o += sc.n
    return res


def test_batch_single_substep_matches_oracle_per_env(M):
    envs = _envs()
    sim = _batch(M, envs)
    start = _split(sim.read(), envs)
    for i, sc in enumerate(envs):
        sim.set_env_tool(i, 0, sc.tools[0].pose(0), sc.tools[0].shape)
    sim.step(1)
    out = _split(sim.read(), envs)
    sim.close()
    for sc, st0, o in zip(envs, start, out):
        if sc.n == 0:
            continue
        st = H.oracle_state(st0)
        prm = O.OracleParams.from_scene(sc)      # friction 0.3: the handle's, shared by all environments
        gm, gmv = O.p2g(prm, st.copy())
        frames, nt = O.frames_for_steps(sc.tools, 0, 1, sc.dt, 1)
        _, _, margin = O.grid_update(prm, gm, gmv, frames, nt)
        skip = H.particles_touching(margin < 1e-5, st.x, sc.n_grid)
        O.run(prm, st, 1, frames, nt)
        ok, errs = H.compare_particles(o, st, sc.dx, skip)
        assert ok, (sc.name, errs)


def test_batch_matches_single_environment_handles(M):
    envs = _envs()
    sim = _batch(M, envs)
    for i, sc in enumerate(envs):
        sim.set_env_tool(i, 0, sc.tools[0].pose(9), sc.tools[0].shape)
    sim.step(10)
    out = _split(sim.read(), envs)
    sim.close()
    for sc, o in zip(envs, out):
        if sc.n == 0:
            continue
        single = M.Sim(M.make_config(32, 1e-4, sc.E, sc.nu, sc.rho, friction=0.3, max_particles=sc.n))
        single.load(sc.x, sc.particle_volume, sc.v, sc.F, sc.C)
        single.set_tool(0, sc.tools[0].pose(-1), sc.tools[0].shape)
        single.set_tool(0, sc.tools[0].pose(9), sc.tools[0].shape)
        single.step(10)
        r = single.read()
        single.close()
        assert np.abs(o["x"] - r["x"]).max() <= 1e-4 * sc.dx, sc.name
        assert np.abs(o["F"] - r["F"]).max() <= 1e-4, sc.name


def test_batch_sort_order(M):
    envs = _envs()
    sim = _batch(M, envs)
    nbe = (32 // 4) ** 3
    ids, keys = sim.read_order()
    prev = None
    for step in range(3):
        x = sim.read()["x"]
        env_of = np.repeat(np.arange(len(envs)), [sc.n for sc in envs])
        k_ref = O.block_keys(32, x).astype(np.int64) + env_of * nbe
        assert np.array_equal(ids, O.sorted_order(k_ref, prev))
        assert np.array_equal(keys, k_ref[ids])
        prev = ids.copy()
        sim.step(1)
        ids, keys = sim.read_order()
    sim.close()


def test_batch256_full_size_sampled_envs_match_oracle(M):
    """The benchmark's batched workload at full size (256 slab environments of
    5K-40K particles on their own 64^3 grids), autotuned as the benchmark runs
    it: after one 25-sub-step frame with every tool moving, one more sub-step
    of eight sampled environments matches the oracle from the same state."""
    envs = scenes.batch_envs(256, seed=0)
    S = 25
    cfg = M.make_config(64, envs[0].dt, 1e4, 0.3, 1e3, friction=0.3, n_envs=len(envs),
                        max_particles=sum(e.n for e in envs))
    sim = M.Sim(cfg)
    for i, sc in enumerate(envs):
        sim.set_env_material(i, sc.E, sc.nu, sc.rho)
    sim.load_batch([sc.x for sc in envs], [sc.particle_volume for sc in envs])
    for i, sc in enumerate(envs):
        sim.set_env_tool(i, 0, sc.tools[0].pose(-1), sc.tools[0].shape)
    best, _ = sim.autotune(S)
    assert sim.kernel_config()["config"] == best
    for i, sc in enumerate(envs):
        sim.set_env_tool(i, 0, sc.tools[0].pose(S - 1), sc.tools[0].shape)
    sim.step(S)
    start = _split(sim.read(), envs)
    for i, sc in enumerate(envs):
        sim.set_env_tool(i, 0, sc.tools[0].pose(S), sc.tools[0].shape)
    sim.step(1)
    out = _split(sim.read(), envs)
    assert sim.status() == M.MPM_OK
    sim.close()
    for e in (0, 37, 74, 111, 148, 185, 222, 255):
        sc = envs[e]
        st = H.oracle_state(start[e])
        mask = H.contact_mask_nodes(sc, st, S)
        skip = H.particles_touching(mask, st.x, sc.n_grid)
        frames, nt = O.frames_for_steps(sc.tools, S, 1, sc.dt, 1)
        O.run(O.OracleParams.from_scene(sc), st, 1, frames, nt)
        ok, errs = H.compare_particles(out[e], st, sc.dx, skip)
        assert ok, (e, errs)
        assert mask.sum() <= 5, e
