"""Sampled distance-field tools (Eqs. 12-14) on the GPU against the FP64
oracle: the grid operation, one sub-step, the slab scene with the paper's
256^3 field, batched environments sharing one field, and the registration
entry point's argument checks.  Tolerances as in the analytic-tool parity
tests; nodes whose FP32 and FP64 decisions may differ (including the cell a
node falls in, within 1e-5 of a cell face) are left out and counted."""
import ctypes as ct

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


def _field(res=64):
    return scenes.grasper_field(res, radius=0.06, half_length=0.05, jaw=(0.04, 0.06, 0.06), gap=0.03)


def _sampled_scene(seed=0, res=64, with_box=True):
    """cube8k particles with random (v, C, F); a grasper field whose jaws cut
    10 cm into the cube, descending and turning, and (optionally) a moving box
    competing with it in the z-buffer; contact threshold theta = 1 cm."""
    sc = H.perturbed_scene(scenes.cube8k(seed), seed=seed + 1)
    fld = _field(res)
    p0 = np.array([0.493, 0.755, 0.508, 0.15, 0.4, -0.1])
    vel = np.array([0.3, -1.5, -0.2, 4.0, 25.0, -6.0])
    dt = sc.dt
    tools = [scenes.Tool(scenes.sampled_shape(), lambda s: p0 + vel * dt * (s + 1), fld)]
    if with_box:
        pb = np.array([0.56, 0.39, 0.45, 0.0, 0.4, 0.1])
        vb = np.array([-0.5, 1.0, 0.3, 0.0, 30.0, -15.0])
        tools.append(scenes.Tool(scenes.box_shape(0.08, 0.05, 0.07), lambda s: pb + vb * dt * (s + 1)))
    sc.tools = tools
    sc.friction = 0.4
    sc.theta = 0.01
    return sc


@pytest.mark.parametrize("pipe", H.PIPELINES)
def test_sampled_grid_operation_parity(M, pipe):
    sc = _sampled_scene()
    sim = M.sim_from_scene(sc, pipeline=H.pipeline_id(pipe))
    for t, tool in enumerate(sc.tools):
        sim.set_tool(t, tool.pose(0), tool.shape, tool.field)
    g = sim.read_grid().astype(np.float64)
    gv = sim.grid_velocity().astype(np.float64)
    sim.close()
    prm = O.OracleParams.from_scene(sc)
    frames, nt = O.frames_for_steps(sc.tools, 0, 1, sc.dt, 1)
    ov, contact, margin = O.grid_update(prm, g[..., 0].copy(), g[..., 1:].copy(), frames, nt)
    mask = margin < 1e-5
    n_sampled = int((contact == 0).sum())
    assert n_sampled > 50, "the sampled tool must touch the material"
    assert int((contact == 1).sum()) > 20, "the box must touch the material"
    assert mask.sum() <= max(5, 0.03 * n_sampled)
    vmax = np.abs(ov).max()
    diff = np.abs(gv - ov).max(axis=-1)
    assert diff[~mask].max() <= 1e-5 * vmax


@pytest.mark.parametrize("pipe", H.PIPELINES)
def test_sampled_single_substep_parity(M, pipe):
    sc = _sampled_scene(seed=4)
    sim = M.sim_from_scene(sc, pipeline=H.pipeline_id(pipe))
    start = sim.read()
    for t, tool in enumerate(sc.tools):
        sim.set_tool(t, tool.pose(0), tool.shape, tool.field)
    sim.step(1)
    out = sim.read()
    sim.close()
    st = H.oracle_state(start)
    mask = H.contact_mask_nodes(sc, st, 0)
    skip = H.particles_touching(mask, st.x, sc.n_grid)
    H.oracle_steps(sc, st, 0, 1, call_len=1)
    assert mask.sum() <= 8
    ok, errs = H.compare_particles(out, st, sc.dx, skip)
    assert ok, errs


def test_sampled_fused_and_split_agree_on_25_substeps(M):
    sc = _sampled_scene(seed=5)
    outs = []
    for pipe in H.PIPELINES:
        sim = M.sim_from_scene(sc, pipeline=H.pipeline_id(pipe))
        for t, tool in enumerate(sc.tools):
            sim.set_tool(t, tool.pose(24), tool.shape, tool.field)
        sim.step(25)
        outs.append(sim.read())
        sim.close()
    st = O.State(sc.x, sc.v, sc.C, sc.F)
    H.oracle_steps(sc, st, 0, 25, call_len=25)
    for out in outs:
        dxp = np.abs(out["x"] - st.x).max(axis=1)
        assert np.quantile(dxp, 0.99) <= 1e-4 * sc.dx
        assert dxp.max() <= 1e-2 * sc.dx


def test_slab30k_sdf_paper_resolution_sampled_single_steps(M):
    """The 30K-particle slab pressed and dragged by the grasper sampled at
    the paper's 256^3; one sub-step from the shared state at sampled
    sub-steps of the 2,000-sub-step script."""
    sc = scenes.slab30k_sdf()
    assert sc.tools[0].field.res == 256
    sim = M.sim_from_scene(sc)
    tool = sc.tools[0]
    s = 0
    touched = 0
    for sample in (100, 900, 1000, 1500, 1975):
        while s < sample:
            m = min(25, sample - s)
            sim.set_tool(0, tool.pose(s + m - 1), tool.shape, tool.field)
            sim.step(m)
            s += m
        state = sim.read()
        sim.set_tool(0, tool.pose(s), tool.shape, tool.field)
        sim.step(1)
        out = sim.read()
        st = H.oracle_state(state)
        prm = O.OracleParams.from_scene(sc)
        gm, gmv = O.p2g(prm, st.copy())
        frames, nt = O.frames_for_steps(sc.tools, s, 1, sc.dt, 1)
        _, contact, margin = O.grid_update(prm, gm, gmv, frames, nt)
        touched += int((contact == 0).sum())
        mask = margin < 1e-5
        skip = H.particles_touching(mask, st.x, sc.n_grid)
        O.run(prm, st, 1, frames, nt)
        ok, errs = H.compare_particles(out, st, sc.dx, skip)
        assert ok, (sample, errs)
        assert mask.sum() <= 5, sample
        s += 1
    sim.close()
    assert touched > 60, "the grasper must press into the slab"


def test_batched_environments_share_one_field(M):
    """Three environments with the same registered field at different poses
    (and one environment with an analytic capsule): the grid operation of
    every environment matches the oracle."""
    fld = _field(48)
    envs = []
    for e in range(4):
        rng = np.random.default_rng(300 + e)
        N = 2500 + 500 * e
        x = (0.35 + 0.3 * rng.random((N, 3))).astype(np.float32)
        v, C, F = scenes.random_state(x, 400 + e, v_scale=0.3, c_scale=1.0, f_dev=0.05)
        p0 = np.array([0.47 + 0.02 * e, 0.70 - 0.01 * e, 0.5, 0.2 * e, 0.3, 0.1])
        vel = np.array([0.1, -1.0, 0.05, 5.0, 0.0, -3.0])
        pose = (lambda p0, vel: (lambda s: p0 + vel * 1e-4 * (s + 1)))(p0, vel)
        tool = (scenes.Tool(scenes.capsule_shape(0.05, 0.06), pose) if e == 2
                else scenes.Tool(scenes.sampled_shape(), pose, fld))
        envs.append(scenes.Scene("e%d" % e, n_grid=32, dt=1e-4, E=5e3, nu=0.3, rho=1e3, x=x,
                                 particle_volume=0.3 ** 3 / N, friction=0.3, v=v, C=C, F=F, tools=[tool]))
    cfg = M.make_config(32, 1e-4, 5e3, 0.3, 1e3, friction=0.3, n_envs=len(envs),
                        max_particles=sum(sc.n for sc in envs))
    sim = M.Sim(cfg)
    sim.load_batch([sc.x for sc in envs], [sc.particle_volume for sc in envs], [sc.v for sc in envs],
                   [sc.F for sc in envs], [sc.C for sc in envs])
    for i, sc in enumerate(envs):
        sim.set_env_tool(i, 0, sc.tools[0].pose(-1), sc.tools[0].shape, sc.tools[0].field)
        sim.set_env_tool(i, 0, sc.tools[0].pose(0), sc.tools[0].shape, sc.tools[0].field)
    assert len(sim._fields) == 1, "one registration for the shared field"
    g = sim.read_grid().astype(np.float64).reshape(len(envs), 32, 32, 32, 4)
    gv = sim.grid_velocity().astype(np.float64).reshape(len(envs), 32, 32, 32, 3)
    sim.close()
    for i, sc in enumerate(envs):
        prm = O.OracleParams.from_scene(sc)
        frames, nt = O.frames_for_steps(sc.tools, 0, 1, sc.dt, 1)
        ov, contact, margin = O.grid_update(prm, g[i, ..., 0].copy(), g[i, ..., 1:].copy(), frames, nt)
        mask = margin < 1e-5
        assert (contact == 0).sum() > 20, sc.name
        assert mask.sum() <= 5, sc.name
        diff = np.abs(gv[i] - ov).max(axis=-1)
        assert diff[~mask].max() <= 1e-5 * np.abs(ov).max(), sc.name


def test_sampled_field_registration_contract(M):
    import torch
    sc = _sampled_scene(with_box=False)
    fld = sc.tools[0].field
    sim = M.sim_from_scene(sc)
    h = sim.h
    o = np.zeros(3)
    fid = ct.c_int32(-1)
    samples = np.zeros(8, np.float32)
    P = samples.ctypes.data_as(ct.c_void_p)
    OD = o.ctypes.data_as(M._DP)
    assert M.mpm_add_sampled_field(h, 0, OD, 0.1, P, 0, ct.byref(fid)) == M.MPM_ERR_ARG
    assert M.mpm_add_sampled_field(h, M.MPM_MAX_FIELD_RES + 1, OD, 0.1, P, 0, ct.byref(fid)) == M.MPM_ERR_ARG
    assert M.mpm_add_sampled_field(h, 2, OD, 0.0, P, 0, ct.byref(fid)) == M.MPM_ERR_ARG
    assert M.mpm_add_sampled_field(h, 2, OD, 0.1, None, 0, ct.byref(fid)) == M.MPM_ERR_ARG
    samples[3] = np.nan
    assert M.mpm_add_sampled_field(h, 2, OD, 0.1, P, 0, ct.byref(fid)) == M.MPM_ERR_ARG
    pose = np.array([0.5, 0.7, 0.5, 0, 0, 0], np.float64)
    bad = scenes.sampled_shape()
    bad[1] = 7                                       # not registered
    assert M.mpm_set_tool_pose(h, 0, pose.ctypes.data_as(M._DP), bad.ctypes.data_as(M._FP)) == M.MPM_ERR_ARG
    bad[1] = 0.5
    assert M.mpm_set_tool_pose(h, 0, pose.ctypes.data_as(M._DP), bad.ctypes.data_as(M._FP)) == M.MPM_ERR_ARG
    # the same field registered from host memory and from device memory gives the same grid operation
    pose0 = sc.tools[0].pose(0)
    sim.set_tool(0, pose0, sc.tools[0].shape, fld)
    gv_host = sim.grid_velocity()
    dev = torch.from_numpy(np.ascontiguousarray(fld.samples)).cuda()
    fid_dev = sim.add_field(dev, fld.origin, fld.h)
    shape = scenes.sampled_shape()
    shape[1] = fid_dev
    sim.set_tool(0, pose0, shape)
    gv_dev = sim.grid_velocity()
    assert np.array_equal(gv_host, gv_dev)
    assert np.abs(gv_host).max() > 0
    for _ in range(M.MPM_MAX_FIELDS - 2):             # two registered so far: fill the table
        sim.add_field(np.zeros(8, np.float32), o, 0.1)
    assert M.mpm_add_sampled_field(h, 2, OD, 0.1, np.zeros(8, np.float32).ctypes.data_as(ct.c_void_p), 0,
                                   ct.byref(fid)) == M.MPM_ERR_CAPACITY
    sim.clear_error()
    sim.close()
