"""The differentiable rollout on the GPU (mpm_tape_record / mpm_tape_backward,
and the torch.autograd binding) against the FP64 oracle's adjoint, which is
pinned by central differences in test_oracle_adjoint_pins.py.

Tolerances (FP32 reverse mode against FP64): one sub-step, element by
element, 2e-4 of each block's largest magnitude (particles whose stencil
touches a node within 1e-5 of a branch point are left out and counted);
material gradients 1e-3 relative; pose gradients 2e-3 of the largest entry.
Rollouts of many sub-steps compare the summed gradients at 1e-2 (two tools,
30 sub-steps) and 3e-2 / 5e-2 (the slab: its loss is a mean of squared
gaps of ~1e-5 m, while FP32 positions near 0.5 resolve 6e-8 m and carry
the rounding of hundreds of sub-steps), and the oracle's own central
differences confirm the GPU gradient."""
import functools

import numpy as np
import pytest

import helpers as H
import test_oracle_adjoint_pins as AP
from oracle import oracle as O
from paper_2402_01181_gb300 import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    import __graft_entry__ as ge
    ge.build()
    from paper_2402_01181_gb300 import mpm
    return mpm


PIPES = ("split", "fused")


def _pipe(M, name):
    return M.MPM_PIPELINE_FUSED if name == "fused" else M.MPM_PIPELINE_SPLIT


def _sim(M, prm, n, pipe="split"):
    cfg = M.make_config(prm.n_grid, prm.dt, prm.E, prm.nu, prm.rho, gravity=tuple(prm.gravity), bound=prm.bound,
                        theta=prm.theta, friction=prm.friction, pipeline=_pipe(M, pipe), max_particles=n)
    return M.Sim(cfg)


def _f32_state(st):
    return {k: getattr(st, k).astype(np.float32) for k in ("x", "v", "F", "C")}


@pytest.mark.parametrize("pipe", PIPES)
def test_single_substep_adjoint_matches_oracle(M, pipe):
    import torch
    prm, st, tools, p0, p1 = AP._scene()
    s32 = _f32_state(st)
    sim = _sim(M, prm, st.n, pipe)
    sim.load(s32["x"], prm.V0, s32["v"], s32["F"], s32["C"])
    for t, tool in enumerate(tools):
        sim.set_tool(t, p0[t], tool.shape)
    sim.tape_record(p1[None], 1)
    rng = np.random.default_rng(21)
    ybar = AP._random_bar(rng, st.n)
    dev = torch.device("cuda")
    g = sim.tape_backward(*[torch.tensor(ybar[k], dtype=torch.float32, device=dev) for k in ("x", "v", "F", "C")],
                          want_state=True)
    sim.close()
    ref_state = O.State(s32["x"], s32["v"], s32["C"], s32["F"])
    frames = AP._frames(tools, p0, p1, prm.dt)
    ybar32 = {k: ybar[k].astype(np.float32).astype(np.float64) for k in ybar}
    rbar, lame, tb = O.step_adjoint(prm, ref_state, frames, 2, ybar32)
    gm, gmv = O.p2g(prm, ref_state.copy())
    _, contact, margin = O.grid_update(prm, gm, gmv, frames, 2)
    assert (contact >= 0).sum() > 20
    skip = H.particles_touching(margin < 1e-5, ref_state.x, prm.n_grid)
    assert skip.sum() <= 0.02 * st.n
    keep = ~skip
    for k in ("x", "v", "F", "C"):
        got = g[k].cpu().numpy().astype(np.float64)
        scale = np.abs(rbar[k]).max()
        err = np.abs(got[keep] - rbar[k][keep]).max() / scale
        assert err <= 2e-4, (k, err)
    Eb, nub = O.lame_vjp(prm.E, prm.nu, lame[0], lame[1])
    assert abs(g["E"] - Eb) <= 1e-3 * abs(Eb), (g["E"], Eb)
    assert abs(g["nu"] - nub) <= 1e-3 * abs(nub), (g["nu"], nub)
    for t, tool in enumerate(tools):
        J = O.frame_jacobian(tool.shape, p0[t], p1[t], prm.dt)
        ref = J[:, 6:].T @ tb[t]
        got = g["poses"][0, t]
        assert np.abs(got - ref).max() <= 2e-3 * np.abs(ref).max(), (t, got, ref)


@pytest.mark.parametrize("pipe", PIPES)
def test_rollout_gradients_match_oracle(M, pipe):
    """30 sub-steps with two moving tools, checkpoints every 8 (a short last
    segment), loss = mean |x(T) - target|^2, through torch.autograd."""
    import torch
    from paper_2402_01181_gb300 import autodiff
    prm, st, tools, p0, p1 = AP._scene(seed=11)
    K = 30
    poses = np.stack([p0 + (k + 1) * 0.5 * (p1 - p0) for k in range(K)])
    s32 = _f32_state(st)
    rng = np.random.default_rng(22)
    target = (st.x + 0.01 * rng.normal(size=st.x.shape)).astype(np.float32)
    dev = torch.device("cuda")
    sim = _sim(M, prm, st.n, pipe)
    for t, tool in enumerate(tools):
        sim.set_tool(t, p0[t], tool.shape)
    E = torch.tensor(prm.E, dtype=torch.float64, requires_grad=True)
    nu = torch.tensor(prm.nu, dtype=torch.float64, requires_grad=True)
    P = torch.tensor(poses, dtype=torch.float64, requires_grad=True)
    x0 = torch.tensor(s32["x"], device=dev, requires_grad=True)
    v0 = torch.tensor(s32["v"], device=dev, requires_grad=True)
    F0 = torch.tensor(s32["F"], device=dev, requires_grad=True)
    C0 = torch.tensor(s32["C"], device=dev, requires_grad=True)
    xT, vT, FT, CT = autodiff.rollout(sim, E, nu, P, x0, prm.V0, v0, F0, C0, checkpoint_every=8)
    loss = ((xT - torch.tensor(target, device=dev)) ** 2).sum(dim=1).mean()
    loss.backward()
    sim.close()
    ref = O.rollout_loss_and_gradients(prm, O.State(s32["x"], s32["v"], s32["C"], s32["F"]), tools, p0, poses,
                                       target.astype(np.float64), checkpoint=8)
    assert abs(loss.item() - ref["loss"]) <= 1e-4 * ref["loss"]
    assert abs(E.grad.item() - ref["E"]) <= 1e-2 * abs(ref["E"]), (E.grad.item(), ref["E"])
    assert abs(nu.grad.item() - ref["nu"]) <= 1e-2 * abs(ref["nu"]), (nu.grad.item(), ref["nu"])
    gp = P.grad.numpy()
    assert np.abs(gp - ref["poses"]).max() <= 1e-2 * np.abs(ref["poses"]).max()
    for k, got in (("x", x0.grad), ("v", v0.grad), ("F", F0.grad), ("C", C0.grad)):
        r = ref["state0"][k]
        assert np.abs(got.cpu().numpy() - r).max() <= 1e-2 * np.abs(r).max(), k


def test_slab30k_rollout_gradient_against_oracle_and_differences(M):
    """The tissue slab pressed by the capsule: 200 sub-steps from the moment
    the capsule reaches the slab (sub-step 90 of its script; 1 cm of
    indentation), checkpoints every 50.  The target comes from an FP64 oracle
    rollout with E = 1.2e4, nu = 0.33 and shifted poses.  The GPU gradients
    with respect to E, nu and the poses match the oracle's adjoint, and the
    oracle's central differences of the loss for E and nu.  The loss is
    small (RMS gap ~1e-5 m) against FP32 positions near 0.5 (resolution 6e-8
    m), which bounds the GPU's agreement near 1%."""
    import torch
    from paper_2402_01181_gb300 import autodiff
    case = scenes.slab30k_diff(steps=200, checkpoint=50, first=90)
    sc = case.scene
    prm = O.OracleParams.from_scene(sc)
    tools = sc.tools
    tprm = O.OracleParams(**{**prm.__dict__, "E": case.target_E, "nu": case.target_nu})
    st0 = O.State(sc.x)
    tgt_state = st0.copy()
    tf, nt = O.rollout_frames(tools, case.pose_init, case.target_poses, prm.dt)
    O.run(tprm, tgt_state, case.poses.shape[0], tf, nt)
    target = tgt_state.x.astype(np.float32)
    dev = torch.device("cuda")
    sim = M.sim_from_scene(sc, pipeline=M.MPM_PIPELINE_SPLIT, load=False)
    sim.set_tool(0, case.pose_init[0], tools[0].shape)      # placed at the start of the stream
    E = torch.tensor(prm.E, dtype=torch.float64, requires_grad=True)
    nu = torch.tensor(prm.nu, dtype=torch.float64, requires_grad=True)
    P = torch.tensor(case.poses, dtype=torch.float64, requires_grad=True)
    x0 = torch.tensor(sc.x, device=dev)
    xT, _, _, _ = autodiff.rollout(sim, E, nu, P, x0, sc.particle_volume, checkpoint_every=case.checkpoint)
    loss = ((xT - torch.tensor(target, device=dev)) ** 2).sum(dim=1).mean()
    loss.backward()
    sim.close()
    ref = O.rollout_loss_and_gradients(prm, st0, tools, case.pose_init, case.poses, target.astype(np.float64),
                                       checkpoint=case.checkpoint)
    assert abs(loss.item() - ref["loss"]) <= 2e-2 * ref["loss"], (loss.item(), ref["loss"])
    assert abs(E.grad.item() - ref["E"]) <= 3e-2 * abs(ref["E"]), (E.grad.item(), ref["E"])
    assert abs(nu.grad.item() - ref["nu"]) <= 3e-2 * abs(ref["nu"]), (nu.grad.item(), ref["nu"])
    gp = P.grad.numpy()
    assert np.abs(gp - ref["poses"]).max() <= 5e-2 * np.abs(ref["poses"]).max()

    def loss_at(E_, nu_, poses_):
        p = O.OracleParams(**{**prm.__dict__, "E": E_, "nu": nu_})
        s = st0.copy()
        fr, n_ = O.rollout_frames(tools, case.pose_init, poses_, prm.dt)
        O.run(p, s, poses_.shape[0], fr, n_)
        return float(np.mean(np.sum((s.x - target) ** 2, axis=1)))

    hE, hn = 1e-3 * prm.E, 1e-3 * prm.nu
    fdE = (loss_at(prm.E + hE, prm.nu, case.poses) - loss_at(prm.E - hE, prm.nu, case.poses)) / (2 * hE)
    fdn = (loss_at(prm.E, prm.nu + hn, case.poses) - loss_at(prm.E, prm.nu - hn, case.poses)) / (2 * hn)
    assert abs(E.grad.item() - fdE) <= 5e-2 * abs(fdE), (E.grad.item(), fdE)
    assert abs(nu.grad.item() - fdn) <= 5e-2 * abs(fdn), (nu.grad.item(), fdn)


@pytest.mark.parametrize("pipe", PIPES)
def test_tape_contract(M, pipe):
    import torch
    sc = scenes.cube8k()
    poses = np.zeros((3, 0, 6))
    cfg = M.make_config(sc.n_grid, sc.dt, sc.E, sc.nu, sc.rho, n_envs=2, max_particles=sc.n)
    batched = M.Sim(cfg)
    batched.load_batch([sc.x[:100], sc.x[100:200]], [sc.particle_volume] * 2)
    with pytest.raises(M.MPMError) as e:           # one environment only
        batched.tape_record(poses, 1)
    assert e.value.status == M.MPM_ERR_STATE
    batched.close()
    sim = M.sim_from_scene(sc, pipeline=_pipe(M, pipe))
    with pytest.raises(M.MPMError) as e:
        sim.tape_backward(torch.zeros((sc.n, 3), device="cuda"))
    assert e.value.status == M.MPM_ERR_STATE
    with pytest.raises(M.MPMError) as e:
        sim.tape_record(poses, 0)
    assert e.value.status == M.MPM_ERR_ARG
    sim.tape_record(poses, 2)
    out = sim.read()
    ref = O.State(sc.x)
    H.oracle_steps(sc, ref, 0, 3)
    assert np.abs(out["x"] - ref.x).max() <= 1e-3 * sc.dx      # the record steps the state like mpm_step
    sim.set_env_material(0, sc.E * 2, sc.nu, sc.rho)
    with pytest.raises(M.MPMError) as e:
        sim.tape_backward(torch.zeros((sc.n, 3), device="cuda"))
    assert e.value.status == M.MPM_ERR_STATE
    sim.close()


def test_tape_read_substep_contract(M):
    """mpm_tape_read_substep returns the states the reverse pass differentiates
    at.  A one-sub-step record starts from the loaded state, so its sub-step 0
    is that state and the load's grid, bit for bit; a record of 7 sub-steps
    with checkpoints every 3 has a last segment of one sub-step (j = 0 only).
    The split pipeline has no such record, and a backward pass ends it."""
    import torch
    sc = scenes.slab30k()
    sim = M.sim_from_scene(sc, pipeline=M.MPM_PIPELINE_FUSED)
    tool = sc.tools[0]
    sim.set_tool(0, tool.pose(0), tool.shape)
    with pytest.raises(M.MPMError) as e:            # nothing recorded yet
        sim.tape_read_substep(0)
    assert e.value.status == M.MPM_ERR_STATE
    before = sim.read()
    grid = sim.read_grid()
    sim.tape_record(np.asarray([tool.pose(1)])[:, None, :], 1)
    got = sim.tape_read_substep(0)
    for k in ("x", "v", "F", "C"):
        assert np.array_equal(got[k], before[k]), k
    assert np.array_equal(got["grid"], grid)
    with pytest.raises(M.MPMError) as e:
        sim.tape_read_substep(1)
    assert e.value.status == M.MPM_ERR_ARG
    sim.tape_record(np.asarray([tool.pose(2 + k) for k in range(7)])[:, None, :], 3)
    last = sim.tape_read_substep(0)                 # sub-step 6: one sub-step before the end
    assert np.isfinite(last["x"]).all() and np.abs(last["x"] - before["x"]).max() > 0
    with pytest.raises(M.MPMError) as e:
        sim.tape_read_substep(1)
    assert e.value.status == M.MPM_ERR_ARG
    sim.tape_backward(torch.zeros((sc.n, 3), device="cuda"))
    with pytest.raises(M.MPMError) as e:            # the reverse pass replays into the record
        sim.tape_read_substep(0)
    assert e.value.status == M.MPM_ERR_STATE
    sim.close()
    split = M.sim_from_scene(sc, pipeline=M.MPM_PIPELINE_SPLIT)
    split.set_tool(0, tool.pose(0), tool.shape)
    split.tape_record(np.asarray([tool.pose(1)])[:, None, :], 1)
    with pytest.raises(M.MPMError) as e:
        split.tape_read_substep(0)
    assert e.value.status == M.MPM_ERR_STATE
    split.close()


def test_segmented_backward_matches_one_segment(M):
    """The fused reverse pass replays segments on a second stream, one segment
    ahead of the reverse sub-steps, into two record buffers in turn.  The same
    rollout (100 sub-steps of the differentiable workload) reversed as five
    segments and as one segment (recorded by the forward pass, no replay)
    must agree: dL/dE, dL/dnu and the initial-state adjoint to 1e-4 (the fused
    forward reproduces to ~1e-7 there), the pose gradients to 2e-2 of their
    largest entry (the stick/slide kink makes them reproducible only to a few
    1e-3).  A buffer overwritten while read, or read before written, would
    break this by orders of magnitude."""
    import torch
    case = scenes.slab30k_diff()
    sc = case.scene
    K = 100
    dev = torch.device("cuda")
    xbar = torch.tensor(np.random.default_rng(5).normal(size=(sc.n, 3)).astype(np.float32) * 1e-4, device=dev)
    out = {}
    for ck in (K, 20):
        sim = M.sim_from_scene(sc, pipeline=M.MPM_PIPELINE_FUSED, load=False)
        sim.load(sc.x, sc.particle_volume)
        sim.set_tool(0, case.pose_init[0], sc.tools[0].shape)
        sim.tape_record(case.poses[:K], ck)
        out[ck] = sim.tape_backward(xbar, want_state=True)
        sim.close()
    a, b = out[K], out[20]
    for k in ("E", "nu"):
        assert abs(a[k] - b[k]) <= 1e-4 * abs(a[k]), (k, a[k], b[k])
    for k in ("x", "v", "F", "C"):
        ga, gb = a[k].cpu().numpy(), b[k].cpu().numpy()
        assert np.abs(ga - gb).max() <= 1e-4 * np.abs(ga).max(), k
    scale = np.maximum(np.abs(a["poses"]).max(axis=0, keepdims=True), 1e-300)
    assert (np.abs(a["poses"] - b["poses"]) / scale).max() <= 2e-2


@functools.lru_cache(maxsize=1)
def _config5_oracle():
    """The differentiable workload's FP32 target (an FP64 oracle rollout with
    E = 1.2e4, nu = 0.33 and shifted poses) and the oracle's loss and
    gradients at the workload's own parameters."""
    case = scenes.slab30k_diff()
    sc = case.scene
    prm = O.OracleParams.from_scene(sc)
    tprm = O.OracleParams(**{**prm.__dict__, "E": case.target_E, "nu": case.target_nu})
    st0 = O.State(sc.x)
    tgt_state = st0.copy()
    tf, nt = O.rollout_frames(sc.tools, case.pose_init, case.target_poses, prm.dt)
    O.run(tprm, tgt_state, case.poses.shape[0], tf, nt)
    target = tgt_state.x.astype(np.float32)
    ref = O.rollout_loss_and_gradients(prm, st0, sc.tools, case.pose_init, case.poses, target.astype(np.float64),
                                       checkpoint=case.checkpoint)
    return case, target, ref


@pytest.mark.parametrize("pipe", PIPES)
def test_config5_full_size_gradients_match_oracle(M, pipe):
    """The full differentiable workload the benchmark times: the 30K slab
    over 500 sub-steps (the capsule descends, touches near sub-step 100 and
    presses 2 cm in), checkpoints every 50.  The GPU loss and its gradients
    with respect to E, nu and all 500 x 6 pose entries against the oracle's
    adjoint, end to end: the FP32 forward trajectory drifts from the FP64 one
    over 500 sub-steps, and the loss is a mean of squared gaps of ~1e-5 m, so
    the bar here is 3e-2 / 5e-2 (the adjoint's own arithmetic is checked at
    1e-3, segment by segment, in the test below)."""
    import torch
    from paper_2402_01181_gb300 import autodiff
    case, target, ref = _config5_oracle()
    sc = case.scene
    prm = O.OracleParams.from_scene(sc)
    dev = torch.device("cuda")
    sim = M.sim_from_scene(sc, pipeline=_pipe(M, pipe), load=False)
    sim.set_tool(0, case.pose_init[0], sc.tools[0].shape)
    E = torch.tensor(prm.E, dtype=torch.float64, requires_grad=True)
    nu = torch.tensor(prm.nu, dtype=torch.float64, requires_grad=True)
    P = torch.tensor(case.poses, dtype=torch.float64, requires_grad=True)
    xT, _, _, _ = autodiff.rollout(sim, E, nu, P, torch.tensor(sc.x, device=dev), sc.particle_volume,
                                   checkpoint_every=case.checkpoint)
    loss = ((xT - torch.tensor(target, device=dev)) ** 2).sum(dim=1).mean()
    loss.backward()
    sim.close()
    err = {"loss": abs(loss.item() - ref["loss"]) / ref["loss"], "E": abs(E.grad.item() - ref["E"]) / abs(ref["E"]),
           "nu": abs(nu.grad.item() - ref["nu"]) / abs(ref["nu"]),
           "poses": np.abs(P.grad.numpy() - ref["poses"]).max() / np.abs(ref["poses"]).max()}
    print("config-5 end-to-end relative errors (%s):" % pipe, err)
    assert err["loss"] <= 2e-2 and err["E"] <= 3e-2 and err["nu"] <= 3e-2 and err["poses"] <= 5e-2, err


def _segment_errors(got, ref):
    """Relative errors of one segment's gradients: E and nu against their own
    magnitude; each pose component (tool, coordinate) against its largest
    magnitude over the segment; each block of the incoming state adjoint
    against its largest magnitude."""
    out = {"E": abs(got["E"] - ref["E"]) / abs(ref["E"]), "nu": abs(got["nu"] - ref["nu"]) / abs(ref["nu"])}
    scale = np.abs(ref["poses"]).max(axis=0, keepdims=True)
    out["poses"] = float((np.abs(got["poses"] - ref["poses"]) / np.maximum(scale, 1e-300)).max())
    for k in ("x", "v", "F", "C"):
        r = ref["state0"][k]
        out[k] = float(np.abs(got[k] - r).max() / np.abs(r).max())
    return out


@pytest.mark.parametrize("pipe", PIPES)
def test_config5_segments_match_oracle_adjoint(M, pipe):
    """The benchmark's differentiable workload (the 30K slab, 500 sub-steps,
    checkpoints every 50) reversed one 50-sub-step segment at a time, on the
    GPU (mpm_tape_record / mpm_tape_backward from the GPU's own checkpoint
    state) and in the FP64 oracle, both seeded with the same incoming adjoint
    (the GPU's, from the segment after it; the loss gradient for the last).
    The oracle reverses each sub-step at the GPU's own forward state and grid
    of that sub-step, so no FP32 drift of the forward trajectory and no
    rounding of the forward grid (the fused pipeline's P2G rounds in 32-bit
    fixed point) enters: what is compared is the adjoint's arithmetic.  Per
    segment, dL/dE, dL/dnu, the outgoing state adjoint and every pose entry
    (against the largest entry of its coordinate in the segment) agree to 1e-3.

    Which states: on the split pipeline, a replay of the segment from its
    checkpoint, one sub-step per call (the split forward is deterministic, so
    it is the trajectory the reverse pass recomputes).  The fused forward is
    not bit-reproducible (its per-block partial grids are added with float
    reductions in any order, and the fixed-point arena turns a last-bit change
    of an input into a step of 2^-22 of the group's bound), which moves nodes
    under the capsule across the stick/slide kink of Eq. 18 from one run to
    the next.  So on the fused pipeline the states are the record of the very
    run that is reversed (mpm_tape_read_substep: a one-segment record is
    reversed without recomputation).  The run-to-run spread of the fused pose
    gradients is measured with a second run and printed."""
    import torch
    case = scenes.slab30k_diff()
    sc = case.scene
    prm = O.OracleParams.from_scene(sc)
    K, ck = case.poses.shape[0], case.checkpoint
    tool = sc.tools[0]
    dev = torch.device("cuda")

    def seg_sim(state, pose_start):
        sim = M.sim_from_scene(sc, pipeline=_pipe(M, pipe), load=False)
        sim.load(state["x"], sc.particle_volume, state["v"], state["F"], state["C"])
        sim.set_tool(0, pose_start, tool.shape)
        return sim

    # the GPU's forward trajectory, one sub-step per recorded call
    sim = M.sim_from_scene(sc, pipeline=_pipe(M, pipe), load=False)
    sim.load(sc.x, sc.particle_volume)
    sim.set_tool(0, case.pose_init[0], tool.shape)
    states = []
    for k in range(K):
        states.append(sim.read())
        sim.tape_record(case.poses[k:k + 1], 1)
    final = sim.read()
    sim.close()
    starts = [case.pose_init[0]] + [case.poses[s * ck - 1, 0] for s in range(1, K // ck)]
    # the loss seed from the FP64 target rollout
    tprm = O.OracleParams(**{**prm.__dict__, "E": case.target_E, "nu": case.target_nu})
    tgt = O.State(sc.x)
    tf, nt = O.rollout_frames(sc.tools, case.pose_init, case.target_poses, prm.dt)
    O.run(tprm, tgt, K, tf, nt)
    seed = {"x": (2.0 * (final["x"].astype(np.float64) - tgt.x) / sc.n).astype(np.float32),
            "v": np.zeros((sc.n, 3), np.float32), "F": np.zeros((sc.n, 9), np.float32),
            "C": np.zeros((sc.n, 9), np.float32)}
    worst = {}
    spreads, pose_errors = [], []
    for s in range(K // ck - 1, -1, -1):
        seg_poses = case.poses[s * ck:(s + 1) * ck]
        runs = []
        seg_states, seg_grids = [], []
        for r in range(2 if pipe == "fused" else 1):
            sim = seg_sim(states[s * ck], starts[s])
            sim.tape_record(seg_poses, ck)
            if pipe == "fused" and r == 0:
                # the states this run's reverse pass differentiates at
                for j in range(ck):
                    st = sim.tape_read_substep(j)
                    seg_states.append(O.State(st["x"], st["v"], st["C"], st["F"]))
                    seg_grids.append(st["grid"])
            runs.append(sim.tape_backward(*[torch.tensor(seed[k], device=dev) for k in ("x", "v", "F", "C")],
                                          want_state=True))
            sim.close()
        g = runs[0]
        got = {"E": g["E"], "nu": g["nu"], "poses": g["poses"]}
        got.update({k: g[k].cpu().numpy().astype(np.float64) for k in ("x", "v", "F", "C")})
        # the GPU's own run-to-run spread of the pose gradients (the fused forward is
        # not bit-reproducible: see the docstring)
        spread = 0.0
        if len(runs) > 1:
            scale = np.abs(g["poses"]).max(axis=0, keepdims=True)
            spread = float((np.abs(runs[1]["poses"] - g["poses"]) / np.maximum(scale, 1e-300)).max())
        spreads.append(spread)
        if pipe == "split":
            # the states the reverse pass differentiates at: its replay of the segment
            # from the checkpoint (a fresh load, then the recorded sub-steps one by one)
            rep = seg_sim(states[s * ck], starts[s])
            for k in range(s * ck, (s + 1) * ck):
                st = rep.read()
                seg_states.append(O.State(st["x"], st["v"], st["C"], st["F"]))
                seg_grids.append(rep.read_grid())
                rep.tape_record(case.poses[k:k + 1], 1)
            rep.close()
        ref = O.reverse_from_states(prm, seg_states, sc.tools, starts[s][None], seg_poses,
                                    {k: seed[k].astype(np.float64) for k in ("x", "v", "F", "C")}, grids=seg_grids)
        err = _segment_errors(got, ref)
        for k, v in err.items():
            worst[k] = max(worst.get(k, 0.0), v)
        assert all(v <= 1e-3 for v in err.values()), (s, err)
        pose_errors.append(err["poses"])
        seed = {k: g[k].cpu().numpy() for k in ("x", "v", "F", "C")}    # the GPU's own adjoint, upstream
    print("config-5 per-segment worst relative errors (%s):" % pipe, worst,
          "largest run-to-run pose spread:", max(spreads))
