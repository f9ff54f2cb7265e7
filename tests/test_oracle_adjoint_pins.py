"""Pins of the oracle's adjoint (reverse mode of one sub-step and of a
rollout) against central finite differences of the oracle's FORWARD step.
The forward step is itself pinned in test_oracle_pins.py; the differences
share no code with the hand-written adjoint, so a dropped term, a wrong sign
or a transposed operand in the adjoint fails here.

The scenes are small (16^3 grid, a few hundred particles) with two tools in
contact, friction on (sliding and sticking nodes), nonzero stress, and
particles moving across cells.  The difference steps are chosen where the
FP64 central differences converge (to 1e-8 relative or better, checked by
shrinking h), and the bar is 1e-5 relative: a planted mistake moves the
result by far more."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2402_01181_gb300 import scenes


def _scene(seed=0, n=16, N=300, dt=1e-3):
    rng = np.random.default_rng(seed)
    x = 0.3 + 0.4 * rng.random((N, 3))
    v, C, F = scenes.random_state(x.astype(np.float32), seed + 1, v_scale=0.4, c_scale=1.5, f_dev=0.12)
    prm = O.OracleParams(n_grid=n, dt=dt, E=3e3, nu=0.32, rho=1e3, V0=(0.4 ** 3) / N, bound=3,
                         theta=0.0, friction=0.35)
    st = O.State(x, v.astype(np.float64), C.astype(np.float64), F.astype(np.float64))
    tools = [scenes.Tool(scenes.capsule_shape(0.09, 0.07), None), scenes.Tool(scenes.box_shape(0.09, 0.08, 0.09), None)]
    pose0 = np.array([[0.47, 0.60, 0.52, 0.3, 0.1, 0.2], [0.56, 0.38, 0.45, 0.0, 0.4, 0.1]])
    pose1 = pose0 + np.array([[0.002, -0.004, 0.001, 0.02, -0.01, 0.015], [-0.003, 0.004, 0.002, 0.0, 0.03, -0.02]])
    return prm, st, tools, pose0, pose1


def _frames(tools, pose0, pose1, dt):
    arr = (O.ToolFrame * len(tools))()
    for t, tool in enumerate(tools):
        arr[t] = O.tool_frames(tool.shape, pose0[t], pose1[t], 1, dt)[0]
    return arr


def _step(prm, st, frames, nt):
    s = st.copy()
    O.run(prm, s, 1, frames, nt)
    return s


def _dot(bar, st):
    return sum(float(np.sum(bar[k] * getattr(st, k))) for k in ("x", "v", "C", "F"))


def _random_bar(rng, n):
    return {"x": rng.normal(size=(n, 3)), "v": rng.normal(size=(n, 3)) * 1e-2,
            "C": rng.normal(size=(n, 9)) * 1e-3, "F": rng.normal(size=(n, 9))}


def test_contact_branches_are_exercised():
    prm, st, tools, p0, p1 = _scene()
    frames = _frames(tools, p0, p1, prm.dt)
    gm, gmv = O.p2g(prm, st.copy())
    _, contact, margin = O.grid_update(prm, gm, gmv, frames, 2)
    assert (contact == 0).sum() > 10 and (contact == 1).sum() > 10
    assert margin[contact >= 0].min() > 1e-6      # no node within FD reach of a branch point


@pytest.mark.parametrize("block", ["x", "v", "C", "F"])
def test_step_adjoint_state_blocks_match_central_differences(block):
    prm, st, tools, p0, p1 = _scene()
    frames = _frames(tools, p0, p1, prm.dt)
    rng = np.random.default_rng(5)
    ybar = _random_bar(rng, st.n)
    xbar, _, _ = O.step_adjoint(prm, st, frames, 2, ybar)
    h = 1e-6 if block == "x" else 1e-5
    for trial in range(3):
        d = rng.normal(size=getattr(st, block).shape)
        a, b = st.copy(), st.copy()
        getattr(a, block)[...] += h * d
        getattr(b, block)[...] -= h * d
        fd = (_dot(ybar, _step(prm, a, frames, 2)) - _dot(ybar, _step(prm, b, frames, 2))) / (2 * h)
        an = float(np.sum(xbar[block] * d))
        assert abs(fd - an) <= 1e-5 * abs(fd), (block, trial, fd, an)


def test_step_adjoint_material_matches_central_differences():
    prm, st, tools, p0, p1 = _scene()
    frames = _frames(tools, p0, p1, prm.dt)
    rng = np.random.default_rng(6)
    ybar = _random_bar(rng, st.n)
    _, lame, _ = O.step_adjoint(prm, st, frames, 2, ybar)
    Eb, nub = O.lame_vjp(prm.E, prm.nu, lame[0], lame[1])
    for name, an, h in (("E", Eb, 1e-3), ("nu", nub, 1e-7)):
        pa = O.OracleParams(**{**prm.__dict__, name: getattr(prm, name) + h})
        pb = O.OracleParams(**{**prm.__dict__, name: getattr(prm, name) - h})
        fd = (_dot(ybar, _step(pa, st, frames, 2)) - _dot(ybar, _step(pb, st, frames, 2))) / (2 * h)
        assert abs(fd - an) <= 1e-5 * abs(fd), (name, fd, an)


@pytest.mark.parametrize("field,sl", [("R", slice(0, 9)), ("T", slice(9, 12)), ("u", slice(12, 15)),
                                      ("w", slice(15, 18))])
def test_step_adjoint_tool_frames_match_central_differences(field, sl):
    prm, st, tools, p0, p1 = _scene()
    frames = _frames(tools, p0, p1, prm.dt)
    rng = np.random.default_rng(7)
    ybar = _random_bar(rng, st.n)
    _, _, tb = O.step_adjoint(prm, st, frames, 2, ybar)
    h = 1e-5 if field in ("R", "T") else 1e-4
    for t in range(2):
        d = rng.normal(size=sl.stop - sl.start)
        fa, fb = _frames(tools, p0, p1, prm.dt), _frames(tools, p0, p1, prm.dt)
        for q in range(len(d)):
            getattr(fa[t], field)[q] += h * d[q]
            getattr(fb[t], field)[q] -= h * d[q]
        fd = (_dot(ybar, _step(prm, st, fa, 2)) - _dot(ybar, _step(prm, st, fb, 2))) / (2 * h)
        an = float(tb[t, sl] @ d)
        assert abs(fd - an) <= 1e-5 * abs(fd), (field, t, fd, an)


def test_rollout_gradients_match_central_differences():
    """Five sub-steps with pose streams, loss = mean |x(T) - target|^2: the
    gradients with respect to E, nu and pose entries of both tools (through
    the frame map, sub-steps inside and at the ends of the stream) against
    central differences of the forward rollout; checkpoints every 2
    sub-steps exercise the segment recomputation."""
    prm, st, tools, p0, p1 = _scene(seed=3, dt=2e-3)
    K = 5
    rng = np.random.default_rng(8)
    vel = p1 - p0
    poses = np.stack([p0 + (k + 1) * vel for k in range(K)])
    target = st.x + 0.01 * rng.normal(size=st.x.shape)
    g = O.rollout_loss_and_gradients(prm, st, tools, p0, poses, target, checkpoint=2)

    def loss(prm_, poses_):
        return O.rollout_loss_and_gradients(prm_, st, tools, p0, poses_, target, checkpoint=K)["loss"]

    for name, h in (("E", 1e-2), ("nu", 1e-7)):
        pa = O.OracleParams(**{**prm.__dict__, name: getattr(prm, name) + h})
        pb = O.OracleParams(**{**prm.__dict__, name: getattr(prm, name) - h})
        fd = (loss(pa, poses) - loss(pb, poses)) / (2 * h)
        assert abs(fd - g[name]) <= 1e-5 * abs(fd), (name, fd, g[name])
    for (k, t, c) in ((0, 0, 1), (2, 0, 4), (4, 0, 0), (1, 1, 2), (3, 1, 5), (4, 1, 3)):
        h = 1e-7
        pa, pb = poses.copy(), poses.copy()
        pa[k, t, c] += h
        pb[k, t, c] -= h
        fd = (loss(prm, pa) - loss(prm, pb)) / (2 * h)
        an = g["poses"][k, t, c]
        assert abs(fd - an) <= 1e-4 * max(abs(fd), 1e-6 * np.abs(g["poses"]).max()), ((k, t, c), fd, an)


def _left_jacobian(r):
    """The left Jacobian of SO(3) in its textbook closed form,
    J(r) = I + (1 - cos t)/t^2 [r]x + (t - sin t)/t^3 [r]x^2, t = |r|: the
    derivative of the rotation vector of R(r + e) R(r)^T at e = 0."""
    t = float(np.linalg.norm(r))
    K = np.array([[0.0, -r[2], r[1]], [r[2], 0.0, -r[0]], [-r[1], r[0], 0.0]])
    return np.eye(3) + (1 - np.cos(t)) / t ** 2 * K + (t - np.sin(t)) / t ** 3 * K @ K


@pytest.mark.parametrize("case", range(6))
def test_frame_jacobian_matches_central_differences(case):
    """The closed-form derivative of the one-sub-step frame map (Rodrigues'
    formula and its inverse) against central differences of the oracle's
    forward frames (orc_tool_frames), from rotations below the series
    threshold of the closed forms to rotations of ~1 rad and relative turns
    of up to 0.4 rad within the call."""
    rng = np.random.default_rng(40 + case)
    rot = (1e-5, 5e-4, 0.3, 1.2, 2.5, 0.05)[case]
    turn = (1e-6, 2e-4, 0.02, 0.4, 0.1, 0.3)[case]
    p0 = np.concatenate([rng.uniform(0.3, 0.7, 3), rot * rng.normal(size=3) / np.sqrt(3)])
    p1 = p0 + np.concatenate([1e-3 * rng.normal(size=3), turn * rng.normal(size=3) / np.sqrt(3)])
    dt = 5e-5
    shape = scenes.capsule_shape(0.02, 0.15)
    Ja = O.frame_jacobian(shape, p0, p1, dt)
    Jd = O.frame_jacobian_differences(shape, p0, p1, dt, h=1e-5)
    for row in range(18):
        scale = max(np.abs(Jd[row]).max(), 1e-12)
        assert np.abs(Ja[row] - Jd[row]).max() <= 1e-6 * scale, (row, Ja[row], Jd[row])


def test_frame_jacobian_closed_forms():
    """Special cases the derivative must reproduce exactly: with one sub-step
    per call the frame's R is R(r1) and T is T1, so neither depends on pose0;
    u = (T1 - T0)/dt; at r0 = r1 = r the angular velocity w = log(R1 R0^T)/dt
    moves by J(r)/dt with r1 and by -J(r)/dt with r0 (J: the left Jacobian
    of SO(3)); at r = 0, dR/dr_i is the generator [e_i]x."""
    dt = 1e-4
    shape = scenes.capsule_shape(0.02, 0.15)
    for r in (np.zeros(3), np.array([0.3, -0.5, 0.8]), np.array([1e-4, 2e-4, -1e-4])):
        p = np.concatenate([[0.4, 0.5, 0.6], r])
        J = O.frame_jacobian(shape, p, p, dt)
        assert np.abs(J[0:12, 0:6]).max() <= 1e-12                       # R, T independent of pose0
        assert np.allclose(J[9:12, 6:9], np.eye(3), atol=0) and np.abs(J[9:12, 9:12]).max() == 0
        assert np.allclose(J[12:15, 0:3], -np.eye(3) / dt, rtol=1e-15) and np.allclose(J[12:15, 6:9], np.eye(3) / dt)
        Jl = np.eye(3) if not r.any() else _left_jacobian(r)
        assert np.abs(J[15:18, 9:12] - Jl / dt).max() <= 1e-9 / dt
        assert np.abs(J[15:18, 3:6] + Jl / dt).max() <= 1e-9 / dt
    J = O.frame_jacobian(shape, np.zeros(6), np.zeros(6), dt)
    for i in range(3):
        gen = np.zeros((3, 3))
        gen[(i + 2) % 3, (i + 1) % 3], gen[(i + 1) % 3, (i + 2) % 3] = 1.0, -1.0
        assert np.array_equal(J[0:9, 9 + i].reshape(3, 3), gen)


@pytest.mark.parametrize("block", ["x", "v"])
def test_step_adjoint_near_the_walls_matches_central_differences(block):
    """Particles resting near the floor and a side wall, whose stencils reach
    the sticky band of the grid operation (Sec. III-B, reading c4): the
    forward step zeroes those nodes' velocities, so nothing flows back
    through them, and the adjoint must agree with central differences."""
    rng = np.random.default_rng(8)
    N, n, dt = 200, 16, 1e-3
    x = np.stack([0.06 + 0.3 * rng.random(N), 0.07 + 0.3 * rng.random(N), 0.3 + 0.4 * rng.random(N)], axis=1)
    v, C, F = scenes.random_state(x.astype(np.float32), 9, v_scale=0.4, c_scale=1.5, f_dev=0.12)
    prm = O.OracleParams(n_grid=n, dt=dt, E=3e3, nu=0.32, rho=1e3, V0=(0.3 ** 3) / N, bound=3,
                         gravity=(0.0, -9.8, 0.0))
    st = O.State(x, v.astype(np.float64), C.astype(np.float64), F.astype(np.float64))
    frames = (O.ToolFrame * 1)()
    base = np.floor(x * n - 0.5).astype(int)
    assert (base.min(axis=1) < 3).sum() > 50                  # stencils inside the wall band
    ybar = _random_bar(rng, N)
    xbar, _, _ = O.step_adjoint(prm, st, frames, 0, ybar)
    h = 1e-6 if block == "x" else 1e-5
    for trial in range(3):
        d = rng.normal(size=getattr(st, block).shape)
        a, b = st.copy(), st.copy()
        getattr(a, block)[...] += h * d
        getattr(b, block)[...] -= h * d
        fd = (_dot(ybar, _step(prm, a, frames, 0)) - _dot(ybar, _step(prm, b, frames, 0))) / (2 * h)
        an = float(np.sum(xbar[block] * d))
        assert abs(fd - an) <= 1e-5 * abs(fd), (block, trial, fd, an)


def test_reverse_from_states_is_the_rollout_reverse():
    """Given the oracle's own forward states, the reverse along a supplied
    trajectory is the checkpointed rollout's reverse: the same sub-step
    adjoints in the same order, so the results are identical."""
    prm, st, tools, p0, p1 = _scene(seed=5, dt=2e-3)
    K = 4
    poses = np.stack([p0 + (k + 1) * (p1 - p0) for k in range(K)])
    target = st.x + 0.01
    ref = O.rollout_loss_and_gradients(prm, st, tools, p0, poses, target, checkpoint=3)
    frames, nt = O.rollout_frames(tools, p0, poses, prm.dt)
    states, s = [], st.copy()
    for k in range(K):
        states.append(s.copy())
        arr = (O.ToolFrame * nt)()
        for t in range(nt):
            arr[t] = frames[k * nt + t]
        O.run(prm, s, 1, arr, nt)
    got = O.reverse_from_states(prm, states, tools, p0, poses, {"x": 2.0 * (s.x - target) / s.n})
    assert got["E"] == ref["E"] and got["nu"] == ref["nu"]
    assert np.array_equal(got["poses"], ref["poses"])
    for k in ("x", "v", "C", "F"):
        assert np.array_equal(got["state0"][k], ref["state0"][k])


def test_step_adjoint_at_its_own_grid_is_the_step_adjoint():
    """Evaluated at a supplied grid that is the P2G of the state itself, the
    reverse sub-step is the plain one, bit for bit; at a perturbed grid the
    grid operation and G2P see the perturbation (the sub-step's forward at
    that grid differs) while the P2G reverse is unchanged in form."""
    prm, st, tools, p0, p1 = _scene(seed=7)
    frames = _frames(tools, p0, p1, prm.dt)
    rng = np.random.default_rng(9)
    bar = _random_bar(rng, st.n)
    gm, gmv = O.p2g(prm, st.copy())
    grid = np.concatenate([gm[..., None], gmv], axis=-1)
    a = O.step_adjoint(prm, st, frames, 2, bar)
    b = O.step_adjoint(prm, st, frames, 2, bar, grid=grid)
    for k in ("x", "v", "C", "F"):
        assert np.array_equal(a[0][k], b[0][k])
    assert np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])
    grid2 = grid.copy()
    grid2[..., 1:] *= 1.001
    c = O.step_adjoint(prm, st, frames, 2, bar, grid=grid2)
    assert not np.array_equal(a[0]["x"], c[0]["x"])
