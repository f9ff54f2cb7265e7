"""Seeded synthetic scenes for the MLS-MPM soft-tissue step.

This module is the one place that both the CUDA path and the FP64 oracle take
their inputs from.  It holds geometry and scripted trajectories only: particle
positions (jittered lattices, uniform boxes), material and grid settings, and
tool poses per sub-step.  It contains none of the method's arithmetic (no
weights, stresses, Lame parameters or collision handling), so sharing it does
not couple the two implementations.

The paper's scenes (a tissue slab of ~24K-30K particles on a table, a 64^3
grid, Sec. IV-A and Table II) are not distributed; these generators stand in
for them with the sizes, densities and tool motions stated per scene below.
Random numbers come from numpy's PCG64 generator with an explicit seed.
"""
from __future__ import annotations

import functools
from dataclasses import dataclass, field
from typing import Callable, List, Optional, Sequence

import numpy as np

# Tool shape kinds, matching the `shape[0]` code of the C ABI.
CAPSULE = 0
BOX = 1
SAMPLED = 2


@dataclass
class SampledField:
    """A distance field precomputed on a cubic lattice in a tool's reference
    frame (the offline SDF of Sec. III-C): samples[k, j, i] is the distance
    at origin + h * (i, j, k); res = samples.shape[0]."""
    samples: np.ndarray                # (res, res, res) float32, x fastest
    origin: np.ndarray                 # (3,) float64
    h: float

    @property
    def res(self) -> int:
        return int(self.samples.shape[0])


@dataclass
class Tool:
    """One rigid collision shape with a scripted pose stream.

    shape: 8 floats -- [kind, a, b, c, 0, 0, 0, 0]; capsule: a = radius,
    b = half-length of the axis segment along local y; box: (a, b, c) = half
    extents; sampled: the distances come from `field`.  pose(s) returns the
    6-vector (T xyz, rotation vector xyz) the tool has at the END of global
    sub-step s (s = 0, 1, ...); pose(-1) is the starting pose.
    """
    shape: np.ndarray
    pose: Callable[[int], np.ndarray]
    field: Optional[SampledField] = None


@dataclass
class Scene:
    name: str
    n_grid: int
    dt: float
    E: float
    nu: float
    rho: float
    x: np.ndarray                      # (N, 3) float32 positions
    particle_volume: float             # initial volume V_p^0 of every particle
    gravity: Sequence[float] = (0.0, -9.8, 0.0)
    bound: int = 3                     # sticky wall band, in nodes
    friction: float = 0.0
    theta: float = 0.0
    tools: List[Tool] = field(default_factory=list)
    v: Optional[np.ndarray] = None     # (N, 3) float32 or None (zero)
    F: Optional[np.ndarray] = None     # (N, 9) float32 or None (identity)
    C: Optional[np.ndarray] = None     # (N, 9) float32 or None (zero)

    @property
    def n(self) -> int:
        return int(self.x.shape[0])

    @property
    def dx(self) -> float:
        return 1.0 / self.n_grid


def jittered_lattice(cell_lo, cell_hi, n_grid, sub, seed):
    """Particles on a jittered sub-lattice of the cells [cell_lo, cell_hi).

    Every cell of the box holds sub[0]*sub[1]*sub[2] particles, one per
    sub-cell, placed uniformly at random inside its sub-cell.  Particles are
    emitted cell by cell (x fastest, then y, then z) and sub-cell by sub-cell
    inside a cell, so consecutive ids are spatial neighbours.
    """
    rng = np.random.default_rng(seed)
    lo = np.asarray(cell_lo, dtype=np.int64)
    hi = np.asarray(cell_hi, dtype=np.int64)
    sub = np.asarray(sub, dtype=np.int64)
    ext = hi - lo
    cz, cy, cx = np.meshgrid(np.arange(ext[2]), np.arange(ext[1]), np.arange(ext[0]), indexing="ij")
    cells = np.stack([cx.ravel(), cy.ravel(), cz.ravel()], axis=1) + lo          # (ncell, 3)
    sz, sy, sx = np.meshgrid(np.arange(sub[2]), np.arange(sub[1]), np.arange(sub[0]), indexing="ij")
    subs = np.stack([sx.ravel(), sy.ravel(), sz.ravel()], axis=1)                # (nsub, 3)
    pos = cells[:, None, :].astype(np.float64) + (subs[None, :, :] + rng.random((cells.shape[0], subs.shape[0], 3))) / sub
    return (pos.reshape(-1, 3) / n_grid).astype(np.float32)


def uniform_box(lo, hi, count, seed):
    rng = np.random.default_rng(seed)
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    return (lo + (hi - lo) * rng.random((count, 3))).astype(np.float32)


def _linear_path(p0, waypoints):
    """Piecewise-linear pose stream.

    waypoints: list of (end_substep, displacement 3-vector) -- the tool moves
    uniformly so that at the end of sub-step end_substep-1 it has reached the
    given displacement from p0; after the last waypoint it keeps the last
    segment's velocity.
    """
    p0 = np.asarray(p0, dtype=np.float64)
    segs = []
    s_prev, d_prev = 0, np.zeros(3)
    for s_end, disp in waypoints:
        disp = np.asarray(disp, dtype=np.float64)
        segs.append((s_prev, s_end, d_prev, disp))
        s_prev, d_prev = s_end, disp

    def pose(s):
        k = s + 1                       # sub-steps completed
        for (a, b, d0, d1) in segs:
            if k <= b or (a, b, d0, d1) == segs[-1]:
                t = (k - a) / float(b - a)
                d = d0 + t * (d1 - d0)
                out = np.zeros(6)
                out[:3] = p0[:3] + d
                out[3:] = p0[3:]
                return out
        raise AssertionError

    return pose


def capsule_shape(radius, half_length):
    s = np.zeros(8, dtype=np.float32)
    s[0] = CAPSULE
    s[1] = radius
    s[2] = half_length
    return s


def box_shape(hx, hy, hz):
    s = np.zeros(8, dtype=np.float32)
    s[0] = BOX
    s[1:4] = (hx, hy, hz)
    return s


def sampled_shape():
    s = np.zeros(8, dtype=np.float32)
    s[0] = SAMPLED
    return s


# --------------------------------------------------------------------------
# Rasterised tool geometry.  The paper's tool meshes are not distributed, so
# sampled fields are made from simple solids: the distance to a union of
# capsules and boxes (exact outside the union, a bound inside it).
# --------------------------------------------------------------------------

def _capsule_distance(p, radius, half_length):
    c = np.clip(p[..., 1], -half_length, half_length)
    q = p.copy()
    q[..., 1] -= c
    return np.linalg.norm(q, axis=-1) - radius


def _box_distance(p, center, half):
    q = np.abs(p - np.asarray(center)) - np.asarray(half)
    outside = np.linalg.norm(np.maximum(q, 0.0), axis=-1)
    inside = np.minimum(q.max(axis=-1), 0.0)
    return outside + inside


def rasterize(distance: Callable[[np.ndarray], np.ndarray], origin, h: float, res: int) -> SampledField:
    """Sample distance(p) at origin + h (i, j, k), one z slab at a time."""
    origin = np.asarray(origin, dtype=np.float64)
    out = np.empty((res, res, res), dtype=np.float32)
    ii = np.arange(res, dtype=np.float64)
    gy, gx = np.meshgrid(ii, ii, indexing="ij")
    for k in range(res):
        p = np.stack([origin[0] + h * gx, origin[1] + h * gy, np.full_like(gx, origin[2] + h * k)], axis=-1)
        out[k] = distance(p)
    return SampledField(out, origin, float(h))


@functools.lru_cache(maxsize=4)
def grasper_field(res: int = 256, radius: float = 0.012, half_length: float = 0.12,
                  jaw=(0.006, 0.02, 0.012), gap: float = 0.008) -> SampledField:
    """A grasper stand-in: a shaft (capsule along local y, centred at the
    origin) ending in two parallel jaws (boxes of half extents `jaw`, 2*gap
    apart in x) below its lower end.  The field covers the cube centred on
    the solid's bounding box with a margin of 3.3 samples (a spacing that is
    no simple fraction of a grid cell, so that grid nodes do not sit on
    sample-cell faces)."""
    jaw_y = -half_length - radius - jaw[1]
    centers = [(gap + jaw[0], jaw_y, 0.0), (-gap - jaw[0], jaw_y, 0.0)]
    lo_y = jaw_y - jaw[1]
    hi_y = half_length + radius
    side = max(hi_y - lo_y, 2 * (gap + 2 * jaw[0]), 2 * radius)
    h = side / (res - 6.6)
    mid_y = 0.5 * (lo_y + hi_y)
    origin = np.array([-0.5 * side - 3.3 * h, mid_y - 0.5 * side - 3.3 * h, -0.5 * side - 3.3 * h])

    def dist(p):
        d = _capsule_distance(p, radius, half_length)
        for c in centers:
            d = np.minimum(d, _box_distance(p, c, jaw))
        return d

    return rasterize(dist, origin, h, res)


# --------------------------------------------------------------------------
# The workloads.  Sizes follow the paper's scale (30K particles, 64^3 grid,
# rho = 1000 kg/m^3, Sec. IV) and the roofline sweep (1M / 8M particles).
# --------------------------------------------------------------------------

def cube8k(seed: int = 0) -> Scene:
    """8,192 particles (16 per cell, 2x2x4 jittered sub-cells) filling the
    cube [0.375, 0.625]^3 on a 32^3 grid; free fall, no tool."""
    n = 32
    x = jittered_lattice((12, 12, 12), (20, 20, 20), n, (2, 2, 4), seed)
    return Scene("cube8k", n_grid=n, dt=1e-4, E=5e3, nu=0.3, rho=1e3, x=x,
                 particle_volume=0.25 ** 3 / x.shape[0])


def slab30k(seed: int = 0) -> Scene:
    """30,000 particles uniform in a 0.6 x 0.1 x 0.6 m tissue slab lying on
    the floor band of a 64^3 grid, pressed and then dragged by a capsule
    (r = 0.02 m, axis segment 0.3 m, vertical).  Sub-steps 0-999: the tip
    descends 0.05 m; sub-steps 1000-1999: it slides 0.10 m along +x."""
    n = 64
    dx = 1.0 / n
    y0 = 3 * dx
    x = uniform_box((0.2, y0, 0.2), (0.8, y0 + 0.1, 0.8), 30000, seed)
    r, h = 0.02, 0.15
    tip0 = y0 + 0.1 + 0.005
    p0 = np.array([0.5, tip0 + r + h, 0.5, 0.0, 0.0, 0.0])
    pose = _linear_path(p0, [(1000, (0.0, -0.05, 0.0)), (2000, (0.10, -0.05, 0.0))])
    return Scene("slab30k", n_grid=n, dt=5e-5, E=1e4, nu=0.35, rho=1e3, x=x,
                 particle_volume=0.6 * 0.1 * 0.6 / 30000, friction=0.3,
                 tools=[Tool(capsule_shape(r, h), pose)])


def _block(n, cells, seed, name):
    lo_xz = n // 2 - cells // 2
    x = jittered_lattice((lo_xz, 3, lo_xz), (lo_xz + cells, 3 + cells, lo_xz + cells), n, (2, 2, 2), seed)
    dx = 1.0 / n
    top = (3 + cells) * dx
    r, h = 0.02, 0.15
    p0 = np.array([0.5, top + r + h, 0.5, 0.0, 0.0, 0.0])
    dt = 2e-5
    speed = 0.5                                  # m/s, downwards
    steps = 1000
    pose = _linear_path(p0, [(steps, (0.0, -speed * dt * steps, 0.0))])
    return Scene(name, n_grid=n, dt=dt, E=1e4, nu=0.3, rho=1e3, x=x,
                 particle_volume=dx ** 3 / 8, friction=0.3,
                 tools=[Tool(capsule_shape(r, h), pose)])


def block1m(seed: int = 0) -> Scene:
    """1,000,000 particles: a 50^3-cell block (8 per cell, 2x2x2 jittered)
    on the floor of a 128^3 grid, centred in x and z; a capsule indents the
    top centre at 0.5 m/s starting from contact."""
    return _block(128, 50, seed, "block1m")


def block8m(seed: int = 0) -> Scene:
    """8,000,000 particles: a 100^3-cell block on a 256^3 grid, otherwise as
    block1m."""
    return _block(256, 100, seed, "block8m")


def slab30k_sdf(seed: int = 0, res: int = 256) -> Scene:
    """slab30k with the capsule replaced by a sampled grasper field (res^3
    samples, the paper's 256 by default): its jaws press 0.05 m into the slab
    over sub-steps 0-999, then it drags 0.10 m along +x while turning 0.3 rad
    about its axis over sub-steps 1000-1999."""
    sc = slab30k(seed)
    field = grasper_field(res, radius=0.02, half_length=0.15, jaw=(0.012, 0.03, 0.02), gap=0.012)
    tip = -field.origin[1] - 3.3 * field.h         # depth of the jaw tips below the origin
    p0 = np.array([0.5013, 3.0 / 64 + 0.1 + 0.005 + tip, 0.4987, 0.0, 0.0, 0.0])
    down = _linear_path(p0, [(1000, (0.0, -0.05, 0.0))])

    def pose(s):
        if s < 1000:
            return down(s)
        t = min((s + 1 - 1000) / 1000.0, 1.0)
        out = down(999).copy()
        out[0] += 0.10 * t
        out[4] = 0.3 * t
        return out

    sc.name = "slab30k_sdf"
    sc.tools = [Tool(sampled_shape(), pose, field)]
    return sc


@dataclass
class DiffCase:
    """A differentiable-rollout workload: the scene, the pose stream of its
    tool (pose_init, then poses[k, t] at the end of sub-step k), and the
    perturbed stream and material a target rollout uses."""
    scene: Scene
    pose_init: np.ndarray              # (n_tools, 6)
    poses: np.ndarray                  # (K, n_tools, 6)
    target_poses: np.ndarray           # (K, n_tools, 6)
    target_E: float
    target_nu: float
    checkpoint: int


def slab30k_diff(seed: int = 0, steps: int = 500, checkpoint: int = 50, first: int = 0) -> DiffCase:
    """The slab30k scene (at rest) over sub-steps first .. first+steps-1 of
    its tool script (from sub-step 0 the capsule descends onto the slab,
    touching it near sub-step 100, and presses in), the rollout checkpointed
    every `checkpoint` sub-steps; the target uses E = 1.2e4, nu = 0.33 and the pose
    stream shifted by one seeded N(0, 1e-3) draw per pose entry (m, rad),
    the same at every sub-step, so that the target tool moves as smoothly as
    the original."""
    sc = slab30k(seed)
    tool = sc.tools[0]
    pose_init = tool.pose(first - 1)[None, :]
    poses = np.stack([tool.pose(first + k) for k in range(steps)])[:, None, :]
    rng = np.random.default_rng(seed + 12345)
    target = poses + rng.normal(0.0, 1e-3, size=(1, 1, 6))
    return DiffCase(sc, pose_init, poses, target, 1.2e4, 0.33, checkpoint)


SCENES = {
    "cube8k": cube8k,
    "slab30k": slab30k,
    "slab30k_sdf": slab30k_sdf,
    "block1m": block1m,
    "block8m": block8m,
}


def random_state(x: np.ndarray, seed: int, v_scale=0.5, c_scale=2.0, f_dev=0.15):
    """Random (v, C, F) for a given set of positions: v uniform in
    [-v_scale, v_scale]^3, C uniform in [-c_scale, c_scale]^(3x3), and
    F = I + uniform noise of amplitude f_dev (so J stays near 1)."""
    rng = np.random.default_rng(seed)
    n = x.shape[0]
    v = (v_scale * (2 * rng.random((n, 3)) - 1)).astype(np.float32)
    C = (c_scale * (2 * rng.random((n, 9)) - 1)).astype(np.float32)
    F = (np.eye(3).reshape(1, 9) + f_dev * (2 * rng.random((n, 9)) - 1)).astype(np.float32)
    return v, C, F


def batch_envs(n_envs: int = 256, seed: int = 0, n_min: int = 5000, n_max: int = 40000) -> List[Scene]:
    """Independent tissue scenes for batched stepping, each on its own 64^3
    grid: N_e uniform in [n_min, n_max], a slab 0.6 s x 0.1 x 0.6 s m with
    s = sqrt(N_e / 30000) (so the particle density matches slab30k),
    E_e in [2e3, 2e4] Pa, nu_e in [0.2, 0.45], and a capsule following the
    slab30k trajectory shifted by an x,z offset in [-0.1, 0.1] m and pressing
    to a depth in [0.02, 0.05] m."""
    rng = np.random.default_rng(seed)
    n = 64
    dx = 1.0 / n
    y0 = 3 * dx
    out = []
    for e in range(n_envs):
        N = int(rng.integers(n_min, n_max + 1))
        sz = 0.6 * np.sqrt(N / 30000.0)
        x = uniform_box((0.5 - sz / 2, y0, 0.5 - sz / 2), (0.5 + sz / 2, y0 + 0.1, 0.5 + sz / 2), N,
                        int(rng.integers(1 << 31)))
        E = float(rng.uniform(2e3, 2e4))
        nu = float(rng.uniform(0.2, 0.45))
        off = rng.uniform(-0.1, 0.1, size=2)
        depth = float(rng.uniform(0.02, 0.05))
        r, h = 0.02, 0.15
        tip0 = y0 + 0.1 + 0.005
        p0 = np.array([0.5 + off[0], tip0 + r + h, 0.5 + off[1], 0.0, 0.0, 0.0])
        pose = _linear_path(p0, [(1000, (0.0, -depth, 0.0)), (2000, (0.10, -depth, 0.0))])
        out.append(Scene("env%d" % e, n_grid=n, dt=5e-5, E=E, nu=nu, rho=1e3, x=x,
                         particle_volume=sz * 0.1 * sz / N, friction=0.3,
                         tools=[Tool(capsule_shape(r, h), pose)]))
    return out
