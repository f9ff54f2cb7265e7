"""Shared helpers of the GPU parity tests: run the oracle on the exact FP32
state the GPU holds, and compare element by element."""
import numpy as np

from oracle import oracle as O
from paper_2402_01181_gb300 import scenes

PIPELINES = ("fused", "split")


def pipeline_id(name):
    from paper_2402_01181_gb300 import mpm
    return mpm.MPM_PIPELINE_FUSED if name == "fused" else mpm.MPM_PIPELINE_SPLIT


def oracle_state(out):
    """FP64 oracle state from a GPU readout dict (x, v, F, C float32)."""
    return O.State(out["x"].astype(np.float64), out["v"].astype(np.float64), out["C"].astype(np.float64),
                   out["F"].astype(np.float64))


def oracle_steps(sc, st, s0, nsteps, call_len=None):
    """Advance an oracle state by nsteps sub-steps of the scene starting at
    global sub-step s0, with tools driven by calls of call_len sub-steps."""
    prm = O.OracleParams.from_scene(sc)
    frames, nt = O.frames_for_steps(sc.tools, s0, nsteps, sc.dt, call_len)
    O.run(prm, st, nsteps, frames, nt)
    return st


def contact_mask_nodes(sc, st, s0, tol=1e-5):
    """Grid nodes whose oracle grid operation at global sub-step s0 (a call of
    one sub-step) sits within tol of a branch point (contact threshold,
    approaching test, friction clamp, z-buffer tie): FP32 and FP64 may take
    different branches there."""
    prm = O.OracleParams.from_scene(sc)
    gm, gmv = O.p2g(prm, st.copy())
    frames, nt = O.frames_for_steps(sc.tools, s0, 1, sc.dt, 1)
    _, _, margin = O.grid_update(prm, gm, gmv, frames, nt)
    return margin < tol


def particles_touching(mask_nodes, x, n_grid):
    """Particles whose 3x3x3 stencil includes a masked node."""
    if not mask_nodes.any():
        return np.zeros(x.shape[0], bool)
    base = np.clip(np.floor(x.astype(np.float64) * n_grid - 0.5).astype(np.int64), 0, n_grid - 3)
    hit = np.zeros(x.shape[0], bool)
    for i in range(3):
        for j in range(3):
            for k in range(3):
                hit |= mask_nodes[base[:, 0] + i, base[:, 1] + j, base[:, 2] + k]
    return hit


def rel_err(a, b, floor=0.0):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    if a.size == 0:
        return 0.0
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), floor))


def compare_particles(out, st, dx, skip=None, tol_x=None, tol_v=1e-5, tol_C=2e-4, tol_F=1e-5):
    """Single-step tolerances for FP32 against FP64 (see the design notes):
    positions to 1e-6 absolute (about 3e-5 dx at dx = 1/32), velocities and
    C relative to the largest reference magnitude, F absolute."""
    keep = np.ones(st.n, bool) if skip is None else ~skip
    tol_x = 1e-6 if tol_x is None else tol_x
    vmax = max(np.abs(st.v).max(), 1e-3)
    ex = np.abs(out["x"][keep] - st.x[keep]).max() if keep.any() else 0.0
    ev = np.abs(out["v"][keep] - st.v[keep]).max() / vmax if keep.any() else 0.0
    cfloor = 4.0 / dx * vmax * 1e-2
    eC = rel_err(out["C"][keep], st.C[keep], cfloor)
    eF = np.abs(out["F"][keep] - st.F[keep]).max() if keep.any() else 0.0
    errs = dict(x=ex, v=ev, C=eC, F=eF)
    ok = ex <= tol_x and ev <= tol_v and eC <= tol_C and eF <= tol_F
    return ok, errs


def perturbed_scene(sc, seed=0, v_scale=0.3, c_scale=2.0, f_dev=0.1):
    v, C, F = scenes.random_state(sc.x, seed, v_scale=v_scale, c_scale=c_scale, f_dev=f_dev)
    sc.v, sc.C, sc.F = v, C, F
    return sc
