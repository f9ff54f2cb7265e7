"""ctypes front end of the FP64 MLS-MPM oracle (oracle/mpm_oracle.c).

TEST INFRASTRUCTURE ONLY: the tests, the package smoke check and the
benchmark's CPU-baseline leg use this module; the CUDA library never does.
It builds the C file with gcc (strict IEEE double: no fast-math, no FMA
contraction, so results agree between x86-64 and aarch64 hosts) into
oracle/_build/ and wraps each entry point with numpy arrays.
"""
from __future__ import annotations

import ctypes as ct
import os
import subprocess
import threading
from dataclasses import dataclass
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mpm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libmpm_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle shared library if it is missing or stale."""
    import fcntl
    os.makedirs(_BUILD, exist_ok=True)
    with open(os.path.join(_BUILD, ".lock"), "w") as fh:
        fcntl.flock(fh, fcntl.LOCK_EX)
        _build_locked(force)
    return _LIB


def _build_locked(force):
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp.%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
                               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)


class Params(ct.Structure):
    _fields_ = [("n_grid", ct.c_int32), ("bound", ct.c_int32), ("dt", ct.c_double),
                ("gravity", ct.c_double * 3), ("E", ct.c_double), ("nu", ct.c_double),
                ("rho", ct.c_double), ("V0", ct.c_double), ("theta", ct.c_double),
                ("friction", ct.c_double)]


class ToolFrame(ct.Structure):
    _fields_ = [("kind", ct.c_int32), ("res", ct.c_int32), ("dims", ct.c_double * 3),
                ("R", ct.c_double * 9), ("T", ct.c_double * 3), ("u", ct.c_double * 3),
                ("w", ct.c_double * 3), ("h", ct.c_double), ("sdf", ct.POINTER(ct.c_float))]


class Counters(ct.Structure):
    _fields_ = [("j_clamped", ct.c_int64), ("out_of_domain", ct.c_int64)]


_D = ct.POINTER(ct.c_double)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            # ORACLE_LIB lets the mutation tests load a deliberately broken copy.
            L = ct.CDLL(os.environ.get("ORACLE_LIB") or build())
            P = ct.POINTER(Params)
            TF = ct.POINTER(ToolFrame)
            CN = ct.POINTER(Counters)
            L.orc_lame.argtypes = [ct.c_double, ct.c_double, _D, _D]
            L.orc_piola.argtypes = [ct.c_double, ct.c_double, _D, _D]
            L.orc_piola.restype = ct.c_int
            L.orc_piola_FT.argtypes = [ct.c_double, ct.c_double, _D, _D]
            L.orc_piola_FT.restype = ct.c_int
            L.orc_weights.argtypes = [ct.c_double, _D]
            L.orc_p2g.argtypes = [P, ct.c_int64, _D, _D, _D, _D, _D, _D, CN]
            L.orc_rotvec_to_matrix.argtypes = [_D, _D]
            L.orc_matrix_to_rotvec.argtypes = [_D, _D]
            L.orc_tool_frames.argtypes = [ct.c_int32, _D, _D, _D, ct.c_int32, ct.c_double, TF]
            L.orc_sdf.argtypes = [ct.c_int32, _D, _D, _D]
            L.orc_sdf.restype = ct.c_double
            L.orc_sdf_sampled.argtypes = [ct.POINTER(ct.c_float), ct.c_int32, _D, ct.c_double, _D, _D, _D]
            L.orc_sdf_sampled.restype = ct.c_double
            L.orc_grid_update.argtypes = [P, TF, ct.c_int32, _D, _D, _D,
                                          ct.POINTER(ct.c_int32), _D]
            L.orc_g2p.argtypes = [P, _D, ct.c_int64, _D, _D, _D, _D, CN]
            L.orc_step.argtypes = [P, TF, ct.c_int32, ct.c_int64, _D, _D, _D, _D, _D, CN]
            L.orc_run.argtypes = [P, TF, ct.c_int32, ct.c_int32, ct.c_int64, _D, _D, _D, _D, CN]
            L.orc_block_keys.argtypes = [ct.c_int32, ct.c_int64, ct.POINTER(ct.c_float),
                                         ct.POINTER(ct.c_uint32)]
            L.orc_step_adjoint.argtypes = [P, TF, ct.c_int32, ct.c_int64, _D, _D, _D, _D, _D, _D, _D, _D,
                                           _D, _D]
            L.orc_step_adjoint.restype = ct.c_int
            L.orc_step_adjoint_at_grid.argtypes = [P, TF, ct.c_int32, ct.c_int64, _D, _D, _D, _D, _D, _D, _D, _D,
                                                   _D, _D, _D, _D]
            L.orc_step_adjoint_at_grid.restype = ct.c_int
            L.orc_lame_vjp.argtypes = [ct.c_double, ct.c_double, ct.c_double, ct.c_double, _D, _D]
            L.orc_surface.argtypes = [ct.c_int32, _D, ct.c_double, ct.c_double, _D, ct.c_int64]
            L.orc_surface.restype = ct.c_int64
            _lib = L
    return _lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_D)


def _f64(a, shape=None):
    out = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if shape is not None:
        out = out.reshape(shape)
    return out


# ------------------------------------------------------------------ params

@dataclass
class OracleParams:
    n_grid: int
    dt: float
    E: float
    nu: float
    rho: float
    V0: float
    gravity: Sequence[float] = (0.0, -9.8, 0.0)
    bound: int = 3
    theta: float = 0.0
    friction: float = 0.0

    def c(self) -> Params:
        p = Params()
        p.n_grid = self.n_grid
        p.bound = self.bound
        p.dt = self.dt
        for i in range(3):
            p.gravity[i] = self.gravity[i]
        p.E, p.nu, p.rho, p.V0 = self.E, self.nu, self.rho, self.V0
        p.theta, p.friction = self.theta, self.friction
        return p

    @property
    def mass(self) -> float:
        return self.rho * self.V0

    @staticmethod
    def from_scene(sc) -> "OracleParams":
        return OracleParams(n_grid=sc.n_grid, dt=sc.dt, E=sc.E, nu=sc.nu, rho=sc.rho,
                            V0=sc.particle_volume, gravity=tuple(sc.gravity), bound=sc.bound,
                            theta=sc.theta, friction=sc.friction)


# -------------------------------------------------------------- primitives

def lame(E, nu):
    mu, lam = ct.c_double(), ct.c_double()
    lib().orc_lame(E, nu, ct.byref(mu), ct.byref(lam))
    return mu.value, lam.value


def piola(mu, lam, F):
    F = _f64(F, (9,))
    P = np.zeros(9)
    lib().orc_piola(mu, lam, _dp(F), _dp(P))
    return P.reshape(3, 3)


def piola_FT(mu, lam, F):
    F = _f64(F, (9,))
    P = np.zeros(9)
    lib().orc_piola_FT(mu, lam, _dp(F), _dp(P))
    return P.reshape(3, 3)


def weights(fx):
    w = np.zeros(3)
    lib().orc_weights(float(fx), _dp(w))
    return w


def rotvec_to_matrix(r):
    r = _f64(r, (3,))
    R = np.zeros(9)
    lib().orc_rotvec_to_matrix(_dp(r), _dp(R))
    return R.reshape(3, 3)


def matrix_to_rotvec(R):
    R = _f64(R, (9,))
    r = np.zeros(3)
    lib().orc_matrix_to_rotvec(_dp(R), _dp(r))
    return r


def sdf(kind, dims, p):
    dims = _f64(dims, (3,))
    p = _f64(p, (3,))
    n = np.zeros(3)
    d = lib().orc_sdf(int(kind), _dp(dims), _dp(p), _dp(n))
    return d, n


def _field_arrays(field):
    samples = np.ascontiguousarray(field.samples, dtype=np.float32)
    res = samples.shape[0]
    assert samples.shape == (res, res, res)
    return samples, res, _f64(field.origin, (3,)), float(field.h)


def sdf_sampled(field, p):
    """Sampled distance field lookup (Eqs. 12-14): (distance, unit normal,
    distance of p from the nearest cell face)."""
    samples, res, origin, h = _field_arrays(field)
    p = _f64(p, (3,))
    n = np.zeros(3)
    cm = np.zeros(1)
    d = lib().orc_sdf_sampled(samples.ctypes.data_as(ct.POINTER(ct.c_float)), res, _dp(origin), h,
                              _dp(p), _dp(n), _dp(cm))
    return d, n, float(cm[0])


def tool_frames(shape, pose0, pose1, nsub, dt, field=None):
    """Frames for one tool over one call of nsub sub-steps (see the C file).
    A sampled tool (shape[0] == 2) takes its samples, origin and spacing from
    field; the returned array keeps the samples alive."""
    shape = np.asarray(shape, dtype=np.float64)
    kind = int(shape[0])
    dims = _f64(shape[1:4])
    if kind == 2:
        samples, res, dims, h = _field_arrays(field)
    arr = (ToolFrame * nsub)()
    lib().orc_tool_frames(kind, _dp(dims), _dp(_f64(pose0, (6,))), _dp(_f64(pose1, (6,))),
                          int(nsub), float(dt), arr)
    if kind == 2:
        ptr = samples.ctypes.data_as(ct.POINTER(ct.c_float))
        for k in range(nsub):
            arr[k].res = res
            arr[k].h = h
            arr[k].sdf = ptr
        arr._keep = [samples]
    return arr


def frames_for_steps(tools, s0, nsub, dt, call_len=None):
    """Sub-step-major ToolFrame array for sub-steps s0 .. s0+nsub-1 of a scene's
    scripted tools, when the simulation is driven by calls of call_len
    sub-steps (default: one call covering all nsub) whose target pose is the
    scripted pose at the end of the call."""
    if not tools:
        return (ToolFrame * 1)(), 0
    call_len = call_len or nsub
    nt = len(tools)
    out = (ToolFrame * (nsub * nt))()
    out._keep = []
    s = s0
    while s < s0 + nsub:
        m = min(call_len, s0 + nsub - s)
        for t, tool in enumerate(tools):
            fr = tool_frames(tool.shape, tool.pose(s - 1), tool.pose(s + m - 1), m, dt,
                             getattr(tool, "field", None))
            out._keep.append(getattr(fr, "_keep", None))
            for k in range(m):
                ct.memmove(ct.byref(out, ((s - s0 + k) * nt + t) * ct.sizeof(ToolFrame)),
                           ct.byref(fr, k * ct.sizeof(ToolFrame)), ct.sizeof(ToolFrame))
        s += m
    return out, nt


# ------------------------------------------------------------- the method

class State:
    """FP64 particle state (x, v, C, F) in particle-id order."""

    def __init__(self, x, v=None, C=None, F=None):
        n = np.asarray(x).shape[0]
        self.x = _f64(x, (n, 3)).copy()
        self.v = np.zeros((n, 3)) if v is None else _f64(v, (n, 3)).copy()
        self.C = np.zeros((n, 9)) if C is None else _f64(C, (n, 9)).copy()
        self.F = np.tile(np.eye(3).reshape(1, 9), (n, 1)) if F is None else _f64(F, (n, 9)).copy()
        self.counters = Counters()

    @property
    def n(self):
        return self.x.shape[0]

    def copy(self):
        s = State(self.x, self.v, self.C, self.F)
        s.counters.j_clamped = self.counters.j_clamped
        s.counters.out_of_domain = self.counters.out_of_domain
        return s


def p2g(prm: OracleParams, st: State):
    n = prm.n_grid
    gm = np.zeros(n ** 3)
    gmv = np.zeros(n ** 3 * 3)
    lib().orc_p2g(ct.byref(prm.c()), st.n, _dp(st.x), _dp(st.v), _dp(st.C), _dp(st.F),
                  _dp(gm), _dp(gmv), ct.byref(st.counters))
    return gm.reshape(n, n, n), gmv.reshape(n, n, n, 3)


def grid_update(prm: OracleParams, gm, gmv, frames=None, ntools=0):
    n = prm.n_grid
    gm = _f64(gm, (n ** 3,))
    gmv = _f64(gmv, (n ** 3 * 3,))
    gv = np.zeros(n ** 3 * 3)
    contact = np.zeros(n ** 3, dtype=np.int32)
    margin = np.zeros(n ** 3)
    if frames is None:
        frames = (ToolFrame * 1)()
        ntools = 0
    lib().orc_grid_update(ct.byref(prm.c()), frames, int(ntools), _dp(gm), _dp(gmv), _dp(gv),
                          contact.ctypes.data_as(ct.POINTER(ct.c_int32)), _dp(margin))
    return gv.reshape(n, n, n, 3), contact.reshape(n, n, n), margin.reshape(n, n, n)


def g2p(prm: OracleParams, st: State, gv):
    n = prm.n_grid
    gv = _f64(gv, (n ** 3 * 3,))
    lib().orc_g2p(ct.byref(prm.c()), _dp(gv), st.n, _dp(st.x), _dp(st.v), _dp(st.C),
                  _dp(st.F), ct.byref(st.counters))


def run(prm: OracleParams, st: State, nsteps: int, frames=None, ntools=0):
    """nsteps sub-steps in place; frames is sub-step-major (nsteps * ntools)."""
    if frames is None or ntools == 0:
        frames = (ToolFrame * 1)()
        ntools = 0
    lib().orc_run(ct.byref(prm.c()), frames, int(ntools), int(nsteps), st.n, _dp(st.x),
                  _dp(st.v), _dp(st.C), _dp(st.F), ct.byref(st.counters))


def block_keys(n_grid: int, x32: np.ndarray) -> np.ndarray:
    x32 = np.ascontiguousarray(x32, dtype=np.float32).reshape(-1, 3)
    keys = np.zeros(x32.shape[0], dtype=np.uint32)
    lib().orc_block_keys(int(n_grid), x32.shape[0], x32.ctypes.data_as(ct.POINTER(ct.c_float)),
                         keys.ctypes.data_as(ct.POINTER(ct.c_uint32)))
    return keys


def sorted_order(keys: np.ndarray, previous: Optional[np.ndarray] = None) -> np.ndarray:
    """Stable counting-sort order of particle ids by block key.

    previous: the logical order before this sort (ids); None means id order.
    Returns the ids in sorted order: ascending key, ties kept in their
    previous relative order.  numpy's stable sort is the library step.
    """
    if previous is None:
        previous = np.arange(keys.shape[0], dtype=np.int64)
    previous = np.asarray(previous, dtype=np.int64)
    idx = np.argsort(keys[previous], kind="stable")
    return previous[idx]


# ------------------------------------------------------------- the adjoint

def step_adjoint(prm: OracleParams, st: State, frames, ntools, bar, grid=None):
    """Reverse mode of one sub-step from state st (unchanged).  bar: dict of
    the adjoints of the state after the sub-step (x, v, C, F; missing keys are
    zero).  Returns (adjoint of the state before it, [dL/dmu, dL/dlam],
    dL/d(frame entries) as (ntools, 18): R row-major, T, u, w).  grid: an
    (n, n, n, 4) array of (mass, momentum) to evaluate the grid operation and
    G2P at instead of the P2G of st (a grid computed elsewhere, e.g. by the
    GPU); the reverse of P2G still differentiates the P2G of st."""
    n = st.n
    out = {k: (np.zeros((n, c)) if bar.get(k) is None else _f64(bar[k], (n, c)).copy())
           for k, c in (("x", 3), ("v", 3), ("C", 9), ("F", 9))}
    lame = np.zeros(2)
    tb = np.zeros((max(ntools, 1), 18))
    if frames is None or ntools == 0:
        frames = (ToolFrame * 1)()
        ntools = 0
    if grid is None:
        rc = lib().orc_step_adjoint(ct.byref(prm.c()), frames, int(ntools), n, _dp(st.x), _dp(st.v), _dp(st.C),
                                    _dp(st.F), _dp(out["x"]), _dp(out["v"]), _dp(out["C"]), _dp(out["F"]),
                                    _dp(lame), _dp(tb))
    else:
        ng = prm.n_grid
        g = _f64(grid, (ng ** 3, 4))
        gm = np.ascontiguousarray(g[:, 0])
        gmv = np.ascontiguousarray(g[:, 1:]).reshape(-1)
        rc = lib().orc_step_adjoint_at_grid(ct.byref(prm.c()), frames, int(ntools), n, _dp(st.x), _dp(st.v),
                                            _dp(st.C), _dp(st.F), _dp(gm), _dp(gmv), _dp(out["x"]), _dp(out["v"]),
                                            _dp(out["C"]), _dp(out["F"]), _dp(lame), _dp(tb))
    if rc != 0:
        raise MemoryError("orc_step_adjoint: out of memory")
    return out, lame, tb[:ntools]


def lame_vjp(E, nu, mu_bar, lam_bar):
    Eb = ct.c_double()
    nb = ct.c_double()
    lib().orc_lame_vjp(float(E), float(nu), float(mu_bar), float(lam_bar), ct.byref(Eb), ct.byref(nb))
    return Eb.value, nb.value


def _frame_vector(fr) -> np.ndarray:
    return np.array(list(fr.R) + list(fr.T) + list(fr.u) + list(fr.w))


def _hat(r):
    """[r]x: the cross-product matrix of a 3-vector."""
    return np.array([[0.0, -r[2], r[1]], [r[2], 0.0, -r[0]], [-r[1], r[0], 0.0]])


def rotvec_to_matrix_derivative(r):
    """dR/dr_i (i = 0, 1, 2; each 3 x 3) of Rodrigues' formula as the oracle
    evaluates it, R = I + a K + b K^2 with K = [r]x, theta = |r|,
    a = sin(theta)/theta and b = (1 - cos(theta))/theta^2, differentiated
    term by term:
        dR/dr_i = (a'/theta) r_i K + a E_i + (b'/theta) r_i K^2 + b (E_i K + K E_i),
    E_i = [e_i]x, a'/theta = (theta cos(theta) - sin(theta))/theta^3,
    b'/theta = (theta sin(theta) - 2 (1 - cos(theta)))/theta^4 (their Taylor
    series below theta = 1e-3, where the closed forms cancel)."""
    r = _f64(r, (3,))
    th = float(np.sqrt(r @ r))
    if th < 1e-3:
        t2 = th * th
        a = 1.0 - t2 / 6.0 + t2 * t2 / 120.0
        b = 0.5 - t2 / 24.0 + t2 * t2 / 720.0
        da = -1.0 / 3.0 + t2 / 30.0 - t2 * t2 / 840.0
        db = -1.0 / 12.0 + t2 / 180.0 - t2 * t2 / 6720.0
    else:
        s, c = np.sin(th), np.cos(th)
        a = s / th
        b = (1.0 - c) / (th * th)
        da = (th * c - s) / th ** 3
        db = (th * s - 2.0 * (1.0 - c)) / th ** 4
    K = _hat(r)
    K2 = K @ K
    out = np.zeros((3, 3, 3))
    for i in range(3):
        Ei = _hat(np.eye(3)[i])
        out[i] = da * r[i] * K + a * Ei + db * r[i] * K2 + b * (Ei @ K + K @ Ei)
    return out


def matrix_to_rotvec_derivative(M):
    """dr/dM (3 x 3 x 3: [component, row, column]) of the oracle's inverse of
    Rodrigues' formula, r = f(theta) s with s = (M21 - M12, M02 - M20,
    M10 - M01), theta = acos((tr M - 1)/2) and f = theta/(2 sin(theta)):
        dr = f'(theta) (dtheta/d tr) s d(tr M) + f ds,
    dtheta/d tr = -1/(2 sin(theta)), f' = (sin(theta) - theta cos(theta))/(2 sin(theta)^2);
    their product g = -(sin(theta) - theta cos(theta))/(4 sin(theta)^3) is
    taken from its Taylor series -1/12 - theta^2/30 below theta = 1e-3.
    Rotations by close to a half turn (another branch of the inverse) are
    not needed by the one-sub-step frames and are refused."""
    M = _f64(M, (3, 3))
    c = min(1.0, max(-1.0, 0.5 * (np.trace(M) - 1.0)))
    th = float(np.arccos(c))
    if th > np.pi - 1e-6:
        raise ValueError("matrix_to_rotvec_derivative: rotation too close to a half turn")
    sv = np.array([M[2, 1] - M[1, 2], M[0, 2] - M[2, 0], M[1, 0] - M[0, 1]])
    if th < 1e-3:
        t2 = th * th
        f = 0.5 + t2 / 12.0 + 7.0 * t2 * t2 / 720.0
        g = -1.0 / 12.0 - t2 / 30.0
    else:
        sn = np.sin(th)
        f = th / (2.0 * sn)
        g = -(sn - th * np.cos(th)) / (4.0 * sn ** 3)
    ds = np.zeros((3, 3, 3))          # ds_a / dM_jk
    for a, (j, k) in enumerate(((2, 1), (0, 2), (1, 0))):
        ds[a, j, k] = 1.0
        ds[a, k, j] = -1.0
    out = f * ds
    for a in range(3):
        out[a] += g * sv[a] * np.eye(3)
    return out


def frame_jacobian(shape, pose0, pose1, dt, field=None):
    """d(frame entries: R row-major, T, u, w) / d(pose0, pose1) of a
    one-sub-step call (18 x 12), in closed form.  The frame map (reading
    r12 of Eq. 11's tool pose stream, as orc_tool_frames computes it) at the
    fraction s = 1 of a call of span dt is
        M = R(r1) R(r0)^T,  phi = log M,  R = exp(s phi) R(r0),
        T = T0 + s (T1 - T0),  u = (T1 - T0)/span,  w = phi/span,
    and its derivative is taken by the chain rule through
    rotvec_to_matrix_derivative (exp) and matrix_to_rotvec_derivative
    (log).  shape and field do not enter the frame."""
    p0, p1 = _f64(pose0, (6,)), _f64(pose1, (6,))
    s, span = 1.0, float(dt)
    R0, R1 = rotvec_to_matrix(p0[3:]), rotvec_to_matrix(p1[3:])
    dR0, dR1 = rotvec_to_matrix_derivative(p0[3:]), rotvec_to_matrix_derivative(p1[3:])
    M = R1 @ R0.T
    phi = matrix_to_rotvec(M)
    dlog = matrix_to_rotvec_derivative(M)
    # dphi/dr0_i and dphi/dr1_i
    dphi0 = np.stack([np.einsum("ajk,jk->a", dlog, R1 @ dR0[i].T) for i in range(3)], axis=1)
    dphi1 = np.stack([np.einsum("ajk,jk->a", dlog, dR1[i] @ R0.T) for i in range(3)], axis=1)
    Es = rotvec_to_matrix(s * phi)
    dEs = rotvec_to_matrix_derivative(s * phi)
    J = np.zeros((18, 12))
    for i in range(3):
        # R = exp(s phi) R0
        dE0 = sum(dEs[a] * s * dphi0[a, i] for a in range(3))
        dE1 = sum(dEs[a] * s * dphi1[a, i] for a in range(3))
        J[0:9, 3 + i] = (dE0 @ R0 + Es @ dR0[i]).reshape(9)
        J[0:9, 9 + i] = (dE1 @ R0).reshape(9)
        # T, u
        J[9 + i, i] = 1.0 - s
        J[9 + i, 6 + i] = s
        J[12 + i, i] = -1.0 / span
        J[12 + i, 6 + i] = 1.0 / span
    # w = phi / span
    J[15:18, 3:6] = dphi0 / span
    J[15:18, 9:12] = dphi1 / span
    return J


def frame_jacobian_differences(shape, pose0, pose1, dt, field=None, h=1e-6):
    """The same 18 x 12 matrix by central differences of orc_tool_frames
    (an independent check of frame_jacobian, used by the pins)."""
    p = np.concatenate([_f64(pose0, (6,)), _f64(pose1, (6,))])
    J = np.zeros((18, 12))
    for c in range(12):
        a, b = p.copy(), p.copy()
        a[c] += h
        b[c] -= h
        fa = _frame_vector(tool_frames(shape, a[:6], a[6:], 1, dt, field)[0])
        fb = _frame_vector(tool_frames(shape, b[:6], b[6:], 1, dt, field)[0])
        J[:, c] = (fa - fb) / (2 * h)
    return J


def rollout_frames(tools, pose_init, poses, dt):
    """Frames of a rollout that moves tool t from pose_init[t] through
    poses[k, t] (the pose at the end of sub-step k), one sub-step per pose."""
    K, nt = poses.shape[0], len(tools)
    out = (ToolFrame * max(1, K * nt))()
    out._keep = []
    for k in range(K):
        for t, tool in enumerate(tools):
            p0 = pose_init[t] if k == 0 else poses[k - 1, t]
            fr = tool_frames(tool.shape, p0, poses[k, t], 1, dt, getattr(tool, "field", None))
            out._keep.append(getattr(fr, "_keep", None))
            ct.memmove(ct.byref(out, (k * nt + t) * ct.sizeof(ToolFrame)), ct.byref(fr, 0), ct.sizeof(ToolFrame))
    return out, nt


def _frames_getter(frames, nt):
    fsz = ct.sizeof(ToolFrame)

    def frames_at(k):
        arr = (ToolFrame * max(1, nt))()
        if nt:
            ct.memmove(arr, ct.byref(frames, k * nt * fsz), nt * fsz)
        return arr
    return frames_at


def _reverse_segment(prm, seg, k0, frames_at, nt, bar, lame, fbar, grids=None):
    """Reverse mode of the sub-steps k0 .. k0+len(seg)-1 whose input states
    are seg[j] (and whose grids are grids[j], if given): the adjoint of the
    state after the last of them (bar) is carried back to the state before
    the first; lame and fbar accumulate the material and frame adjoints."""
    for j in range(len(seg) - 1, -1, -1):
        k = k0 + j
        bar, lb, tb = step_adjoint(prm, seg[j], frames_at(k), nt, bar, None if grids is None else grids[j])
        lame += lb
        if nt:
            fbar[k] = tb
    return bar


def _gradients(prm, tools, pose_init, poses, lame, fbar):
    """dL/dE, dL/dnu from the Lame adjoints (Eq. 6) and dL/dposes from the
    frame adjoints through the frame map (each sub-step's frame depends on
    the pose before it and its own pose)."""
    Eb, nub = lame_vjp(prm.E, prm.nu, lame[0], lame[1])
    pose_bar = np.zeros_like(poses)
    for k in range(poses.shape[0]):
        for t, tool in enumerate(tools):
            p0 = pose_init[t] if k == 0 else poses[k - 1, t]
            J = frame_jacobian(tool.shape, p0, poses[k, t], prm.dt, getattr(tool, "field", None))
            g = J.T @ fbar[k, t]
            pose_bar[k, t] += g[6:]
            if k > 0:
                pose_bar[k - 1, t] += g[:6]
    return Eb, nub, pose_bar


def rollout_loss_and_gradients(prm: OracleParams, st0: State, tools, pose_init, poses, target,
                               checkpoint=50, final_bar=None):
    """A rollout of K = len(poses) sub-steps from st0 (unchanged) and the
    gradients of L = mean_p |x_p(K) - target_p|^2 (or of the loss whose
    final-state adjoint final_bar(state) returns) with respect to E, nu, the
    poses (K, ntools, 6) and the initial state.  Forward states are kept at
    every `checkpoint`-th sub-step and recomputed per segment."""
    poses = np.asarray(poses, dtype=np.float64)
    K = poses.shape[0]
    frames, nt = rollout_frames(tools, pose_init, poses, prm.dt)
    frames_at = _frames_getter(frames, nt)
    cps = {}
    st = st0.copy()
    for k in range(K):
        if k % checkpoint == 0:
            cps[k] = st.copy()
        run(prm, st, 1, frames_at(k), nt)
    final = st
    if final_bar is None:
        diff = final.x - _f64(target, final.x.shape)
        loss = float(np.mean(np.sum(diff * diff, axis=1)))
        bar = {"x": 2.0 * diff / final.n}
    else:
        loss, bar = final_bar(final)
    lame = np.zeros(2)
    fbar = np.zeros((K, nt, 18))
    for c0 in sorted(cps, reverse=True):
        seg = [cps[c0].copy()]
        for k in range(c0, min(c0 + checkpoint, K) - 1):
            s = seg[-1].copy()
            run(prm, s, 1, frames_at(k), nt)
            seg.append(s)
        bar = _reverse_segment(prm, seg, c0, frames_at, nt, bar, lame, fbar)
    Eb, nub, pose_bar = _gradients(prm, tools, pose_init, poses, lame, fbar)
    return {"loss": loss, "E": Eb, "nu": nub, "poses": pose_bar, "state0": bar, "final": final,
            "lame": lame, "frames": fbar}


def reverse_from_states(prm: OracleParams, states, tools, pose_init, poses, bar, grids=None):
    """Reverse mode of K = len(poses) sub-steps along a given forward
    trajectory: states[k] is the state before sub-step k (k = 0 .. K-1),
    bar the adjoint of the state after the last sub-step.  Each sub-step's
    adjoint is evaluated at its given input state (its forward pass is
    recomputed from that state alone), so a trajectory computed elsewhere --
    in another precision -- enters only through the states it supplies.
    grids[k], if given, is the (n, n, n, 4) grid sub-step k's grid operation
    read there (see step_adjoint).  Returns the gradients with respect to E,
    nu, the poses and states[0]."""
    poses = np.asarray(poses, dtype=np.float64)
    K = poses.shape[0]
    assert len(states) == K
    frames, nt = rollout_frames(tools, pose_init, poses, prm.dt)
    frames_at = _frames_getter(frames, nt)
    bar = {k: _f64(v).copy() for k, v in bar.items()}
    lame = np.zeros(2)
    fbar = np.zeros((K, nt, 18))
    bar = _reverse_segment(prm, list(states), 0, frames_at, nt, bar, lame, fbar, grids)
    Eb, nub, pose_bar = _gradients(prm, tools, pose_init, poses, lame, fbar)
    return {"E": Eb, "nu": nub, "poses": pose_bar, "state0": bar, "lame": lame, "frames": fbar}


# ----------------------------------------------------------- the surface

def surface(field, iso, dx):
    """Triangles (T, 3, 3) of the iso-surface field >= iso of an n^3 node
    field ([i, j, k], node (i, j, k) at (i, j, k) dx), in cell order (i
    fastest, then j, then k)."""
    f = np.ascontiguousarray(field, dtype=np.float64)
    n = f.shape[0]
    assert f.shape == (n, n, n)
    total = lib().orc_surface(n, _dp(f.reshape(-1)), float(iso), float(dx), ct.cast(None, _D), 0)
    out = np.zeros(max(total, 1) * 9)
    lib().orc_surface(n, _dp(f.reshape(-1)), float(iso), float(dx), _dp(out), total)
    return out[:total * 9].reshape(total, 3, 3)
