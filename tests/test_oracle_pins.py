"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these re-evaluates the oracle's own formulas: each compares it with
a closed form, an invariant, a hand-computed case, a brute-force sum over all
grid nodes, or a finite difference of an energy, so that a dropped term, a
wrong sign or index, or a transposed operand in the oracle fails one of them.
"""
import json
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2402_01181_gb300 import scenes

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rand_F(rng, n, jlo=0.5, jhi=2.0):
    """Random deformation gradients with J in [jlo, jhi]."""
    out = []
    while len(out) < n:
        F = np.eye(3) + 0.4 * (2 * rng.random((3, 3)) - 1)
        J = np.linalg.det(F)
        if jlo <= J <= jhi:
            out.append(F)
    return np.array(out)


def _rand_rotation(rng):
    q, r = np.linalg.qr(rng.normal(size=(3, 3)))
    q = q @ np.diag(np.sign(np.diag(r)))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


def neo_hookean_energy(mu, lam, F):
    """Compressible Neo-Hookean energy density whose first Piola stress is
    mu (F - F^-T) + lam ln(J) F^-T (the Eq. 5 form of the cited MLS-MPM)."""
    J = np.linalg.det(F)
    return 0.5 * mu * (np.trace(F.T @ F) - 3.0) - mu * math.log(J) + 0.5 * lam * math.log(J) ** 2


def bspline(u):
    """Closed-form quadratic B-spline N(u), zero outside |u| < 1.5."""
    a = abs(u)
    if a < 0.5:
        return 0.75 - a * a
    if a < 1.5:
        return 0.5 * (1.5 - a) ** 2
    return 0.0


def _params(n=16, E=0.0, nu=0.3, dt=1e-3, bound=0, gravity=(0.0, 0.0, 0.0), V0=None, rho=1e3,
            friction=0.0, theta=0.0):
    dx = 1.0 / n
    return O.OracleParams(n_grid=n, dt=dt, E=E, nu=nu, rho=rho, V0=V0 if V0 is not None else dx ** 3 / 8,
                          gravity=gravity, bound=bound, friction=friction, theta=theta)


# ------------------------------------------------------------------ weights

def test_weights_moments():
    """Quadratic B-spline: partition of unity, linear reproduction and second
    moment 1/4 (the MLS inertia D_p = dx^2/4 I) for every fx in [0.5, 1.5)."""
    for fx in np.linspace(0.5, 1.5, 101)[:-1]:
        w = O.weights(fx)
        o = np.arange(3) - fx
        assert abs(w.sum() - 1.0) < 1e-15
        assert abs((w * o).sum()) < 1e-15
        assert abs((w * o * o).sum() - 0.25) < 1e-15
        for k in range(3):
            assert abs(w[k] - bspline(o[k])) < 1e-15


# ----------------------------------------------------------------- material

def test_lame_golden_and_bulk_identity():
    """Eq. 6 values for the workloads, and the bulk modulus identity
    K = E / (3(1-2 nu)) = lam + 2 mu / 3."""
    golden = {(5e3, 0.3): (1923.0769230769231, 2884.6153846153848),
              (1e4, 0.35): (3703.7037037037035, 8641.975308641975),
              (1e4, 0.3): (3846.153846153846, 5769.2307692307695)}
    for (E, nu), (mu_g, lam_g) in golden.items():
        mu, lam = O.lame(E, nu)
        assert mu == pytest.approx(mu_g, rel=1e-14)
        assert lam == pytest.approx(lam_g, rel=1e-14)
        assert E / (3 * (1 - 2 * nu)) == pytest.approx(lam + 2 * mu / 3, rel=1e-14)
        assert E == pytest.approx(mu * (3 * lam + 2 * mu) / (lam + mu), rel=1e-14)


def test_piola_is_energy_gradient():
    """P(F) equals the central finite difference of the Neo-Hookean energy."""
    rng = np.random.default_rng(1)
    mu, lam = O.lame(1e4, 0.3)
    for F in _rand_F(rng, 20):
        P = O.piola(mu, lam, F)
        h = 1e-6
        G = np.zeros((3, 3))
        for a in range(3):
            for b in range(3):
                Fp, Fm = F.copy(), F.copy()
                Fp[a, b] += h
                Fm[a, b] -= h
                G[a, b] = (neo_hookean_energy(mu, lam, Fp) - neo_hookean_energy(mu, lam, Fm)) / (2 * h)
        assert np.max(np.abs(P - G)) <= 1e-6 * max(1.0, np.max(np.abs(G)))


def test_stress_free_at_rest_and_under_rotation():
    """No stress at F = I and under any rigid rotation; P F^T symmetric."""
    rng = np.random.default_rng(2)
    mu, lam = O.lame(5e3, 0.3)
    assert np.max(np.abs(O.piola(mu, lam, np.eye(3)))) == 0.0
    for _ in range(20):
        R = _rand_rotation(rng)
        assert np.max(np.abs(O.piola(mu, lam, R))) < 1e-10 * mu
    for F in _rand_F(rng, 20):
        tau = O.piola_FT(mu, lam, F)
        assert np.max(np.abs(tau - tau.T)) < 1e-10 * mu


# --------------------------------------------------------------------- P2G

def _rand_particles(rng, n, ngrid, margin=4):
    lo, hi = margin / ngrid, 1 - margin / ngrid
    return lo + (hi - lo) * rng.random((n, 3))


def test_p2g_brute_force_over_all_nodes():
    """Without stress, P2G equals the sum over every node of the closed-form
    B-spline times m_p (v_p + C_p (x_i - x_p)) (Eqs. 1-2)."""
    rng = np.random.default_rng(3)
    prm = _params(n=12)
    n, dx, m = prm.n_grid, 1.0 / prm.n_grid, prm.mass
    for npart in (1, 3, 8):
        x = _rand_particles(rng, npart, n)
        v = rng.normal(size=(npart, 3))
        C = rng.normal(size=(npart, 9))
        st = O.State(x, v, C)
        gm, gmv = O.p2g(prm, st)
        bm = np.zeros((n, n, n))
        bmv = np.zeros((n, n, n, 3))
        for p in range(npart):
            for i in range(n):
                for j in range(n):
                    for k in range(n):
                        d = np.array([i, j, k]) * dx - x[p]
                        w = bspline(d[0] / dx) * bspline(d[1] / dx) * bspline(d[2] / dx)
                        if w == 0.0:
                            continue
                        bm[i, j, k] += w * m
                        bmv[i, j, k] += w * m * (v[p] + C[p].reshape(3, 3) @ d)
        assert np.max(np.abs(gm - bm)) < 1e-15
        assert np.max(np.abs(gmv - bmv)) < 1e-13


def test_p2g_conserves_mass_linear_and_angular_momentum():
    """Grid mass = particle mass; grid momentum = particle momentum (the
    stress impulse sums to zero); grid angular momentum = the APIC particle
    angular momentum x_p x m v_p + m dx^2/4 eps:C_p^T, with the stress term
    contributing nothing because P F^T is symmetric."""
    rng = np.random.default_rng(4)
    prm = _params(n=16, E=2e4, nu=0.3, dt=1e-3)
    n, dx, m = prm.n_grid, 1.0 / prm.n_grid, prm.mass
    N = 200
    x = _rand_particles(rng, N, n)
    v = rng.normal(size=(N, 3))
    C = rng.normal(size=(N, 9)) * 3
    F = _rand_F(rng, N).reshape(N, 9)
    gm, gmv = O.p2g(prm, O.State(x, v, C, F))
    assert gm.sum() == pytest.approx(N * m, rel=1e-13)
    P_lin = m * v.sum(axis=0)
    assert np.max(np.abs(gmv.reshape(-1, 3).sum(axis=0) - P_lin)) < 1e-12 * max(1, np.abs(P_lin).max()) + 1e-14
    I, J, K = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    xi = np.stack([I, J, K], axis=-1).reshape(-1, 3) * dx
    L_grid = np.cross(xi, gmv.reshape(-1, 3)).sum(axis=0)
    Cm = C.reshape(N, 3, 3)
    spin = np.stack([Cm[:, 2, 1] - Cm[:, 1, 2], Cm[:, 0, 2] - Cm[:, 2, 0], Cm[:, 1, 0] - Cm[:, 0, 1]], axis=1)
    L_part = (np.cross(x, m * v) + m * dx * dx / 4 * spin).sum(axis=0)
    assert np.max(np.abs(L_grid - L_part)) < 1e-12


def test_p2g_stress_impulse_is_energy_gradient():
    """The stress impulse of P2G (Eq. 3, with v = C = 0) equals minus the
    gradient of the total Neo-Hookean energy with respect to the grid
    velocities, where the energy is taken after the G2P update of F
    (Eqs. 4 and 9) -- the variational consistency of MLS-MPM.  The gradient
    is a central finite difference through the oracle's own G2P."""
    rng = np.random.default_rng(5)
    n = 8
    prm = _params(n=n, E=3e3, nu=0.3, dt=1e-3)
    mu, lam = O.lame(prm.E, prm.nu)
    x = 0.5 + (rng.random((2, 3)) - 0.5) * 0.1
    F = _rand_F(rng, 2, 0.7, 1.4).reshape(2, 9)
    gm, gmv = O.p2g(prm, O.State(x, None, None, F))
    prm_g = _params(n=n, E=0.0, dt=prm.dt)   # G2P itself does not depend on E

    def energy(gv):
        st = O.State(x, None, None, F)
        O.g2p(prm_g, st, gv)
        return sum(prm.V0 * neo_hookean_energy(mu, lam, st.F[p].reshape(3, 3)) for p in range(2))

    gv0 = np.zeros((n, n, n, 3))
    nodes = np.argwhere(gm > 0)
    h = 1e-4
    for (i, j, k) in nodes:
        for a in range(3):
            gp, gmn = gv0.copy(), gv0.copy()
            gp[i, j, k, a] += h
            gmn[i, j, k, a] -= h
            dE = (energy(gp) - energy(gmn)) / (2 * h)
            assert gmv[i, j, k, a] == pytest.approx(-dE, rel=1e-6, abs=1e-13)


# --------------------------------------------------------------------- G2P

def test_g2p_brute_force_over_all_nodes():
    """v_p and C_p from a random grid velocity field equal the brute-force
    sums over every node with the closed-form B-spline (Eqs. 8-9)."""
    rng = np.random.default_rng(6)
    prm = _params(n=10, dt=1e-3)
    n, dx = prm.n_grid, 1.0 / prm.n_grid
    gv = rng.normal(size=(n, n, n, 3))
    x = _rand_particles(rng, 5, n)
    st = O.State(x)
    O.g2p(prm, st, gv)
    for p in range(5):
        vb = np.zeros(3)
        B = np.zeros((3, 3))
        for i in range(n):
            for j in range(n):
                for k in range(n):
                    d = np.array([i, j, k]) * dx - x[p]
                    w = bspline(d[0] / dx) * bspline(d[1] / dx) * bspline(d[2] / dx)
                    vb += w * gv[i, j, k]
                    B += w * np.outer(gv[i, j, k], d)
        assert np.max(np.abs(st.v[p] - vb)) < 1e-13
        assert np.max(np.abs(st.C[p].reshape(3, 3) - 4 / dx ** 2 * B)) < 1e-10
        assert np.max(np.abs(st.x[p] - (x[p] + prm.dt * vb))) < 1e-15
        Fn = (np.eye(3) + prm.dt * 4 / dx ** 2 * B)
        assert np.max(np.abs(st.F[p].reshape(3, 3) - Fn)) < 1e-12


def test_g2p_reproduces_affine_fields():
    """For a grid velocity field v(x) = v0 + G x, APIC recovers v_p = v(x_p)
    and C_p = G exactly (a closed form of Eqs. 8-9)."""
    rng = np.random.default_rng(7)
    prm = _params(n=16, dt=1e-3)
    n, dx = prm.n_grid, 1.0 / prm.n_grid
    v0 = rng.normal(size=3)
    G = rng.normal(size=(3, 3))
    I, J, K = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    xi = np.stack([I, J, K], axis=-1) * dx
    gv = v0 + xi @ G.T
    x = _rand_particles(rng, 50, n)
    st = O.State(x)
    O.g2p(prm, st, gv)
    assert np.max(np.abs(st.v - (v0 + x @ G.T))) < 1e-12
    assert np.max(np.abs(st.C.reshape(-1, 3, 3) - G)) < 1e-9


def test_g2p_conserves_angular_momentum():
    """Particle APIC angular momentum after G2P (at the pre-advection
    positions) equals the grid angular momentum sum m_i x_i x v_i."""
    rng = np.random.default_rng(8)
    prm = _params(n=16, E=0.0, dt=1e-3)
    n, dx, m = prm.n_grid, 1.0 / prm.n_grid, prm.mass
    x = _rand_particles(rng, 300, n)
    st = O.State(x)
    gm, _ = O.p2g(prm, st)
    gv = rng.normal(size=(n, n, n, 3))
    O.g2p(prm, st, gv)
    I, J, K = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    xi = np.stack([I, J, K], axis=-1).reshape(-1, 3) * dx
    L_grid = np.cross(xi, gm.reshape(-1, 1) * gv.reshape(-1, 3)).sum(axis=0)
    L_lin_grid = (gm.reshape(-1, 1) * gv.reshape(-1, 3)).sum(axis=0)
    Cm = st.C.reshape(-1, 3, 3)
    spin = np.stack([Cm[:, 2, 1] - Cm[:, 1, 2], Cm[:, 0, 2] - Cm[:, 2, 0], Cm[:, 1, 0] - Cm[:, 0, 1]], axis=1)
    L_part = (np.cross(x, m * st.v) + m * dx * dx / 4 * spin).sum(axis=0)
    assert np.max(np.abs(L_grid - L_part)) < 1e-11
    assert np.max(np.abs(L_lin_grid - m * st.v.sum(axis=0))) < 1e-11


# ------------------------------------------------------------- whole steps

def test_free_fall_closed_form():
    """The 8,192-particle cube falls freely for 200 steps: symplectic Euler
    gives v_k = k g dt and x_k = x_0 + g dt^2 k(k+1)/2, with C = 0, F = I."""
    sc = scenes.cube8k()
    prm = O.OracleParams.from_scene(sc)
    st = O.State(sc.x)
    x0 = st.x.copy()
    k = 200
    O.run(prm, st, k)
    g = np.array(sc.gravity)
    assert np.max(np.abs(st.v - k * g * sc.dt)) < 1e-12
    assert np.max(np.abs(st.x - (x0 + g * sc.dt ** 2 * k * (k + 1) / 2))) < 1e-13
    assert np.max(np.abs(st.C)) < 1e-9
    assert np.max(np.abs(st.F - np.eye(3).reshape(1, 9))) < 1e-12
    assert st.counters.j_clamped == 0 and st.counters.out_of_domain == 0


def test_stretched_block_contracts():
    """A block stretched along x (F = diag(1.2, 1, 1)) with no gravity: the
    stress impulses point inward along x on the two x faces and the block's
    x extent shrinks in the first steps."""
    sc = scenes.cube8k()
    prm = O.OracleParams.from_scene(sc)
    prm.gravity = (0.0, 0.0, 0.0)
    F = np.tile(np.diag([1.2, 1.0, 1.0]).reshape(1, 9), (sc.n, 1))
    st = O.State(sc.x, None, None, F)
    w0 = st.x[:, 0].max() - st.x[:, 0].min()
    O.run(prm, st, 20)
    left = st.x[:, 0] < 0.45
    right = st.x[:, 0] > 0.55
    assert st.v[left, 0].mean() > 0 and st.v[right, 0].mean() < 0
    assert st.x[:, 0].max() - st.x[:, 0].min() < w0


# ------------------------------------------------------------ tools, grid

def _one_node_grid(case, n=8):
    m = np.zeros((n, n, n))
    mv = np.zeros((n, n, n, 3))
    m[4, 4, 4] = 1.0
    mv[4, 4, 4] = case["v_in"]
    return m, mv


def _frames_from_case(tools):
    arr = (O.ToolFrame * max(1, len(tools)))()
    for t, tl in enumerate(tools):
        f = arr[t]
        f.kind = int(tl["shape"][0])
        for d in range(3):
            f.dims[d] = tl["shape"][1 + d]
            f.T[d] = tl["T"][d]
            f.u[d] = tl["u"][d]
            f.w[d] = tl["w"][d]
        R = tl.get("R", [1.0 if i % 4 == 0 else 0.0 for i in range(9)])
        for i in range(9):
            f.R[i] = R[i]
    return arr


def test_grid_operation_golden_cases():
    with open(os.path.join(GOLDEN, "friction_cases.json")) as fh:
        cases = json.load(fh)["cases"]
    for case in cases:
        prm = _params(n=8, dt=case.get("dt", 1e-3), gravity=tuple(case.get("gravity", (0, 0, 0))),
                      bound=case.get("bound", 0), friction=case["friction"])
        m, mv = _one_node_grid(case)
        gv, contact, _ = O.grid_update(prm, m, mv, _frames_from_case(case["tools"]), len(case["tools"]))
        assert np.allclose(gv[4, 4, 4], case["v_out"], atol=1e-12), case["name"]
        assert contact[4, 4, 4] == case["contact"], case["name"]
        other = np.ones((8, 8, 8), bool)
        other[4, 4, 4] = False
        assert np.all(gv[other] == 0.0), case["name"]          # massless nodes stay at rest


def test_grid_operation_rigid_motion_is_kept():
    """A node that already moves with the tool's rigid velocity is left as is
    (v_rel = 0), for a translating and spinning capsule."""
    rng = np.random.default_rng(9)
    prm = _params(n=8, friction=0.4)
    for _ in range(10):
        T = np.array([0.5, 0.5, 0.5]) + 0.02 * rng.normal(size=3)
        u = rng.normal(size=3)
        w = rng.normal(size=3)
        tl = {"shape": [0, 0.2, 0.1, 0], "T": T, "u": u, "w": w}
        vco = u + np.cross(w, np.array([0.5, 0.5, 0.5]) - T)
        m, mv = _one_node_grid({"v_in": vco})
        gv, contact, _ = O.grid_update(prm, m, mv, _frames_from_case([tl]), 1)
        assert contact[4, 4, 4] == 0
        assert np.allclose(gv[4, 4, 4], vco, atol=1e-12)


def _surface_samples(kind, dims, k=60):
    pts = []
    if kind == scenes.CAPSULE:
        r, h = dims[0], dims[1]
        th = np.linspace(0, 2 * np.pi, k, endpoint=False)
        for y in np.linspace(-h, h, k):
            pts += [(r * np.cos(t), y, r * np.sin(t)) for t in th]
        for s in (-1, 1):
            for ph in np.linspace(0, np.pi / 2, k // 2):
                pts += [(r * np.cos(ph) * np.cos(t), s * (h + r * np.sin(ph)), r * np.cos(ph) * np.sin(t)) for t in th]
    else:
        g = np.linspace(-1, 1, k)
        for ax in range(3):
            for s in (-1, 1):
                for a in g:
                    for b in g:
                        p = np.zeros(3)
                        p[ax] = s
                        o = [i for i in range(3) if i != ax]
                        p[o[0]], p[o[1]] = a, b
                        pts.append(tuple(p * dims))
    return np.array(pts)


def _inside(kind, dims, p):
    if kind == scenes.CAPSULE:
        c = np.clip(p[1], -dims[1], dims[1])
        return np.linalg.norm(p - np.array([0, c, 0])) < dims[0]
    return np.all(np.abs(p) < dims)


def test_sdf_against_sampled_surfaces():
    """Analytic capsule and box distances agree with the distance to a dense
    sampling of the surface (sign from a point-in-shape test), and the normal
    agrees with the finite-difference gradient of the distance."""
    rng = np.random.default_rng(10)
    for kind, dims in ((scenes.CAPSULE, np.array([0.05, 0.1, 0.0])), (scenes.BOX, np.array([0.06, 0.1, 0.04]))):
        surf = _surface_samples(kind, dims)
        spacing = 2.5 * (dims.max() * 2) / 60
        for _ in range(60):
            p = rng.normal(size=3) * 0.12
            d, nrm = O.sdf(kind, dims, p)
            db = np.min(np.linalg.norm(surf - p, axis=1)) * (-1 if _inside(kind, dims, p) else 1)
            assert abs(d - db) < spacing, (kind, p, d, db)
            h = 1e-7
            gfd = np.array([(O.sdf(kind, dims, p + h * e)[0] - O.sdf(kind, dims, p - h * e)[0]) / (2 * h)
                            for e in np.eye(3)])
            if abs(np.linalg.norm(gfd) - 1.0) < 1e-4:          # away from kinks / medial axis
                assert np.allclose(nrm, gfd, atol=1e-5)


def test_rotation_maps_and_tool_frames():
    rng = np.random.default_rng(11)
    for _ in range(30):
        r = rng.normal(size=3)
        r *= rng.random() * 3.0 / np.linalg.norm(r)
        R = O.rotvec_to_matrix(r)
        assert np.allclose(R @ R.T, np.eye(3), atol=1e-14)
        assert np.linalg.det(R) == pytest.approx(1.0, abs=1e-14)
        assert np.allclose(R @ r, r, atol=1e-14)                 # the axis is fixed
        assert np.allclose(O.matrix_to_rotvec(R), r, atol=1e-9)
    shape = np.array([0, 0.02, 0.15, 0, 0, 0, 0, 0])
    p0 = np.array([0.4, 0.5, 0.6, 0.1, -0.2, 0.05])
    p1 = np.array([0.43, 0.48, 0.6, 0.15, -0.1, 0.0])
    dt, nsub = 1e-3, 5
    fr = O.tool_frames(shape, p0, p1, nsub, dt)
    assert np.allclose(np.array(fr[nsub - 1].T), p1[:3], atol=1e-15)
    assert np.allclose(np.array(fr[nsub - 1].R).reshape(3, 3), O.rotvec_to_matrix(p1[3:]), atol=1e-13)
    assert np.allclose(np.array(fr[0].u), (p1[:3] - p0[:3]) / (nsub * dt), atol=1e-12)
    # angular velocity: R_{k+1} R_k^T = exp(w dt)
    R0 = np.array(fr[1].R).reshape(3, 3)
    R1 = np.array(fr[2].R).reshape(3, 3)
    assert np.allclose(O.matrix_to_rotvec(R1 @ R0.T) / dt, np.array(fr[0].w), atol=1e-9)
    # kinematic consistency inside the call: every sub-step's pose moves on from
    # the previous one (from pose0 for the first) by the frame's own velocities
    prevT, prevR = p0[:3], O.rotvec_to_matrix(p0[3:])
    for k in range(nsub):
        Tk, Rk = np.array(fr[k].T), np.array(fr[k].R).reshape(3, 3)
        assert np.allclose(Tk - prevT, np.array(fr[k].u) * dt, atol=1e-15), k
        assert np.allclose(O.matrix_to_rotvec(Rk @ prevR.T), np.array(fr[k].w) * dt, atol=1e-12), k
        prevT, prevR = Tk, Rk


# --------------------------------------------------------------- sort keys

def test_block_keys_brute_force():
    rng = np.random.default_rng(12)
    n = 32
    x = (0.1 + 0.8 * rng.random((500, 3))).astype(np.float32)
    keys = O.block_keys(n, x)
    nb = n // 4
    for p in range(500):
        c = [min(max(int(math.floor(float(x[p, d]) * n - 0.5)), 0), n - 3) // 4 for d in range(3)]
        assert keys[p] == c[0] + nb * (c[1] + nb * c[2])
    order = O.sorted_order(keys)
    assert np.all(np.diff(keys[order].astype(np.int64)) >= 0)
    for kv in np.unique(keys):                                  # stable: ids ascending inside a key
        ids = order[keys[order] == kv]
        assert np.all(np.diff(ids) > 0)
    prev = rng.permutation(500)
    order2 = O.sorted_order(keys, prev)
    pos = np.empty(500, int)
    pos[prev] = np.arange(500)
    for kv in np.unique(keys):
        ids = order2[keys[order2] == kv]
        assert np.all(np.diff(pos[ids]) > 0)


def test_inverted_particles_are_counted():
    prm = _params(n=16, E=1e3)
    x = np.full((1, 3), 0.5)
    F = np.diag([1.0, 1.0, -1.0]).reshape(1, 9)
    st = O.State(x, None, None, F)
    O.p2g(prm, st)
    assert st.counters.j_clamped == 1


# ------------------------------------------------- sampled distance fields

def _field(fn, origin, h, res):
    """Samples fn at origin + h (i, j, k), x fastest -- written out here so
    the pins do not lean on the scene module's rasteriser."""
    out = np.empty((res, res, res), dtype=np.float32)
    for k in range(res):
        for j in range(res):
            for i in range(res):
                out[k, j, i] = fn(np.asarray(origin) + h * np.array([i, j, k], dtype=np.float64))
    return scenes.SampledField(out, np.asarray(origin, dtype=np.float64), h)


def test_sampled_field_reads_the_lower_sample_of_a_linear_field():
    """Eq. 12 reads the sample at floor((x_ref - o) / h); Eq. 14's central
    difference of a linear field is its exact gradient, also one-sided at the
    faces, so the unit normal is a / |a| everywhere inside the field; outside
    it there is no contact (+inf)."""
    a = np.array([0.3, -1.7, 0.9])
    c = 0.05
    o = np.array([-0.125, 0.0625, -0.25])                # powers of two: sample positions are exact
    h, res = 1.0 / 64, 10
    fld = _field(lambda q: a @ q + c, o, h, res)
    rng = np.random.default_rng(13)
    unit = a / np.linalg.norm(a)
    pts = [o + h * res * rng.random(3) for _ in range(200)]
    for ax in range(3):                                    # first and last cell on each axis
        for cell in (0, res - 1):
            p = o + h * res * rng.random(3)
            p[ax] = o[ax] + h * (cell + 0.37)
            pts.append(p)
    for p in pts:
        d, nrm, _ = O.sdf_sampled(fld, p)
        corner = o + h * np.floor((p - o) / h)
        assert abs(d - (a @ corner + c)) < 1e-6, p
        assert np.allclose(nrm, unit, atol=1e-6), (p, nrm)
    for i in range(res):                                   # exactly on a sample, and just below it
        p = o + h * np.array([i, 3, 5], dtype=np.float64)
        assert O.sdf_sampled(fld, p)[0] == pytest.approx(a @ p + c, abs=1e-6)
        if i > 0:
            q = p.copy()
            q[0] -= 1e-12
            assert O.sdf_sampled(fld, q)[0] == pytest.approx(a @ (p - h * np.array([1, 0, 0])) + c, abs=1e-6)
    for ax in range(3):
        for p_ax in (o[ax] - 1e-9, o[ax] + h * res, o[ax] + h * res + 0.3):
            p = o + 0.5 * h * res
            p[ax] = p_ax
            assert O.sdf_sampled(fld, p)[0] == np.inf


def test_sampled_sphere_field_converges_to_the_sphere():
    """A sampled sphere's distance is within sqrt(3) h of the exact one (the
    field is 1-Lipschitz and the sample lies in the same cell), and its
    central-difference normal points radially from that sample."""
    R, h, res = 0.1, 0.3 / 24, 24
    o = np.array([-0.15, -0.15, -0.15])
    fld = _field(lambda q: np.linalg.norm(q) - R, o, h, res)
    rng = np.random.default_rng(14)
    for _ in range(300):
        u = rng.normal(size=3)
        u /= np.linalg.norm(u)
        p = u * rng.uniform(0.07, 0.13)
        d, nrm, _ = O.sdf_sampled(fld, p)
        assert abs(d - (np.linalg.norm(p) - R)) <= math.sqrt(3) * h + 1e-7
        corner = o + h * np.floor((p - o) / h)              # the sample the normal is taken at
        assert nrm @ (corner / np.linalg.norm(corner)) > 0.999


def test_sampled_tool_contact_removes_the_normal_velocity():
    """A static sampled tool whose field is the plane 2 (q_y - y0) (gradient
    of length 2, so the normal must be normalised), turned about z by phi:
    with mu = 0 a node moving into it keeps exactly its velocity minus the
    component along the world normal R e_y; a separating node is untouched.
    x_ref of the node is (0, -0.003, 0), well inside a cell."""
    fld = _field(lambda q: 2.0 * (q[1] - 0.013), np.array([-0.0625] * 3), 1.0 / 128, 16)
    prm = _params(n=8, friction=0.0)
    node = np.array([0.5, 0.5, 0.5])
    for phi in (0.0, 0.7, -2.1):
        pose = np.zeros(6)
        pose[5] = phi
        R = O.rotvec_to_matrix(pose[3:]).reshape(3, 3)
        pose[:3] = node - R @ np.array([0.0, -0.003, 0.0])
        frames = O.tool_frames(scenes.sampled_shape(), pose, pose, 1, 1e-3, fld)
        n_w = R @ np.array([0.0, 1.0, 0.0])
        t_w = R @ np.array([1.0, 0.0, 0.2])
        for v_in, touches in ((-0.5 * n_w + t_w, True), (0.4 * n_w + t_w, False)):
            m, mv = _one_node_grid({"v_in": v_in})
            gv, contact, _ = O.grid_update(prm, m, mv, frames, 1)
            assert contact[4, 4, 4] == 0
            want = v_in - (v_in @ n_w) * n_w if touches else v_in
            assert np.allclose(gv[4, 4, 4], want, atol=1e-12), (phi, gv[4, 4, 4], want)


def test_sampled_capsule_agrees_with_the_analytic_capsule():
    """The grid operation with a sampled capsule (h = dx / 4) finds the same
    contacts as with the analytic capsule wherever the analytic distance is
    more than sqrt(3) h from the threshold."""
    n, r, hl = 32, 0.06, 0.08
    prm = _params(n=n, friction=0.3, theta=0.0)
    h, res = (1.0 / n) / 4, 48
    o = np.full(3, -0.5 * h * res) + np.array([0.0013, -0.0021, 0.0007])
    dims = np.array([r, hl, 0.0])
    fld = _field(lambda q: O.sdf(scenes.CAPSULE, dims, q)[0], o, h, res)
    rng = np.random.default_rng(15)
    pose = np.array([0.51, 0.49, 0.5, 0.3, -0.2, 0.5])
    m = np.zeros((n, n, n))
    mv = np.zeros((n, n, n, 3))
    m[8:24, 8:24, 8:24] = 1.0
    mv[8:24, 8:24, 8:24] = rng.normal(size=(16, 16, 16, 3))
    fa = O.tool_frames(scenes.capsule_shape(r, hl), pose, pose, 1, 1e-3)
    fs = O.tool_frames(scenes.sampled_shape(), pose, pose, 1, 1e-3, fld)
    _, ca, _ = O.grid_update(prm, m, mv, fa, 1)
    _, cs, _ = O.grid_update(prm, m, mv, fs, 1)
    R = O.rotvec_to_matrix(pose[3:]).reshape(3, 3)
    ii = np.argwhere(m > 0)
    far = 0
    for i, j, k in ii:
        xr = R.T @ (np.array([i, j, k]) / n - pose[:3])
        da = O.sdf(scenes.CAPSULE, dims, xr)[0]
        if abs(da) > math.sqrt(3) * h:
            far += 1
            assert ca[i, j, k] == cs[i, j, k], (i, j, k, da)
    assert far > 1000 and (ca == 0).sum() > 50


def test_wall_band_is_three_nodes_deep_on_every_face():
    """Sec. III-B boundary condition, reading c4: sticky walls zero the velocity
    of every node within 3 nodes of any face.  Checked by closed forms rather
    than by the band test itself: the zeroed set holds n^3 - (n - 6)^3 nodes,
    it is mirror-symmetric on every axis (node i <-> n - 1 - i, the domain
    [0, 1) seen from either end), and no interior node is touched."""
    n = 16
    prm = O.OracleParams(n_grid=n, dt=1e-3, E=1e3, nu=0.3, rho=1e3, V0=1e-6, gravity=(0.0, 0.0, 0.0))
    gm = np.ones(n ** 3)
    gmv = np.tile([1.0, 2.0, 3.0], n ** 3)
    v, _, _ = O.grid_update(prm, gm, gmv)
    zero = np.all(v == 0.0, axis=-1)
    assert zero.sum() == n ** 3 - (n - 6) ** 3
    for ax in range(3):
        assert np.array_equal(zero, np.flip(zero, axis=ax))
    assert not zero[3:n - 3, 3:n - 3, 3:n - 3].any()
    assert np.allclose(v[~zero], [1.0, 2.0, 3.0])


def test_zbuffer_tie_goes_to_the_lower_tool_index():
    """Sec. III-C's multi-object merge, reading c11: on a tie of the closest
    distance, the lower object index wins.  Two capsules at the same pose with
    different velocities tie at every node; the pair must act exactly as the
    first capsule alone, and not as the second."""
    rng = np.random.default_rng(21)
    prm = _params(n=16, friction=0.3)
    n = prm.n_grid
    m = np.zeros((n, n, n))
    mv = np.zeros((n, n, n, 3))
    m[4:12, 4:12, 4:12] = 1.0 + rng.random((8, 8, 8))
    mv[4:12, 4:12, 4:12] = rng.normal(size=(8, 8, 8, 3))
    base = {"shape": [scenes.CAPSULE, 0.12, 0.1, 0.0], "T": [0.5, 0.52, 0.48], "w": [0.0, 0.0, 0.0],
            "R": list(O.rotvec_to_matrix(np.array([0.3, -0.2, 0.4])).reshape(9))}
    t0 = dict(base, u=[0.4, -1.0, 0.2])
    t1 = dict(base, u=[-0.7, 0.5, 0.9])
    v01, c01, _ = O.grid_update(prm, m, mv, _frames_from_case([t0, t1]), 2)
    v0, c0, _ = O.grid_update(prm, m, mv, _frames_from_case([t0]), 1)
    v1, _, _ = O.grid_update(prm, m, mv, _frames_from_case([t1]), 1)
    hit = c0 == 0
    assert hit.sum() > 20
    assert np.array_equal(v01, v0) and np.array_equal(c01, c0)
    assert np.abs(v01[hit] - v1[hit]).max() > 0.1
