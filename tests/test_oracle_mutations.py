"""The oracle's pins have teeth: plant a plausible mistake in a copy of the
oracle source (a dropped term, a wrong sign, a transposed operand, a wrong
index, the garbled printed form of Eq. 5; in the forward step and in its
adjoint), build it, and check that the pin suites fail on it.  The same for
the Python part of the oracle (the closed-form derivative of the tool frame
map used by the rollout gradients), loaded in place of oracle/oracle.py in a
child process.  Runs on the CPU only; the real oracle is untouched."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "mpm_oracle.c")

MUTATIONS = {
    "Eq5 printed F - F^T": ("mu * (F[i] - FiT[i])", "mu * (F[i] - F[3 * (i % 3) + i / 3])"),
    "stress impulse sign": ("const double f = -(4.0 / (dx * dx))", "const double f = (4.0 / (dx * dx))"),
    "stress uses F^T F": ("mat_mul(P, FT, out);", "mat_mul(FT, P, out);"),
    "dropped affine term": ("mom[a] = mp * vp[a] + mp * Cd + f * p->dt;", "mom[a] = mp * vp[a] + f * p->dt;"),
    "transposed C in P2G": ("Cd += Cp[3 * a + b] * xi_xp[b];", "Cd += Cp[3 * b + a] * xi_xp[b];"),
    "transposed C in G2P": ("B[3 * a + b] += wip * vi[a] * xi_xp[b];", "B[3 * b + a] += wip * vi[a] * xi_xp[b];"),
    "F update order": ("mat_mul(IdtC, Fp, Fn);", "mat_mul(Fp, IdtC, Fn);"),
    "weight w2": ("w[2] = 0.5 * (fx - 0.5) * (fx - 0.5);", "w[2] = 0.5 * (fx - 0.4) * (fx - 0.4);"),
    "node index order": ("return ((int64_t)i * n + j) * n + k;", "return ((int64_t)k * n + j) * n + i;"),
    "no gravity": ("+ p->dt * p->gravity[a];  /* Eq. 7", ";  /* Eq. 7"),
    "advect with old v": ("vp[a] = vnew[a];\n            xp[a] += p->dt * vnew[a];",
                          "xp[a] += p->dt * vp[a];\n            vp[a] = vnew[a];"),
    "x_ref uses R not R^T": ("s += tl->R[3 * b + a] * (xw[b] - tl->T[b]);", "s += tl->R[3 * a + b] * (xw[b] - tl->T[b]);"),
    "friction not clamped": ("c->scale = c->s > 0.0 ? c->s / c->vtn : 0.0;", "c->scale = c->s / c->vtn;"),
    "projects separating nodes": ("if (c->vn < 0.0) {", "if (c->vn < 1e30) {"),
    "normal not rotated": ("c->nw[a] += tl->R[3 * a + b] * nref[b];", "c->nw[a] += tl->R[3 * b + a] * nref[b];"),
    "tool velocity drops spin": ("c->vco[0] = tl->u[0] + tl->w[1] * c->r[2] - tl->w[2] * c->r[1];", "c->vco[0] = tl->u[0];"),
    "z-buffer picks farthest": ("if (d < dmin) {", "if (d > dmin || dmin == INFINITY) {"),
    "walls ignored": ("v[0] = v[1] = v[2] = 0.0;          /* sticky walls */", ";"),
    "sampled index rounds": ("const double f = floor(u);", "const double f = floor(u + 0.5);"),
    "sampled axis order": ("#define ORC_SDF_AT(i, j, k) ((double)sdf[((int64_t)(k) * res + (j)) * res + (i)])",
                           "#define ORC_SDF_AT(i, j, k) ((double)sdf[((int64_t)(i) * res + (j)) * res + (k)])"),
    "sampled normal not normalised": ("if (gn > 0.0) { nrm[0] = g[0] / gn; nrm[1] = g[1] / gn; nrm[2] = g[2] / gn; }",
                                      "if (gn > 0.0) { nrm[0] = g[0]; nrm[1] = g[1]; nrm[2] = g[2]; }"),
    "sampled difference reversed": ("(ORC_SDF_AT(hi[0], hi[1], hi[2]) - ORC_SDF_AT(lo[0], lo[1], lo[2])) / span",
                                    "(ORC_SDF_AT(lo[0], lo[1], lo[2]) - ORC_SDF_AT(hi[0], hi[1], hi[2])) / span"),
    "sampled faces not one-sided": ("const double span = (double)(hi[a] - lo[a]) * h;", "const double span = 2.0 * h;"),
    "sampled outside counts as contact": ("            return INFINITY;\n        }\n        c[a] = (int64_t)f;",
                                          "            return -1.0;\n        }\n        c[a] = (int64_t)f;"),
    "adjoint drops dt x_bar": ("vbt[a] = vbo[a] + dt * xbo[a];", "vbt[a] = vbo[a];"),
    "adjoint F update transposed": ("sF += IdtC[3 * c + a] * Fbo[3 * c + b];", "sF += IdtC[3 * a + c] * Fbo[3 * c + b];"),
    "adjoint C from F product transposed": ("sC += Fbo[3 * a + c] * Fp[3 * b + c];", "sC += Fbo[3 * a + c] * Fp[3 * c + b];"),
    "adjoint weight slope sign": ("    dw[0] = -(1.5 - fx);", "    dw[0] = (1.5 - fx);"),
    "adjoint grid mass sign": ("gmb[I] = -dotv / (gm[I] * gm[I]);", "gmb[I] = dotv / (gm[I] * gm[I]);"),
    "adjoint friction slope dropped": ("vnb += p->friction * scb / c.vtn;", "vnb += 0.0;"),
    "adjoint tool spin dropped": ("tb[15] += c.r[1] * vcob[2] - c.r[2] * vcob[1];", "tb[15] += 0.0;"),
    "adjoint normal curvature dropped": ("if (tl->kind != 2) sdf_normal_jacobian(tl->kind, tl->dims, xref, Jn);",
                                         "if (0) sdf_normal_jacobian(tl->kind, tl->dims, xref, Jn);"),
    "adjoint stress uses tau not its symmetrisation": ("s += (taub[3 * a + c] + taub[3 * c + a]) * Fp[3 * c + b];",
                                                       "s += 2.0 * taub[3 * a + c] * Fp[3 * c + b];"),
    "adjoint lambda uses J": ("lame_bar[1] += trb * (J > 0.0 ? log(J) : log(1e-6));", "lame_bar[1] += trb * J;"),
    "adjoint dpos term dropped in P2G": ("xbp[b] -= wip * am;", "xbp[b] -= 0.0 * am;"),
    "surface tetrahedra do not tile the cell": ("{{1, 3}, {1, 5}, {2, 3}, {2, 6}, {4, 5}, {4, 6}}",
                                                "{{1, 3}, {1, 5}, {2, 3}, {2, 6}, {4, 5}, {4, 5}}"),
    "surface edge point from either end": ("    if (a > b) { const int t = a; a = b; b = t; }\n    int pa[3], pb[3];",
                                           "    int pa[3], pb[3];"),
    "surface lone vertex odd permutation": ("{1, 0, 3, 2}, {2, 0, 1, 3}", "{1, 0, 2, 3}, {2, 0, 1, 3}"),
    "surface quad parity ignored": ("if (inv & 1) { const int x = perm[2];", "if (0) { const int x = perm[2];"),
    "surface interpolation from the wrong end": ("const double t = (iso - f[a]) / (f[b] - f[a]);",
                                                 "const double t = (f[b] - iso) / (f[b] - f[a]);"),
    "wall band one node narrower at the top": ("i >= n - b || j >= n - b || k >= n - b;", "i > n - b || j > n - b || k > n - b;"),
    "friction with the wrong sign": ("c->s = c->vtn + p->friction * c->vn;", "c->s = c->vtn - p->friction * c->vn;"),
    "Lame lambda with 1 + 2 nu": ("*lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));", "*lam = E * nu / ((1.0 + nu) * (1.0 + 2.0 * nu));"),
    "C scaled by 3 / dx^2": ("Cp[a] = 4.0 / (dx * dx) * B[a];     /* Eq. 9 */", "Cp[a] = 3.0 / (dx * dx) * B[a];     /* Eq. 9 */"),
    "stencil base without the half-cell shift": ("int b = (int)floor(s - 0.5);\n        if (b < 0) { b = 0; bad = 1; }",
                                                 "int b = (int)floor(s);\n        if (b < 0) { b = 0; bad = 1; }"),
    "volumetric stress term dropped": ("P[i] = mu * (F[i] - FiT[i]) + lam * lnJ * FiT[i];", "P[i] = mu * (F[i] - FiT[i]);"),
    "empty nodes get gravity": ("                if (grid_m[I] > 0.0) {\n                    for (int a = 0; a < 3; ++a)",
                                "                if (grid_m[I] >= 0.0) {\n                    for (int a = 0; a < 3; ++a)"),
    "particle mass without density": ("    const double dx = 1.0 / n;\n    const double mp = p->rho * p->V0;",
                                      "    const double dx = 1.0 / n;\n    const double mp = p->V0;"),
    "z-buffer tie goes to the later tool": ("        if (d < dmin) {\n            *d2 = dmin;", "        if (d <= dmin) {\n            *d2 = dmin;"),
    "tool velocity over one sub-step, not the call": ("t->u[d] = (pose1[d] - pose0[d]) / span;", "t->u[d] = (pose1[d] - pose0[d]) / dt;"),
    "tool poses not interpolated within a call": ("t->T[d] = pose0[d] + s * (pose1[d] - pose0[d]);", "t->T[d] = pose1[d];"),
    "box interior normal on the wrong axis": ("    if (q[1] > q[a]) a = 1;\n    if (q[2] > q[a]) a = 2;", "    if (q[1] < q[a]) a = 1;\n    if (q[2] < q[a]) a = 2;"),
    "capsule segment not clamped": ("        if (c > dims[1]) c = dims[1];\n", ""),
    "adjoint flows through the walls": ("                if (in_wall_band(p, i, j, k)) continue;\n                double vf[3], vbar[3];",
                                        "                double vf[3], vbar[3];"),
    "surface skips the last cell layer": ("    for (int k = 0; k + 1 < n; ++k)\n        for (int j = 0; j + 1 < n; ++j)",
                                          "    for (int k = 0; k + 2 < n; ++k)\n        for (int j = 0; j + 1 < n; ++j)"),
    "surface tetrahedron orientation ignored": ("if (tet_orientation(t[0], t[1], t[2], t[3]) < 0) {", "if (0) {"),
    "surface nin = 3 winding not flipped": ("if (nin == 3) { int s0 = e[1][0]", "if (0) { int s0 = e[1][0]"),
    "tool contact at cell centres, not nodes": ("const double xw[3] = {i * dx, j * dx, k * dx};\n                        double nref[3]",
                                                "const double xw[3] = {(i + 0.5) * dx, (j + 0.5) * dx, (k + 0.5) * dx};\n                        double nref[3]"),
    "gravity added to momentum before the division": ("v[a] = grid_mv[3 * I + a] / grid_m[I] + p->dt * p->gravity[a];  /* Eq. 7 + gravity */",
                                                      "v[a] = (grid_mv[3 * I + a] + p->dt * p->gravity[a]) / grid_m[I];  /* Eq. 7 + gravity */"),
    "block key axis order": ("keys[q] = (uint32_t)(b[0] + nb * (b[1] + nb * b[2]));", "keys[q] = (uint32_t)(b[2] + nb * (b[1] + nb * b[0]));"),
}


PINS = {"forward": "test_oracle_pins.py", "adjoint": "test_oracle_adjoint_pins.py",
        "surface": "test_oracle_surface_pins.py"}


def _suite(name):
    """The pin file a mistake must fail: the adjoint's and the surface's own
    pins for mistakes in those parts, the forward pins otherwise."""
    if name.startswith("adjoint"):
        return PINS["adjoint"]
    if name.startswith("surface"):
        return PINS["surface"]
    return PINS["forward"]


def _run_c_mutant(name, work):
    """Build the oracle with planted mistake `name` and run its pin suite;
    returns (anchor found once, pin-suite exit code, output)."""
    old, new = MUTATIONS[name]
    src = open(SRC).read()
    if src.count(old) != 1:
        return False, None, ""
    os.makedirs(work, exist_ok=True)
    mutated = os.path.join(work, "mut.c")
    with open(mutated, "w") as fh:
        fh.write(src.replace(old, new))
    lib = os.path.join(work, "libmut.so")
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                           "-o", lib, mutated, "-lm"])
    env = dict(os.environ, ORACLE_LIB=lib)
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", _suite(name))],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    return True, r.returncode, r.stdout[-2000:] + r.stderr[-2000:]


def _in_parallel(fn, names, base):
    """fn(name, work dir) for every name, the independent child processes
    running side by side on the host's cores."""
    from concurrent.futures import ThreadPoolExecutor
    workers = max(1, min(len(names), os.cpu_count() or 1))
    with ThreadPoolExecutor(max_workers=workers) as ex:
        futs = {n: ex.submit(fn, n, os.path.join(str(base), "m%02d" % i)) for i, n in enumerate(names)}
        return {n: f.result() for n, f in futs.items()}


@pytest.fixture(scope="module")
def c_mutants(tmp_path_factory):
    return _in_parallel(_run_c_mutant, sorted(MUTATIONS), tmp_path_factory.mktemp("c_mutants"))


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_catch_planted_mistake(name, c_mutants):
    unique, rc, out = c_mutants[name]
    assert unique, "mutation anchor must be unique: " + name
    assert rc != 0, "planted mistake '%s' passed every pin" % name


PY_SRC = os.path.join(ROOT, "oracle", "oracle.py")

PY_MUTATIONS = {
    "adjoint frame: Rodrigues slope term dropped": ("out[i] = da * r[i] * K + a * Ei + db * r[i] * K2",
                                                    "out[i] = a * Ei + db * r[i] * K2"),
    "adjoint frame: R0 derivative not transposed": ("np.einsum(\"ajk,jk->a\", dlog, R1 @ dR0[i].T)",
                                                    "np.einsum(\"ajk,jk->a\", dlog, R1 @ dR0[i])"),
    "adjoint frame: log trace term dropped": ("out[a] += g * sv[a] * np.eye(3)", "out[a] += 0.0 * sv[a] * np.eye(3)"),
    "adjoint frame: linear velocity sign": ("J[12 + i, i] = -1.0 / span", "J[12 + i, i] = 1.0 / span"),
    "adjoint frame: exp(s phi) R0 drops the R0 derivative": ("J[0:9, 3 + i] = (dE0 @ R0 + Es @ dR0[i]).reshape(9)",
                                                              "J[0:9, 3 + i] = (dE0 @ R0).reshape(9)"),
}

_DRIVER = """
import importlib.util, sys
sys.path.insert(0, %r)
import oracle as pkg
spec = importlib.util.spec_from_file_location("oracle.oracle", %r)
mod = importlib.util.module_from_spec(spec)
sys.modules["oracle.oracle"] = mod
spec.loader.exec_module(mod)
pkg.oracle = mod
import pytest
sys.exit(pytest.main(["-q", "-x", "-p", "no:cacheprovider", %r]))
"""


def _run_py_mutant(name, work):
    """Load oracle/oracle.py with planted mistake `name` in a child process
    and run its pin suite; returns (anchor found once, exit code, output)."""
    from oracle import oracle as O
    old, new = PY_MUTATIONS[name]
    src = open(PY_SRC).read()
    if src.count(old) != 1:
        return False, None, ""
    os.makedirs(work, exist_ok=True)
    mutated = os.path.join(work, "oracle.py")
    with open(mutated, "w") as fh:
        fh.write(src.replace(old, new))
    env = dict(os.environ, ORACLE_LIB=O.build())
    code = _DRIVER % (ROOT, mutated, os.path.join(ROOT, "tests", _suite(name)))
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    return True, r.returncode, r.stdout + r.stderr


@pytest.fixture(scope="module")
def py_mutants(tmp_path_factory):
    from oracle import oracle as O
    O.build()                    # once, before the children share the library
    return _in_parallel(_run_py_mutant, sorted(PY_MUTATIONS), tmp_path_factory.mktemp("py_mutants"))


@pytest.mark.parametrize("name", sorted(PY_MUTATIONS))
def test_pins_catch_planted_python_mistake(name, py_mutants):
    unique, rc, out = py_mutants[name]
    assert unique, "mutation anchor must be unique: " + name
    assert "passed" in out or "failed" in out, out
    assert rc != 0, "planted mistake '%s' passed every pin" % name
