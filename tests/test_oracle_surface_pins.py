"""Pins of the oracle's surface extraction (the renderer's Marching Cubes
step, in its tetrahedral form) against geometry: a sampled sphere gives a
closed, consistently oriented surface of Euler characteristic 2 whose area
and enclosed volume approach the sphere's; a linear field gives the exact
plane; random closed fields give closed surfaces."""
import math

import numpy as np

from oracle import oracle as O


def _edges(tris):
    """Directed edges keyed by exact vertex coordinates."""
    keys = [tuple(v) for v in tris.reshape(-1, 3)]
    ids = {}
    vid = np.array([ids.setdefault(k, len(ids)) for k in keys]).reshape(-1, 3)
    directed = [(t[a], t[(a + 1) % 3]) for t in vid for a in range(3)]
    return vid, directed, len(ids)


def _closed_and_oriented(tris):
    vid, directed, nv = _edges(tris)
    ds = {}
    for e in directed:
        ds[e] = ds.get(e, 0) + 1
    for (a, b), c in ds.items():
        if c != 1 or ds.get((b, a), 0) != 1:      # each edge once each way: closed and consistently oriented
            return False, None
    und = {tuple(sorted(e)) for e in directed}
    return True, nv - len(und) + len(tris)        # Euler characteristic


def _normals(tris):
    return np.cross(tris[:, 1] - tris[:, 0], tris[:, 2] - tris[:, 0])


def test_sphere_is_closed_oriented_and_converges():
    c = np.array([0.5013, 0.4987, 0.5021])
    R = 0.3
    for n in (24, 48):
        dx = 1.0 / (n - 1)
        g = np.arange(n) * dx
        X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
        field = R - np.sqrt((X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Z - c[2]) ** 2)
        tris = O.surface(field, 0.0, dx)
        closed, chi = _closed_and_oriented(tris)
        assert closed and chi == 2, n
        r = np.linalg.norm(tris.reshape(-1, 3) - c, axis=1)
        assert np.abs(r - R).max() <= 0.1 * dx
        nrm = _normals(tris)
        area = 0.5 * np.linalg.norm(nrm, axis=1).sum()
        vol = np.einsum("ij,ij->i", tris[:, 0] - c, np.cross(tris[:, 1] - c, tris[:, 2] - c)).sum() / 6.0
        assert abs(area / (4 * math.pi * R * R) - 1) < (0.02 if n == 24 else 0.01), (n, area)
        assert abs(vol / (4 / 3 * math.pi * R ** 3) - 1) < (0.015 if n == 24 else 0.004), (n, vol)   # inscribed: O(dx^2)
        cen = tris.mean(axis=1) - c
        assert np.all(np.einsum("ij,ij->i", cen, nrm) > 0)        # every triangle faces outward


def test_linear_field_gives_the_exact_plane():
    n, z0 = 12, 0.4371
    dx = 1.0 / (n - 1)
    g = np.arange(n) * dx
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    tris = O.surface(z0 - Z, 0.0, dx)
    assert np.abs(tris[..., 2] - z0).max() < 1e-14
    nrm = _normals(tris)
    assert np.all(nrm[:, 2] > 0) and np.abs(nrm[:, :2]).max() < 1e-12    # facing the outside, z > z0
    assert abs(0.5 * nrm[:, 2].sum() - 1.0) < 1e-12                       # the unit cross-section


def test_random_closed_fields_give_closed_surfaces():
    rng = np.random.default_rng(3)
    for trial in range(5):
        n = 10
        field = rng.random((n, n, n))
        field[0, :, :] = field[-1, :, :] = field[:, 0, :] = field[:, -1, :] = field[:, :, 0] = field[:, :, -1] = 0.0
        tris = O.surface(field, 0.5, 0.1)
        closed, chi = _closed_and_oriented(tris)
        assert closed and chi % 2 == 0, trial
