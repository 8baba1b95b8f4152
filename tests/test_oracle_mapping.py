"""Pins of the oracle's particle generation (Sec. 3.2, Figs. 6, 8, 9):
closed-form counts and positions on the cube, containment on the sphere,
ray parity against the analytic inside test, band layers."""
import numpy as np

import oracle as O
from paper_2501_03056_gb300 import workloads as W


def test_cube_generation_closed_form():
    v, t = W.cube_mesh()
    o = O.Oracle(v, t, 0.05, 0.065)
    o.extract_features(30.0)
    x, c, cons = o.map_particles()
    counts = np.bincount(c, minlength=5)
    # the triangle grid puts cell centres on the faces: 21^3 - 19^3 surface
    # cells, all projectable; 19^3 interior cells; 12 x 19 edge + 8 corners
    assert counts[W.CLS_S] == 21 ** 3 - 19 ** 3
    assert counts[W.CLS_V] == 19 ** 3
    assert counts[W.CLS_F] == 12 * 19 and counts[W.CLS_P] == 8
    S = x[c == W.CLS_S]
    assert np.all(np.abs(np.abs(S).max(axis=1) - 0.5) < 1e-15)
    # S particles on the face lattice (k + 1/2) dx or on the edges
    assert np.all(cons[c == W.CLS_S] >= 0)
    V = x[c == W.CLS_V]
    grid = (V + 0.45) / 0.05
    assert np.all(np.abs(V) <= 0.45 + 1e-7) and np.all(np.abs(grid - np.round(grid)) < 1e-5)
    # features first, then surface, then volume
    order = np.r_[np.where(np.isin(c, [W.CLS_F, W.CLS_P]))[0].max(), np.where(c == W.CLS_S)[0].min()]
    assert order[0] < order[1] < np.where(c == W.CLS_V)[0].min()


def test_cube_band_layers():
    v, t = W.cube_mesh()
    o = O.Oracle(v, t, 0.05, 0.065)
    x, c, _ = o.map_particles(features=False, band_cells=2)
    V, I = x[c == W.CLS_V], x[c == W.CLS_I]
    # interior cell centres at |x|_inf <= 0.45; within 2 cells of the shell
    # (centres at 0.5) means |x|_inf >= 0.40
    assert len(V) == 19 ** 3 - 15 ** 3 and len(I) == 15 ** 3
    assert np.all(np.abs(V).max(axis=1) >= 0.40 - 1e-7) and np.all(np.abs(I).max(axis=1) <= 0.35 + 1e-7)


def test_sphere_generation_is_inside_and_body_fitted():
    v, t = W.icosphere_mesh(3)
    dx = 0.06
    o = O.Oracle(v, t, dx, 1.3 * dx)
    x, c, cons = o.map_particles(features=False)
    V, S = x[c == W.CLS_V], x[c == W.CLS_S]
    r = np.linalg.norm(V, axis=1)
    assert r.max() < 1.0 and len(V) > 0.8 * (4 / 3) * np.pi * (1 - dx) ** 3 / dx ** 3
    # every lattice centre well inside the sphere is a volume particle
    org, inv, n = o.tri_grid()
    g = [org[a] + (np.arange(n[a]) + 0.5) * dx for a in range(3)]
    P = np.stack(np.meshgrid(*g, indexing="ij"), -1).reshape(-1, 3)
    deep = P[np.linalg.norm(P, axis=1) < 1 - 2 * dx]
    assert len(V) >= len(deep)
    # surface particles lie on their triangle's plane, near the sphere
    vv = v.astype(np.float64)
    tri = t[cons[c == W.CLS_S]]
    nrm = np.cross(vv[tri[:, 1]] - vv[tri[:, 0]], vv[tri[:, 2]] - vv[tri[:, 0]])
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    assert np.abs(np.einsum("ij,ij->i", S - vv[tri[:, 0]], nrm)).max() < 1e-14
    assert np.all(np.abs(np.linalg.norm(S, axis=1) - 1.0) < 0.02)


def test_generation_ray_parity_matches_the_analytic_torus():
    v, t = W.torus_mesh(1.0, 0.3, 96, 32)
    dx = 0.05
    o = O.Oracle(v, t, dx, 1.3 * dx)
    x, c, _ = o.map_particles(surface=False, features=False)
    tube = np.sqrt((np.sqrt(x[:, 0] ** 2 + x[:, 1] ** 2) - 1.0) ** 2 + x[:, 2] ** 2)
    assert tube.max() < 0.3 and len(x) > 0
