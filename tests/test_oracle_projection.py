"""Pins of the oracle's constraint step (Sec. 3.2.1, 3.3.3, 3.3.4, Fig. 6, 8).

Closed-form feet on flat faces, brute-force all-triangle search, the
triangle-box binning against polygon clipping, and the pseudonormal inside
test against ray parity and the analytic sphere."""
import numpy as np
import pytest

import oracle as O
from paper_2501_03056_gb300 import workloads as W


def surface_points_cube(n, seed, spread=0.3):
    rng = np.random.default_rng(seed)
    axis = rng.integers(0, 3, n)
    sgn = rng.choice([-1.0, 1.0], n)
    p = rng.uniform(-0.49, 0.49, (n, 3))
    p[np.arange(n), axis] = sgn * 0.5 + rng.uniform(-spread, spread, n) * 0.05
    return p.astype(np.float32), axis, sgn


def test_surface_projection_on_cube_faces_is_the_closed_form_foot():
    v, t = W.cube_mesh()
    o = O.Oracle(v, t, 0.05, 0.065)
    y, axis, sgn = surface_points_cube(3000, 0)
    x, tri, ok = o.project_points(y, np.zeros(len(y), np.int32))
    assert ok.all()
    # closed form: among the faces whose square contains the foot, the
    # nearest plane wins
    yd = y.astype(np.float64)
    best = np.full(len(y), np.inf)
    expect = yd.copy()
    for ax in range(3):
        others = [k for k in range(3) if k != ax]
        inside = np.all(np.abs(yd[:, others]) <= 0.5, axis=1)
        for s_ in (-0.5, 0.5):
            d = np.abs(yd[:, ax] - s_)
            take = inside & (d < best)
            best[take] = d[take]
            expect[take] = yd[take]
            expect[take, ax] = s_
            axis = np.where(take, ax, axis)
    np.testing.assert_allclose(x, expect, atol=1e-15)
    # the chosen triangle lies on that face
    nrm = np.cross(v[t[tri, 1]] - v[t[tri, 0]], v[t[tri, 2]] - v[t[tri, 0]])
    assert np.all(np.argmax(np.abs(nrm), axis=1) == axis)


@pytest.mark.parametrize("mesh", ["cube", "ico2", "torus"])
def test_binned_search_equals_brute_force_near_the_surface(mesh):
    if mesh == "cube":
        v, t = W.cube_mesh()
        dx = 0.05
    elif mesh == "ico2":
        v, t = W.icosphere_mesh(2)
        dx = 0.1
    else:
        v, t = W.torus_mesh(1.0, 0.3, 24, 12)
        dx = 0.08
    o = O.Oracle(v, t, dx, 1.3 * dx)
    rng = np.random.default_rng(5)
    # points within dx / 2 of a random surface point
    tri = rng.integers(0, len(t), 2000)
    bc = rng.dirichlet([1, 1, 1], 2000)
    p = np.einsum("ij,ijk->ik", bc, v[t[tri]].astype(np.float64))
    p += rng.normal(size=p.shape) * 0.2 * dx
    y = p.astype(np.float32)
    x, co, ok = o.project_points(y, np.zeros(len(y), np.int32))
    bt, bd = o.brute_surface(y)
    # the closest projectable triangle is within the 27 cells whenever its
    # foot is closer than dx
    near = (bt >= 0) & (bd < 0.99 * dx)
    assert near.sum() > 1500
    assert np.array_equal(co[near], bt[near])
    assert np.all(ok[near])


def test_projected_surface_points_lie_on_their_triangle():
    v, t = W.icosphere_mesh(3)
    o = O.Oracle(v, t, 0.05, 0.065)
    rng = np.random.default_rng(2)
    d = rng.normal(size=(2000, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    y = (d * rng.uniform(0.985, 1.01, (2000, 1))).astype(np.float32)
    x, tri, ok = o.project_points(y, np.zeros(len(y), np.int32))
    assert ok.mean() > 0.99
    vv = v.astype(np.float64)
    a, b, c = vv[t[tri[ok], 0]], vv[t[tri[ok], 1]], vv[t[tri[ok], 2]]
    n = np.cross(b - a, c - a)
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    assert np.max(np.abs(np.einsum("ij,ij->i", x[ok] - a, n))) < 1e-14
    r = np.linalg.norm(x[ok], axis=1)
    assert r.max() <= 1.0 + 1e-12 and r.min() > 0.995


def test_revert_when_nothing_is_projectable():
    v, t = W.cube_mesh()
    o = O.Oracle(v, t, 0.05, 0.065)
    # beyond a convex corner no face's foot is inside
    y = np.array([[0.53, 0.53, 0.53]], np.float32)
    x, tri, ok = o.project_points(y, np.zeros(1, np.int32), np.array([7], np.int32))
    assert not ok[0] and tri[0] == 7
    np.testing.assert_array_equal(x[0], y[0].astype(np.float64))


def _clip_nonempty(tri, lo, hi):
    poly = [np.asarray(p, np.float64) for p in tri]
    for ax in range(3):
        for bound, keep in ((lo[ax], lambda q: q >= lo[ax]), (hi[ax], lambda q: q <= hi[ax])):
            out = []
            for i in range(len(poly)):
                p, q = poly[i], poly[(i + 1) % len(poly)]
                ip, iq = keep(p[ax]), keep(q[ax])
                if ip:
                    out.append(p)
                if ip != iq:
                    s = (bound - p[ax]) / (q[ax] - p[ax])
                    out.append(p + s * (q - p))
            poly = out
            if not poly:
                return False
    return True


def test_triangle_binning_matches_polygon_clipping():
    v, t = W.icosphere_mesh(1)
    dx = 0.21
    o = O.Oracle(v, t, dx, 1.3 * dx)
    org, inv, n = o.tri_grid()
    keys, tris = o.tri_bins()
    binned = set(zip(keys.tolist(), tris.tolist()))
    vv = v.astype(np.float64)
    slack = 1e-6 * dx
    for ti in range(len(t)):
        tri = vv[t[ti]]
        lo = np.floor((tri.min(0) - org) / dx).astype(int) - 1
        hi = np.floor((tri.max(0) - org) / dx).astype(int) + 1
        for z in range(max(lo[2], 0), min(hi[2], n[2] - 1) + 1):
            for y in range(max(lo[1], 0), min(hi[1], n[1] - 1) + 1):
                for x in range(max(lo[0], 0), min(hi[0], n[0] - 1) + 1):
                    c0 = org.astype(np.float64) + np.array([x, y, z]) * dx
                    key = x + n[0] * (y + n[1] * z)
                    inner = _clip_nonempty(tri, c0 + 1e-9, c0 + dx - 1e-9)
                    outer = _clip_nonempty(tri, c0 - 2 * slack, c0 + dx + 2 * slack)
                    if inner:
                        assert (key, ti) in binned
                    if not outer:
                        assert (key, ti) not in binned


@pytest.mark.parametrize("mesh", ["ico3", "torus"])
def test_pseudonormal_sign_agrees_with_ray_parity(mesh):
    if mesh == "ico3":
        v, t = W.icosphere_mesh(3)
        dx = 0.05
    else:
        v, t = W.torus_mesh(1.0, 0.3, 48, 16)
        dx = 0.05
    o = O.Oracle(v, t, dx, 1.3 * dx)
    rng = np.random.default_rng(11)
    tri = rng.integers(0, len(t), 3000)
    bc = rng.dirichlet([1, 1, 1], 3000)
    p = np.einsum("ij,ijk->ik", bc, v[t[tri]].astype(np.float64))
    p += rng.normal(size=p.shape) * 0.3 * dx
    y = p.astype(np.float32)
    ins = o.volume_inside(y)
    par = o.ray_parity(y.astype(np.float64))
    assert 0.3 < par.mean() < 0.7
    assert np.array_equal(ins, par)


def test_volume_inside_on_the_sphere_closed_form():
    v, t = W.icosphere_mesh(4)
    o = O.Oracle(v, t, 0.04, 0.052)
    rng = np.random.default_rng(4)
    d = rng.normal(size=(4000, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    r = rng.uniform(0.97, 1.03, (4000, 1))
    y = (d * r).astype(np.float32)
    ins = o.volume_inside(y)
    # level-4 icosphere: faces lie between radius cos(edge / 2) ~ 0.9995 and 1
    assert np.all(ins[r[:, 0] < 0.999])
    assert not np.any(ins[r[:, 0] > 1.0005])


def test_feature_projection_on_cube_edges():
    a = W.cube_workload()[0]
    o = O.from_assembly(a)
    rng = np.random.default_rng(9)
    t = rng.uniform(-0.45, 0.45, 500)
    y = np.stack([t, np.full(500, 0.5), np.full(500, -0.5)], 1) + rng.normal(size=(500, 3)) * 0.003
    x, seg, ok = o.project_points(y.astype(np.float32), np.full(500, W.CLS_F, np.int32))
    assert ok.all()
    np.testing.assert_allclose(x[:, 1], 0.5, atol=1e-15)
    np.testing.assert_allclose(x[:, 2], -0.5, atol=1e-15)
    np.testing.assert_allclose(x[:, 0], y[:, 0].astype(np.float32), atol=1e-7)
    assert len(np.unique(seg)) == 1


def test_zero_area_triangles_are_never_projection_targets():
    # a cube whose top face carries an extra zero-area sliver
    v, t = W.cube_mesh()
    v = np.vstack([v, [[0.0, 0.0, 0.5]]]).astype(np.float32)
    top = [i for i in range(len(t)) if np.all(v[t[i], 2] == 0.5)][0]
    a, b = t[top, 0], t[top, 1]
    t = np.vstack([t, [[a, b, a]]]).astype(np.int32)       # degenerate (repeated vertex)
    o = O.Oracle(v, t, 0.05, 0.065)
    rng = np.random.default_rng(0)
    y = np.stack([rng.uniform(-0.45, 0.45, 500), rng.uniform(-0.45, 0.45, 500),
                  np.full(500, 0.51)], 1).astype(np.float32)
    x, tri, ok = o.project_points(y, np.zeros(500, np.int32))
    assert ok.all() and np.all(tri != len(t) - 1)
    np.testing.assert_allclose(x[:, 2], 0.5, atol=1e-15)
    assert o.volume_inside(y - np.array([0, 0, 0.02], np.float32)).all()
