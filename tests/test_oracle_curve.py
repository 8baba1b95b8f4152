"""Pins of the intersection curve of two bodies (the crease of a Boolean
result, Sec. 3.2.3; reading: it carries feature particles like a feature
line, Sec. 3.2.2).  Two unit icospheres whose centres are 1.2 apart meet on
the circle x = 0.6, r = 0.8 (up to the facets' chord error); every curve
point lies on a triangle of both meshes (brute force), the curve is one
closed line, and its particles are spaced L / ceil(L / dx)."""
import numpy as np
import pytest

import oracle as O
from paper_2501_03056_gb300 import workloads as W


def two_spheres(offset, level=4, dx=0.03):
    v, t = W.icosphere_mesh(level)
    v2 = (v.astype(np.float64) + np.asarray(offset)).astype(np.float32)
    h = float(np.float32(1.3 * dx))
    a, b = O.Oracle(v, t, dx, h), O.Oracle(v2, t, dx, h)
    a.set_particles(np.zeros((0, 3), np.float32), np.zeros(0, np.int32))
    return a, b, (v, t), (v2, t)


def point_triangle_distance(p, V, T):
    """Brute-force distance from each point to the closest point of any
    triangle (interior foot or the closest point of an edge)."""
    out = np.full(len(p), np.inf)
    A, B, C = V[T[:, 0]].astype(np.float64), V[T[:, 1]].astype(np.float64), V[T[:, 2]].astype(np.float64)
    n = np.cross(B - A, C - A)
    n /= np.linalg.norm(n, axis=1)[:, None]

    def seg_dist(q, P0, P1):
        e = P1 - P0
        t = np.clip(np.einsum("ij,ij->i", q - P0, e) / np.einsum("ij,ij->i", e, e), 0.0, 1.0)
        return np.linalg.norm(q - (P0 + t[:, None] * e), axis=1)

    for i, q in enumerate(p.astype(np.float64)):
        d = np.einsum("ij,ij->i", q - A, n)
        f = q - d[:, None] * n
        v0, v1, v2 = B - A, C - A, f - A
        d00, d01, d11 = (v0 * v0).sum(1), (v0 * v1).sum(1), (v1 * v1).sum(1)
        d20, d21 = (v2 * v0).sum(1), (v2 * v1).sum(1)
        den = d00 * d11 - d01 * d01
        bv = (d11 * d20 - d01 * d21) / den
        bw = (d00 * d21 - d01 * d20) / den
        inside = (bv >= 0) & (bw >= 0) & (bv + bw <= 1)
        best = np.abs(d[inside]).min() if inside.any() else np.inf
        qq = np.broadcast_to(q, A.shape)
        edges = np.minimum(np.minimum(seg_dist(qq, A, B), seg_dist(qq, B, C)), seg_dist(qq, C, A))
        out[i] = min(best, edges.min())
    return out


@pytest.mark.parametrize("offset", [(1.2, 0.0137, 0.0291), (1.2, 0.0, 0.0)])
def test_two_spheres_meet_on_one_closed_circle(offset):
    a, b, (va, ta), (vb, tb) = two_spheres(offset)
    n = a.boolean_curve(b)
    pts = a.curve_points()
    first, nseg, closed, segv = a.feature_lines()
    assert len(nseg) == 1 and closed[0] == 1 and nseg[0] == len(pts)
    # on both surfaces (FP32 rounding of the points)
    assert point_triangle_distance(pts, va, ta).max() < 1e-6
    assert point_triangle_distance(pts, vb, tb).max() < 1e-6
    # near the analytic circle: the plane halfway between the centres, radius
    # sqrt(1 - 0.6^2 - ...) up to the chord error of the level-4 facets
    c = np.asarray(offset) / 2
    u = np.asarray(offset) / np.linalg.norm(offset)
    rel = pts.astype(np.float64) - c
    axial = rel @ u
    radial = np.linalg.norm(rel - np.outer(axial, u), axis=1)
    r_exact = np.sqrt(1 - (np.linalg.norm(offset) / 2) ** 2)
    assert np.abs(axial).max() < 2e-3 and np.abs(radial - r_exact).max() < 3e-3
    # particles: L / ceil(L / dx) along a loop of length L, all feature class
    x, cls, cons = a.get_particles()
    L = np.linalg.norm(np.diff(np.vstack([pts, pts[:1]]).astype(np.float64), axis=0), axis=1).sum()
    assert n == len(x) == int(np.ceil(L / 0.03 - 1e-12)) and np.all(cls == W.CLS_F)
    assert np.all((cons >= 0) & (cons < len(pts)))
    gaps = np.linalg.norm(np.diff(x, axis=0), axis=1)
    assert np.abs(gaps - L / n).max() < 0.02 * L / n       # chords of equal arcs on a fine polyline


def test_curve_particles_slide_along_the_curve_and_stay_on_it():
    # the union of the two spheres relaxed: the curve particles move only
    # along their line (they are exempt from the partner's side rule, lying
    # on both surfaces) and stay on both meshes
    a, b, (va, ta), (vb, tb) = two_spheres((1.2, 0.0137, 0.0291), level=3, dx=0.05)
    a.boolean_curve(b)
    x0, _, _ = a.get_particles()
    b.set_particles(np.zeros((0, 3), np.float32), np.zeros(0, np.int32))
    O.boolean_relax(a, b, O.UNION, 5)
    x, cls, cons = a.get_particles()
    assert np.abs(x - x0).max() > 0                              # they moved
    assert point_triangle_distance(x.astype(np.float32), va, ta).max() < 1e-5
    assert point_triangle_distance(x.astype(np.float32), vb, tb).max() < 1e-5
