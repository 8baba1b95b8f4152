"""Pins of the oracle's Boolean union (Sec. 3.2.3, Fig. 10): which particles
stay (ray parity against the other mesh), against the closed forms of the
cube and of the icosphere's inscribed and circumscribed balls; surfaces kept
out of the partner during the union's relaxation; a union with a far-away
partner relaxes exactly as the body alone."""
import numpy as np

import oracle as O
from paper_2501_03056_gb300 import workloads as W


def _pair():
    a, b = W.union_pair_workload()
    return a, b, O.from_assembly(a), O.from_assembly(b)


def _ball_radii(b):
    """Inscribed and circumscribed radius of the (convex) icosphere about its centre."""
    v = b.verts.astype(np.float64)
    c = np.array([0.45, 0.05, -0.03])
    p = v[b.tris]
    n = np.cross(p[:, 1] - p[:, 0], p[:, 2] - p[:, 0])
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    r_in = np.abs(np.einsum("ij,ij->i", n, p[:, 0] - c)).min()
    r_out = np.linalg.norm(v - c, axis=1).max()
    return c, r_in, r_out


def test_union_keep_matches_the_closed_forms():
    a, b, oa, ob = _pair()
    c, r_in, r_out = _ball_radii(b)
    # cube particles inside the sphere go, whatever their class
    ka = oa.union_keep(ob, volume_stays=False)
    xa = oa.get_particles()[0]
    d = np.linalg.norm(xa - c, axis=1)
    assert not ka[d < r_in - 1e-9].any() and ka[d > r_out + 1e-9].all()
    assert (d < r_in - 1e-9).sum() > 500
    # sphere particles inside the cube: surface ones go, volume ones stay
    kb = ob.union_keep(oa, volume_stays=True)
    xb, cb, _ = ob.get_particles()
    inside = np.abs(xb).max(axis=1) < 0.5 - 1e-9
    outside = np.abs(xb).max(axis=1) > 0.5 + 1e-9
    vol = np.isin(cb, [W.CLS_V, W.CLS_I])
    assert kb[inside & vol].all() and not kb[inside & ~vol].any() and kb[outside].all()
    assert (inside & vol).sum() > 100 and (inside & ~vol).sum() > 100


def test_union_relaxation_keeps_surfaces_out_of_the_partner():
    a, b, oa, ob = _pair()
    O.keep_rows(oa, oa.union_keep(ob, False))
    O.keep_rows(ob, ob.union_keep(oa, True))
    c, r_in, r_out = _ball_radii(b)
    O.union_relax(oa, ob, 5)
    xa, ca, _ = oa.get_particles()
    xb, cb, _ = ob.get_particles()
    surf_a = np.isin(ca, [W.CLS_S, W.CLS_F])
    surf_b = np.isin(cb, [W.CLS_S, W.CLS_F])
    assert not (np.linalg.norm(xa[surf_a] - c, axis=1) < r_in - 1e-9).any()
    assert not (np.abs(xb[surf_b]).max(axis=1) < 0.5 - 1e-9).any()
    # volume particles stay inside the union
    in_cube = lambda x: np.abs(x).max(axis=1) <= 0.5 + 1e-9
    in_ball = lambda x: np.linalg.norm(x - c, axis=1) <= r_out + 1e-9
    assert (in_cube(xa) | in_ball(xa)).all() and (in_cube(xb) | in_ball(xb)).all()
    # the union moved: one shared time step over both bodies
    assert oa.last_iteration()[0] == ob.last_iteration()[0] > 0


def test_union_with_a_far_partner_relaxes_as_the_body_alone():
    # the partner is a cube 4 units away holding a few volume particles 5 dx
    # apart: no pair within 2h, zero force, so the shared amax is the
    # cube's own and the cube must relax exactly as alone
    a = W.cube_workload()[0]
    shift = np.array([4.0, 0.0, 0.0])
    g = (np.arange(3) - 1) * 5 * a.dx
    far = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3) + shift
    b = W.Assembly("cube_far", (a.verts + shift).astype(np.float32), a.tris, a.dx, a.h,
                   far.astype(np.float32), np.full(len(far), W.CLS_V, np.int32), 30.0, {})
    oa, ob, alone = O.from_assembly(a), O.from_assembly(b), O.from_assembly(a)
    assert oa.union_keep(ob, False).all() and ob.union_keep(oa, True).all()
    O.union_relax(oa, ob, 3)
    alone.relax(3)
    assert np.array_equal(oa.get_particles()[0], alone.get_particles()[0])
    assert np.array_equal(ob.get_particles()[0], far.astype(np.float32).astype(np.float64))


def test_union_keep_on_rays_through_mesh_edges():
    # points straight below the cap's fan edges of a 48-gon cylinder: an
    # undisplaced +z ray would cross both faces of each edge (even parity)
    v, t = W.cylinder_mesh(0.2, 0.5, 48, 6)
    dx, h = 0.01, 0.013
    cyl = O.Oracle(v, t, dx, h)
    ang = np.arange(48) * 2 * np.pi / 48
    r = np.repeat([0.1, 0.3], 48)
    pts = np.stack([r * np.cos(np.tile(ang, 2)), r * np.sin(np.tile(ang, 2)), np.zeros(96)], 1)
    bv, bt = W.cube_mesh(0.5)
    box = O.Oracle(bv, bt, dx, h)
    box.set_particles(pts.astype(np.float32), np.full(96, W.CLS_S, np.int32))
    keep = box.union_keep(cyl, volume_stays=False)
    assert np.array_equal(keep, r > 0.2)


def _classes(o):
    x, c, _ = o.get_particles()
    return x, c, np.isin(c, [W.CLS_S, W.CLS_F]), np.isin(c, [W.CLS_V, W.CLS_I])


def test_difference_and_intersection_keep_match_the_closed_forms():
    a, b, oa, ob = _pair()
    c, r_in, r_out = _ball_radii(b)
    xa, ca, _, vola = _classes(oa)
    xb, cb, surfb, volb = _classes(ob)
    da = np.linalg.norm(xa - c, axis=1)
    in_cube_b = np.abs(xb).max(axis=1) < 0.5 - 1e-9
    out_cube_b = np.abs(xb).max(axis=1) > 0.5 + 1e-9
    sure_in, sure_out = da < r_in - 1e-9, da > r_out + 1e-9
    # difference cube - sphere: the cube keeps what is outside the sphere,
    # the sphere keeps only its surface inside the cube (the cavity wall)
    ka, kb = oa.boolean_keep(ob, O.DIFFERENCE, True), ob.boolean_keep(oa, O.DIFFERENCE, False)
    assert not ka[sure_in].any() and ka[sure_out].all()
    assert not kb[volb].any() and kb[~volb & in_cube_b].all() and not kb[out_cube_b].any()
    # intersection: the cube keeps what is inside the sphere, the sphere its
    # surface inside the cube
    ka, kb = oa.boolean_keep(ob, O.INTERSECTION, True), ob.boolean_keep(oa, O.INTERSECTION, False)
    assert ka[sure_in].all() and not ka[sure_out].any()
    assert not kb[volb].any() and kb[~volb & in_cube_b].all() and not kb[out_cube_b].any()


def test_difference_relaxation_keeps_the_cavity():
    a, b, oa, ob = _pair()
    c, r_in, r_out = _ball_radii(b)
    O.keep_rows(oa, oa.boolean_keep(ob, O.DIFFERENCE, True))
    O.keep_rows(ob, ob.boolean_keep(oa, O.DIFFERENCE, False))
    O.boolean_relax(oa, ob, O.DIFFERENCE, 5)
    xa, _, _, _ = _classes(oa)
    xb, _, _, _ = _classes(ob)
    assert not (np.linalg.norm(xa - c, axis=1) < r_in - 1e-9).any()      # nothing of the cube in the cavity
    assert (np.abs(xb).max(axis=1) <= 0.5 + 1e-9).all()                    # the wall stays inside the cube
    assert (np.abs(xa).max(axis=1) <= 0.5 + 1e-9).all()


def test_intersection_relaxation_stays_in_both():
    a, b, oa, ob = _pair()
    c, r_in, r_out = _ball_radii(b)
    O.keep_rows(oa, oa.boolean_keep(ob, O.INTERSECTION, True))
    O.keep_rows(ob, ob.boolean_keep(oa, O.INTERSECTION, False))
    O.boolean_relax(oa, ob, O.INTERSECTION, 5)
    for o in (oa, ob):
        x = o.get_particles()[0]
        assert (np.abs(x).max(axis=1) <= 0.5 + 1e-9).all()
        assert (np.linalg.norm(x - c, axis=1) <= r_out + 1e-9).all()
