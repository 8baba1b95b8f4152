"""Pins of Boolean chains on the oracle (Sec. 3.2.3, Fig. 10 combines several
bodies): a body may take part in several operations, keeps what each of them
keeps, and relaxes under the rules of all of them.  Checked against the
closed forms of the icospheres' inscribed and circumscribed balls and of
the cube, which do not come from the oracle's rules: a union chain of three
spheres in a row (the middle one in two unions), a cube with two separate
spherical cavities (the cube in two differences), and the intersection
curves of the union chain, whose particles stay on both surfaces of their
own pair and outside the third sphere."""
import numpy as np
import pytest

import oracle as O
from paper_2501_03056_gb300 import workloads as W

S, V, F, I, P = W.CLS_S, W.CLS_V, W.CLS_F, W.CLS_I, W.CLS_P
DX = 0.05
H = float(np.float32(1.3 * DX))
R = 0.5
CENTRES = [np.array([0.0, 0.0, 0.0]), np.array([0.7, 0.0131, 0.0217]), np.array([1.4, 0.0297, -0.0113])]


def sphere(c, level=3):
    v, t = W.icosphere_mesh(level, R)
    v = (v.astype(np.float64) + c).astype(np.float32)
    p = v.astype(np.float64)[t]
    n = np.cross(p[:, 1] - p[:, 0], p[:, 2] - p[:, 0])
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    r_in = np.abs(np.einsum("ij,ij->i", n, p[:, 0] - c)).min()
    r_out = np.linalg.norm(v.astype(np.float64) - c, axis=1).max()
    return v, t, r_in, r_out


def generated(v, t, features=False):
    o = O.Oracle(v, t, DX, H)
    if features:
        o.extract_features(30.0)
    x, c, cons = o.map_particles()
    x32 = x.astype(np.float32)
    o.set_particles(x32, c)
    o.set_state(x32.astype(np.float64), cons)
    return o


def apply_op(oa, ob, op):
    """One Boolean operation on the current particle sets (oa first)."""
    ka, kb = oa.boolean_keep(ob, op, True), ob.boolean_keep(oa, op, False)
    O.keep_rows(oa, ka)
    O.keep_rows(ob, kb)


def union_chain():
    sp = [sphere(c) for c in CENTRES]
    bodies = [generated(v, t) for v, t, _, _ in sp]
    apply_op(bodies[0], bodies[1], O.UNION)
    apply_op(bodies[1], bodies[2], O.UNION)
    return sp, bodies


def surface_mask(c):
    return np.isin(c, [S, F, P])


def test_union_chain_keeps_every_surface_out_of_its_partners():
    sp, bodies = union_chain()
    x0 = [b.get_particles()[0].copy() for b in bodies]
    O.boolean_relax_many(bodies, [(0, 1, O.UNION), (1, 2, O.UNION)], 8)
    moved = 0.0
    for i, b in enumerate(bodies):
        x, c, _ = b.get_particles()
        moved = max(moved, np.abs(x - x0[i]).max())
        s = surface_mask(c)
        for j in (i - 1, i + 1):                  # the partners of body i
            if not 0 <= j < 3:
                continue
            d = np.linalg.norm(x[s] - CENTRES[j], axis=1)
            assert (d >= sp[j][2] - 1e-9).all(), (i, j, (d < sp[j][2]).sum())
    assert moved > 1e-3 * DX
    # the middle sphere lost surface on both sides: none of its surface
    # particles lies in the outer spheres' circumscribed balls' far halves
    xb, cb, _ = bodies[1].get_particles()
    s = surface_mask(cb)
    assert (np.linalg.norm(xb[s] - CENTRES[0], axis=1) >= sp[0][2] - 1e-9).all()
    assert (np.linalg.norm(xb[s] - CENTRES[2], axis=1) >= sp[2][2] - 1e-9).all()


def test_a_single_pair_through_the_chain_form_equals_the_pair_form():
    sp = [sphere(c) for c in CENTRES[:2]]
    one = [generated(v, t) for v, t, _, _ in sp]
    two = [generated(v, t) for v, t, _, _ in sp]
    apply_op(one[0], one[1], O.UNION)
    apply_op(two[0], two[1], O.UNION)
    O.boolean_relax(one[0], one[1], O.UNION, 4)
    O.boolean_relax_many(two, [(0, 1, O.UNION)], 4)
    for a, b in zip(one, two):
        assert np.array_equal(a.get_particles()[0], b.get_particles()[0])


def test_cube_with_two_cavities_keeps_both_walls():
    v, t = W.cube_mesh(0.5)
    cube = generated(v, t, features=True)
    cav = [np.array([0.55, 0.05, -0.02]), np.array([-0.55, -0.03, 0.04])]   # cutting the faces x = +-0.5
    sp = [sphere(c, level=3) for c in cav]
    holes = [generated(sv, st) for sv, st, _, _ in sp]
    apply_op(cube, holes[0], O.DIFFERENCE)
    apply_op(cube, holes[1], O.DIFFERENCE)
    O.boolean_relax_many([cube, holes[0], holes[1]], [(0, 1, O.DIFFERENCE), (0, 2, O.DIFFERENCE)], 8)
    xc, cc, _ = cube.get_particles()
    for q in range(2):
        # the cube keeps nothing inside either cavity
        d = np.linalg.norm(xc - cav[q], axis=1)
        assert (d >= sp[q][2] - 1e-9).all(), (q, (d < sp[q][2]).sum())
        # each cavity wall stays inside the cube and has no volume particles
        xh, ch, _ = holes[q].get_particles()
        assert len(xh) > 100 and not np.isin(ch, [V, I]).any()
        assert (np.abs(xh).max(axis=1) <= 0.5 + 1e-6).all()


def _dist_to_mesh(p, v, t):
    A, B, Cc = (v[t[:, k]].astype(np.float64) for k in range(3))
    n = np.cross(B - A, Cc - A)
    n /= np.linalg.norm(n, axis=1)[:, None]

    def seg(q, P0, P1):
        e = P1 - P0
        s = np.clip(np.einsum("ij,ij->i", q - P0, e) / np.einsum("ij,ij->i", e, e), 0.0, 1.0)
        return np.linalg.norm(q - (P0 + s[:, None] * e), axis=1)

    out = np.empty(len(p))
    for i, q in enumerate(p.astype(np.float64)):
        d = np.einsum("ij,ij->i", q - A, n)
        f = q - d[:, None] * n
        v0, v1, v2 = B - A, Cc - A, f - A
        d00, d01, d11 = (v0 * v0).sum(1), (v0 * v1).sum(1), (v1 * v1).sum(1)
        d20, d21 = (v2 * v0).sum(1), (v2 * v1).sum(1)
        den = d00 * d11 - d01 * d01
        bv, bw = (d11 * d20 - d01 * d21) / den, (d00 * d21 - d01 * d20) / den
        inside = (bv >= 0) & (bw >= 0) & (bv + bw <= 1)
        best = np.abs(d[inside]).min() if inside.any() else np.inf
        qq = np.broadcast_to(q, A.shape)
        out[i] = min(best, np.minimum(np.minimum(seg(qq, A, B), seg(qq, B, Cc)), seg(qq, Cc, A)).min())
    return out


def test_curves_of_a_chain_stay_on_their_own_pair():
    sp, bodies = union_chain()
    n_before = [b.n for b in bodies]
    assert bodies[0].boolean_curve(bodies[1]) > 0       # the A-B curve, on A
    assert bodies[1].boolean_curve(bodies[2]) > 0       # the B-C curve, on B
    O.boolean_relax_many(bodies, [(0, 1, O.UNION), (1, 2, O.UNION)], 6)
    for i, j in ((0, 1), (1, 2)):
        x, c, _ = bodies[i].get_particles()
        xc = x[n_before[i]:]
        assert len(xc) > 10 and np.all(c[n_before[i]:] == F)
        for k in (i, j):                               # on both surfaces of the pair
            assert _dist_to_mesh(xc.astype(np.float32), sp[k][0], sp[k][1]).max() < 1e-5
        other = 2 if i == 0 else 0                     # and outside the third sphere
        assert (np.linalg.norm(xc - CENTRES[other], axis=1) > sp[other][3]).all()
    # B's own surface particles still keep out of A and C
    xb, cb, _ = bodies[1].get_particles()
    s = surface_mask(cb[:n_before[1]])
    for j in (0, 2):
        assert (np.linalg.norm(xb[:n_before[1]][s] - CENTRES[j], axis=1) >= sp[j][2] - 1e-9).all()


def test_more_operations_than_a_body_takes_are_refused():
    sp = sphere(CENTRES[0])
    bodies = [generated(sp[0], sp[1]) for _ in range(6)]
    with pytest.raises(ValueError):
        O.boolean_relax_many(bodies, [(0, k, O.UNION) for k in range(1, 6)], 1)
    with pytest.raises(ValueError):
        O.boolean_relax_many(bodies[:2], [(0, 0, O.UNION)], 1)
