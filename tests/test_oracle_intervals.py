"""Oracle pins for the C_compact interval form of cell sets (Sec. 3.1.3:
C_compact begin / length over Morton codes of Eq. 9) and its Boolean
algebra (Sec. 3.2.3, Fig. 10: union, difference and intersection of two
bodies' grid sets as intervals).  Pinned on closed forms of aligned Morton
blocks, on brute-force set algebra over explicit code sets, on set
identities, and on a body's own generated volume particles."""
import numpy as np
import pytest

import oracle
from paper_2501_03056_gb300 import workloads as W

UNION, DIFFERENCE, INTERSECTION = 0, 1, 2


def runs_brute(codes):
    """Maximal runs of a set of integers, by walking the sorted set."""
    out = []
    for c in sorted(set(int(x) for x in codes)):
        if out and out[-1][0] + out[-1][1] == c:
            out[-1][1] += 1
        else:
            out.append([c, 1])
    return [tuple(r) for r in out]


def as_pairs(runs):
    return list(zip((int(x) for x in runs[0]), (int(x) for x in runs[1])))


def expand(runs):
    return {c for b, n in as_pairs(runs) for c in range(b, b + n)}


def centres(cells, o, d):
    return (o + (cells.astype(np.float64) + 0.5) * d).astype(np.float32)


def test_aligned_morton_block_is_one_run():
    # an aligned 2^k cube of cells fills the low 3k bits of Eq. 9's code:
    # one run of 8^k codes starting at the code of its low corner
    for k in range(4):
        s = 1 << k
        for corner in [(0, 0, 0), (s, 0, 0), (0, 2 * s, s), (3 * s, s, 5 * s)]:
            ijk = np.stack(np.meshgrid(*[np.arange(c, c + s) for c in corner], indexing="ij"), -1).reshape(-1, 3)
            b, n = oracle.lattice_intervals(ijk + 0.5, [0, 0, 0], 1.0)
            assert as_pairs((b, n)) == [(oracle.morton3(*corner), 8 ** k)]


def test_square_in_a_plane_is_runs_of_four():
    # a 4 x 4 square at z = 0: code = x0 + 2 y0 + 8 x1 + 16 y1, so four runs
    # of the four (x0, y0) at begins 0, 8, 16, 24
    ij = np.stack(np.meshgrid(np.arange(4), np.arange(4), indexing="ij"), -1).reshape(-1, 2)
    pts = np.c_[ij, np.zeros(len(ij))] + 0.5
    b, n = oracle.lattice_intervals(pts, [0, 0, 0], 1.0)
    assert as_pairs((b, n)) == [(0, 4), (8, 4), (16, 4), (24, 4)]


@pytest.mark.parametrize("seed", range(5))
def test_lattice_intervals_against_brute_force(seed):
    rng = np.random.default_rng(seed)
    d = 0.37
    o = rng.uniform(-3, 3, 3).astype(np.float32)
    cells = rng.integers(0, 12, (400, 3))
    cells = np.r_[cells, cells[:50]]                          # repeated cells
    # anywhere inside the cell, away from its faces
    pts = (o + (cells + rng.uniform(0.05, 0.95, cells.shape)) * d).astype(np.float32)
    b, n = oracle.lattice_intervals(pts, o, d)
    want = runs_brute(oracle.morton3(*map(int, c)) for c in cells)
    assert as_pairs((b, n)) == want


def random_runs(rng, n, span, canonical):
    if canonical:
        cells = rng.choice(span, size=n, replace=False)
        r = runs_brute(cells)
        return np.array([x[0] for x in r], np.uint64), np.array([x[1] for x in r], np.uint64)
    # any order, overlapping, touching and empty runs
    b = rng.integers(0, span, n)
    ln = rng.integers(0, 9, n)
    return b.astype(np.uint64), ln.astype(np.uint64)


@pytest.mark.parametrize("seed", range(8))
@pytest.mark.parametrize("canonical", [True, False])
def test_interval_boolean_against_set_algebra(seed, canonical):
    rng = np.random.default_rng(100 + seed)
    A = random_runs(rng, 60, 300, canonical)
    B = random_runs(rng, 60, 300, canonical)
    sa, sb = expand(A), expand(B)
    for op, want in ((UNION, sa | sb), (DIFFERENCE, sa - sb), (INTERSECTION, sa & sb)):
        got = oracle.interval_boolean(A, B, op)
        assert as_pairs(got) == runs_brute(want)       # the same set, as maximal runs


def test_interval_boolean_identities():
    rng = np.random.default_rng(7)
    A = random_runs(rng, 80, 500, False)
    B = random_runs(rng, 80, 500, False)
    empty = (np.zeros(0, np.uint64), np.zeros(0, np.uint64))
    canon = runs_brute(expand(A))
    assert as_pairs(oracle.interval_boolean(A, empty, UNION)) == canon
    assert as_pairs(oracle.interval_boolean(empty, A, UNION)) == canon
    assert as_pairs(oracle.interval_boolean(A, A, INTERSECTION)) == canon
    assert as_pairs(oracle.interval_boolean(A, A, DIFFERENCE)) == []
    assert as_pairs(oracle.interval_boolean(A, empty, INTERSECTION)) == []
    # (A - B) u (A n B) = A and |A u B| = |A| + |B| - |A n B|
    d = oracle.interval_boolean(A, B, DIFFERENCE)
    i = oracle.interval_boolean(A, B, INTERSECTION)
    assert as_pairs(oracle.interval_boolean(d, i, UNION)) == canon
    u = oracle.interval_boolean(A, B, UNION)
    assert len(expand(u)) == len(expand(A)) + len(expand(B)) - len(expand(i))


def test_quadrilateral_and_circle():
    # the two shapes of Fig. 10 in the z = 0 plane of a 16 x 16 grid: a
    # quadrilateral of cells and a disc of cells overlapping it
    ij = np.stack(np.meshgrid(np.arange(16), np.arange(16), indexing="ij"), -1).reshape(-1, 2)
    quad = ij[(ij[:, 0] >= 2) & (ij[:, 0] < 10) & (ij[:, 1] >= 3) & (ij[:, 1] < 9)]
    disc = ij[((ij[:, 0] + 0.5 - 10) ** 2 + (ij[:, 1] + 0.5 - 8) ** 2) < 4.5 ** 2]
    to3 = lambda c: np.c_[c, np.zeros(len(c))] + 0.5
    A = oracle.lattice_intervals(to3(quad), [0, 0, 0], 1.0)
    B = oracle.lattice_intervals(to3(disc), [0, 0, 0], 1.0)
    code = lambda cells: {oracle.morton3(int(x), int(y), 0) for x, y in cells}
    qa, qb = code(quad), code(disc)
    for op, want in ((UNION, qa | qb), (DIFFERENCE, qa - qb), (INTERSECTION, qa & qb)):
        r = oracle.interval_boolean(A, B, op)
        assert expand(r) == want
        x = oracle.interval_cells(r, [0, 0, 0], 1.0)
        assert len(x) == len(want) and (x[:, 2] == 0.5).all()


def test_interval_cells_round_trip():
    rng = np.random.default_rng(11)
    o = np.array([-1.25, 0.5, 3.0], np.float32)
    d = np.float32(0.05)
    cells = np.unique(rng.integers(0, 40, (3000, 3)), axis=0)
    x = centres(cells, o, d)
    runs = oracle.lattice_intervals(x, o, d)
    back = oracle.interval_cells(runs, o, d)
    order = np.argsort([oracle.morton3(*map(int, c)) for c in cells])
    # codes ascending, each cell once, at its centre in FP64 rounded once
    assert np.array_equal(back, x[order])


def test_interval_errors():
    with pytest.raises(ValueError):
        oracle.lattice_intervals(np.array([[-1.0, 0.5, 0.5]], np.float32), [0, 0, 0], 1.0)
    with pytest.raises(ValueError):
        oracle.lattice_intervals(np.array([[2.0 ** 22, 0.5, 0.5]], np.float32), [0, 0, 0], 1.0)
    one = (np.array([3], np.uint64), np.array([2], np.uint64))
    with pytest.raises(ValueError):
        oracle.interval_boolean(one, one, 3)
    past = (np.array([2 ** 63 - 1], np.uint64), np.array([2], np.uint64))
    with pytest.raises(ValueError):
        oracle.interval_boolean(one, past, UNION)
    with pytest.raises(ValueError):
        oracle.interval_cells(past, [0, 0, 0], 1.0)


def test_volume_grid_set_of_a_body_reproduces_its_volume_particles():
    # the interior grids of a generated body (Sec. 3.2: one volume particle
    # at the centre of every interior cell) as C_compact, and back: the same
    # particles, bit for bit
    a = W.cube_workload()[0]
    o = oracle.Oracle(a.verts, a.tris, a.dx, a.h)
    o.extract_features(30.0)
    x, c, _ = o.map_particles()
    tg_o, _, _ = o.tri_grid()
    vol = x[c == 1].astype(np.float32)
    assert len(vol) > 1000
    runs = oracle.lattice_intervals(vol, tg_o, a.dx)
    back = oracle.interval_cells(runs, tg_o, a.dx)
    key = lambda p: sorted(map(tuple, p.tolist()))
    assert len(back) == len(vol) and key(back) == key(vol)


def _sphere_and_box(dx):
    """An icosphere and a box with the same lower bounding-box corner, so
    that their generation lattices (triangle-grid origin and dx) coincide."""
    v1, t1 = W.icosphere_mesh(3, 0.5)
    lo = v1.min(axis=0)
    v2, t2 = W.cube_mesh(0.5)
    v2 = ((v2 + np.float32(0.5)) * np.float32(0.6) + lo).astype(np.float32)
    h = W.smoothing_length(dx)
    gen = {"generate": {"band_cells": 0, "inner_cells": 0}}
    return [W.Assembly("sphere", v1, t1, dx, h, None, None, 30.0, dict(gen)),
            W.Assembly("box", v2, t2, dx, h, None, None, 30.0, dict(gen))]


def test_interval_algebra_and_the_particle_rule_differ_only_on_the_other_surface():
    # two readings of the Boolean operation on the volume particles of two
    # bodies that share a lattice: the interval algebra of their interior
    # grid sets (Fig. 10) and the particle rule of the relaxed operation
    # (each particle tested against the other mesh by ray parity).  Cells
    # without the cutter's triangles are inside it exactly when they are in
    # its interior set, so the two agree everywhere off the cells that hold
    # the second body's triangles.
    dx = float(np.float32(0.04))
    a, b = _sphere_and_box(dx)
    oa, ob = oracle.from_assembly(a), oracle.from_assembly(b)
    (o1, _, _), (o2, _, nb) = oa.tri_grid(), ob.tri_grid()
    assert np.array_equal(o1, o2)

    def cells(x):
        return {tuple(t) for t in np.floor((x.astype(np.float32) - o1) / np.float32(dx)).astype(np.int64).tolist()}

    xa, ca, _ = oa.get_particles()
    xb, cb, _ = ob.get_particles()
    va, vb = ca == 1, cb == 1                         # volume particles
    ra = oracle.lattice_intervals(xa[va].astype(np.float32), o1, dx)
    rb = oracle.lattice_intervals(xb[vb].astype(np.float32), o1, dx)
    keys, _ = ob.tri_bins()                           # cells that hold the box's triangles
    k = keys.astype(np.int64)
    surf_b = set(zip((k % nb[0]).tolist(), ((k // nb[0]) % nb[1]).tolist(), (k // (nb[0] * nb[1])).tolist()))
    assert cells(xa[va]) & surf_b                     # the box's surface crosses the sphere's interior
    for op in (UNION, DIFFERENCE, INTERSECTION):
        ka = oa.boolean_keep(ob, op, True)
        kb = ob.boolean_keep(oa, op, False)
        by_particles = cells(xa[va & ka]) | cells(xb[vb & kb])
        by_intervals = cells(oracle.interval_cells(oracle.interval_boolean(ra, rb, op), o1, dx))
        assert by_particles - surf_b == by_intervals - surf_b, op
