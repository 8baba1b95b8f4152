"""Pins of the Morton order of the grid rows (Eq. 9 over y and z, x the
fastest axis inside a row) on the oracle: the rows of a 4 x 4 corner of the
grid come in the textbook Z order, every key still names its cell's x and
slab, the row ranks are a permutation, and the relaxation does not depend
on the order (each particle sums its stencil cells in the same order)."""
import numpy as np
import pytest

import oracle as O
from paper_2501_03056_gb300 import workloads as W

# the Z order of the rows (y, z) of a 4 x 4 block, from Eq. 9 with z's bit
# above y's at every level: code = y0 + 2 z0 + 4 y1 + 8 z1
Z_ORDER_4X4 = [(0, 0), (1, 0), (0, 1), (1, 1), (2, 0), (3, 0), (2, 1), (3, 1),
               (0, 2), (1, 2), (0, 3), (1, 3), (2, 2), (3, 2), (2, 3), (3, 3)]


def cube_oracle():
    v, t = W.cube_mesh(0.5)
    dx = 0.05
    return O.Oracle(v, t, dx, float(np.float32(1.3 * dx)))


def test_rows_of_a_corner_come_in_z_order():
    o = cube_oracle()
    org, inv, cell, n, _ = o.nbr_grid()
    assert n[1] >= 4 and n[2] >= 4
    # one particle at the centre of cell (1, y, z) for the 16 rows, given in
    # reverse so that id order says nothing
    rows = [(y, z) for z in range(4) for y in range(4)][::-1]
    xyz = np.array([[org[0] + 1.5 * cell, org[1] + (y + 0.5) * cell, org[2] + (z + 0.5) * cell] for y, z in rows],
                   np.float32)
    o.set_particles(xyz, np.full(len(rows), W.CLS_V, np.int32))
    o.set_cell_order(1)
    key, perm = o.keys()
    assert [rows[i] for i in perm] == Z_ORDER_4X4
    # row-major: z outer, y inner
    o.set_cell_order(0)
    key, perm = o.keys()
    assert [rows[i] for i in perm] == [(y, z) for z in range(4) for y in range(4)]


def test_keys_keep_the_cell_x_and_slab_and_ranks_are_a_permutation():
    o = cube_oracle()
    rng = np.random.default_rng(4)
    org, inv, cell, n, _ = o.nbr_grid()
    xyz = rng.uniform(-0.5, 0.5, (20000, 3)).astype(np.float32)
    o.set_particles(xyz, np.full(len(xyz), W.CLS_V, np.int32))
    k0, _ = o.keys()
    o.set_cell_order(1)
    k1, p1 = o.keys()
    nx = int(n[0])
    # x cell and slab are the low part of both keys
    assert np.array_equal(k0 % (8 * nx), k1 % (8 * nx))
    # the row part maps rows one to one
    r0, r1 = k0 // (8 * nx), k1 // (8 * nx)
    pairs = {}
    for a, b in zip(r0.tolist(), r1.tolist()):
        assert pairs.setdefault(a, b) == b
    assert len(set(pairs.values())) == len(pairs)
    assert max(pairs.values()) < int(n[1]) * int(n[2])
    # the permutation sorts by (key, id)
    assert np.all(np.diff(k1[p1].astype(np.int64)) >= 0)


def test_relaxation_does_not_depend_on_the_row_order():
    a = W.cube_workload()[0]
    o0, o1 = O.from_assembly(a), O.from_assembly(a)
    o1.set_cell_order(1)
    o0.relax(5)
    o1.relax(5)
    assert np.array_equal(o0.get_particles()[0], o1.get_particles()[0])


def test_unknown_order_is_refused():
    o = cube_oracle()
    with pytest.raises(ValueError):
        o.set_cell_order(2)
