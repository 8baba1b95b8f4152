"""Pins of the paper-literal options of the oracle: the surface-then-volume
schedule (Algorithm 1 for surface particles, then the intermediate volume
particles, Sec. 3.3.4) through the mobile-class mask, and the re-projection
cascade of Sec. 3.3.3 (own triangle, own cell, 27 cells) against the
canonical closest projectable triangle, on meshes built so that the two
rules choose differently."""
import numpy as np

import oracle as O
from paper_2501_03056_gb300 import workloads as W


def test_surface_then_volume_schedule():
    a = W.cube_workload()[0]
    o = O.from_assembly(a)
    x0, c, _ = o.get_particles()
    surf, vol = np.isin(c, [W.CLS_S, W.CLS_F]), c == W.CLS_V
    o.set_mobile_classes([W.CLS_S, W.CLS_F])
    o.relax(3)
    x1 = o.get_particles()[0]
    assert np.array_equal(x1[vol], x0[vol]) and (np.abs(x1[surf] - x0[surf]).max(axis=1) > 0).mean() > 0.9
    o.set_mobile_classes([W.CLS_V])
    o.relax(3)
    x2 = o.get_particles()[0]
    assert np.array_equal(x2[surf], x1[surf]) and (np.abs(x2[vol] - x1[vol]).max(axis=1) > 0).mean() > 0.9
    # the default mask moves every class, as before
    o2, o3 = O.from_assembly(a), O.from_assembly(a)
    o2.set_mobile_classes([W.CLS_S, W.CLS_V, W.CLS_F])
    o2.relax(2)
    o3.relax(2)
    assert np.array_equal(o2.get_particles()[0], o3.get_particles()[0])


def _two_sheets(z_top, top_box):
    """A large triangle in z = 0 and a small one in z = z_top over top_box
    (x0, x1, y0, y1); both facing +z."""
    v = np.array([[-1, -1, 0], [3, -1, 0], [-1, 3, 0],
                  [top_box[0], top_box[2], z_top], [top_box[1], top_box[2], z_top], [top_box[0], top_box[3], z_top]],
                 np.float32)
    t = np.array([[0, 1, 2], [3, 4, 5]], np.int32)
    return v, t


def test_cascade_keeps_a_particle_on_its_triangle():
    # the small sheet hovers 0.002 above the big one: a point 0.0015 up is
    # closer to the small sheet, but its foot is still on the big one
    v, t = _two_sheets(0.002, (0.0, 0.2, 0.0, 0.2))
    o = O.Oracle(v, t, 0.05, 0.065)
    y = np.array([[0.03, 0.03, 0.0015]], np.float32)
    s = np.array([W.CLS_S], np.int32)
    _, co, ok = o.project_points(y, s, np.array([0], np.int32))
    assert ok[0] and co[0] == 1                      # canonical: the closer small sheet
    o.set_cascade(True)
    _, co, ok = o.project_points(y, s, np.array([0], np.int32))
    assert ok[0] and co[0] == 0                      # cascade: still on its triangle
    _, co, ok = o.project_points(y, s, np.array([-1], np.int32))
    assert ok[0] and co[0] == 1                      # no triangle yet: own cell, closest


def test_cascade_prefers_the_own_cell():
    # a point near the top of its triangle cell: the big sheet lies in the
    # cell (z = 0.05 below it), a small sheet just above the cell is closer
    dx = 0.1
    v0, t0 = _two_sheets(0.3, (0.0, 0.2, 0.0, 0.2))
    probe = O.Oracle(v0, t0, dx, 0.13)
    o_, inv, n = probe.tri_grid()
    cz = int(np.floor((0.0 - o_[2]) * inv))                   # cell holding z = 0
    top = o_[2] + (cz + 1) / inv                              # its upper face
    y = np.array([[0.05, 0.05, top - 0.01 * dx]], np.float32)
    v, t = _two_sheets(float(top + 0.2 * dx), (0.0, 0.2, 0.0, 0.2))
    o = O.Oracle(v, t, dx, 0.13)
    assert np.array_equal(o.tri_grid()[0], o_)                # same origin: y is in the same cell
    s = np.array([W.CLS_S], np.int32)
    _, co, ok = o.project_points(y, s, np.array([-1], np.int32))
    assert ok[0] and co[0] == 1                      # canonical: the closer sheet in the cell above
    o.set_cascade(True)
    _, co, ok = o.project_points(y, s, np.array([-1], np.int32))
    assert ok[0] and co[0] == 0                      # cascade: the own cell's sheet first
