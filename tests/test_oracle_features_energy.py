"""Pins of the oracle's feature extraction (Sec. 3.2.2) and of the
uniformity energy with its analytic gradient (through the surface
projection), and a few end-to-end properties of Algorithm 1."""
import numpy as np
import pytest

import oracle as O
from paper_2501_03056_gb300 import workloads as W


def test_cube_features_at_30_degrees():
    v, t = W.cube_mesh()
    o = O.Oracle(v, t, 0.05, 0.065)
    assert o.extract_features(30.0) == 12
    fe = o.feature_edges()
    d = np.abs(v[fe[:, 0]].astype(np.float64) - v[fe[:, 1]])
    # the 12 cube edges: axis aligned, unit length
    assert np.all(np.sort(d, axis=1) == np.array([0.0, 0.0, 1.0]))
    assert len({tuple(e) for e in fe.tolist()}) == 12 and np.all(fe[:, 0] < fe[:, 1])
    sing = o.singular_points()
    assert np.array_equal(sing, np.arange(8))       # every corner has degree 3
    first, nseg, closed, segv = o.feature_lines()
    assert len(first) == 12 and np.all(nseg == 1) and not closed.any()
    # above 90 degrees nothing is a feature
    assert o.extract_features(100.0) == 0


@pytest.mark.parametrize("mesh", ["ico3", "torus"])
def test_smooth_meshes_have_no_features(mesh):
    v, t = W.icosphere_mesh(3) if mesh == "ico3" else W.torus_mesh(1.0, 0.3, 64, 32)
    o = O.Oracle(v, t, 0.05, 0.065)
    assert o.extract_features(30.0) == 0
    assert len(o.singular_points()) == 0


def test_boundary_edges_form_a_loop():
    v = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0]], np.float32)
    t = np.array([[0, 1, 2]], np.int32)
    o = O.Oracle(v, t, 0.1, 0.13)
    assert o.extract_features(30.0) == 3          # single face edges are features
    assert len(o.singular_points()) == 0          # each corner has degree 2
    first, nseg, closed, segv = o.feature_lines()
    assert len(first) == 1 and nseg[0] == 3 and closed[0] == 1
    xyz, cls = o.feature_particles(0.1)
    L = 2.0 + np.sqrt(2.0)
    assert len(xyz) == int(np.ceil(L / 0.1)) and np.all(cls == W.CLS_F)


def test_cylinder_rims_are_loops():
    v, t = W.cylinder_mesh(0.5, 1.0, 64, 4)
    o = O.Oracle(v, t, 0.05, 0.065)
    assert o.extract_features(30.0) == 128
    first, nseg, closed, segv = o.feature_lines()
    assert len(first) == 2 and np.all(closed == 1) and np.all(nseg == 64)


def test_feature_particle_spacing_is_length_over_ceil():
    v, t = W.cube_mesh()
    o = O.Oracle(v, t, 0.05, 0.065)
    o.extract_features(30.0)
    for dx in (0.05, 0.07, 0.3):
        xyz, cls = o.feature_particles(dx)
        n = int(np.ceil(1.0 / dx))
        assert (cls == W.CLS_P).sum() == 8
        assert (cls == W.CLS_F).sum() == 12 * (n - 1)
        # points along the edge through (-0.5, -0.5, z): spacing 1 / n exactly
        on = (np.abs(xyz[:, 0] + 0.5) < 1e-12) & (np.abs(xyz[:, 1] + 0.5) < 1e-12)
        z = np.sort(xyz[on, 2])
        np.testing.assert_allclose(np.diff(z), 1.0 / n, rtol=1e-12)
    # the cube workload's hand-placed edge points are exactly these
    xyz, cls = o.feature_particles(0.05)
    a = W.cube_workload()[0]
    ref = a.xyz[(a.cls == W.CLS_F) | (a.cls == W.CLS_P)]
    assert len(ref) == len(xyz)


def _small_state(seed=0):
    """Cube crop: particles after a few iterations, so surface particles
    carry a triangle."""
    a = W.cube_workload(seed=seed)[0]
    o = O.from_assembly(a)
    o.relax(3)
    return a, o


def test_energy_gradient_matches_central_differences():
    a, o = _small_state()
    x, cls, cons = o.get_particles()
    E, g = o.energy(grad=True)
    rng = np.random.default_rng(1)
    idx = rng.choice(np.where(np.isin(cls, [0, 1, 2]))[0], 25, replace=False)
    eps = 1e-6 * a.dx
    for i in idx:
        for k in range(3):
            xp = x.copy()
            xp[i, k] += eps
            o.set_state(xp)
            ep = o.energy()
            xp[i, k] -= 2 * eps
            o.set_state(xp)
            em = o.energy()
            fd = (ep - em) / (2 * eps)
            assert g[i, k] == pytest.approx(fd, rel=1e-6, abs=1e-7 * np.abs(g).max())
    o.set_state(x)


def test_projected_energy_gradients_match_central_differences():
    a, o = _small_state(1)
    x, cls, cons = o.get_particles()
    assert (cons[cls == W.CLS_S] >= 0).all()
    rng = np.random.default_rng(3)
    y = x.copy()
    s = cls == W.CLS_S
    y[s] += rng.normal(size=(s.sum(), 3)) * 0.01 * a.dx     # off the surface
    E, gy, gV = o.energy_projected(y)
    assert E == pytest.approx(o.energy_projected(y, grad=False), rel=1e-15)
    eps = 1e-6 * a.dx
    for i in rng.choice(np.where(s)[0], 12, replace=False):
        for k in range(3):
            yp = y.copy(); yp[i, k] += eps
            ym = y.copy(); ym[i, k] -= eps
            fd = (o.energy_projected(yp, grad=False) - o.energy_projected(ym, grad=False)) / (2 * eps)
            assert gy[i, k] == pytest.approx(fd, rel=1e-6, abs=1e-7 * np.abs(gy).max())
    V0 = a.verts.astype(np.float64)
    for vi in range(8):
        for k in range(3):
            vp = V0.copy(); vp[vi, k] += eps
            vm = V0.copy(); vm[vi, k] -= eps
            fd = (o.energy_projected(y, vp, grad=False) - o.energy_projected(y, vm, grad=False)) / (2 * eps)
            assert gV[vi, k] == pytest.approx(fd, rel=1e-6, abs=1e-7 * np.abs(gV).max())


def test_w0_are_the_lattice_sums():
    v, t = W.cube_mesh()
    o = O.Oracle(v, t, 0.05, 0.065)
    w0 = o.w0()
    h, dx = float(np.float32(0.065)), float(np.float32(0.05))
    assert w0[W.CLS_V] == pytest.approx(O.lattice_sum(dx, h, 3), rel=1e-14)
    assert w0[W.CLS_S] == pytest.approx(O.lattice_sum(dx, h, 2), rel=1e-14)
    assert w0[W.CLS_F] == pytest.approx(O.lattice_sum(dx, h, 1), rel=1e-14)


def test_cube_relaxation_keeps_constraints_and_improves_uniformity():
    a = W.cube_workload()[0]
    o = O.from_assembly(a)
    s0 = o.stats()
    o.relax(100)
    s1 = o.stats()
    x, cls, cons = o.get_particles()
    # surface particles sit on a face, feature particles on an edge
    S = x[cls == W.CLS_S]
    assert np.all(np.max(np.abs(S), axis=1) == 0.5)
    F = x[cls == W.CLS_F]
    assert np.all(np.sort(np.abs(F), axis=1)[:, 1:] == 0.5)
    P = x[cls == W.CLS_P]
    np.testing.assert_array_equal(P, a.xyz[a.cls == W.CLS_P])
    V = x[cls == W.CLS_V]
    assert np.all(np.abs(V) <= 0.5)
    assert s1["std_S"] < 0.5 * s0["std_S"] and s1["std_V"] < 0.5 * s0["std_V"]


def test_energy_descent_lowers_the_energy():
    a = W.cube_workload()[0]
    o = O.from_assembly(a)
    o.relax(2)
    e0 = o.energy()
    o.relax_energy(20)
    assert o.energy() < e0
