"""Pins of the oracle's neighbour grid, force and step (Sec. 3.1.3, Eqs. 15,
22-25, Algorithm 1).

Brute force O(N^2) neighbour sets, the two-particle closed form, pair
antisymmetry, lattice symmetry and the exact h/16 limited step."""
import numpy as np
import pytest

import oracle as O
from paper_2501_03056_gb300 import workloads as W


def big_box(half=2.0):
    v, t = W.cube_mesh(half)
    return v, t


def cloud(n, seed, lo=-0.3, hi=0.3):
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, size=(n, 3)).astype(np.float32)


def test_keys_follow_the_row_major_cell_rule():
    v, t = big_box(1.0)
    o = O.Oracle(v, t, 0.05, 0.065)
    org, inv, cell, n, r2 = o.nbr_grid()
    assert cell >= 2 * 0.065 and cell == pytest.approx(2 * np.float32(0.065) * (1 + 1 / 256), rel=1e-6)
    assert r2 == np.float32((2 * np.float32(0.065)) ** 2)
    # particles at 0.55 of their cell along each axis: x-slab floor(8 * 0.55) = 4
    idx = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1], [3, 7, 2], [n[0] - 1, n[1] - 1, n[2] - 1]])
    xyz = (org[None, :].astype(np.float64) + (idx + 0.55) * cell).astype(np.float32)
    o.set_particles(xyz, np.full(len(idx), W.CLS_V, np.int32))
    key, perm = o.keys()
    expect = 8 * (idx[:, 0] + n[0] * (idx[:, 1] + n[1] * idx[:, 2])) + 4
    assert np.array_equal(key, expect.astype(np.uint32))
    assert np.array_equal(perm, np.argsort(expect, kind="stable").astype(np.uint32))


def test_keys_order_a_cell_by_x_slab():
    # inside one cell the key's low 3 bits are floor(8 * fractional x); y and
    # z fractions do not enter; fractions kept away from slab boundaries
    v, t = big_box(1.0)
    o = O.Oracle(v, t, 0.05, 0.065)
    org, inv, cell, n, r2 = o.nbr_grid()
    frac = np.array([0.99, 0.01, 0.51, 0.13, 0.9, 0.3, 0.49, 0.6])
    base = np.array([5, 3, 4])
    xyz = org[None, :].astype(np.float64) + (base[None, :] + 0.5) * cell + np.zeros((len(frac), 3))
    xyz[:, 0] = org[0] + (base[0] + frac) * cell
    xyz[:, 1] += (frac - 0.5) * 0.8 * cell                 # moves inside the cell along y
    o.set_particles(xyz.astype(np.float32), np.full(len(frac), W.CLS_V, np.int32))
    key, perm = o.keys()
    c = base[0] + n[0] * (base[1] + n[1] * base[2])
    assert np.array_equal(key, (8 * c + np.floor(8 * frac)).astype(np.uint32))
    # stable: equal slabs (0.9 and 0.99) keep id order
    assert np.array_equal(perm, np.argsort(np.floor(8 * frac), kind="stable").astype(np.uint32))
    cells, s, e = o.cell_ranges()
    assert list(cells) == [c] and s[0] == 0 and e[0] == len(frac)


def test_points_outside_the_grid_are_clamped():
    v, t = big_box(1.0)
    o = O.Oracle(v, t, 0.05, 0.065)
    org, inv, cell, n, r2 = o.nbr_grid()
    xyz = np.array([[-50, -50, -50], [50, 50, 50]], np.float32)
    o.set_particles(xyz, np.full(2, W.CLS_V, np.int32))
    key, _ = o.keys()
    assert key[0] == 0 and key[1] == 8 * n[0] * n[1] * n[2] - 1


def test_stable_permutation_and_cell_ranges():
    a = W.cube_workload()[0]
    o = O.from_assembly(a)
    key, perm = o.keys()
    assert np.array_equal(perm, np.argsort(key, kind="stable").astype(np.uint32))
    cells, s, e = o.cell_ranges()
    ks = key[perm]
    assert np.all(np.diff(cells.astype(np.int64)) > 0)
    assert s[0] == 0 and e[-1] == a.n and np.array_equal(s[1:], e[:-1])
    for c, b, f in zip(cells[::37], s[::37], e[::37]):
        assert np.all(ks[b:f] // 8 == c)


@pytest.mark.parametrize("seed", [0, 1])
def test_cell_scan_equals_brute_force_neighbours(seed):
    a = W.cube_workload(seed=seed)[0]
    o = O.from_assembly(a)
    _, cnt, _ = o.forces()
    assert np.array_equal(cnt, o.brute_neighbours())
    # a random cloud of every class
    v, t = big_box(1.0)
    o2 = O.Oracle(v, t, 0.02, 0.026)
    xyz = cloud(1500, seed, -0.12, 0.12)
    cls = np.random.default_rng(seed).integers(0, 5, 1500).astype(np.int32)
    o2.set_particles(xyz, cls)
    _, cnt2, _ = o2.forces()
    assert np.array_equal(cnt2, o2.brute_neighbours())
    assert cnt2.max() > 20


def test_two_particles_closed_form():
    v, t = big_box()
    h = float(np.float32(0.1))
    o = O.Oracle(v, t, 0.077, h)
    for r in (0.03, 0.05, 0.1, 0.15, 0.19):
        xyz = np.array([[0, 0, 0], [r, 0, 0]], np.float32)
        o.set_particles(xyz, np.full(2, W.CLS_V, np.int32))
        acc, cnt, amax = o.forces()
        rr = float(np.float32(r))
        # a_0 = -dW/dr e_01 with e_01 pointing from 1 to 0: repulsion along -x
        assert acc[0, 0] == pytest.approx(O.dW(rr, h), rel=1e-12)
        assert acc[1, 0] == pytest.approx(-O.dW(rr, h), rel=1e-12)
        assert np.all(acc[:, 1:] == 0) and np.all(cnt == 1)
        assert amax == pytest.approx(abs(O.dW(rr, h)), rel=1e-12)


def test_pair_forces_sum_to_zero():
    v, t = big_box()
    o = O.Oracle(v, t, 0.02, 0.026)
    o.set_particles(cloud(3000, 7, -0.15, 0.15), np.full(3000, W.CLS_V, np.int32))
    acc, cnt, _ = o.forces()
    tot = np.abs(acc).sum()
    assert tot > 0 and cnt.mean() > 30
    assert np.all(np.abs(acc.sum(axis=0)) < 1e-12 * tot)


def test_interior_of_a_perfect_lattice_feels_no_force():
    v, t = big_box()
    dx = 0.02
    k = np.arange(-6, 7) * dx
    g = np.stack(np.meshgrid(k, k, k, indexing="ij"), -1).reshape(-1, 3)
    o = O.Oracle(v, t, dx, 1.3 * dx)
    o.set_particles(g.astype(np.float32), np.full(len(g), W.CLS_V, np.int32))
    acc, _, _ = o.forces()
    centre = np.argmin(np.linalg.norm(g, axis=1))
    scale = abs(O.dW(0.5 * 1.3 * dx, 1.3 * dx))
    assert np.linalg.norm(acc[centre]) < 1e-10 * scale
    # density of that particle equals the cubic lattice sum W0
    rho = o.density()
    # (the lattice is stored in FP32, so agreement is to FP32 rounding)
    assert rho[centre] == pytest.approx(O.lattice_sum(dx, np.float32(1.3 * dx), 3), rel=1e-6)


def test_class_mask():
    v, t = big_box()
    h = 0.1
    o = O.Oracle(v, t, 0.077, h)
    # surface particle surrounded only by volume and innermost particles
    xyz = np.array([[0, 0, 0], [0.05, 0, 0], [0, 0.05, 0], [0, 0, 0.07]], np.float32)
    cls = np.array([W.CLS_S, W.CLS_V, W.CLS_I, W.CLS_V], np.int32)
    o.set_particles(xyz, cls)
    acc, cnt, _ = o.forces()
    assert cnt[0] == 0 and np.all(acc[0] == 0)
    assert cnt[1] == 3 and cnt[3] == 3   # volume feels everything
    assert cnt[2] == 0 and np.all(acc[2] == 0)   # innermost is fixed


def test_limited_step_moves_the_fastest_particle_by_h_over_16():
    # volume particles deep inside a large box: no triangle within reach,
    # so the trial point is accepted and the move is a dt^2 with
    # dt = 0.25 sqrt(h / amax): exactly (h / 16) a / amax.
    v, t = big_box(2.0)
    dx = 0.02
    h = float(np.float32(1.3 * dx))
    o = O.Oracle(v, t, dx, h)
    xyz = cloud(2000, 3, -0.2, 0.2)
    o.set_particles(xyz, np.full(2000, W.CLS_V, np.int32))
    acc, _, amax = o.forces()
    o.relax(1)
    x1, _, _ = o.get_particles()
    disp = x1 - xyz.astype(np.float64)
    np.testing.assert_allclose(disp, (h / 16.0) * acc / amax, rtol=1e-12, atol=1e-15)
    assert np.max(np.linalg.norm(disp, axis=1)) == pytest.approx(h / 16.0, rel=1e-12)


def test_deterministic_across_thread_counts():
    a = W.cube_workload()[0]
    res = []
    for th in (1, 3):
        O.set_threads(th)
        o = O.from_assembly(a)
        o.relax(5)
        res.append(o.get_particles())
    O.set_threads(0)
    assert np.array_equal(res[0][0], res[1][0]) and np.array_equal(res[0][2], res[1][2])
