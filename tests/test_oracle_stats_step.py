"""Pins of the oracle's uniformity statistics, of the tangential step of
Eqs. 24-25 and of the inside test's edge tolerance (Fig. 8).

Each case is built so that the statistic or the step has a closed form that
does not come from the oracle: a single particle's kernel sum is W(0) =
alpha_3 (Eq. 17, normalised to a unit integral over the support 2h), three
particles give a known population
standard deviation, an exact FP32 lattice has one density and a smallest
pair of exactly dx, and on a folded surface the step of a surface particle
that crosses the fold lands where removing the normal part of the
displacement (and only that) puts it."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2501_03056_gb300 import workloads as W

S, V, F, I, P = W.CLS_S, W.CLS_V, W.CLS_F, W.CLS_I, W.CLS_P
DX = 0.0625                      # a power of two: lattice coordinates are exact in FP32
H = float(np.float32(1.3 * DX))


def box_oracle(half=1.0, dx=DX, h=H):
    v, t = W.cube_mesh(half)
    return O.Oracle(v, t, dx, h)


def stats_of(xyz, cls, **kw):
    o = box_oracle(**kw)
    o.set_particles(np.asarray(xyz, np.float32), np.asarray(cls, np.int32))
    return o.stats()


def alpha3(h):
    # Eq. 17 with the normalisation that makes the 3-D kernel integrate to
    # one over its support 2h (the printed 21 / (6 pi h^3) integrates to 8/3)
    return 21.0 / (16.0 * math.pi * h ** 3)


def test_single_particle_density_is_w_zero():
    st = stats_of([[0.1, 0.2, -0.3]], [V])
    assert st["mean_V"] == pytest.approx(alpha3(H), rel=1e-14)
    assert st["std_V"] == 0.0 and st["n_V"] == 1
    assert st["n_S"] == 0 and st["mean_S"] == 0.0
    assert math.isinf(st["min_pair_over_dx"])      # no neighbour at all


def test_standard_deviation_is_the_population_one():
    # densities {a, a + w, a + w}: an isolated particle and a pair at r < 2h.
    # mean = a + 2w / 3 and the population deviation is w sqrt(2) / 3, so
    # std = (mean - a) / sqrt(2) whatever W(r) is (a sample deviation would
    # give (mean - a) sqrt(3) / 2)
    r = 1.7 * DX
    xyz = [[-0.6, -0.6, -0.6], [0.2, 0.0, 0.0], [0.2 + r, 0.0, 0.0]]
    st = stats_of(xyz, [V, V, V])
    a = alpha3(H)
    assert st["n_V"] == 3
    assert st["std_V"] == pytest.approx((st["mean_V"] - a) / math.sqrt(2.0), rel=1e-12)
    assert st["mean_V"] > a
    # the pair is the smallest masked pair of a mobile particle
    r32 = float(np.float32(0.2 + r)) - float(np.float32(0.2))
    assert st["min_pair_over_dx"] == pytest.approx(r32 / DX, rel=1e-14)


def test_smallest_pair_is_masked_and_over_mobile_particles_only():
    xyz, cls = [], []

    def put(p, c):
        xyz.append(p)
        cls.append(c)

    # two surface particles exactly dx apart (the answer)
    put([0.0, 0.0, 0.0], S)
    put([DX, 0.0, 0.0], S)
    # an innermost particle 0.25 dx from the first: innermost particles do
    # not act on surface ones (S <- S, F, P), and they never move
    put([0.0, 0.25 * DX, 0.0], I)
    # two innermost particles 0.125 dx apart, far away: fixed, not counted
    put([0.5, 0.5, 0.5], I)
    put([0.5 + 0.125 * DX, 0.5, 0.5], I)
    # two singular points 0.0625 dx apart: fixed as well
    put([-0.5, 0.5, -0.5], P)
    put([-0.5, 0.5 + 0.0625 * DX, -0.5], P)
    # a volume particle 1.5 dx from a surface particle: volume particles feel
    # every class, so this pair counts through the volume particle
    put([-0.5, -0.5, 0.0], S)
    put([-0.5 + 1.5 * DX, -0.5, 0.0], V)
    st = stats_of(xyz, cls)
    assert st["min_pair_over_dx"] == 1.0
    # with the volume particle closer than dx to a fixed innermost one, that
    # pair becomes the smallest (V <- I)
    xyz.append([-0.5 + 1.5 * DX, -0.5 + 0.5 * DX, 0.0])
    cls.append(I)
    st = stats_of(xyz, cls)
    assert st["min_pair_over_dx"] == 0.5


def test_perfect_lattice_has_one_density_and_pairs_of_dx():
    # a 12^3 cubic lattice at spacing dx: the central 6^3 are volume
    # particles, the three outer layers innermost (fixed) ones, so every
    # volume particle sees the complete lattice within 2h = 2.6 dx
    k = np.arange(12) - 5.5
    g = np.stack(np.meshgrid(k, k, k, indexing="ij"), -1).reshape(-1, 3)
    xyz = (g * DX).astype(np.float32)
    inner = np.all(np.abs(g) < 3, axis=1)
    cls = np.where(inner, V, I).astype(np.int32)
    o = box_oracle()
    o.set_particles(xyz, cls)
    st = o.stats()
    assert st["n_V"] == 216
    assert st["std_V"] <= 1e-13 * st["mean_V"]
    assert st["min_pair_over_dx"] == 1.0
    # and that density is the cubic lattice sum at spacing dx (the W0 of
    # the volume class)
    assert st["mean_V"] == pytest.approx(O.lattice_sum(DX, H, 3), rel=1e-12)


def folded_sheet(phi_deg, dx):
    """Two flat pieces meeting along the y axis: z = 0 for x in [-1, 0], and
    a piece tilted down by phi for x >= 0 (unit slope length)."""
    phi = math.radians(phi_deg)
    c, s = math.cos(phi), math.sin(phi)
    v = np.array([[-1, -1, 0], [0, -1, 0], [0, 1, 0], [-1, 1, 0],
                  [c, -1, -s], [c, 1, -s]], np.float32)
    t = np.array([[0, 1, 2], [0, 2, 3], [1, 4, 5], [1, 5, 2]], np.int32)
    return v, t


@pytest.mark.parametrize("phi_deg", [20.0, 35.0])
def test_surface_step_removes_the_normal_part_of_the_displacement(phi_deg):
    # One surface particle on the flat piece just before the fold, pushed
    # forward and up by a singular point behind it.  It is the only mobile
    # particle, so its displacement is exactly h / 16 along its force (dt =
    # 0.25 sqrt(h / amax) with the velocity reset); Eqs. 24-25, read as acting
    # on the displacement, drop the part along the flat
    # piece's normal, so the trial point stays in the plane z = 0, crosses
    # the fold by delta, and its only projectable foot is on the tilted
    # piece, delta cos(phi) down the slope.  Keeping the normal part would
    # put the trial point above the plane and the foot elsewhere.
    dx, h = 0.05, float(np.float32(0.065))
    v, t = folded_sheet(phi_deg, dx)
    o = O.Oracle(v, t, dx, h)
    theta = math.radians(30.0)
    eps = 0.3 * h / 16
    s0 = np.array([-eps, 0.0, 0.0], np.float32)
    p0 = (s0.astype(np.float64) - 1.2 * dx * np.array([math.cos(theta), 0.0, math.sin(theta)])).astype(np.float32)
    o.set_particles(np.stack([s0, p0]), np.array([S, P], np.int32))
    o.set_state(None, np.array([0, -1], np.int32))        # the particle sits on triangle 0 (z = 0)
    o.relax(1)
    x, _, cons = o.get_particles()
    # closed form from the FP32 inputs
    a = s0.astype(np.float64) - p0.astype(np.float64)
    a /= np.linalg.norm(a)
    dr = (h / 16.0) * a
    dr[2] = 0.0                                           # flat piece normal is +z exactly
    y = s0.astype(np.float64) + dr
    delta = y[0]
    assert delta > 1e-4 * dx                              # it does cross the fold
    vv = v.astype(np.float64)
    n2 = np.cross(vv[4] - vv[1], vv[5] - vv[1])
    n2 /= np.linalg.norm(n2)
    expect = y - np.dot(y - vv[1], n2) * n2
    assert cons[0] in (2, 3)                              # now on the tilted piece
    np.testing.assert_allclose(x[0], expect, atol=1e-12 * dx)
    phi = math.radians(phi_deg)
    assert x[0][0] == pytest.approx(delta * math.cos(phi) ** 2, rel=1e-5)
    # the singular point has not moved
    np.testing.assert_array_equal(x[1], p0.astype(np.float64))


def test_feature_step_moves_along_its_segment_by_the_limited_step():
    # a feature particle on a cube edge, pushed by a singular point off the
    # edge: the only mobile particle moves h / 16 along its force, of which
    # only the part along the edge is kept
    dx, h = 0.05, float(np.float32(0.065))
    v, t = W.cube_mesh()
    o = O.Oracle(v, t, dx, h)
    o.extract_features(30.0)
    first, nseg, closed, segv = o.feature_lines()
    vv = v.astype(np.float64)
    # a segment along x (an edge of the cube)
    q = next(i for i, (a, b) in enumerate(segv) if abs(vv[b][0] - vv[a][0]) == 1.0)
    a_, b_ = vv[segv[q][0]], vv[segv[q][1]]
    tau = (b_ - a_) / np.linalg.norm(b_ - a_)
    f0 = (a_ + 0.37 * (b_ - a_)).astype(np.float32)
    push = np.array([0.8, 0.3, -0.52])
    push /= np.linalg.norm(push)
    p0 = (f0.astype(np.float64) - 1.1 * dx * push).astype(np.float32)
    o.set_particles(np.stack([f0, p0]), np.array([F, P], np.int32))
    o.set_state(None, np.array([q, -1], np.int32))
    o.relax(1)
    x, _, cons = o.get_particles()
    a = f0.astype(np.float64) - p0.astype(np.float64)
    a /= np.linalg.norm(a)
    expect = f0.astype(np.float64) + (h / 16.0) * np.dot(a, tau) * tau
    np.testing.assert_allclose(x[0], expect, atol=1e-12 * dx)
    assert cons[0] == q


def test_edge_tolerance_of_the_inside_test():
    # A unit square split along its diagonal (extent 1, so the tolerance is
    # 2^-20).  A foot exactly on the shared diagonal is inside both
    # triangles (zero counts as inside) and the lower index wins the tie; a
    # foot 2^-21 outside the square's edge x = 0 still projects; one 2^-19
    # outside does not (the particle would revert).
    v = np.array([[0, 0, 0], [1, 0, 0], [1, 1, 0], [0, 1, 0]], np.float32)
    t = np.array([[0, 1, 2], [0, 2, 3]], np.int32)
    o = O.Oracle(v, t, 0.05, 0.065)
    y = np.array([[0.375, 0.375, 0.01],                 # above the diagonal
                  [-2.0 ** -21, 0.5, 0.02],              # half the tolerance outside x = 0
                  [-2.0 ** -19, 0.5, 0.02],              # twice the tolerance outside
                  [0.25, 0.75, -0.03]], np.float32)      # plainly inside triangle 1
    x, tri, ok = o.project_points(y, np.full(len(y), S, np.int32))
    assert ok.tolist() == [True, True, False, True]
    assert tri[0] == 0 and tri[1] == 1 and tri[3] == 1
    np.testing.assert_array_equal(x[0], [0.375, 0.375, 0.0])
    np.testing.assert_array_equal(x[1], [-2.0 ** -21, 0.5, 0.0])
    # a brute-force check of both sides of the tie: the foot lies on both
    # triangles' planes at the same distance
    assert abs(float(y[0, 2])) == pytest.approx(0.01, rel=1e-6)
