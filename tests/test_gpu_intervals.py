"""C_compact interval form of grid sets on the GPU (fppg_lattice_intervals,
fppg_interval_boolean, fppg_interval_cells; Sec. 3.1.3, Sec. 3.2.3, Fig. 10)
against the oracle: the same runs and the same cell centres, bit for bit,
on random sets that span many tiles, on the edge cases, and on the volume
grid sets of two generated bodies that share a lattice."""
import ctypes as C

import numpy as np
import pytest

import oracle
import paper_2501_03056_gb300 as pkg
from paper_2501_03056_gb300 import workloads as W

pytestmark = pytest.mark.gpu
OPS = (pkg.UNION, pkg.DIFFERENCE, pkg.INTERSECTION)


@pytest.fixture(scope="module")
def torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2501_03056_gb300 import _build
    _build.build()
    return torch


def dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(a).astype(np.int64))).cuda()


def host(t):
    return t.cpu().numpy().astype(np.uint64)


def same_runs(got, want):
    assert len(got[0]) == len(want[0])
    assert np.array_equal(host(got[0]), want[0]) and np.array_equal(host(got[1]), want[1])


def random_runs(rng, n, span, canonical):
    if canonical:
        cells = np.sort(rng.choice(span, size=n, replace=False))
        r = oracle.interval_boolean((cells.astype(np.uint64), np.ones(n, np.uint64)),
                                    (np.zeros(0, np.uint64), np.zeros(0, np.uint64)), pkg.UNION)
        return r
    return rng.integers(0, span, n).astype(np.uint64), rng.integers(0, 12, n).astype(np.uint64)


@pytest.mark.parametrize("canonical", [True, False])
def test_interval_boolean_matches_oracle(torch, canonical):
    rng = np.random.default_rng(21 if canonical else 22)
    A = random_runs(rng, 30000, 200000, canonical)
    B = random_runs(rng, 25000, 200000, canonical)
    for op in OPS:
        got = pkg.interval_boolean((dev(torch, A[0]), dev(torch, A[1])), (dev(torch, B[0]), dev(torch, B[1])), op)
        same_runs(got, oracle.interval_boolean(A, B, op))


def test_interval_boolean_edge_cases(torch):
    e = (np.zeros(0, np.uint64), np.zeros(0, np.uint64))
    one = (np.array([5], np.uint64), np.array([3], np.uint64))
    touch = (np.array([8, 2], np.uint64), np.array([4, 3], np.uint64))      # [8, 12) and [2, 5): touching one
    zero = (np.array([6, 7], np.uint64), np.array([0, 0], np.uint64))
    block = (np.array([oracle.morton3(8, 8, 8)], np.uint64), np.array([512], np.uint64))
    big = (np.array([2 ** 62], np.uint64), np.array([2 ** 62], np.uint64))  # up to 2^63 exactly
    cases = [e, one, touch, zero, block, big]
    for A in cases:
        for B in cases:
            for op in OPS:
                got = pkg.interval_boolean((dev(torch, A[0]), dev(torch, A[1])),
                                           (dev(torch, B[0]), dev(torch, B[1])), op)
                same_runs(got, oracle.interval_boolean(A, B, op))


def test_interval_errors_and_capacity(torch):
    L = pkg.lib()
    past = (dev(torch, [2 ** 63 - 1]), dev(torch, [2]))
    one = (dev(torch, [3]), dev(torch, [2]))
    with pytest.raises(pkg.FPPGError):
        pkg.interval_boolean(one, past, pkg.UNION)
    with pytest.raises(pkg.FPPGError):
        pkg.interval_boolean(one, one, 3)
    with pytest.raises(pkg.FPPGError):
        pkg.interval_cells(past, [0, 0, 0], 1.0)
    with pytest.raises(pkg.FPPGError):
        pkg.lattice_intervals(torch.tensor([[-1.0, 0.5, 0.5]], device="cuda"), [0, 0, 0], 1.0)
    # a capacity below the count: FPPG_ERR_ARG with the count, nothing
    # written ([0, 2) and [10, 12) with [3, 5): three runs, code 2 between)
    two = (dev(torch, [0, 10]), dev(torch, [2, 2]))
    out_b, out_l = dev(torch, [77]), dev(torch, [77])
    n = C.c_int64()
    r = L.fppg_interval_boolean(two[0].data_ptr(), two[1].data_ptr(), 2, one[0].data_ptr(), one[1].data_ptr(), 1,
                                pkg.UNION, out_b.data_ptr(), out_l.data_ptr(), 1, C.byref(n), None)
    assert r == pkg.ERR_ARG and n.value == 3 and int(out_b[0]) == 77 and int(out_l[0]) == 77


@pytest.mark.parametrize("seed", [0, 1])
def test_lattice_intervals_and_cells_match_oracle(torch, seed):
    rng = np.random.default_rng(40 + seed)
    d = np.float32(0.013)
    o = rng.uniform(-2, 2, 3).astype(np.float32)
    cells = rng.integers(0, 90, (200000, 3))
    pts = (o + (cells + rng.uniform(0.0, 1.0, cells.shape)) * d).astype(np.float32)   # anywhere in the cell
    x = torch.from_numpy(pts).cuda()
    got = pkg.lattice_intervals(x, o, d)
    want = oracle.lattice_intervals(pts, o, d)
    same_runs(got, want)
    xc = pkg.interval_cells(got, o, d).cpu().numpy()
    assert np.array_equal(xc, oracle.interval_cells(want, o, d))


def _sphere_and_box(dx):
    v1, t1 = W.icosphere_mesh(3, 0.5)
    lo = v1.min(axis=0)
    v2, t2 = W.cube_mesh(0.5)
    v2 = ((v2 + np.float32(0.5)) * np.float32(0.6) + lo).astype(np.float32)   # the same lower corner
    assert np.array_equal(v2.min(axis=0), lo)
    h = W.smoothing_length(dx)
    gen = {"generate": {"band_cells": 0, "inner_cells": 0}}
    return [W.Assembly("sphere", v1, t1, dx, h, None, None, 30.0, dict(gen)),
            W.Assembly("box", v2, t2, dx, h, None, None, 30.0, dict(gen))]


def test_volume_grid_sets_of_two_bodies(torch):
    # two generated bodies on one lattice (same dx, same lower corner): their
    # interior grid sets combined as intervals (Fig. 10), on the GPU and in
    # the oracle, and against explicit cell-set algebra
    dx = float(np.float32(0.02))
    asm = _sphere_and_box(dx)
    bodies = [pkg.Body.from_assembly(a) for a in asm]
    (o1, d1), (o2, d2) = bodies[0].grid_lattice(), bodies[1].grid_lattice()
    assert np.array_equal(o1, o2) and d1 == d2 == dx
    runs, vols = [], []
    for b in bodies:
        x, c, _ = b.get_particles()
        v = np.ascontiguousarray(x[c == pkg.V])
        assert len(v) > 10000
        vols.append(v)
        r = pkg.lattice_intervals(torch.from_numpy(v).cuda(), o1, d1)
        same_runs(r, oracle.lattice_intervals(v, o1, d1))
        # the runs give the body's volume particles back, bit for bit
        back = pkg.interval_cells(r, o1, d1).cpu().numpy()
        assert len(back) == len(v)
        assert sorted(map(tuple, back.tolist())) == sorted(map(tuple, v.tolist()))
        runs.append(r)
    cell = lambda p: {tuple(t) for t in np.floor((p - o1) / np.float32(d1)).astype(np.int64).tolist()}
    s1, s2 = cell(vols[0]), cell(vols[1])
    for op, want in ((pkg.UNION, s1 | s2), (pkg.DIFFERENCE, s1 - s2), (pkg.INTERSECTION, s1 & s2)):
        got = pkg.interval_boolean(runs[0], runs[1], op)
        same_runs(got, oracle.interval_boolean((host(runs[0][0]), host(runs[0][1])),
                                               (host(runs[1][0]), host(runs[1][1])), op))
        xc = pkg.interval_cells(got, o1, d1).cpu().numpy()
        assert cell(xc) == want and len(xc) == len(want)
    assert 0 < len(s1 & s2) < min(len(s1), len(s2))          # the two really overlap
    for b in bodies:
        b.close()
