"""The seeded synthetic inputs (CPU): the meshes are closed and outward
oriented, the counter-based jitter is deterministic and bounded, and the
workloads have the sizes the benchmark and the parity tests are quoted on."""
import numpy as np
import pytest

from paper_2501_03056_gb300 import workloads as W


def _closed_and_outward(v, t):
    v = np.asarray(v, np.float64)
    t = np.asarray(t, np.int64)
    # every directed edge appears once and its reverse once
    e = np.concatenate([t[:, [0, 1]], t[:, [1, 2]], t[:, [2, 0]]])
    fwd = {tuple(x) for x in e.tolist()}
    assert len(fwd) == len(e), "a directed edge repeats (inconsistent orientation)"
    assert all((b, a) in fwd for a, b in fwd), "an edge without its reverse (open mesh)"
    # positive signed volume (divergence theorem over the faces)
    a, b, c = v[t[:, 0]], v[t[:, 1]], v[t[:, 2]]
    vol = np.einsum("ij,ij->i", a, np.cross(b, c)).sum() / 6.0
    assert vol > 0.0
    return vol


@pytest.mark.parametrize("name", ["cube", "icosphere", "torus", "cylinder", "gear"])
def test_meshes_are_closed_and_outward(name):
    if name == "cube":
        v, t = W.cube_mesh()
        assert _closed_and_outward(v, t) == pytest.approx(1.0, rel=1e-12)
    elif name == "icosphere":
        v, t = W.icosphere_mesh(3)
        assert len(t) == 20 * 4 ** 3
        vol = _closed_and_outward(v, t)
        assert 0.95 * 4.0 / 3.0 * np.pi < vol < 4.0 / 3.0 * np.pi   # inscribed polyhedron
    elif name == "torus":
        v, t = W.torus_mesh(1.0, 0.3, 64, 24)
        assert len(t) == 2 * 64 * 24
        vol = _closed_and_outward(v, t)
        assert vol == pytest.approx(2 * np.pi ** 2 * 1.0 * 0.3 ** 2, rel=0.02)
    elif name == "cylinder":
        v, t = W.cylinder_mesh()
        vol = _closed_and_outward(v, t)
        assert vol == pytest.approx(np.pi * 0.25 * 1.0, rel=0.01)
    else:
        v, t = W.gear_mesh()
        assert len(t) == 51840
        _closed_and_outward(v, t)


def test_jitter_is_deterministic_and_bounded():
    ids = np.arange(100000, dtype=np.uint64)
    a = W.jitter(7, ids, 1, 0.25)
    b = W.jitter(7, ids, 1, 0.25)
    assert np.array_equal(a, b)
    assert np.abs(a).max() <= 0.25 and abs(a.mean()) < 0.01
    assert not np.array_equal(a, W.jitter(8, ids, 1, 0.25))       # the seed matters
    assert not np.array_equal(a, W.jitter(7, ids, 2, 0.25))       # so does the axis
    u = W.uniform01(3, ids, 0)
    assert u.min() >= 0.0 and u.max() < 1.0


def test_workload_sizes_and_classes():
    cube = W.cube_workload()[0]
    assert cube.n == 10636
    counts = np.bincount(cube.cls, minlength=5)
    assert counts[W.CLS_S] == 2400 and counts[W.CLS_F] == 228 and counts[W.CLS_P] == 8 and counts[W.CLS_V] == 8000
    st = W.sphere_torus_workload()
    assert [a.n for a in st] == [539787, 237428] and sum(a.n for a in st) == 777215
    again = W.sphere_torus_workload()
    for x, y in zip(st, again):
        assert np.array_equal(x.xyz, y.xyz) and np.array_equal(x.cls, y.cls)
