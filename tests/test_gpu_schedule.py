"""The paper-literal options on the GPU against the oracle: the
re-projection cascade of Sec. 3.3.3 (own triangle, own cell, 27 cells) and
the surface-then-volume schedule (Algorithm 1, then Sec. 3.3.4) through the
mobile-class mask, plain and batched (a captured graph sees a new mask)."""
import numpy as np
import pytest

import oracle as O
import paper_2501_03056_gb300 as pkg
from paper_2501_03056_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2501_03056_gb300 import _build
    _build.build()


def _sheets(z_top):
    v = np.array([[-1, -1, 0], [3, -1, 0], [-1, 3, 0], [0, 0, z_top], [0.2, 0, z_top], [0, 0.2, z_top]], np.float32)
    return v, np.array([[0, 1, 2], [3, 4, 5]], np.int32)


def test_cascade_on_stacked_sheets():
    v, t = _sheets(0.002)
    b = pkg.Body(v, t, 0.05, 0.065)
    y = np.array([[0.03, 0.03, 0.0015]], np.float32)
    s = np.array([W.CLS_S], np.int32)
    assert b.project_points(y, s, np.array([0], np.int32))[1][0] == 1
    b.set_projection_rule(cascade=True)
    assert b.project_points(y, s, np.array([0], np.int32))[1][0] == 0
    assert b.project_points(y, s, np.array([-1], np.int32))[1][0] == 1


@pytest.mark.parametrize("mesh", ["ico4", "torus", "cube"])
def test_cascade_projection_matches_oracle(mesh):
    if mesh == "cube":
        v, t = W.cube_mesh()
        dx = 0.05
    elif mesh == "ico4":
        v, t = W.icosphere_mesh(4)
        dx = 0.03
    else:
        v, t = W.torus_mesh(1.0, 0.3, 128, 32)
        dx = 0.03
    b, o = pkg.Body(v, t, dx, 1.3 * dx), O.Oracle(v, t, dx, 1.3 * dx)
    b.set_projection_rule(cascade=True)
    o.set_cascade(True)
    rng = np.random.default_rng(9)
    tri = rng.integers(0, len(t), 20000)
    bc = rng.dirichlet([1, 1, 1], 20000)
    p = np.einsum("ij,ijk->ik", bc, v[t[tri]].astype(np.float64))
    y = (p + rng.normal(size=p.shape) * 0.3 * dx).astype(np.float32)
    # the particles' current triangles: where they came from, half of them
    # replaced by a neighbour's (so the cascade's first test fails there)
    cons = np.where(rng.random(20000) < 0.5, tri, (tri + 1) % len(t)).astype(np.int32)
    cls = np.zeros(len(y), np.int32)
    x, gt, ok = b.project_points(y, cls, cons)
    ox, ot, ook = o.project_points(y, cls, cons)
    agree = (gt == ot) & (ok == ook)
    assert agree.mean() > 0.999
    both = ok & ook
    assert np.abs(x[both].astype(np.float64) - ox[both]).max() < 1e-4 * dx
    kept = (gt == cons) & ok
    assert 0.2 < kept.mean() < 0.9          # the cascade's first stage decides a good share


def test_surface_then_volume_schedule_matches_oracle():
    a = W.cube_workload()[0]
    b, o = pkg.Body.from_assembly(a), O.from_assembly(a)
    x0 = b.get_particles()[0]
    surf, vol = np.isin(a.cls, [W.CLS_S, W.CLS_F]), a.cls == W.CLS_V
    for classes, moving, still in (([W.CLS_S, W.CLS_F], surf, vol), ([W.CLS_V], vol, surf)):
        b.set_mobile_classes(classes)
        o.set_mobile_classes(classes)
        b.relax(3)
        o.relax(3)
        x = b.get_particles()[0]
        assert np.array_equal(x[still], x0[still])
        assert (np.abs(x[moving] - x0[moving]).max(axis=1) > 0).mean() > 0.9
        err = np.abs(x.astype(np.float64) - o.get_particles()[0]).max(axis=1) / a.dx
        assert np.quantile(err, 0.999) < 1e-4 and err.max() < 1e-3, err.max()
        x0 = x


def test_batch_mobile_mask_reaches_a_captured_graph():
    a = W.cube_workload()[0]
    plain, batched = pkg.Body.from_assembly(a), pkg.Body.from_assembly(a)
    bt = pkg.Batch([batched])
    bt.set_graph_iters(2)
    bt.relax(2, use_graph=True)                 # graph captured with every class mobile
    plain.relax(2)
    bt.set_mobile_classes([W.CLS_V])
    plain.set_mobile_classes([W.CLS_V])
    bt.relax(4, use_graph=True)
    plain.relax(4)
    bt.store()
    assert np.array_equal(plain.get_particles()[0], batched.get_particles()[0])
