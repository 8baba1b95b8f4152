"""The intersection curve of a Boolean pair (Sec. 3.2.3, read as a feature
line of Sec. 3.2.2) on the library against the oracle: the curve points,
lines and particles of fppg_boolean_curve (set-up in FP64, the same
decisions on both sides), the union relaxed with them as one assembly in
the batched form, the curve particles staying on both surfaces, and the
calls that must fail."""
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


def _meshes(offset, level):
    v, t = W.icosphere_mesh(level)
    v2 = (v.astype(np.float64) + np.asarray(offset)).astype(np.float32)
    return (v, t), (v2, t)


def _dist_to_mesh(p, V, T):
    """Brute-force distance from each point to the closest point of any
    triangle (interior foot or the closest point of an edge)."""
    A, B, Cc = (V[T[:, k]].astype(np.float64) for k in range(3))
    n = np.cross(B - A, Cc - A)
    n /= np.linalg.norm(n, axis=1)[:, None]

    def seg(q, P0, P1):
        e = P1 - P0
        t = np.clip(np.einsum("ij,ij->i", q - P0, e) / np.einsum("ij,ij->i", e, e), 0.0, 1.0)
        return np.linalg.norm(q - (P0 + t[:, None] * e), axis=1)

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


@pytest.mark.parametrize("offset", [(1.2, 0.0137, 0.0291), (1.2, 0.0, 0.0), (0.37, -0.81, 0.52)])
def test_curve_of_two_spheres_matches_the_oracle(offset):
    (va, ta), (vb, tb) = _meshes(offset, 4)
    dx = 0.03
    h = float(np.float32(1.3 * dx))
    ga, gb = pkg.Body(va, ta, dx, h), pkg.Body(vb, tb, dx, h)
    oa, ob = O.Oracle(va, ta, dx, h), O.Oracle(vb, tb, dx, h)
    empty = (np.zeros((0, 3), np.float32), np.zeros(0, np.int32))
    for x in (ga, gb, oa):
        x.set_particles(*empty)
    pkg.union(ga, gb)
    n = pkg.boolean_curve(ga, gb)
    on = oa.boolean_curve(ob)
    assert n == on > 0
    # the same FP64 decisions: points, lines and particles alike
    pts, opts = ga.curve_points(), oa.curve_points()
    assert np.array_equal(pts, opts)
    ln, lc, ls = ga.feature_lines()
    first, onseg, oclosed, osegv = oa.feature_lines()
    assert np.array_equal(ln, onseg) and np.array_equal(lc, oclosed) and np.array_equal(ls, osegv)
    x, c, cons = ga.get_particles()
    ox, oc, ocons = oa.get_particles()
    assert np.array_equal(c, oc) and np.array_equal(cons, ocons)
    assert np.abs(x.astype(np.float64) - ox).max() <= 1e-6
    # on both surfaces
    assert _dist_to_mesh(pts, va, ta).max() < 1e-6 and _dist_to_mesh(pts, vb, tb).max() < 1e-6
    # the curve comes once
    with pytest.raises(pkg.FPPGError) as e:
        pkg.boolean_curve(ga, gb)
    assert e.value.code == pkg.ERR_STATE


def _generated(mesh, dx, h):
    o = O.Oracle(*mesh, dx, h)
    x, c, cons = o.map_particles()
    x32 = x.astype(np.float32)
    o.set_particles(x32, c)
    o.set_state(x32.astype(np.float64), cons)
    g = pkg.Body(*mesh, dx, h)
    g.set_particles(x32, c)
    g.set_constraints(cons)
    return g, o


@pytest.mark.parametrize("graph", [False, True])
def test_union_with_its_curve_relaxes_like_the_oracle(graph):
    offset = (1.2, 0.0137, 0.0291)
    (va, ta), (vb, tb) = _meshes(offset, 3)
    dx = 0.06
    h = float(np.float32(1.3 * dx))
    (ga, oa), (gb, ob) = _generated((va, ta), dx, h), _generated((vb, tb), dx, h)
    ka, kb = oa.union_keep(ob, False), ob.union_keep(oa, True)
    O.keep_rows(oa, ka)
    O.keep_rows(ob, kb)
    na, nb = pkg.union(ga, gb)
    assert (na, nb) == (ka.sum(), kb.sum())
    n = pkg.boolean_curve(ga, gb)
    assert n == oa.boolean_curve(ob) > 0
    x0, c0, _ = ga.get_particles()
    curve = np.arange(len(x0)) >= na
    assert np.all(c0[curve] == W.CLS_F)
    bt = pkg.Batch([ga, gb])
    bt.set_graph_iters(5)
    bt.relax(10, use_graph=graph)
    bt.store()
    O.boolean_relax(oa, ob, O.UNION, 10)
    for g, o in ((ga, oa), (gb, ob)):
        x, c, _ = g.get_particles()
        ox, oc, _ = o.get_particles()
        assert np.array_equal(c, oc)
        err = np.abs(x.astype(np.float64) - ox).max(axis=1) / dx
        assert np.quantile(err, 0.999) < 1e-4 and err.max() < 1.3 / 16.0, err.max()
    # the curve particles slid along the curve (no partner rule holds them)
    # and stayed on both surfaces
    x, _, _ = ga.get_particles()
    assert np.abs(x[curve] - x0[curve]).max() > 1e-4 * dx
    assert _dist_to_mesh(x[curve], va, ta).max() < 1e-5
    assert _dist_to_mesh(x[curve], vb, tb).max() < 1e-5


def test_curve_needs_the_boolean_pair():
    (va, ta), (vb, tb) = _meshes((1.2, 0.0137, 0.0291), 2)
    dx = 0.1
    h = float(np.float32(1.3 * dx))
    ga, gb = pkg.Body(va, ta, dx, h), pkg.Body(vb, tb, dx, h)
    empty = (np.zeros((0, 3), np.float32), np.zeros(0, np.int32))
    ga.set_particles(*empty)
    gb.set_particles(*empty)
    for a, b in ((ga, gb), (ga, ga)):
        with pytest.raises(pkg.FPPGError) as e:
            pkg.boolean_curve(a, b)
        assert e.value.code in (pkg.ERR_STATE, pkg.ERR_ARG)
    assert pkg.lib().fppg_boolean_curve(None, gb.handle, None) == pkg.ERR_ARG


def test_every_allocation_of_the_curve_can_fail_cleanly():
    (va, ta), (vb, tb) = _meshes((1.2, 0.0137, 0.0291), 3)
    dx = 0.06
    h = float(np.float32(1.3 * dx))
    L = pkg.lib()
    ref = None
    for k in range(64):
        ga, gb = pkg.Body(va, ta, dx, h), pkg.Body(vb, tb, dx, h)
        x = np.array([[0.0, 0.0, 0.0], [-0.5, 0.0, 0.0]], np.float32)
        ga.set_particles(x, np.array([W.CLS_V, W.CLS_V], np.int32))
        gb.set_particles(x[:0], np.zeros(0, np.int32))
        pkg.union(ga, gb)
        assert L.fppg_debug_fail_allocation(k) == pkg.OK
        try:
            n = pkg.boolean_curve(ga, gb)
        except pkg.FPPGError as e:
            L.fppg_debug_fail_allocation(-1)
            assert e.code == pkg.ERR_OOM, (k, str(e))
            # no curve lines left behind
            ln, _, _ = ga.feature_lines()
            assert len(ln) == 0 and len(ga.curve_points()) == 0
            continue
        L.fppg_debug_fail_allocation(-1)
        ref = (n, ga.get_particles())
        break
    assert ref is not None and ref[0] > 0
    ga, gb = pkg.Body(va, ta, dx, h), pkg.Body(vb, tb, dx, h)
    ga.set_particles(x, np.array([W.CLS_V, W.CLS_V], np.int32))
    gb.set_particles(x[:0], np.zeros(0, np.int32))
    pkg.union(ga, gb)
    assert pkg.boolean_curve(ga, gb) == ref[0]
    assert np.array_equal(ga.get_particles()[0], ref[1][0])
