"""Boolean chains on the GPU against the FP64 oracle (Sec. 3.2.3, Fig. 10):
a body in several operations keeps what every one of them keeps and relaxes
under all their rules, in one assembly with its partners.  A union chain of
three spheres (the middle one in two unions), a cube with two cavities (the
cube in two differences), the chain's intersection curves, and the calls
that must fail."""
import numpy as np
import pytest

import oracle as O
import paper_2501_03056_gb300 as pkg
from paper_2501_03056_gb300 import workloads as W

pytestmark = pytest.mark.gpu

S, V, F, I, P = W.CLS_S, W.CLS_V, W.CLS_F, W.CLS_I, W.CLS_P
DX = 0.05
H = float(np.float32(1.3 * DX))
CENTRES = [np.array([0.0, 0.0, 0.0]), np.array([0.7, 0.0131, 0.0217]), np.array([1.4, 0.0297, -0.0113])]


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2501_03056_gb300 import _build
    _build.build()


def sphere(c, level=3, r=0.5):
    v, t = W.icosphere_mesh(level, r)
    return (v.astype(np.float64) + c).astype(np.float32), t


def both(v, t, features=False):
    """The oracle's generated body on both sides (the same particles and
    constraints)."""
    o = O.Oracle(v, t, DX, H)
    g = pkg.Body(v, t, DX, H)
    if features:
        o.extract_features(30.0)
        g.extract_features(30.0)
    x, c, cons = o.map_particles()
    x32 = x.astype(np.float32)
    o.set_particles(x32, c)
    o.set_state(x32.astype(np.float64), cons)
    g.set_particles(x32, c)
    g.set_constraints(cons)
    return g, o


def apply_op(ga, gb, oa, ob, op):
    ka, kb = oa.boolean_keep(ob, op, True), ob.boolean_keep(oa, op, False)
    O.keep_rows(oa, ka)
    O.keep_rows(ob, kb)
    na, nb = pkg.boolean(ga, gb, op)
    assert (na, nb) == (ka.sum(), kb.sum())


def same_particles(g, o):
    x, c, _ = g.get_particles()
    ox, oc, _ = o.get_particles()
    assert np.array_equal(c, oc) and np.array_equal(x, ox.astype(np.float32))


def relaxed_alike(gs, os_, pairs, iters=10, graph=True):
    bt = pkg.Batch(gs)
    bt.set_graph_iters(5)
    bt.relax(iters, use_graph=graph)
    bt.store()
    O.boolean_relax_many(os_, pairs, iters)
    for g, o in zip(gs, os_):
        x, c, _ = g.get_particles()
        ox, oc, _ = o.get_particles()
        assert np.array_equal(c, oc)
        err = np.abs(x.astype(np.float64) - ox).max(axis=1) / DX
        assert np.quantile(err, 0.999) < 1e-4 and err.max() < 1.3 / 16.0, err.max()


def union_chain():
    bodies = [both(*sphere(c)) for c in CENTRES]
    gs, os_ = [b[0] for b in bodies], [b[1] for b in bodies]
    apply_op(gs[0], gs[1], os_[0], os_[1], pkg.UNION)
    apply_op(gs[1], gs[2], os_[1], os_[2], pkg.UNION)
    for g, o in zip(gs, os_):
        same_particles(g, o)
    return gs, os_


@pytest.mark.parametrize("graph", [False, True])
def test_union_chain_relaxes_like_the_oracle(graph):
    gs, os_ = union_chain()
    relaxed_alike(gs, os_, [(0, 1, O.UNION), (1, 2, O.UNION)], graph=graph)


def test_cube_with_two_cavities_relaxes_like_the_oracle():
    gc, oc = both(*W.cube_mesh(0.5), features=True)
    cav = [np.array([0.55, 0.05, -0.02]), np.array([-0.55, -0.03, 0.04])]
    holes = [both(*sphere(c)) for c in cav]
    for gh, oh in holes:
        apply_op(gc, gh, oc, oh, pkg.DIFFERENCE)
    same_particles(gc, oc)
    relaxed_alike([gc] + [h[0] for h in holes], [oc] + [h[1] for h in holes],
                  [(0, 1, O.DIFFERENCE), (0, 2, O.DIFFERENCE)])


def test_chain_curves_match_the_oracle_and_relax_alike():
    gs, os_ = union_chain()
    for i, j in ((0, 1), (1, 2)):
        n = pkg.boolean_curve(gs[i], gs[j])
        assert n == os_[i].boolean_curve(os_[j]) > 0
        assert np.array_equal(gs[i].curve_points(), os_[i].curve_points())
        same_particles(gs[i], os_[i])
    relaxed_alike(gs, os_, [(0, 1, O.UNION), (1, 2, O.UNION)])


def test_chain_calls_that_must_fail():
    gs, _ = union_chain()
    # the same pair twice
    with pytest.raises(pkg.FPPGError) as e:
        pkg.union(gs[0], gs[1])
    assert e.value.code == pkg.ERR_STATE
    # a batch without every partner of its operands
    with pytest.raises(pkg.FPPGError) as e:
        pkg.Batch(gs[:2])
    assert e.value.code == pkg.ERR_STATE
    # at most four operations per body
    v, t = sphere(CENTRES[1])
    extra = [both(v, t)[0] for _ in range(3)]
    for x in extra[:2]:
        pkg.union(gs[1], x)                         # gs[1]: operations 3 and 4
    with pytest.raises(pkg.FPPGError) as e:
        pkg.union(gs[1], extra[2])
    assert e.value.code == pkg.ERR_STATE
    # the curve of a pair once
    pkg.boolean_curve(gs[0], gs[1])
    for a, b in ((gs[0], gs[1]), (gs[1], gs[0])):
        with pytest.raises(pkg.FPPGError) as e:
            pkg.boolean_curve(a, b)
        assert e.value.code == pkg.ERR_STATE
