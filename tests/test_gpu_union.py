"""Boolean union (Sec. 3.2.3, Fig. 10) on the GPU against the FP64 oracle:
the particles that stay (bit-exact), the union relaxed as one assembly in
the batched form, surfaces kept out of the partner, the calls that must
fail, and the 64-body batch's gear-shaft unions at full size."""
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


def _pair():
    a, b = W.union_pair_workload()
    return a, b, pkg.Body.from_assembly(a), pkg.Body.from_assembly(b), O.from_assembly(a), O.from_assembly(b)


def _united(a, b, ga, gb, oa, ob):
    ka, kb = oa.union_keep(ob, False), ob.union_keep(oa, True)
    O.keep_rows(oa, ka)
    O.keep_rows(ob, kb)
    na, nb = pkg.union(ga, gb)
    return ka, kb, na, nb


def test_union_keeps_the_oracle_particles():
    a, b, ga, gb, oa, ob = _pair()
    ka, kb, na, nb = _united(a, b, ga, gb, oa, ob)
    assert (na, nb) == (ka.sum(), kb.sum()) and 0 < na < a.n and 0 < nb < b.n
    for g, asm, k in ((ga, a, ka), (gb, b, kb)):
        x, c, _ = g.get_particles()
        assert np.array_equal(x, asm.xyz[k]) and np.array_equal(c, asm.cls[k])


def _sphere_frame(b):
    c = np.array([0.45, 0.05, -0.03])
    p = b.verts.astype(np.float64)[b.tris]
    n = np.cross(p[:, 1] - p[:, 0], p[:, 2] - p[:, 0])
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    r_in = np.abs(np.einsum("ij,ij->i", n, p[:, 0] - c)).min()
    r_out = np.linalg.norm(b.verts.astype(np.float64) - c, axis=1).max()
    return c, r_in, r_out


@pytest.mark.parametrize("graph", [False, True])
def test_union_relaxation_matches_the_oracle(graph):
    a, b, ga, gb, oa, ob = _pair()
    _united(a, b, ga, gb, oa, ob)
    bt = pkg.Batch([ga, gb])
    bt.set_graph_iters(5)
    bt.relax(10, use_graph=graph)
    bt.store()
    O.union_relax(oa, ob, 10)
    for g, o, asm in ((ga, oa, a), (gb, ob, b)):
        x, c, _ = g.get_particles()
        ox, oc, _ = o.get_particles()
        assert np.array_equal(c, oc)
        err = np.abs(x.astype(np.float64) - ox).max(axis=1) / asm.dx
        assert np.quantile(err, 0.999) < 1e-4 and err.max() < 1.3 / 16.0, (asm.name, err.max())


def test_union_surfaces_stay_out_of_the_partner():
    a, b, ga, gb, oa, ob = _pair()
    _united(a, b, ga, gb, oa, ob)
    c, r_in, r_out = _sphere_frame(b)
    bt = pkg.Batch([ga, gb])
    bt.set_graph_iters(20)
    bt.relax(60, use_graph=True)
    bt.store()
    xa, ca, _ = ga.get_particles()
    xb, cb, _ = gb.get_particles()
    sa, sb = np.isin(ca, [W.CLS_S, W.CLS_F]), np.isin(cb, [W.CLS_S, W.CLS_F])
    assert not (np.linalg.norm(xa[sa] - c, axis=1) < r_in - 1e-6).any()
    assert not (np.abs(xb[sb]).max(axis=1) < 0.5 - 1e-6).any()
    tol = 1e-6
    for x in (xa, xb):
        assert ((np.abs(x).max(axis=1) <= 0.5 + tol) | (np.linalg.norm(x - c, axis=1) <= r_out + tol)).all()


def test_union_members_relax_only_together():
    a, b, ga, gb, oa, ob = _pair()
    pkg.union(ga, gb)
    with pytest.raises(pkg.FPPGError):
        ga.relax(1)                                 # alone
    with pytest.raises(pkg.FPPGError):
        pkg.Batch([ga])                             # without its partner
    with pytest.raises(pkg.FPPGError):
        pkg.union(ga, gb)                           # already united
    v, t = W.cube_mesh()
    open_cube = pkg.Body(v, t[:-1], a.dx, a.h)      # a face half open
    open_cube.set_particles(a.xyz, a.cls)
    other = pkg.Body.from_assembly(b)
    with pytest.raises(pkg.FPPGError):
        pkg.union(open_cube, other)


def test_config4_gear_shaft_unions_at_full_size():
    asm = W.batch_union_workload()
    pairs = [(i, a.meta["union_with"]) for i, a in enumerate(asm) if a.meta.get("union_with", -1) > i]
    assert len(pairs) >= 8
    bodies = [pkg.Body.from_assembly(a) for a in asm]
    before = sum(g.n for g in bodies)
    for i, j in pairs:
        pkg.union(bodies[i], bodies[j])
    n = sum(g.n for g in bodies)
    assert 6.5e6 < n < before
    bt = pkg.Batch(bodies)
    bt.autotune(1)
    bt.set_graph_iters(4)
    bt.relax(8, use_graph=True)
    bt.store()
    for i, j in pairs:           # no gear surface inside its shaft, no shaft surface inside its gear's hub ring
        s = asm[i].meta["scale"]
        xg, cg, _ = bodies[i].get_particles()
        xs, cs, _ = bodies[j].get_particles()
        sg = np.isin(cg, [W.CLS_S, W.CLS_F])
        r_in = 0.2 * s * np.cos(np.pi / 48)
        inside_shaft = (np.hypot(xg[:, 0], xg[:, 1]) < r_in - 1e-5) & (np.abs(xg[:, 2]) < 0.25 * s - 1e-5)
        assert not (sg & inside_shaft).any(), asm[i].name
        ss = np.isin(cs, [W.CLS_S, W.CLS_F])
        r = np.hypot(xs[:, 0], xs[:, 1])
        in_hub = (r > 0.15 * s + 1e-4) & (r < 0.45 * s * 0.9) & (np.abs(xs[:, 2]) < 0.1 * s - 1e-4)
        assert not (ss & in_hub).any(), asm[j].name
    # the smallest pair against the oracle, from the oracle's own generation
    i, j = min(pairs, key=lambda p: asm[p[0]].meta["scale"])
    oa, ob = O.from_assembly(asm[i]), O.from_assembly(asm[j])
    ga, gb = pkg.Body.from_assembly(asm[i]), pkg.Body.from_assembly(asm[j])
    for g, o in ((ga, oa), (gb, ob)):
        x, c, cons = o.get_particles()
        g.set_particles(x.astype(np.float32), c)
        g.set_constraints(cons)
    ka, kb, na, nb = _united(asm[i], asm[j], ga, gb, oa, ob)
    assert (na, nb) == (ka.sum(), kb.sum())
    pair = pkg.Batch([ga, gb])
    pair.relax(3, use_graph=False)
    pair.store()
    O.union_relax(oa, ob, 3)
    for g, o, a in ((ga, oa, asm[i]), (gb, ob, asm[j])):
        err = np.abs(g.get_particles()[0].astype(np.float64) - o.get_particles()[0]).max(axis=1) / a.dx
        assert (err < 1e-4).mean() > 0.999 and err.max() < 1.3 / 16.0, (a.name, err.max())


@pytest.mark.parametrize("op", [pkg.DIFFERENCE, pkg.INTERSECTION])
def test_difference_and_intersection_match_the_oracle(op):
    a, b, ga, gb, oa, ob = _pair()
    ka, kb = oa.boolean_keep(ob, op, True), ob.boolean_keep(oa, op, False)
    O.keep_rows(oa, ka)
    O.keep_rows(ob, kb)
    na, nb = pkg.boolean(ga, gb, op)
    assert (na, nb) == (ka.sum(), kb.sum()) and na > 0 and nb > 0
    for g, asm, k in ((ga, a, ka), (gb, b, kb)):
        x, c, _ = g.get_particles()
        assert np.array_equal(x, asm.xyz[k]) and np.array_equal(c, asm.cls[k])
    bt = pkg.Batch([ga, gb])
    bt.set_graph_iters(5)
    bt.relax(10, use_graph=True)
    bt.store()
    O.boolean_relax(oa, ob, op, 10)
    for g, o, asm in ((ga, oa, a), (gb, ob, b)):
        err = np.abs(g.get_particles()[0].astype(np.float64) - o.get_particles()[0]).max(axis=1) / asm.dx
        assert np.quantile(err, 0.999) < 1e-4 and err.max() < 1.3 / 16.0, (asm.name, err.max())
    c, r_in, r_out = _sphere_frame(b)
    xa, xb = ga.get_particles()[0], gb.get_particles()[0]
    assert (np.abs(xb).max(axis=1) <= 0.5 + 1e-6).all()          # b's surface stays inside the cube
    if op == pkg.DIFFERENCE:
        assert not (np.linalg.norm(xa - c, axis=1) < r_in - 1e-6).any()
    else:
        assert (np.linalg.norm(xa - c, axis=1) <= r_out + 1e-6).all()
