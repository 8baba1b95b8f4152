"""The Morton order of the grid rows (Eq. 9 over y and z, x fastest inside a
row) on the GPU: keys, permutation and cell ranges bit-exact against the
oracle in that order (both the full sort and the incremental repair);
relaxations equal to the row-major order's up to the FP32 rounding of the
two partial sums a row's slots are split between (their absolute parity
moves with the order) in the plain form and a Boolean assembly, the
batched graph form bit-identical to the plain form in the same order; the
energy and its gradients the same in both orders; the autotuner choosing
between the two orders."""
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


def small_sphere_torus(seed=1):
    return W.sphere_torus_workload(seed=seed, dx=0.06, level=3, torus_nu=64, torus_nv=24)


@pytest.mark.parametrize("inc", [False, True])
def test_keys_permutation_and_ranges_in_morton_row_order(inc):
    for a in W.cube_workload(seed=2) + small_sphere_torus(2):
        b, o = pkg.Body.from_assembly(a), O.from_assembly(a)
        b.set_incremental(inc)
        b.set_cell_order(pkg.ORDER_MORTON_ROWS)
        o.set_cell_order(1)
        for _ in range(2):                  # the second build repairs the first order
            key, perm, cells, st, en = b.debug_grid()
            okey, operm = o.keys()
            assert np.array_equal(key, okey) and np.array_equal(perm, operm)
            oc, os_, oe = o.cell_ranges()
            assert np.array_equal(cells, oc) and np.array_equal(st, os_) and np.array_equal(en, oe)
            b.relax(1)
            o.relax(1)
        assert np.abs(b.get_particles()[0].astype(np.float64) - o.get_particles()[0]).max() < 1e-4 * a.dx


def close(x0, x1, dx):
    err = np.abs(x0.astype(np.float64) - x1).max(axis=1) / dx
    return np.quantile(err, 0.999) < 1e-5 and err.max() < 1e-4


def test_plain_and_batched_relaxations_do_not_depend_on_the_row_order():
    asm = small_sphere_torus(3)
    ref = [pkg.Body.from_assembly(a) for a in asm]
    mor = [pkg.Body.from_assembly(a) for a in asm]
    for a, r, m in zip(asm, ref, mor):
        m.set_cell_order(pkg.ORDER_MORTON_ROWS)
        r.relax(6)
        m.relax(6)
        assert close(r.get_particles()[0], m.get_particles()[0], a.dx)
    # the batched graph form in Morton order gives the plain body's bits
    bodies = [pkg.Body.from_assembly(a) for a in asm[:1]]
    bt = pkg.Batch(bodies)
    bt.set_cell_order(pkg.ORDER_MORTON_ROWS)
    bt.set_graph_iters(3)
    bt.relax(6, use_graph=True)
    bt.store()
    assert np.array_equal(mor[0].get_particles()[0], bodies[0].get_particles()[0])


def test_boolean_assembly_in_morton_row_order():
    a, b = W.union_pair_workload()
    runs = []
    for order in (pkg.ORDER_ROWS, pkg.ORDER_MORTON_ROWS):
        ga, gb = pkg.Body.from_assembly(a), pkg.Body.from_assembly(b)
        pkg.union(ga, gb)
        bt = pkg.Batch([ga, gb])
        bt.set_cell_order(order)
        bt.set_incremental(True)
        bt.relax(6, use_graph=False)
        bt.store()
        runs.append([g.get_particles()[0] for g in (ga, gb)])
    for asm_, x0, x1 in zip((a, b), *runs):
        assert close(x0, x1, asm_.dx)


def test_full_size_icosphere_torus_keys_and_autotune():
    asm = W.sphere_torus_workload()
    a = asm[0]
    b, o = pkg.Body.from_assembly(a), O.from_assembly(a)
    b.set_cell_order(pkg.ORDER_MORTON_ROWS)
    o.set_cell_order(1)
    key, perm, *_ = b.debug_grid()
    okey, operm = o.keys()
    assert np.array_equal(key, okey) and np.array_equal(perm, operm)
    bodies = [pkg.Body.from_assembly(x) for x in asm]
    snap = [g.get_particles()[0].copy() for g in bodies]
    bt = pkg.Batch(bodies)
    choice = bt.autotune(2)
    assert choice["cell_order"] in (0, 1)
    bt.store()
    for g, x in zip(bodies, snap):                 # tuning restores the state
        assert np.array_equal(g.get_particles()[0], x)


def test_bad_order_is_an_argument_error():
    a = W.cube_workload()[0]
    b = pkg.Body.from_assembly(a)
    assert pkg.lib().fppg_set_cell_order(b.handle, 2) == pkg.ERR_ARG
    assert pkg.lib().fppg_set_cell_order(None, 1) == pkg.ERR_ARG


def test_energy_and_backward_in_morton_row_order():
    import torch
    a = W.cube_workload(seed=1)[0]
    b = pkg.Body.from_assembly(a)
    b.relax(2)
    x, c, cons = b.get_particles()
    res = []
    for order in (pkg.ORDER_ROWS, pkg.ORDER_MORTON_ROWS):
        g = pkg.Body(a.verts, a.tris, a.dx, a.h)
        g.extract_features(a.dihedral_deg)
        g.set_particles(x, c)
        g.set_constraints(cons)
        g.set_cell_order(order)
        y = torch.from_numpy(np.ascontiguousarray(x)).cuda()
        v = torch.from_numpy(np.ascontiguousarray(a.verts)).cuda()
        gy, gv = torch.empty_like(y), torch.empty_like(v)
        E = g.energy_ptr(y.data_ptr(), v.data_ptr(), gy.data_ptr(), gv.data_ptr())
        res.append((E, gy.cpu().numpy(), gv.cpu().numpy()))
    (E0, gy0, gv0), (E1, gy1, gv1) = res
    # the same energy and gradients up to the FP32 sums, within the bounds the
    # energy test holds against the oracle
    assert E1 == pytest.approx(E0, rel=1e-5)
    assert np.abs(gy1 - gy0).max() <= 1e-4 * np.abs(gy0).max()
    assert np.abs(gv1 - gv0).max() <= 1e-4 * np.abs(gv0).max()
