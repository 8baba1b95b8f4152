"""Checkpoint and resume (Algorithm 1 has no random draws): relaxing n
iterations equals relaxing k, saving the particles (positions, classes,
constraints), loading them into a fresh body and relaxing n - k more, bit
for bit.  The fresh body has no previous key order and no inside or surface
certificates, so this also shows that the incremental ordering and both
kinds of certificates change no result: the resumed run takes the full
searches where the continued one took certified shortcuts."""
import numpy as np
import pytest

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


def resumed(a, k, n, incremental):
    b = pkg.Body.from_assembly(a)
    b.set_incremental(incremental)
    b.relax(k)
    x, c, cons = b.get_particles()
    r = pkg.Body(a.verts, a.tris, a.dx, a.h)
    if a.dihedral_deg is not None:
        r.extract_features(a.dihedral_deg)
    r.set_incremental(incremental)
    r.set_particles(x, c)
    r.set_constraints(cons)
    r.relax(n - k)
    return r.get_particles()


@pytest.mark.parametrize("incremental", [False, True])
def test_resume_is_bit_exact(incremental):
    for a in W.cube_workload(seed=4) + small_sphere_torus(4):
        full = pkg.Body.from_assembly(a)
        full.set_incremental(incremental)
        full.relax(12)
        x, c, cons = full.get_particles()
        rx, rc, rcons = resumed(a, 5, 12, incremental)
        assert np.array_equal(x, rx), (a.name, np.abs(x - rx).max())
        assert np.array_equal(c, rc) and np.array_equal(cons, rcons)


def test_resume_of_a_batched_graph_run_is_bit_exact():
    asm = small_sphere_torus(5)
    full = [pkg.Body.from_assembly(a) for a in asm]
    bt = pkg.Batch(full)
    bt.set_graph_iters(4)
    bt.relax(12, use_graph=True)
    bt.store()
    half = [pkg.Body.from_assembly(a) for a in asm]
    bt2 = pkg.Batch(half)
    bt2.set_graph_iters(4)
    bt2.relax(4, use_graph=True)
    bt2.store()
    fresh = []
    for a, h in zip(asm, half):
        x, c, cons = h.get_particles()
        r = pkg.Body(a.verts, a.tris, a.dx, a.h)
        r.set_particles(x, c)
        r.set_constraints(cons)
        fresh.append(r)
    bt3 = pkg.Batch(fresh)
    bt3.set_graph_iters(4)
    bt3.relax(8, use_graph=True)
    bt3.store()
    for f, r in zip(full, fresh):
        assert np.array_equal(f.get_particles()[0], r.get_particles()[0])
