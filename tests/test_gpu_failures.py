"""Out-of-memory paths, made on the host: fppg_debug_fail_allocation makes
the k-th device allocation from now fail as cudaMalloc does when the device
is full.  Every entry point that allocates must then return FPPG_ERR_OOM
(never crash, never report success), and the library must work normally
afterwards, with the same results as a run that saw no failure."""
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
    yield
    pkg.lib().fppg_debug_fail_allocation(-1)


def _sweep(call, limit=400):
    """Fail allocation k = 0, 1, ... of `call` until it succeeds; returns how
    many allocations it made (the failing ones all raised FPPG_ERR_OOM)."""
    L = pkg.lib()
    for k in range(limit):
        assert L.fppg_debug_fail_allocation(k) == pkg.OK
        try:
            out = call()
        except pkg.FPPGError as e:
            assert e.code == pkg.ERR_OOM, (k, str(e))
            continue
        L.fppg_debug_fail_allocation(-1)
        return k, out
    L.fppg_debug_fail_allocation(-1)
    raise AssertionError("the call did not succeed within the sweep")


def _reference(a, iters):
    b = pkg.Body.from_assembly(a)
    b.relax(iters)
    return b.get_particles()


def test_every_allocation_of_the_main_path_can_fail_cleanly():
    a = W.cube_workload()[0]
    ref = _reference(a, 3)
    # body creation (mesh, grids, candidate lists)
    n_create, body = _sweep(lambda: pkg.Body(a.verts, a.tris, a.dx, a.h))
    assert n_create > 10
    # features, then the particles (device staging), then a relaxation
    _sweep(lambda: body.extract_features(a.dihedral_deg))
    _sweep(lambda: body.set_particles(a.xyz, a.cls))
    _sweep(lambda: body.relax(3))
    x, c, cons = body.get_particles()
    assert np.array_equal(x, ref[0]) and np.array_equal(cons, ref[2])


def test_generation_batches_graphs_and_energy_fail_cleanly():
    import torch
    v, t = W.cylinder_mesh(0.5, 1.0, 64, 4)
    b = pkg.Body(v, t, 0.04, float(np.float32(1.3 * 0.04)))
    b.extract_features(30.0)
    _, n = _sweep(lambda: b.map_particles(band_cells=2))
    ref = pkg.Body(v, t, 0.04, float(np.float32(1.3 * 0.04)))
    ref.extract_features(30.0)
    assert ref.map_particles(band_cells=2) == n
    assert np.array_equal(b.get_particles()[0], ref.get_particles()[0])
    # a batch of two bodies, its CUDA graph and the autotuner
    asm = W.cube_workload(seed=2)
    bodies = [pkg.Body.from_assembly(x) for x in asm + W.cube_workload(seed=3)]
    _, batch = _sweep(lambda: pkg.Batch(bodies))
    batch.set_graph_iters(2)
    _sweep(lambda: batch.relax(4, use_graph=True))
    _sweep(lambda: batch.autotune(1))
    # the energy and its backward
    y = torch.from_numpy(np.ascontiguousarray(ref.get_particles()[0])).cuda()
    vt = torch.from_numpy(np.ascontiguousarray(v)).cuda()
    gy, gv = torch.empty_like(y), torch.empty_like(vt)
    _, E = _sweep(lambda: ref.energy_ptr(y.data_ptr(), vt.data_ptr(), gy.data_ptr(), gv.data_ptr()))
    assert E == ref.energy_ptr(y.data_ptr(), vt.data_ptr(), gy.data_ptr(), gv.data_ptr())


def test_the_hook_rejects_bad_arguments():
    assert pkg.lib().fppg_debug_fail_allocation(-2) == pkg.ERR_ARG
    assert pkg.lib().fppg_debug_fail_allocation(-1) == pkg.OK
