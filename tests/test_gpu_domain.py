"""The spatial decomposition on the GPU path: two ranks (processes) drive
their own bodies through the C ABI (ghosts, the two halves of an
iteration) and exchange over gloo; the run on one GPU holds both ranks, as
the ranks never wait on each other inside a kernel (every exchange is on the
host between launches).  Against one body relaxed alone: the same
neighbours, time step and projections, so the positions agree to the FP32
rounding of the force sums, whose order differs."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

pytestmark = pytest.mark.gpu


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, iters, out):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    torch.cuda.set_device(0)
    import paper_2501_03056_gb300 as pkg
    from paper_2501_03056_gb300 import domain as D
    from paper_2501_03056_gb300 import workloads as W
    a = W.cube_workload()[0]
    b = pkg.Body.from_assembly(a)
    x0, c0, cons0 = b.get_particles()
    dom = D.SlabDomain(D.BodyEngine(b), x0, c0, cons0, a.h)
    dom.relax(iters)
    x, cons = dom.gather()
    out[rank] = (x, cons, dom.ghosts_received, dom.migrated_in)
    dist.barrier()
    dist.destroy_process_group()


def test_decomposed_relaxation_on_the_gpu_matches_one_body():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2501_03056_gb300 import _build
    _build.build()
    import paper_2501_03056_gb300 as pkg
    from paper_2501_03056_gb300 import workloads as W
    iters = 10
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, iters, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(600)
    assert all(p.exitcode == 0 for p in procs)
    a = W.cube_workload()[0]
    ref = pkg.Body.from_assembly(a)
    ref.relax(iters)
    rx, _, rcons = ref.get_particles()
    x, cons, gh, mig = out[0]
    assert np.array_equal(x, out[1][0])
    assert gh > 0 and out[1][2] > 0
    err = np.abs(x.astype(np.float64) - rx).max(axis=1) / a.dx
    assert np.quantile(err, 0.999) < 2e-5 and err.max() < 1e-3, err.max()
    assert (cons == rcons).mean() > 0.999
