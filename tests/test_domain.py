"""Spatial decomposition over ranks (host logic on CPU, world size 2 over
gloo): slabs along z, ghosts within 2h of each shared face, the largest
force reduced over the ranks, migration across faces.  Each rank's engine
is the FP64 oracle here, so the decomposed relaxation must equal the
single-domain oracle up to the order of the force sums."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle as O
from paper_2501_03056_gb300 import domain as D
from paper_2501_03056_gb300 import workloads as W


class OracleEngine:
    """The oracle as a rank's engine (test only)."""

    def __init__(self, a):
        self.o = O.Oracle(a.verts, a.tris, a.dx, a.h)
        if a.dihedral_deg is not None:
            self.o.extract_features(a.dihedral_deg)

    def set(self, xyz, cls, cons, n_ghost):
        self.o.set_particles(np.asarray(xyz, np.float32), cls)
        self.o.set_state(np.asarray(xyz, np.float64), cons)
        self.o.set_ghost_count(n_ghost)

    def forces(self):
        return self.o.relax_forces()

    def step(self, amax):
        self.o.relax_step(amax)

    def get(self):
        x, _, cons = self.o.get_particles()
        return x, cons


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, iters, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    O.set_threads(2)
    a = W.cube_workload()[0]
    ref = O.from_assembly(a)
    x0, c0, cons0 = ref.get_particles()
    dom = D.SlabDomain(OracleEngine(a), x0, c0, cons0, a.h)
    owned0 = len(dom.gid)
    dom.relax(iters)
    x, cons = dom.gather()
    out[rank] = (x, cons, owned0, dom.ghosts_received, dom.migrated_in)
    dist.barrier()
    dist.destroy_process_group()


def test_decomposed_relaxation_equals_one_domain():
    iters = 20
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, iters, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(300)
    assert all(p.exitcode == 0 for p in procs)
    a = W.cube_workload()[0]
    ref = O.from_assembly(a)
    ref.relax(iters)
    rx, _, rcons = ref.get_particles()
    x0, cons0, own0, gh0, mig0 = out[0]
    x1, cons1, own1, gh1, mig1 = out[1]
    assert np.array_equal(x0, x1) and np.array_equal(cons0, cons1)   # every rank gathers the same
    assert own0 + own1 == a.n and min(own0, own1) > 0.4 * a.n         # balanced slabs
    assert min(gh0, gh1) > 20 * 1000                                 # ghosts every iteration
    assert mig0 + mig1 > 0                                           # and particles crossed the face
    err = np.abs(x0 - rx).max(axis=1) / a.dx
    # the same neighbours, time step and projections; only the order of the
    # FP64 force sums differs
    assert err.max() < 1e-9, err.max()
    assert np.array_equal(cons0, rcons)


def test_slab_faces_and_owners():
    z = np.linspace(-1, 1, 1001)
    f = D.slab_faces(z, 4)
    assert f[0] == -np.inf and f[-1] == np.inf and np.all(np.diff(f) > 0)
    own = D.owner_of(z, f)
    counts = np.bincount(own, minlength=4)
    assert counts.sum() == len(z) and counts.min() >= 240
    assert D.owner_of([f[2]], f)[0] == 2          # a point on a face belongs to the slab above it
