"""Spatial decomposition of one body over several processes (one per GPU).

The relaxation is local: a particle feels only the particles within 2h
(Eq. 15), and the only global quantity of an iteration is the largest force,
which fixes the shared time step (Eqs. 22-23).  So the body is cut into
slabs along z, one per rank, and every iteration of Algorithm 1 becomes:

1. halo exchange: each rank sends the particles it owns within ``halo``
   (>= 2h) of a face it shares to the neighbour behind that face, which
   appends them to its own particles as ghosts (they act by their class and
   never move);
2. the force half of the iteration (grid, Eq. 15) on every rank, then the
   largest force reduced over the ranks (all-reduce max);
3. the step half with that maximum (Eqs. 22-25 and the projections);
4. migration: an owned particle whose z left the slab goes to the rank whose
   slab holds it.

Every owned particle therefore sees exactly the neighbours it sees in one
domain, moves with the same time step and is projected on the same mesh:
the result equals the single-domain relaxation up to the order of the force
sums.  The engine of a rank is anything with ``set(xyz, cls, cons,
n_ghost)``, ``forces() -> amax``, ``step(amax)`` and ``get() -> (xyz,
cons)``; ``BodyEngine`` drives this library's C ABI on the rank's GPU.
Exchanges go through ``torch.distributed`` (any backend).
"""
from __future__ import annotations

import numpy as np


class BodyEngine:
    """A rank's engine on a ``Body`` (fppg_set_ghost_count,
    fppg_relax_forces, fppg_relax_step)."""

    def __init__(self, body):
        self.body = body

    def set(self, xyz, cls, cons, n_ghost):
        self.body.set_particles(xyz, cls)
        self.body.set_constraints(cons)
        self.body.set_ghost_count(n_ghost)

    def forces(self) -> float:
        return self.body.relax_forces()

    def step(self, amax: float):
        self.body.relax_step(amax)

    def get(self):
        x, _, cons = self.body.get_particles()
        return x, cons


def slab_faces(z, world):
    """z planes of `world` slabs holding about equal numbers of particles
    (faces[0] = -inf, faces[world] = +inf)."""
    z = np.asarray(z, np.float64)
    inner = np.quantile(z, np.arange(1, world) / world) if len(z) else np.zeros(world - 1)
    return np.concatenate([[-np.inf], inner, [np.inf]])


def owner_of(z, faces):
    """Rank whose slab [faces[r], faces[r + 1]) holds each z."""
    return np.searchsorted(faces, np.asarray(z, np.float64), side="right") - 1


class SlabDomain:
    """The particles this rank owns, with their global ids, and the
    exchanges of an iteration.

    xyz, cls, cons: the whole initial set (every rank passes the same);
    h: the smoothing length (the halo is 2h times (1 + 2^-8));
    group: a ``torch.distributed`` process group (None: the default).
    """

    def __init__(self, engine, xyz, cls, cons, h, group=None):
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)
        self.engine = engine
        xyz = np.ascontiguousarray(xyz)           # the engine's precision (FP32 on a GPU)
        self.faces = slab_faces(xyz[:, 2], self.world)
        self.halo = 2.0 * float(h) * (1.0 + 2.0 ** -8)
        inner = np.diff(self.faces[1:-1])
        if len(inner) and inner.min() <= self.halo:
            raise ValueError("slabs thinner than 2h: use fewer ranks for this body")
        own = owner_of(xyz[:, 2], self.faces) == self.rank
        self.gid = np.nonzero(own)[0].astype(np.int64)
        self.xyz = xyz[own]
        self.cls = np.ascontiguousarray(cls, np.int32)[own]
        self.cons = np.ascontiguousarray(cons, np.int32)[own]
        self.n_total = len(xyz)
        self.ghosts_received = 0     # ghosts received over all iterations
        self.migrated_in = 0         # particles that moved into this slab

    # ---- exchanges ----------------------------------------------------------
    def _exchange(self, outgoing):
        """outgoing: {rank: payload}; returns the payloads sent to this rank."""
        got = [None] * self.world
        self.dist.all_gather_object(got, outgoing, group=self.group)
        return [g[self.rank] for g in got if g is not None and self.rank in g]

    def _max(self, v):
        import torch
        backend = self.dist.get_backend(self.group)
        t = torch.tensor([float(v)], dtype=torch.float64, device="cuda" if backend == "nccl" else "cpu")
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX, group=self.group)
        return float(t.item())

    def halo_out(self):
        """The owned particles within the halo of each shared face, per
        neighbour rank."""
        out = {}
        z = self.xyz[:, 2].astype(np.float64)
        for nb in (self.rank - 1, self.rank + 1):
            if nb < 0 or nb >= self.world:
                continue
            face = self.faces[self.rank] if nb < self.rank else self.faces[self.rank + 1]
            near = np.abs(z - face) <= self.halo
            out[nb] = (self.xyz[near], self.cls[near])
        return out

    # ---- one iteration ------------------------------------------------------
    def iterate(self):
        ghosts = self._exchange(self.halo_out())
        gx = [self.xyz] + [g[0] for g in ghosts]
        gc = [self.cls] + [g[1] for g in ghosts]
        n_ghost = sum(len(g[1]) for g in ghosts)
        self.ghosts_received += n_ghost
        xyz = np.concatenate(gx)
        cls = np.concatenate(gc).astype(np.int32)
        cons = np.concatenate([self.cons, np.full(n_ghost, -1, np.int32)])
        self.engine.set(xyz, cls, cons, n_ghost)
        amax = self._max(self.engine.forces())
        self.engine.step(amax)
        x, c = self.engine.get()
        n_own = len(self.gid)
        self.xyz, self.cons = np.ascontiguousarray(x[:n_own]), np.ascontiguousarray(c[:n_own])
        self._migrate()
        return amax

    def _migrate(self):
        dest = owner_of(self.xyz[:, 2], self.faces)
        stay = dest == self.rank
        out = {}
        for r in np.unique(dest[~stay]):
            m = dest == r
            out[int(r)] = (self.gid[m], self.xyz[m], self.cls[m], self.cons[m])
        arrivals = self._exchange(out)
        self.migrated_in += sum(len(a[0]) for a in arrivals)
        self.gid = np.concatenate([self.gid[stay]] + [a[0] for a in arrivals])
        self.xyz = np.concatenate([self.xyz[stay]] + [a[1] for a in arrivals])
        self.cls = np.concatenate([self.cls[stay]] + [a[2] for a in arrivals]).astype(np.int32)
        self.cons = np.concatenate([self.cons[stay]] + [a[3] for a in arrivals]).astype(np.int32)

    def relax(self, n_iter):
        for _ in range(int(n_iter)):
            self.iterate()

    def gather(self):
        """(xyz, cons) of every particle in global id order, on every rank."""
        got = [None] * self.world
        self.dist.all_gather_object(got, (self.gid, self.xyz, self.cons), group=self.group)
        xyz = np.zeros((self.n_total, 3), self.xyz.dtype)
        cons = np.zeros(self.n_total, np.int32)
        for gid, x, c in got:
            xyz[gid] = x
            cons[gid] = c
        return xyz, cons
