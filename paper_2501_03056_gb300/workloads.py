"""Seeded synthetic inputs for the FPPG relaxation path.

This module only *makes inputs*: triangle meshes (cube, icosphere, torus,
cylinder, spur gear) and the initial particle sets that sit on or inside them
(lattices plus a counter-based jitter).  It holds none of the relaxation
arithmetic -- no kernel, no force, no projection onto triangles, no feature
extraction.  Both the CUDA library and the FP64 oracle consume exactly the
arrays produced here, so the two sides always see identical data.

Particle classes (shared vocabulary of the whole package, Sec. 3.3 and
Sec. 3.3.4 of the paper):

* ``S`` = 0  surface particle (mapped to the closest projectable triangle)
* ``V`` = 1  volume particle that relaxes (the "intermediate" layer)
* ``F`` = 2  feature-line particle (moves along its polyline)
* ``I`` = 3  innermost volume particle (fixed)
* ``P`` = 4  singular feature point (fixed)

Jitter is a counter-based stream: splitmix64 (Steele, Lea and Flood, 2014) of
the 64-bit counter ``seed * 2**32 + 4 * id + axis``; the top 53 bits give a
uniform number in [0, 1).
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np

CLS_S, CLS_V, CLS_F, CLS_I, CLS_P = 0, 1, 2, 3, 4
CLASS_NAMES = {CLS_S: "S", CLS_V: "V", CLS_F: "F", CLS_I: "I", CLS_P: "P"}

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)


# --------------------------------------------------------------------------
# counter-based random numbers
# --------------------------------------------------------------------------
def splitmix64(x: np.ndarray) -> np.ndarray:
    """splitmix64 finaliser applied element-wise to uint64 counters."""
    x = np.asarray(x, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = x + np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, ids: np.ndarray, axis: int) -> np.ndarray:
    """U[0,1) for each particle id on one axis (0, 1, 2), counter-based."""
    ids = np.asarray(ids, dtype=np.uint64)
    with np.errstate(over="ignore"):
        ctr = np.uint64(seed) * np.uint64(1 << 32) + ids * np.uint64(4) + np.uint64(axis)
    z = splitmix64(ctr)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def jitter(seed: int, ids: np.ndarray, axis: int, amp: float) -> np.ndarray:
    """Uniform offsets in [-amp, amp)."""
    return (2.0 * uniform01(seed, ids, axis) - 1.0) * amp


# --------------------------------------------------------------------------
# meshes (outward-facing, counter-clockwise seen from outside)
# --------------------------------------------------------------------------
def _orient_outward(verts: np.ndarray, tris: np.ndarray, inside_point) -> np.ndarray:
    """Flip triangles whose winding points towards ``inside_point``."""
    v = verts.astype(np.float64)
    a, b, c = v[tris[:, 0]], v[tris[:, 1]], v[tris[:, 2]]
    nrm = np.cross(b - a, c - a)
    cen = (a + b + c) / 3.0
    flip = np.einsum("ij,ij->i", nrm, cen - np.asarray(inside_point, dtype=np.float64)) < 0
    out = tris.copy()
    out[flip, 1], out[flip, 2] = tris[flip, 2], tris[flip, 1]
    return out


def cube_mesh(half: float = 0.5):
    """Axis-aligned cube [-half, half]^3 as 12 triangles."""
    verts = np.array([[(i & 1) * 2 - 1, ((i >> 1) & 1) * 2 - 1, ((i >> 2) & 1) * 2 - 1]
                      for i in range(8)], dtype=np.float64) * half
    tris = []
    for axis in range(3):
        for sgn in (0, 1):
            quad = [i for i in range(8) if ((i >> axis) & 1) == sgn]
            o1, o2 = [ax for ax in range(3) if ax != axis]
            # order the four corners around the face
            ang = [math.atan2(verts[i, o2], verts[i, o1]) for i in quad]
            quad = [q for _, q in sorted(zip(ang, quad))]
            tris.append([quad[0], quad[1], quad[2]])
            tris.append([quad[0], quad[2], quad[3]])
    tris = np.array(tris, dtype=np.int32)
    tris = _orient_outward(verts, tris, (0.0, 0.0, 0.0))
    return verts.astype(np.float32), tris.astype(np.int32)


def icosphere_mesh(level: int, radius: float = 1.0):
    """Icosahedron refined ``level`` times by edge midpoints pushed to the sphere."""
    phi = (1.0 + 5.0 ** 0.5) / 2.0
    base = []
    for s1 in (-1.0, 1.0):
        for s2 in (-1.0, 1.0):
            base += [(0.0, s1, s2 * phi), (s1, s2 * phi, 0.0), (s2 * phi, 0.0, s1)]
    v = np.array(base, dtype=np.float64)
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    # faces: triples of mutually adjacent vertices (edge = shortest distance)
    d = np.linalg.norm(v[:, None, :] - v[None, :, :], axis=2)
    emin = np.min(d[d > 1e-9])
    adj = np.abs(d - emin) < 1e-6
    faces = []
    for i in range(12):
        for j in range(i + 1, 12):
            if not adj[i, j]:
                continue
            for k in range(j + 1, 12):
                if adj[i, k] and adj[j, k]:
                    faces.append([i, j, k])
    tris = _orient_outward(v, np.array(faces, dtype=np.int64), (0.0, 0.0, 0.0))
    verts = [tuple(p) for p in v]
    for _ in range(level):
        cache = {}

        def mid(a, b):
            key = (a, b) if a < b else (b, a)
            if key not in cache:
                p = (np.asarray(verts[a]) + np.asarray(verts[b])) * 0.5
                p /= np.linalg.norm(p)
                cache[key] = len(verts)
                verts.append(tuple(p))
            return cache[key]

        new = []
        for a, b, c in tris:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            new += [[a, ab, ca], [b, bc, ab], [c, ca, bc], [ab, bc, ca]]
        tris = np.array(new, dtype=np.int64)
    verts = np.array(verts, dtype=np.float64) * radius
    return verts.astype(np.float32), tris.astype(np.int32)


def torus_mesh(R: float = 1.0, r: float = 0.3, nu: int = 256, nv: int = 64):
    """Torus around the z axis from an nu x nv grid of (u, v) quads."""
    u = 2.0 * np.pi * np.arange(nu) / nu
    v = 2.0 * np.pi * np.arange(nv) / nv
    uu, vv = np.meshgrid(u, v, indexing="ij")
    rho = R + r * np.cos(vv)
    verts = np.stack([rho * np.cos(uu), rho * np.sin(uu), r * np.sin(vv)], axis=-1).reshape(-1, 3)
    idx = lambda i, j: (i % nu) * nv + (j % nv)  # noqa: E731
    tris = []
    for i in range(nu):
        for j in range(nv):
            a, b, c, d = idx(i, j), idx(i + 1, j), idx(i + 1, j + 1), idx(i, j + 1)
            tris += [[a, b, c], [a, c, d]]
    return verts.astype(np.float32), np.array(tris, dtype=np.int32)


def cylinder_mesh(radius: float = 0.5, height: float = 1.0, n: int = 64, nz: int = 8):
    """Closed cylinder along z with capped ends (fan around the cap centres)."""
    ang = 2.0 * np.pi * np.arange(n) / n
    zs = np.linspace(-height / 2, height / 2, nz + 1)
    verts = [(radius * math.cos(a), radius * math.sin(a), z) for z in zs for a in ang]
    tris = []
    for k in range(nz):
        for i in range(n):
            a, b = k * n + i, k * n + (i + 1) % n
            c, d = (k + 1) * n + (i + 1) % n, (k + 1) * n + i
            tris += [[a, b, c], [a, c, d]]
    bot = len(verts)
    verts.append((0.0, 0.0, -height / 2))
    top = len(verts)
    verts.append((0.0, 0.0, height / 2))
    for i in range(n):
        tris.append([bot, (i + 1) % n, i])
        tris.append([top, nz * n + i, nz * n + (i + 1) % n])
    verts = np.array(verts, dtype=np.float64)
    tris = _orient_outward(verts, np.array(tris, dtype=np.int64), (0.0, 0.0, 0.0))
    return verts.astype(np.float32), tris.astype(np.int32)


def gear_profile(teeth: int = 40, r_out: float = 1.0, r_root: float = 0.9,
                 pts_per_tooth: int = 4):
    """Closed 2-D outline of a spur gear with trapezoidal teeth.

    Each tooth pitch is split into root land, rising flank, tip land and
    falling flank (equal angular quarters); returns (x, y) vertices in
    counter-clockwise order."""
    pitch = 2.0 * np.pi / teeth
    out = []
    for t in range(teeth):
        a0 = t * pitch
        # root land: quarter pitch; flank; tip land; flank
        for k in range(pts_per_tooth):
            out.append((r_root, a0 + 0.25 * pitch * k / pts_per_tooth))
        out.append((r_root, a0 + 0.25 * pitch))
        for k in range(pts_per_tooth):
            out.append((r_out, a0 + 0.5 * pitch + 0.25 * pitch * k / pts_per_tooth))
        out.append((r_out, a0 + 0.75 * pitch))
    xy = np.array([(r * math.cos(a), r * math.sin(a)) for r, a in out], dtype=np.float64)
    return xy


def _zipper(inner, outer, ai, ao):
    """Triangles between two closed rings whose angles increase from 0 to
    2 pi (star-shaped about the axis): walk both rings in angle order."""
    ni, no = len(inner), len(outer)
    ti = np.r_[ai, ai[0] + 2 * np.pi]
    to = np.r_[ao, ao[0] + 2 * np.pi]
    i = j = 0
    tris = []
    while i < ni or j < no:
        if j >= no or (i < ni and ti[i + 1] <= to[j + 1]):
            tris.append([inner[i % ni], outer[j % no], inner[(i + 1) % ni]])
            i += 1
        else:
            tris.append([inner[i % ni], outer[j % no], outer[(j + 1) % no]])
            j += 1
    return tris


def gear_mesh(teeth: int = 40, r_out: float = 1.0, r_root: float = 0.9, r_bore: float = 0.3,
              height: float = 0.3, pts_per_tooth: int = 6, rings: int = 20, nz: int = 12,
              bore_points: int = 240):
    """Closed spur gear: trapezoidal teeth extruded along z, with a bore.

    Top and bottom faces are rings of points (bore circle, intermediate
    circles, tooth outline) joined by a zipper; the outer wall and the bore
    wall are nz layers of quads.  Outward orientation by construction."""
    outline = gear_profile(teeth, r_out, r_root, pts_per_tooth)
    ang_o = np.mod(np.arctan2(outline[:, 1], outline[:, 0]), 2 * np.pi)
    ring_xy, ring_ang = [], []
    radii = np.linspace(r_bore, 0.98 * r_root, rings)
    for k, r in enumerate(radii):
        n = int(round(bore_points + (len(outline) - bore_points) * k / max(rings - 1, 1)))
        a = 2.0 * np.pi * np.arange(n) / n
        ring_xy.append(np.stack([r * np.cos(a), r * np.sin(a)], 1))
        ring_ang.append(a)
    ring_xy.append(outline)
    ring_ang.append(ang_o)
    verts, tris = [], []
    zs = np.linspace(-height / 2, height / 2, nz + 1)
    # face rings at the two ends
    face_ids = {}
    for side, z in ((0, zs[0]), (1, zs[-1])):
        ids = []
        for xy in ring_xy:
            start = len(verts)
            verts.extend([(x, y, z) for x, y in xy])
            ids.append(np.arange(start, start + len(xy)))
        face_ids[side] = ids
        for k in range(len(ring_xy) - 1):
            t = _zipper(ids[k], ids[k + 1], ring_ang[k], ring_ang[k + 1])
            # zipper triangles are counter-clockwise seen from +z
            tris.extend(t if side == 1 else [[a, c, b] for a, b, c in t])
    # walls: interior layers get new vertices, the end layers reuse the rings
    def wall(ring, outward):
        m = len(ring_xy[ring])
        layers = [face_ids[0][ring]]
        for z in zs[1:-1]:
            start = len(verts)
            verts.extend([(x, y, z) for x, y in ring_xy[ring]])
            layers.append(np.arange(start, start + m))
        layers.append(face_ids[1][ring])
        for k in range(nz):
            lo, hi = layers[k], layers[k + 1]
            for i in range(m):
                a, b, c, d = lo[i], lo[(i + 1) % m], hi[(i + 1) % m], hi[i]
                tris.extend([[a, b, c], [a, c, d]] if outward else [[a, c, b], [a, d, c]])
    wall(len(ring_xy) - 1, True)      # tooth outline: counter-clockwise ring, outward
    wall(0, False)                    # bore: the solid lies outside the circle
    return np.array(verts, dtype=np.float32), np.array(tris, dtype=np.int32)


# --------------------------------------------------------------------------
# particle sets
# --------------------------------------------------------------------------
@dataclass
class Assembly:
    """One body: its mesh, spacing and initial particles.

    ``xyz``/``cls`` are None for bodies whose initial particles come from
    the method's own generation (Sec. 3.2); ``meta["generate"]`` then holds
    its options (band_cells, inner_cells)."""
    name: str
    verts: np.ndarray          # float32 [nv, 3]
    tris: np.ndarray           # int32 [nt, 3]
    dx: float
    h: float
    xyz: np.ndarray | None     # float32 [n, 3]
    cls: np.ndarray | None     # int32 [n]
    dihedral_deg: float | None = None   # feature threshold; None = no features
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return 0 if self.xyz is None else int(self.xyz.shape[0])


def smoothing_length(dx: float, factor: float = 1.3) -> float:
    """h = 1.3 dx rounded to FP32 (the value both sides receive)."""
    return float(np.float32(factor * dx))


def cube_particles(dx: float = 0.05, seed: int = 0, half: float = 0.5):
    """Face lattices (S), edge points (F), corners (P) and a volume lattice (V).

    S: n x n per face at (k + 1/2) dx with in-plane jitter; F: the n - 1
    interior edge points at k dx with jitter along the edge; P: the 8 corners;
    V: the n^3 lattice at (k + 1/2) dx with 3-D jitter; jitter +-0.25 dx."""
    n = int(round(2 * half / dx))
    amp = 0.25 * dx
    xyz, cls = [], []
    # S
    k = (np.arange(n) + 0.5) * dx - half
    g1, g2 = np.meshgrid(k, k, indexing="ij")
    g1, g2 = g1.ravel(), g2.ravel()
    for axis in range(3):
        for sgn in (-1.0, 1.0):
            o1, o2 = [ax for ax in range(3) if ax != axis]
            p = np.zeros((g1.size, 3))
            p[:, axis] = sgn * half
            p[:, o1] = g1
            p[:, o2] = g2
            xyz.append(p)
            cls.append(np.full(g1.size, CLS_S))
    # F (interior points of the 12 edges)
    t = np.arange(1, n) * dx - half
    for axis in range(3):
        o1, o2 = [ax for ax in range(3) if ax != axis]
        for s1 in (-1.0, 1.0):
            for s2 in (-1.0, 1.0):
                p = np.zeros((t.size, 3))
                p[:, axis] = t
                p[:, o1] = s1 * half
                p[:, o2] = s2 * half
                xyz.append(p)
                cls.append(np.full(t.size, CLS_F))
    # P (corners)
    corners = np.array([[(i & 1) * 2 - 1, ((i >> 1) & 1) * 2 - 1, ((i >> 2) & 1) * 2 - 1]
                        for i in range(8)], dtype=np.float64) * half
    xyz.append(corners)
    cls.append(np.full(8, CLS_P))
    # V
    gx, gy, gz = np.meshgrid(k, k, k, indexing="ij")
    xyz.append(np.stack([gx.ravel(), gy.ravel(), gz.ravel()], axis=1))
    cls.append(np.full(gx.size, CLS_V))

    xyz = np.concatenate(xyz).astype(np.float64)
    cls = np.concatenate(cls).astype(np.int32)
    ids = np.arange(xyz.shape[0])
    jit = np.stack([jitter(seed, ids, a, amp) for a in range(3)], axis=1)
    # S: in-plane jitter only; F: along-edge jitter only; P: none; V: 3-D.
    on_face = np.abs(np.abs(xyz) - half) < 1e-12
    mask = np.ones_like(xyz)
    mask[cls == CLS_P] = 0.0
    sel = (cls == CLS_S) | (cls == CLS_F)
    mask[sel] = (~on_face[sel]).astype(np.float64)
    xyz = xyz + jit * mask
    return xyz.astype(np.float32), cls


def _tangent_frame(p: np.ndarray):
    """Two unit tangents orthogonal to the unit radial direction of p."""
    nrm = p / np.linalg.norm(p, axis=1, keepdims=True)
    ref = np.where(np.abs(nrm[:, 2:3]) < 0.9, np.array([[0.0, 0.0, 1.0]]), np.array([[1.0, 0.0, 0.0]]))
    e1 = np.cross(ref, nrm)
    e1 /= np.linalg.norm(e1, axis=1, keepdims=True)
    e2 = np.cross(nrm, e1)
    return e1, e2


def _lattice_box(lo, hi, dx):
    ax = [np.arange(math.floor(lo[i] / dx), math.ceil(hi[i] / dx) + 1) * dx for i in range(3)]
    g = np.meshgrid(*ax, indexing="ij")
    return np.stack([c.ravel() for c in g], axis=1)


def sphere_particles(dx: float = 0.02, seed: int = 1, radius: float = 1.0,
                     band: float | None = None):
    """Fibonacci points on the sphere (S) plus a cubic volume lattice (V/I).

    Volume points keep at least dx/2 from the analytic surface.  With
    ``band`` set, points deeper than ``band`` below the surface are class I
    (fixed innermost layer); otherwise every volume point is V."""
    amp = 0.25 * dx
    ns = int(round(4.0 * np.pi * radius * radius / (dx * dx)))
    k = np.arange(ns, dtype=np.float64)
    z = 1.0 - (2.0 * k + 1.0) / ns
    rho = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    ga = np.pi * (3.0 - 5.0 ** 0.5)
    phi = k * ga
    s = np.stack([rho * np.cos(phi), rho * np.sin(phi), z], axis=1) * radius
    ids = np.arange(ns)
    e1, e2 = _tangent_frame(s)
    s = s + e1 * jitter(seed, ids, 0, amp)[:, None] + e2 * jitter(seed, ids, 1, amp)[:, None]
    s *= radius / np.linalg.norm(s, axis=1, keepdims=True)

    v = _lattice_box((-radius,) * 3, (radius,) * 3, dx)
    depth = radius - np.linalg.norm(v, axis=1)
    keep = depth >= 0.5 * dx
    v, depth = v[keep], depth[keep]
    ids = np.arange(ns, ns + v.shape[0])
    v = v + np.stack([jitter(seed, ids, a, amp) for a in range(3)], axis=1)
    vcls = np.full(v.shape[0], CLS_V, dtype=np.int32)
    if band is not None:
        vcls[depth >= band] = CLS_I
    xyz = np.concatenate([s, v]).astype(np.float32)
    cls = np.concatenate([np.full(ns, CLS_S, dtype=np.int32), vcls])
    return xyz, cls


def torus_particles(dx: float = 0.02, seed: int = 2, R: float = 1.0, r: float = 0.3,
                    band: float | None = None):
    """Rings of surface points of equal spacing (S) plus a volume lattice (V/I)."""
    amp = 0.25 * dx
    nv = int(round(2.0 * np.pi * r / dx))
    pts = []
    for j in range(nv):
        v = 2.0 * np.pi * (j + 0.5) / nv
        rho = R + r * math.cos(v)
        nu = max(3, int(round(2.0 * np.pi * rho / dx)))
        u = 2.0 * np.pi * (np.arange(nu) + 0.5 * (j % 2)) / nu
        pts.append(np.stack([u, np.full(nu, v)], axis=1))
    uv = np.concatenate(pts)
    ns = uv.shape[0]
    ids = np.arange(ns)
    u, v = uv[:, 0], uv[:, 1]
    rho = R + r * np.cos(v)
    u = u + jitter(seed, ids, 0, amp) / rho
    v = v + jitter(seed, ids, 1, amp) / r
    rho = R + r * np.cos(v)
    s = np.stack([rho * np.cos(u), rho * np.sin(u), r * np.sin(v)], axis=1)

    vol = _lattice_box((-(R + r), -(R + r), -r), (R + r, R + r, r), dx)
    tube = np.sqrt((np.sqrt(vol[:, 0] ** 2 + vol[:, 1] ** 2) - R) ** 2 + vol[:, 2] ** 2)
    depth = r - tube
    keep = depth >= 0.5 * dx
    vol, depth = vol[keep], depth[keep]
    ids = np.arange(ns, ns + vol.shape[0])
    vol = vol + np.stack([jitter(seed, ids, a, amp) for a in range(3)], axis=1)
    vcls = np.full(vol.shape[0], CLS_V, dtype=np.int32)
    if band is not None:
        vcls[depth >= band] = CLS_I
    xyz = np.concatenate([s, vol]).astype(np.float32)
    cls = np.concatenate([np.full(ns, CLS_S, dtype=np.int32), vcls])
    return xyz, cls


# --------------------------------------------------------------------------
# named workloads
# --------------------------------------------------------------------------
def cube_workload(seed: int = 0, dx: float = 0.05) -> list[Assembly]:
    """Unit cube, 12 triangles, dx = 0.05, h = 1.3 dx, 100 iterations.

    ~2,400 surface, 228 edge, 8 corner and 8,000 volume particles with
    +-0.25 dx jitter; features at a 30 degree threshold (the 12 cube edges)."""
    v, t = cube_mesh()
    xyz, cls = cube_particles(dx, seed)
    return [Assembly("cube", v, t, float(np.float32(dx)), smoothing_length(dx), xyz, cls,
                     dihedral_deg=30.0, meta={"n_iter": 100})]


def sphere_torus_workload(seed: int = 1, dx: float = 0.02, level: int = 5,
                          torus_nu: int = 256, torus_nv: int = 64) -> list[Assembly]:
    """Icosphere r = 1 (level 5, 20,480 triangles) and torus R = 1, r = 0.3
    (256 x 64 quads, 32,768 triangles) at dx = 0.02, relaxed for 500 iterations."""
    sv, st = icosphere_mesh(level)
    sx, sc = sphere_particles(dx, seed)
    tv, tt = torus_mesh(1.0, 0.3, torus_nu, torus_nv)
    tx, tc = torus_particles(dx, seed + 100)
    dxf = float(np.float32(dx))
    return [Assembly("icosphere", sv, st, dxf, smoothing_length(dx), sx, sc, None, {"n_iter": 500}),
            Assembly("torus", tv, tt, dxf, smoothing_length(dx), tx, tc, None, {"n_iter": 500})]


def gear_workload(dx: float = 0.004) -> list[Assembly]:
    """Spur gear: 40 trapezoidal teeth, outer r = 1, root r = 0.9, bore
    r = 0.3, height 0.3 (51,840 triangles), 30 degree features, dx = 0.004;
    particles from the generation of Sec. 3.2 with a band of 2 cells of
    relaxing volume particles and 1 cell of fixed innermost ones (~2.4 M)."""
    v, t = gear_mesh()
    dxf = float(np.float32(dx))
    return [Assembly("gear", v, t, dxf, smoothing_length(dx), None, None, 30.0,
                     {"n_iter": 500, "generate": {"band_cells": 2, "inner_cells": 1}})]


def batch_workload(seed: int = 3, bodies: int = 64, dx: float = 0.008) -> list[Assembly]:
    """Batch of bodies of uneven size: cubes, cylinders, icospheres and gears
    at seeded scales 0.1-1 (uniform), one spacing dx; particles from the
    generation of Sec. 3.2 with a 3-cell relaxing band and a 1-cell fixed
    innermost layer (a few thousand to ~470 k particles per body)."""
    shapes = ("cube", "cylinder", "sphere", "gear")
    u = uniform01(seed, np.arange(bodies), 0)
    kind = (uniform01(seed, np.arange(bodies), 1) * len(shapes)).astype(int)
    dxf = float(np.float32(dx))
    meshes = {"cube": cube_mesh(0.5), "cylinder": cylinder_mesh(0.5, 1.0, 64, 8), "sphere": icosphere_mesh(4, 0.5),
              "gear": gear_mesh(teeth=24, r_out=0.5, r_root=0.45, r_bore=0.15, height=0.2, pts_per_tooth=4,
                                rings=8, nz=6, bore_points=96)}
    out = []
    for b in range(bodies):
        scale = 0.1 + 0.9 * float(u[b])
        name = shapes[kind[b]]
        v, t = meshes[name]
        out.append(Assembly(f"{name}{b}", (v.astype(np.float64) * scale).astype(np.float32), t, dxf,
                            smoothing_length(dx), None, None, 30.0,
                            {"n_iter": 50, "scale": scale, "generate": {"band_cells": 3, "inner_cells": 1}}))
    return out


def union_pair_workload(seed: int = 5, dx: float = 0.05) -> list[Assembly]:
    """Two overlapping bodies for the Boolean union (Sec. 3.2.3): the unit
    cube [-0.5, 0.5]^3 (lattice particles as the unit cube workload, 30 degree features)
    and an icosphere of level 3, r = 0.35, centred at (0.45, 0.05, -0.03)
    (Fibonacci surface points and a volume lattice), so that the sphere pokes
    out of the cube's +x face.  meta["union_with"] names the partner."""
    dxf = float(np.float32(dx))
    cv, ct = cube_mesh()
    cx, cc = cube_particles(dx, seed)
    sv, st = icosphere_mesh(3, 0.35)
    sx, sc = sphere_particles(dx, seed + 1, radius=0.35)
    centre = np.array([0.45, 0.05, -0.03])
    sv = (sv.astype(np.float64) + centre).astype(np.float32)
    sx = (sx.astype(np.float64) + centre).astype(np.float32)
    return [Assembly("cube", cv, ct, dxf, smoothing_length(dx), cx, cc, 30.0, {"n_iter": 100, "union_with": 1}),
            Assembly("sphere", sv, st, dxf, smoothing_length(dx), sx, sc, None, {"n_iter": 100, "union_with": 0})]


def batch_union_workload(seed: int = 3, bodies: int = 64, dx: float = 0.008) -> list[Assembly]:
    """The 64-body batch with its Boolean unions: the 64 bodies of batch_workload,
    except that the body after each gear becomes a shaft through that gear
    (a cylinder of radius 0.2 and height 0.5 at the gear's scale, through the
    bore of radius 0.15, so it overlaps the hub and sticks out on both
    sides); each gear-shaft pair is one union (meta["union_with"])."""
    out = batch_workload(seed, bodies, dx)
    shaft_v, shaft_t = cylinder_mesh(0.2, 0.5, 48, 6)
    b = 0
    while b < len(out) - 1:
        a = out[b]
        if a.name.startswith("gear"):
            scale = a.meta["scale"]
            out[b + 1] = Assembly(f"shaft{b + 1}", (shaft_v.astype(np.float64) * scale).astype(np.float32), shaft_t,
                                  a.dx, a.h, None, None, 30.0,
                                  {"n_iter": 50, "scale": scale, "union_with": b,
                                   "generate": dict(a.meta["generate"])})
            a.meta["union_with"] = b + 1
            b += 2
        else:
            b += 1
    return out


# --------------------------------------------------------------------------
# vehicle-like shell (union of rounded boxes and wheels)
# --------------------------------------------------------------------------
def _sd_round_box(p, centre, half, radius):
    q = np.abs(p - np.asarray(centre)) - (np.asarray(half) - radius)
    outside = np.linalg.norm(np.maximum(q, 0.0), axis=-1)
    inside = np.minimum(np.max(q, axis=-1), 0.0)
    return outside + inside - radius


def _sd_cylinder_y(p, centre, radius, half_width):
    d = p - np.asarray(centre)
    r = np.sqrt(d[..., 0] ** 2 + d[..., 2] ** 2) - radius
    w = np.abs(d[..., 1]) - half_width
    return np.minimum(np.maximum(r, w), 0.0) + np.sqrt(np.maximum(r, 0.0) ** 2 + np.maximum(w, 0.0) ** 2)


def vehicle_sdf(p):
    """Signed distance (approximate inside the union) of a car-like body:
    chassis and cabin as rounded boxes, four wheels as cylinders along y."""
    d = _sd_round_box(p, (0.0, 0.0, 0.55), (2.0, 0.9, 0.3), 0.15)
    d = np.minimum(d, _sd_round_box(p, (-0.2, 0.0, 1.05), (1.1, 0.75, 0.25), 0.2))
    for x in (-1.3, 1.3):
        for y in (-0.85, 0.85):
            d = np.minimum(d, _sd_cylinder_y(p, (x, y, 0.38), 0.36, 0.16))
    return d


def surface_nets(sdf, lo, hi, spacing):
    """Closed triangle mesh of {sdf = 0} by surface nets: one vertex per grid
    cell whose corners change sign (mean of the edge crossings), one quad
    (two triangles) per grid edge that changes sign, wound so that the
    normal points from negative (inside) to positive values."""
    axes = [np.arange(lo[a], hi[a] + spacing, spacing) for a in range(3)]
    n = [len(x) for x in axes]
    G = np.stack(np.meshgrid(*axes, indexing="ij"), -1)
    f = sdf(G)
    f[f == 0.0] = 1e-12
    inside = f < 0
    # cells with a sign change
    cs = np.zeros((n[0] - 1, n[1] - 1, n[2] - 1), dtype=np.int8)
    corners = [(i, j, k) for i in (0, 1) for j in (0, 1) for k in (0, 1)]
    for (i, j, k) in corners:
        cs += inside[i:n[0] - 1 + i, j:n[1] - 1 + j, k:n[2] - 1 + k]
    active = (cs > 0) & (cs < 8)
    idx = -np.ones(active.shape, dtype=np.int64)
    cells = np.argwhere(active)
    idx[active] = np.arange(len(cells))
    # vertex = mean of the crossings on the 12 cell edges
    acc = np.zeros((len(cells), 3))
    cnt = np.zeros(len(cells))
    ci, cj, ck = cells[:, 0], cells[:, 1], cells[:, 2]
    for (a, b) in [((0, 0, 0), (1, 0, 0)), ((0, 1, 0), (1, 1, 0)), ((0, 0, 1), (1, 0, 1)), ((0, 1, 1), (1, 1, 1)),
                   ((0, 0, 0), (0, 1, 0)), ((1, 0, 0), (1, 1, 0)), ((0, 0, 1), (0, 1, 1)), ((1, 0, 1), (1, 1, 1)),
                   ((0, 0, 0), (0, 0, 1)), ((1, 0, 0), (1, 0, 1)), ((0, 1, 0), (0, 1, 1)), ((1, 1, 0), (1, 1, 1))]:
        fa = f[ci + a[0], cj + a[1], ck + a[2]]
        fb = f[ci + b[0], cj + b[1], ck + b[2]]
        ch = (fa < 0) != (fb < 0)
        with np.errstate(divide="ignore", invalid="ignore"):
            t = np.where(ch, fa / np.where(ch, fa - fb, 1.0), 0.0)
        pa = G[ci + a[0], cj + a[1], ck + a[2]]
        pb = G[ci + b[0], cj + b[1], ck + b[2]]
        acc[ch] += (pa + t[:, None] * (pb - pa))[ch]
        cnt[ch] += 1
    verts = acc / cnt[:, None]
    tris = []
    # a grid edge along axis a between points p and p + e_a is shared by the
    # four cells around it; those cells' vertices form the quad
    for a in range(3):
        b, c = (a + 1) % 3, (a + 2) % 3
        sl0 = [slice(None)] * 3
        sl1 = [slice(None)] * 3
        sl0[a] = slice(0, n[a] - 1)
        sl1[a] = slice(1, n[a])
        ch = inside[tuple(sl0)] != inside[tuple(sl1)]
        e = np.argwhere(ch)
        # the four cells: offsets 0/-1 along b and c
        ok = (e[:, b] >= 1) & (e[:, b] <= n[b] - 2) & (e[:, c] >= 1) & (e[:, c] <= n[c] - 2)
        e = e[ok]
        flip = inside[tuple(e.T)]          # inside at the lower end: normal along +a
        def cell(db, dc):
            q = e.copy()
            q[:, b] -= db
            q[:, c] -= dc
            return idx[q[:, 0], q[:, 1], q[:, 2]]
        v00, v10, v11, v01 = cell(1, 1), cell(0, 1), cell(0, 0), cell(1, 0)
        q1 = np.stack([v00, v10, v11], 1)
        q2 = np.stack([v00, v11, v01], 1)
        r1 = np.stack([v00, v11, v10], 1)
        r2 = np.stack([v00, v01, v11], 1)
        tris.append(np.where(flip[:, None], q1, r1))
        tris.append(np.where(flip[:, None], q2, r2))
    return verts, np.concatenate(tris).astype(np.int64)


def loop_subdivide(verts, tris):
    """One step of Loop subdivision (Loop, 1987): edge points 3/8 (a + b) +
    1/8 (c + d), vertex points (1 - n beta) v + beta sum(neighbours) with
    beta = (5/8 - (3/8 + cos(2 pi / n) / 4)^2) / n; each triangle -> 4."""
    v = np.asarray(verts, dtype=np.float64)
    t = np.asarray(tris, dtype=np.int64)
    nv = len(v)
    e = np.concatenate([t[:, [0, 1]], t[:, [1, 2]], t[:, [2, 0]]])
    opp = np.concatenate([t[:, 2], t[:, 0], t[:, 1]])
    key = np.minimum(e[:, 0], e[:, 1]) * nv + np.maximum(e[:, 0], e[:, 1])
    uk, inv = np.unique(key, return_inverse=True)
    ne = len(uk)
    a, b = uk // nv, uk % nv
    osum = np.zeros((ne, 3))
    ocnt = np.zeros(ne)
    np.add.at(osum, inv, v[opp])
    np.add.at(ocnt, inv, 1)
    ep = np.where((ocnt == 2)[:, None], 0.375 * (v[a] + v[b]) + 0.125 * osum, 0.5 * (v[a] + v[b]))
    nsum = np.zeros((nv, 3))
    deg = np.zeros(nv)
    np.add.at(nsum, a, v[b])
    np.add.at(nsum, b, v[a])
    np.add.at(deg, a, 1)
    np.add.at(deg, b, 1)
    beta = (0.625 - (0.375 + 0.25 * np.cos(2 * np.pi / np.maximum(deg, 3))) ** 2) / np.maximum(deg, 1)
    vp = (1 - deg * beta)[:, None] * v + beta[:, None] * nsum
    mid = nv + inv.reshape(3, -1).T             # edge point ids of (ab, bc, ca)
    ab, bc, ca = mid[:, 0], mid[:, 1], mid[:, 2]
    new = np.concatenate([np.stack([t[:, 0], ab, ca], 1), np.stack([t[:, 1], bc, ab], 1),
                          np.stack([t[:, 2], ca, bc], 1), np.stack([ab, bc, ca], 1)])
    return np.vstack([vp, ep]), new


def vehicle_mesh(spacing: float = 0.021, noise: float = 1e-3, seed: int = 5, subdivide: int = 2):
    """Closed vehicle-like shell: surface nets of vehicle_sdf, Loop
    subdivision, then seeded vertex noise of amplitude `noise` along the
    vertex normals (counter-based jitter)."""
    v, t = surface_nets(vehicle_sdf, (-2.4, -1.2, -0.2), (2.4, 1.2, 1.6), spacing)
    for _ in range(subdivide):
        v, t = loop_subdivide(v, t)
    nrm = np.zeros_like(v)
    fn = np.cross(v[t[:, 1]] - v[t[:, 0]], v[t[:, 2]] - v[t[:, 0]])
    for k in range(3):
        np.add.at(nrm, t[:, k], fn)
    nrm /= np.maximum(np.linalg.norm(nrm, axis=1, keepdims=True), 1e-30)
    v = v + nrm * jitter(seed, np.arange(len(v)), 0, noise)[:, None]
    return v.astype(np.float32), t.astype(np.int32)


def vehicle_workload(dx: float = 0.0068, spacing: float = 0.021) -> list[Assembly]:
    """Vehicle-like closed shell (~2 M triangles after two Loop steps, 1e-3
    vertex noise, 30 degree features) at a spacing giving ~20 M surface and
    volume particles from the generation of Sec. 3.2 (every interior cell
    relaxes)."""
    v, t = vehicle_mesh(spacing)
    dxf = float(np.float32(dx))
    return [Assembly("vehicle", v, t, dxf, smoothing_length(dx), None, None, 30.0,
                     {"n_iter": 1000, "generate": {"band_cells": 0, "inner_cells": 0}})]


def sphere_1e8_workload(dx: float = 0.00175, level: int = 7) -> list[Assembly]:
    """The sphere of the paper's scaling table (1 x 1 x 1, Table
    tab-generate) at about 10^8 particles: an icosphere of level 7 (r = 0.5,
    327,680 triangles, edges ~2.7 dx) with surface, feature and every
    interior cell generated by Sec. 3.2 at dx = 0.00175 (about 9.8e7 volume
    and 1.0e6 surface particles)."""
    v, t = icosphere_mesh(level, 0.5)
    dxf = float(np.float32(dx))
    return [Assembly("sphere_1e8", v, t, dxf, smoothing_length(dx), None, None, 30.0,
                     {"n_iter": 50, "generate": {"band_cells": 0, "inner_cells": 0}})]
