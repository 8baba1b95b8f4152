"""ctypes binding of the FP64 CPU oracle (``fppg_oracle.c``).

Test infrastructure only: the test-suite, the smoke check and the benchmark's
CPU-baseline leg use it; the product path never imports it.  The shared
object is compiled with gcc on first use (``-ffp-contract=off`` so that the
FP32 decision arithmetic is never fused).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fppg_oracle.c")
_LIBDIR = os.path.join(_HERE, "_lib")
_LIB = os.path.join(_LIBDIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

CFLAGS = ["-O2", "-std=gnu11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off", "-fno-fast-math"]


def build(force: bool = False) -> str:
    """Compile the oracle if the library is missing or older than its source."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.run(["gcc", *CFLAGS, _SRC, "-o", tmp, "-lm"], check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _p(a, ct):
    return a.ctypes.data_as(C.POINTER(ct)) if a is not None else None


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            vp, i64, i32, f32, f64 = C.c_void_p, C.c_int64, C.c_int32, C.c_float, C.c_double
            P = C.POINTER
            sig = {
                "oracle_alpha3": (f64, [f64]),
                "oracle_W": (f64, [f64, f64]),
                "oracle_dW": (f64, [f64, f64]),
                "oracle_lattice_sum": (f64, [f64, f64, C.c_int]),
                "oracle_morton3": (C.c_uint64, [C.c_uint32, C.c_uint32, C.c_uint32]),
                "oracle_create": (vp, [P(f32), i64, P(i32), i64, f32, f32]),
                "oracle_destroy": (None, [vp]),
                "oracle_set_threads": (None, [C.c_int]),
                "oracle_get_threads": (C.c_int, []),
                "oracle_set_fixed_features": (None, [vp, C.c_int]),
                "oracle_set_mobile_classes": (None, [vp, C.c_int]),
                "oracle_set_cascade": (None, [vp, C.c_int]),
                "oracle_tri_grid": (None, [vp, P(f32), P(f32), P(i32)]),
                "oracle_nbr_grid": (None, [vp, P(f32), P(f32), P(f32), P(i32), P(f32)]),
                "oracle_tri_bins": (i64, [vp, P(i64), P(i32), i64]),
                "oracle_pseudonormals": (None, [vp, P(f32), P(f32), P(f32)]),
                "oracle_extract_features": (i64, [vp, f64]),
                "oracle_feature_edges": (i64, [vp, P(i32), i64]),
                "oracle_singular_points": (i64, [vp, P(i32), i64]),
                "oracle_feature_lines": (i64, [vp, P(i64), P(i64), P(i32), P(i32), P(i64)]),
                "oracle_feature_particles": (i64, [vp, f64, P(f64), P(i32), i64]),
                "oracle_set_particles": (C.c_int, [vp, P(f32), P(i32), i64]),
                "oracle_set_state": (None, [vp, P(f64), P(i32)]),
                "oracle_get_particles": (None, [vp, P(f64), P(i32), P(i32)]),
                "oracle_keys": (None, [vp, P(C.c_uint32), P(C.c_uint32)]),
                "oracle_cell_ranges": (i64, [vp, P(C.c_uint32), P(C.c_uint32), P(C.c_uint32), i64]),
                "oracle_forces": (f64, [vp, P(f64), P(i32)]),
                "oracle_brute_neighbours": (None, [vp, P(i32)]),
                "oracle_project_points": (None, [vp, P(f32), P(i32), P(i32), i64, P(f64), P(i32), P(i32)]),
                "oracle_brute_surface": (None, [vp, P(f32), i64, P(i32), P(f32)]),
                "oracle_volume_inside": (None, [vp, P(f32), i64, P(i32)]),
                "oracle_ray_parity": (None, [vp, P(f64), i64, P(i32)]),
                "oracle_relax": (C.c_int, [vp, i32]),
                "oracle_set_ghost_count": (None, [vp, i64]),
                "oracle_boolean_curve": (i64, [vp, vp]),
                "oracle_curve_points": (i64, [vp, P(f32), i64]),
                "oracle_relax_forces": (f64, [vp]),
                "oracle_relax_step": (C.c_int, [vp, f64]),
                "oracle_boolean_keep": (None, [vp, vp, C.c_int, C.c_int, P(i32)]),
                "oracle_boolean_relax": (C.c_int, [vp, vp, C.c_int, i32]),
                "oracle_boolean_relax_many": (C.c_int, [C.POINTER(vp), i32, P(i32), i32, i32]),
                "oracle_set_cell_order": (C.c_int, [vp, i32]),
                "oracle_relax_energy": (C.c_int, [vp, i32]),
                "oracle_last_iteration": (None, [vp, P(f64), P(f64), P(i64)]),
                "oracle_w0": (None, [vp, P(f64)]),
                "oracle_density": (None, [vp, P(f64)]),
                "oracle_energy": (f64, [vp, P(f64)]),
                "oracle_energy_projected": (f64, [vp, P(f64), P(f64), P(f64), P(f64)]),
                "oracle_stats": (None, [vp, P(f64)]),
                "oracle_map_particles": (i64, [vp, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, P(f64), P(i32), P(i32),
                                                i64]),
                "oracle_lattice_intervals": (i64, [P(f32), i64, P(f32), f32, P(C.c_uint64), P(C.c_uint64), i64]),
                "oracle_interval_boolean": (i64, [P(C.c_uint64), P(C.c_uint64), i64, P(C.c_uint64), P(C.c_uint64), i64,
                                                  C.c_int, P(C.c_uint64), P(C.c_uint64), i64]),
                "oracle_interval_cells": (i64, [P(C.c_uint64), P(C.c_uint64), i64, P(f32), f32, P(f32), i64]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def alpha3(h):
    return lib().oracle_alpha3(h)


def W(r, h):
    return lib().oracle_W(r, h)


def dW(r, h):
    return lib().oracle_dW(r, h)


def lattice_sum(dx, h, dim):
    return lib().oracle_lattice_sum(dx, h, dim)


def morton3(x, y, z):
    return int(lib().oracle_morton3(x, y, z))


def _u64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.uint64).reshape(-1))


def lattice_intervals(xyz, origin, d):
    """C_compact (begin, length) of the lattice cells holding the points:
    Morton codes (Eq. 9) of the cells, ascending, as maximal runs."""
    x = np.ascontiguousarray(np.asarray(xyz, np.float32).reshape(-1, 3))
    o = np.ascontiguousarray(np.asarray(origin, np.float32).reshape(3))
    n = lib().oracle_lattice_intervals(_p(x, C.c_float), len(x), _p(o, C.c_float), float(d), None, None, 0)
    if n < 0:
        raise ValueError("a point lies outside the lattice")
    b, l_ = np.zeros(n, np.uint64), np.zeros(n, np.uint64)
    lib().oracle_lattice_intervals(_p(x, C.c_float), len(x), _p(o, C.c_float), float(d), _p(b, C.c_uint64),
                                   _p(l_, C.c_uint64), n)
    return b, l_


def interval_boolean(a, b, op):
    """op(A, B) of two run lists ((begin, length) pairs of arrays): union 0,
    difference 1, intersection 2, as maximal runs (Fig. 10)."""
    ab, al, bb, bl = _u64(a[0]), _u64(a[1]), _u64(b[0]), _u64(b[1])
    args = (_p(ab, C.c_uint64), _p(al, C.c_uint64), len(ab), _p(bb, C.c_uint64), _p(bl, C.c_uint64), len(bb), int(op))
    n = lib().oracle_interval_boolean(*args, None, None, 0)
    if n < 0:
        raise ValueError("unknown op or a run past 2^63")
    ob, ol = np.zeros(n, np.uint64), np.zeros(n, np.uint64)
    lib().oracle_interval_boolean(*args, _p(ob, C.c_uint64), _p(ol, C.c_uint64), n)
    return ob, ol


def interval_cells(runs, origin, d):
    """The cell centres of a run list, in run order and code order."""
    b, l_ = _u64(runs[0]), _u64(runs[1])
    o = np.ascontiguousarray(np.asarray(origin, np.float32).reshape(3))
    n = lib().oracle_interval_cells(_p(b, C.c_uint64), _p(l_, C.c_uint64), len(b), _p(o, C.c_float), float(d), None, 0)
    if n < 0:
        raise ValueError("a run past 2^63")
    x = np.zeros((n, 3), np.float32)
    lib().oracle_interval_cells(_p(b, C.c_uint64), _p(l_, C.c_uint64), len(b), _p(o, C.c_float), float(d),
                                _p(x, C.c_float), n)
    return x


def set_threads(n: int):
    lib().oracle_set_threads(int(n))


def get_threads() -> int:
    return int(lib().oracle_get_threads())


STATS_KEYS = ("mean_S", "mean_V", "mean_F", "std_S", "std_V", "std_F", "min_pair_over_dx",
              "max_disp_over_dx", "n_S", "n_V", "n_F")


class Oracle:
    """One body: its mesh, grids, features and particles, all FP64 on the CPU."""

    def __init__(self, verts, tris, dx, h):
        L = lib()
        self.verts = np.ascontiguousarray(verts, dtype=np.float32)
        self.tris = np.ascontiguousarray(tris, dtype=np.int32)
        self.dx, self.h = float(dx), float(h)
        self._c = L.oracle_create(_p(self.verts, C.c_float), self.verts.shape[0], _p(self.tris, C.c_int32),
                                  self.tris.shape[0], C.c_float(dx), C.c_float(h))
        if not self._c:
            raise ValueError("oracle_create rejected the mesh")
        self.n = 0

    def __del__(self):
        c = getattr(self, "_c", None)
        if c:
            lib().oracle_destroy(c)
            self._c = None

    # grids --------------------------------------------------------------
    def tri_grid(self):
        o, inv, n = np.zeros(3, np.float32), np.zeros(1, np.float32), np.zeros(3, np.int32)
        lib().oracle_tri_grid(self._c, _p(o, C.c_float), _p(inv, C.c_float), _p(n, C.c_int32))
        return o, float(inv[0]), n

    def nbr_grid(self):
        o, inv, cell, n, r2 = (np.zeros(3, np.float32), np.zeros(1, np.float32), np.zeros(1, np.float32),
                               np.zeros(3, np.int32), np.zeros(1, np.float32))
        lib().oracle_nbr_grid(self._c, _p(o, C.c_float), _p(inv, C.c_float), _p(cell, C.c_float),
                              _p(n, C.c_int32), _p(r2, C.c_float))
        return o, float(inv[0]), float(cell[0]), n, float(r2[0])

    def tri_bins(self):
        m = lib().oracle_tri_bins(self._c, None, None, 0)
        k, t = np.zeros(max(m, 1), np.int64), np.zeros(max(m, 1), np.int32)
        lib().oracle_tri_bins(self._c, _p(k, C.c_int64), _p(t, C.c_int32), m)
        return k[:m], t[:m]

    def pseudonormals(self):
        nt, nv = self.tris.shape[0], self.verts.shape[0]
        f, e, v = np.zeros((nt, 3), np.float32), np.zeros((nt, 3, 3), np.float32), np.zeros((nv, 3), np.float32)
        lib().oracle_pseudonormals(self._c, _p(f, C.c_float), _p(e, C.c_float), _p(v, C.c_float))
        return f, e, v

    # features -----------------------------------------------------------
    def extract_features(self, deg):
        return int(lib().oracle_extract_features(self._c, float(deg)))

    def feature_edges(self):
        m = lib().oracle_feature_edges(self._c, None, 0)
        out = np.zeros((max(m, 1), 2), np.int32)
        lib().oracle_feature_edges(self._c, _p(out, C.c_int32), m)
        return out[:m]

    def singular_points(self):
        m = lib().oracle_singular_points(self._c, None, 0)
        out = np.zeros(max(m, 1), np.int32)
        lib().oracle_singular_points(self._c, _p(out, C.c_int32), m)
        return out[:m]

    def feature_lines(self):
        ns = np.zeros(1, np.int64)
        nl = lib().oracle_feature_lines(self._c, None, None, None, None, _p(ns, C.c_int64))
        first, nseg = np.zeros(max(nl, 1), np.int64), np.zeros(max(nl, 1), np.int64)
        closed, segv = np.zeros(max(nl, 1), np.int32), np.zeros((max(int(ns[0]), 1), 2), np.int32)
        lib().oracle_feature_lines(self._c, _p(first, C.c_int64), _p(nseg, C.c_int64), _p(closed, C.c_int32),
                                   _p(segv, C.c_int32), _p(ns, C.c_int64))
        return first[:nl], nseg[:nl], closed[:nl], segv[:int(ns[0])]

    def feature_particles(self, dx=None):
        dx = self.dx if dx is None else dx
        m = lib().oracle_feature_particles(self._c, float(dx), None, None, 0)
        xyz, cls = np.zeros((max(m, 1), 3)), np.zeros(max(m, 1), np.int32)
        lib().oracle_feature_particles(self._c, float(dx), _p(xyz, C.c_double), _p(cls, C.c_int32), m)
        return xyz[:m], cls[:m]

    def map_particles(self, surface=True, volume=True, features=True, band_cells=0, inner_cells=0):
        """Initial particles of Sec. 3.2 (feature, surface-cell, interior-cell)."""
        args = (int(surface), int(volume), int(features), int(band_cells), int(inner_cells))
        m = lib().oracle_map_particles(self._c, *args, None, None, None, 0)
        xyz, cls, cons = np.zeros((max(m, 1), 3)), np.zeros(max(m, 1), np.int32), np.zeros(max(m, 1), np.int32)
        lib().oracle_map_particles(self._c, *args, _p(xyz, C.c_double), _p(cls, C.c_int32), _p(cons, C.c_int32), m)
        return xyz[:m], cls[:m], cons[:m]

    def set_mobile_classes(self, classes):
        """Only these classes move (e.g. (S, F) then (V,) for the paper's
        surface-then-volume schedule)."""
        lib().oracle_set_mobile_classes(self._c, sum(1 << int(c) for c in classes))

    def set_cascade(self, on: bool):
        """Surface re-projection by the cascade of Sec. 3.3.3 instead of the
        closest projectable triangle over the 27 cells."""
        lib().oracle_set_cascade(self._c, int(bool(on)))

    def set_fixed_features(self, fixed: bool):
        lib().oracle_set_fixed_features(self._c, int(bool(fixed)))

    # particles ----------------------------------------------------------
    def set_particles(self, xyz, cls):
        xyz = np.ascontiguousarray(xyz, dtype=np.float32)
        cls = np.ascontiguousarray(cls, dtype=np.int32)
        if lib().oracle_set_particles(self._c, _p(xyz, C.c_float), _p(cls, C.c_int32), xyz.shape[0]) != 0:
            raise ValueError("bad particle class")
        self.n = xyz.shape[0]

    def set_state(self, xyz=None, cons=None):
        x = None if xyz is None else np.ascontiguousarray(xyz, dtype=np.float64)
        c = None if cons is None else np.ascontiguousarray(cons, dtype=np.int32)
        lib().oracle_set_state(self._c, _p(x, C.c_double), _p(c, C.c_int32))

    def get_particles(self):
        x, cl, cs = np.zeros((self.n, 3)), np.zeros(self.n, np.int32), np.zeros(self.n, np.int32)
        lib().oracle_get_particles(self._c, _p(x, C.c_double), _p(cl, C.c_int32), _p(cs, C.c_int32))
        return x, cl, cs

    # hot path pieces ------------------------------------------------------
    def keys(self):
        k, p = np.zeros(self.n, np.uint32), np.zeros(self.n, np.uint32)
        lib().oracle_keys(self._c, _p(k, C.c_uint32), _p(p, C.c_uint32))
        return k, p

    def cell_ranges(self):
        m = lib().oracle_cell_ranges(self._c, None, None, None, 0)
        c, s, e = (np.zeros(max(m, 1), np.uint32) for _ in range(3))
        lib().oracle_cell_ranges(self._c, _p(c, C.c_uint32), _p(s, C.c_uint32), _p(e, C.c_uint32), m)
        return c[:m], s[:m], e[:m]

    def forces(self):
        acc, cnt = np.zeros((self.n, 3)), np.zeros(self.n, np.int32)
        amax = lib().oracle_forces(self._c, _p(acc, C.c_double), _p(cnt, C.c_int32))
        return acc, cnt, amax

    def brute_neighbours(self):
        cnt = np.zeros(self.n, np.int32)
        lib().oracle_brute_neighbours(self._c, _p(cnt, C.c_int32))
        return cnt

    def project_points(self, y, cls, cons=None):
        y = np.ascontiguousarray(y, dtype=np.float32)
        cls = np.ascontiguousarray(cls, dtype=np.int32)
        m = y.shape[0]
        cons = None if cons is None else np.ascontiguousarray(cons, dtype=np.int32)
        x, co, ok = np.zeros((m, 3)), np.zeros(m, np.int32), np.zeros(m, np.int32)
        lib().oracle_project_points(self._c, _p(y, C.c_float), _p(cls, C.c_int32), _p(cons, C.c_int32), m,
                                    _p(x, C.c_double), _p(co, C.c_int32), _p(ok, C.c_int32))
        return x, co, ok.astype(bool)

    def brute_surface(self, y):
        y = np.ascontiguousarray(y, dtype=np.float32)
        m = y.shape[0]
        t, d = np.zeros(m, np.int32), np.zeros(m, np.float32)
        lib().oracle_brute_surface(self._c, _p(y, C.c_float), m, _p(t, C.c_int32), _p(d, C.c_float))
        return t, d

    def volume_inside(self, y):
        y = np.ascontiguousarray(y, dtype=np.float32)
        out = np.zeros(y.shape[0], np.int32)
        lib().oracle_volume_inside(self._c, _p(y, C.c_float), y.shape[0], _p(out, C.c_int32))
        return out.astype(bool)

    def ray_parity(self, p):
        p = np.ascontiguousarray(p, dtype=np.float64)
        out = np.zeros(p.shape[0], np.int32)
        lib().oracle_ray_parity(self._c, _p(p, C.c_double), p.shape[0], _p(out, C.c_int32))
        return out.astype(bool)

    def relax(self, n_iter):
        lib().oracle_relax(self._c, int(n_iter))

    def boolean_curve(self, other: "Oracle") -> int:
        """Feature lines along the curve where this body's surface crosses
        `other`'s, with their feature particles appended to this body;
        returns the particles added."""
        n = int(lib().oracle_boolean_curve(self._c, other._c))
        self.n += n
        return n

    def curve_points(self):
        m = lib().oracle_curve_points(self._c, None, 0)
        out = np.zeros((max(m, 1), 3), np.float32)
        lib().oracle_curve_points(self._c, _p(out, C.c_float), m)
        return out[:m]

    def set_cell_order(self, order: int):
        """Order of the grid rows in the cell key: 0 row-major, 1 Morton
        order of (y, z) (Eq. 9); forces and steps do not depend on it."""
        if lib().oracle_set_cell_order(self._c, int(order)) != 0:
            raise ValueError("unknown cell order, or a grid of more than 2^26 rows")

    def set_ghost_count(self, n_ghost):
        """The last n_ghost particles are ghosts (act on neighbours, never move)."""
        lib().oracle_set_ghost_count(self._c, int(n_ghost))

    def relax_forces(self) -> float:
        """First half of an iteration: forces; returns this body's amax."""
        return float(lib().oracle_relax_forces(self._c))

    def relax_step(self, amax: float):
        """Second half: the step with the given amax, then the projections."""
        if lib().oracle_relax_step(self._c, float(amax)) != 0:
            raise ValueError("relax_step needs relax_forces first")

    def boolean_keep(self, other: "Oracle", op: int, first: bool) -> np.ndarray:
        """Which of this body's particles stay in Boolean operation `op`
        (0 union, 1 difference first - second, 2 intersection) with `other`;
        `first` says whether this body is the first operand."""
        keep = np.zeros(max(self.n, 1), np.int32)
        lib().oracle_boolean_keep(self._c, other._c, int(op), int(bool(first)), _p(keep, C.c_int32))
        return keep[:self.n].astype(bool)

    def union_keep(self, other: "Oracle", volume_stays: bool) -> np.ndarray:
        """boolean_keep for the union: volume_stays marks the second body."""
        return self.boolean_keep(other, 0, not volume_stays)

    def relax_energy(self, n_iter):
        lib().oracle_relax_energy(self._c, int(n_iter))

    def last_iteration(self):
        a, d, r = np.zeros(1), np.zeros(1), np.zeros(1, np.int64)
        lib().oracle_last_iteration(self._c, _p(a, C.c_double), _p(d, C.c_double), _p(r, C.c_int64))
        return float(a[0]), float(d[0]), int(r[0])

    # energy -------------------------------------------------------------
    def w0(self):
        out = np.zeros(5)
        lib().oracle_w0(self._c, _p(out, C.c_double))
        return out

    def density(self):
        rho = np.zeros(self.n)
        lib().oracle_density(self._c, _p(rho, C.c_double))
        return rho

    def energy(self, grad=False):
        g = np.zeros((self.n, 3)) if grad else None
        E = lib().oracle_energy(self._c, _p(g, C.c_double))
        return (E, g) if grad else E

    def energy_projected(self, y, verts=None, grad=True):
        y = np.ascontiguousarray(y, dtype=np.float64)
        v = None if verts is None else np.ascontiguousarray(verts, dtype=np.float64)
        gy = np.zeros((self.n, 3)) if grad else None
        gV = np.zeros((self.verts.shape[0], 3)) if grad else None
        E = lib().oracle_energy_projected(self._c, _p(y, C.c_double), _p(v, C.c_double), _p(gy, C.c_double),
                                          _p(gV, C.c_double))
        return (E, gy, gV) if grad else E

    def stats(self):
        out = np.zeros(len(STATS_KEYS))
        lib().oracle_stats(self._c, _p(out, C.c_double))
        return dict(zip(STATS_KEYS, out.tolist()))


UNION, DIFFERENCE, INTERSECTION = 0, 1, 2


def boolean_relax(a: Oracle, b: Oracle, op: int, n_iter: int):
    """Relax the result of Boolean operation `op` on bodies a (first) and b
    as one assembly (shared forces and time step, partner rules of `op`)."""
    if lib().oracle_boolean_relax(a._c, b._c, int(op), int(n_iter)) != 0:
        raise ValueError("Boolean members need the same dx, h and feature setting")


def boolean_relax_many(bodies, pairs, n_iter: int):
    """Relax bodies joined by several Boolean operations as one assembly;
    pairs = [(first, second, op), ...] indexes `bodies` (a body keeps to the
    sides of every operation it takes part in)."""
    arr = (C.c_void_p * len(bodies))(*[b._c for b in bodies])
    pr = np.ascontiguousarray(np.asarray(pairs, np.int32).reshape(-1, 3))
    r = lib().oracle_boolean_relax_many(arr, len(bodies), _p(pr, C.c_int32), pr.shape[0], int(n_iter))
    if r != 0:
        raise ValueError("Boolean members need the same dx, h and options, valid pairs, at most 4 operations each")


def union_relax(a: Oracle, b: Oracle, n_iter: int):
    boolean_relax(a, b, UNION, n_iter)


def keep_rows(o: Oracle, keep: np.ndarray):
    """Keep only the particles (and their constraints) marked in `keep`."""
    x, c, cons = o.get_particles()
    o.set_particles(x[keep].astype(np.float32), c[keep])
    o.set_state(x[keep], cons[keep])


def from_assembly(a, features=True) -> Oracle:
    """Oracle body for a workloads.Assembly, features extracted, particles set
    (generated by the oracle's own Sec. 3.2 generation when it carries none;
    the constraints of the generated surface particles are kept)."""
    o = Oracle(a.verts, a.tris, a.dx, a.h)
    if features and a.dihedral_deg is not None:
        o.extract_features(a.dihedral_deg)
    if a.xyz is None:
        x, c, cons = o.map_particles(**a.meta.get("generate", {}))
        o.set_particles(x.astype(np.float32), c)
        o.set_state(x.astype(np.float32).astype(np.float64), cons)
    else:
        o.set_particles(a.xyz, a.cls)
    return o
