"""GB300-native relaxation path of Feature-Preserving Particle Generation.

Thin ctypes binding of the C ABI in ``include/fppg.h`` (the CUDA library
``_lib/libfppg.so``).  It only marshals arguments; every step of the path
runs in the library's CUDA kernels.  Importing works without a GPU; any call
that needs the library raises ``FPPGError`` when it has not been built
(``__graft_entry__.build()``) -- there is no fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import workloads  # noqa: F401  (seeded synthetic inputs)

__all__ = ["Body", "Batch", "FPPGError", "lib", "library_path", "workloads", "S", "V", "F", "I", "P"]

S, V, F, I, P = 0, 1, 2, 3, 4
OK, ERR_ARG, ERR_STATE, ERR_OOM, ERR_CUDA, ERR_TIMEOUT, ERR_INTERNAL = range(7)
_HERE = os.path.dirname(os.path.abspath(__file__))
# FPPG_CHECKED=1 in the environment loads the bounds-checked build instead
_LIBPATH = os.path.join(_HERE, "_lib", "libfppg_checked.so" if os.environ.get("FPPG_CHECKED") == "1" else "libfppg.so")
_lock = threading.Lock()
_lib = None


class FPPGError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"fppg error {code}: {msg}")
        self.code = code


class _MapOpts(C.Structure):
    _fields_ = [("surface", C.c_int32), ("volume", C.c_int32), ("features", C.c_int32), ("band_cells", C.c_int32),
                ("inner_cells", C.c_int32)]


class _Stats(C.Structure):
    _fields_ = [("mean_rho", C.c_double * 3), ("std_rho", C.c_double * 3), ("min_pair_over_dx", C.c_double),
                ("max_disp_over_dx", C.c_double), ("count", C.c_int64 * 3)]


def library_path() -> str:
    return _LIBPATH


def lib():
    """The loaded CUDA library (raises FPPGError when it is missing)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(_LIBPATH):
                raise FPPGError(-1, f"{_LIBPATH} is missing: build it with __graft_entry__.build()")
            L = C.CDLL(_LIBPATH)
            vp, i32, i64, f32, f64 = C.c_void_p, C.c_int32, C.c_int64, C.c_float, C.c_double
            P_ = C.POINTER
            sig = {
                "fppg_create": [P_(f32), i64, P_(i32), i64, f32, f32, P_(vp)],
                "fppg_destroy": [vp],
                "fppg_set_stream": [vp, vp],
                "fppg_set_fixed_features": [vp, i32],
                "fppg_extract_features": [vp, f32, P_(i64)],
                "fppg_get_feature_edges": [vp, P_(i32), i64, P_(i64)],
                "fppg_get_feature_lines": [vp, P_(i64), P_(i32), i64, P_(i32), i64, P_(i64), P_(i64)],
                "fppg_set_particles": [vp, P_(f32), P_(i32), i64],
                "fppg_get_particles": [vp, P_(f32), P_(i32), P_(i32), i64, P_(i64)],
                "fppg_set_constraints": [vp, P_(i32), i64],
                "fppg_map_particles": [vp, P_(_MapOpts), P_(i64)],
                "fppg_relax": [vp, i32],
                "fppg_relax_energy": [vp, i32],
                "fppg_stats": [vp, P_(_Stats)],
                "fppg_debug_grid": [vp, P_(C.c_uint32), P_(C.c_uint32), P_(C.c_uint32), P_(C.c_uint32),
                                    P_(C.c_uint32), i64, P_(i64)],
                "fppg_debug_forces": [vp, P_(f32), P_(i32), P_(f32)],
                "fppg_project_points": [vp, P_(f32), P_(i32), P_(i32), i64, P_(f32), P_(i32), P_(i32)],
                "fppg_energy": [vp, vp, vp, P_(f64), vp, vp],
                "fppg_work_counts": [vp, P_(i64), P_(i64), P_(i64)],
                "fppg_debug_search": [vp, P_(i64), P_(i32)],
                "fppg_debug_cell_lists": [vp, P_(i64), P_(i64), P_(i64)],
                "fppg_batch_load": [vp],
                "fppg_copy_positions_dev": [vp, vp],
                "fppg_batch_create": [P_(vp), i32, P_(vp)],
                "fppg_batch_destroy": [vp],
                "fppg_batch_set_stream": [vp, vp],
                "fppg_batch_relax": [vp, i32, i32],
                "fppg_batch_set_graph_iters": [vp, i32],
                "fppg_batch_store": [vp],
                "fppg_batch_time_force": [vp, i32],
                "fppg_batch_force_ms": [vp, P_(f64)],
                "fppg_batch_autotune": [vp, i32, P_(i32), P_(i32), P_(i32), P_(i32), P_(i32), P_(f64)],
                "fppg_batch_set_incremental": [vp, i32],
                "fppg_set_incremental": [vp, i32],
                "fppg_set_cell_order": [vp, i32],
                "fppg_batch_set_cell_order": [vp, i32],
                "fppg_set_ghost_count": [vp, i64],
                "fppg_relax_forces": [vp, P_(f32)],
                "fppg_relax_step": [vp, f32],
                "fppg_batch_configure": [vp, i32, i32, i32],
                "fppg_set_mobile_classes": [vp, i32],
                "fppg_set_projection_rule": [vp, i32],
                "fppg_batch_set_mobile_classes": [vp, i32],
                "fppg_union": [vp, vp, P_(i64), P_(i64)],
                "fppg_boolean": [vp, vp, i32, P_(i64), P_(i64)],
                "fppg_boolean_curve": [vp, vp, P_(i64)],
                "fppg_get_curve_points": [vp, P_(f32), i64, P_(i64)],
                "fppg_batch_phase_ms": [vp, P_(f64)],
                "fppg_device_sm_count": [P_(i32)],
                "fppg_debug_fail_allocation": [i64],
                "fppg_check_status": [P_(C.c_uint32), P_(i32)],
                "fppg_grid_lattice": [vp, P_(f32), P_(f32)],
                "fppg_lattice_intervals": [vp, i64, P_(f32), f32, vp, vp, i64, P_(i64), vp],
                "fppg_interval_boolean": [vp, vp, i64, vp, vp, i64, i32, vp, vp, i64, P_(i64), vp],
                "fppg_interval_cells": [vp, vp, i64, P_(f32), f32, vp, i64, P_(i64), vp],
            }
            for name, args in sig.items():
                fn = getattr(L, name)
                fn.argtypes = args
                fn.restype = C.c_int
            L.fppg_last_error.argtypes = [vp]
            L.fppg_last_error.restype = C.c_char_p
            L.fppg_batch_last_error.argtypes = [vp]
            L.fppg_batch_last_error.restype = C.c_char_p
            L.fppg_batch_kernels_per_iter.argtypes = [vp]
            L.fppg_batch_kernels_per_iter.restype = C.c_int32
            L.fppg_batch_size.argtypes = [vp]
            L.fppg_batch_size.restype = C.c_int64
            _lib = L
    return _lib


def _ptr(a, ct):
    return None if a is None else a.ctypes.data_as(C.POINTER(ct))


def _f32(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float32)
    if shape is not None:
        a = a.reshape(shape)
    return a


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _stream_ptr(stream):
    if stream is None:
        return None
    return C.c_void_p(int(getattr(stream, "cuda_stream", stream)))


class Body:
    """One body: ``fppg_create`` on its mesh (the handle lives until close())."""

    def __init__(self, verts, tris, dx, h, stream=None):
        L = lib()
        self.verts = _f32(verts, (-1, 3))
        self.tris = _i32(tris).reshape(-1, 3)
        self.dx, self.h = float(np.float32(dx)), float(np.float32(h))
        h_ = C.c_void_p()
        r = L.fppg_create(_ptr(self.verts, C.c_float), self.verts.shape[0], _ptr(self.tris, C.c_int32),
                          self.tris.shape[0], C.c_float(dx), C.c_float(h), C.byref(h_))
        if r != OK:
            raise FPPGError(r, L.fppg_last_error(None).decode())
        self._h = h_
        self.n = 0
        if stream is not None:
            self.set_stream(stream)

    @classmethod
    def from_assembly(cls, a, features=True, stream=None):
        """Body of a workloads.Assembly: its mesh, its features, and its given
        particles -- or, when it carries none, the generation of Sec. 3.2."""
        b = cls(a.verts, a.tris, a.dx, a.h, stream=stream)
        if features and a.dihedral_deg is not None:
            b.extract_features(a.dihedral_deg)
        if a.xyz is None:
            b.map_particles(**a.meta.get("generate", {}))
        else:
            b.set_particles(a.xyz, a.cls)
        return b

    def _chk(self, r):
        if r != OK:
            raise FPPGError(r, lib().fppg_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            lib().fppg_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    def set_stream(self, stream):
        self._chk(lib().fppg_set_stream(self._h, _stream_ptr(stream)))

    def set_mobile_classes(self, classes):
        """Only these classes move (e.g. (S, F) then (V,) for the paper's
        surface-then-volume schedule)."""
        self._chk(lib().fppg_set_mobile_classes(self._h, sum(1 << int(c) for c in classes)))

    def set_projection_rule(self, cascade: bool):
        """Surface re-projection by the cascade of Sec. 3.3.3 (own triangle,
        own cell, 27 cells) instead of the closest over the 27 cells."""
        self._chk(lib().fppg_set_projection_rule(self._h, 1 if cascade else 0))

    def set_incremental(self, on: bool):
        """Order the keys by repairing the previous order (True) or by a full
        stable sort (False); both give the same bits."""
        self._chk(lib().fppg_set_incremental(self._h, int(bool(on))))

    def set_cell_order(self, order: int):
        """Order of the grid rows in the cell key (fppg_set_cell_order)."""
        self._chk(lib().fppg_set_cell_order(self._h, int(order)))

    def set_fixed_features(self, fixed: bool):
        self._chk(lib().fppg_set_fixed_features(self._h, int(bool(fixed))))

    def extract_features(self, dihedral_deg) -> int:
        n = C.c_int64()
        self._chk(lib().fppg_extract_features(self._h, C.c_float(dihedral_deg), C.byref(n)))
        return n.value

    def feature_edges(self):
        n = C.c_int64()
        self._chk(lib().fppg_get_feature_edges(self._h, None, 0, C.byref(n)))
        out = np.zeros((max(n.value, 1), 2), np.int32)
        self._chk(lib().fppg_get_feature_edges(self._h, _ptr(out, C.c_int32), n.value, C.byref(n)))
        return out[:n.value]

    def feature_lines(self):
        nl, ns = C.c_int64(), C.c_int64()
        self._chk(lib().fppg_get_feature_lines(self._h, None, None, 0, None, 0, C.byref(nl), C.byref(ns)))
        nseg = np.zeros(max(nl.value, 1), np.int64)
        closed = np.zeros(max(nl.value, 1), np.int32)
        segv = np.zeros((max(ns.value, 1), 2), np.int32)
        self._chk(lib().fppg_get_feature_lines(self._h, _ptr(nseg, C.c_int64), _ptr(closed, C.c_int32), nl.value,
                                               _ptr(segv, C.c_int32), ns.value, C.byref(nl), C.byref(ns)))
        return nseg[:nl.value], closed[:nl.value], segv[:ns.value]

    def curve_points(self) -> np.ndarray:
        """Intersection-curve points (fppg_get_curve_points), FP32 [m, 3]."""
        m = C.c_int64()
        self._chk(lib().fppg_get_curve_points(self._h, None, 0, C.byref(m)))
        out = np.zeros((max(m.value, 1), 3), np.float32)
        self._chk(lib().fppg_get_curve_points(self._h, _ptr(out, C.c_float), m.value, C.byref(m)))
        return out[:m.value]

    def map_particles(self, surface=True, volume=True, features=True, band_cells=0, inner_cells=0) -> int:
        """Replace the particles by the initial set of Sec. 3.2 (on the GPU)."""
        o = _MapOpts(int(surface), int(volume), int(features), int(band_cells), int(inner_cells))
        n = C.c_int64()
        self._chk(lib().fppg_map_particles(self._h, C.byref(o), C.byref(n)))
        self.n = n.value
        return self.n

    def set_particles(self, xyz, cls):
        xyz = _f32(xyz, (-1, 3))
        cls = _i32(cls)
        self._chk(lib().fppg_set_particles(self._h, _ptr(xyz, C.c_float), _ptr(cls, C.c_int32), xyz.shape[0]))
        self.n = xyz.shape[0]

    def set_constraints(self, cons):
        cons = _i32(cons)
        self._chk(lib().fppg_set_constraints(self._h, _ptr(cons, C.c_int32), cons.shape[0]))

    def get_particles(self):
        xyz = np.zeros((max(self.n, 1), 3), np.float32)
        cls = np.zeros(max(self.n, 1), np.int32)
        cons = np.zeros(max(self.n, 1), np.int32)
        n = C.c_int64()
        self._chk(lib().fppg_get_particles(self._h, _ptr(xyz, C.c_float), _ptr(cls, C.c_int32),
                                           _ptr(cons, C.c_int32), self.n, C.byref(n)))
        return xyz[:self.n], cls[:self.n], cons[:self.n]

    def get_positions_into(self, xyz_out: np.ndarray):
        """Positions into a caller buffer (e.g. pinned host memory)."""
        n = C.c_int64()
        self._chk(lib().fppg_get_particles(self._h, _ptr(xyz_out, C.c_float), None, None, self.n, C.byref(n)))

    def relax(self, n_iter: int):
        self._chk(lib().fppg_relax(self._h, int(n_iter)))

    def set_ghost_count(self, n_ghost: int):
        """The last n_ghost particles become ghosts (they act, never move)."""
        self._chk(lib().fppg_set_ghost_count(self._h, int(n_ghost)))

    def relax_forces(self) -> float:
        """First half of an iteration (grid and forces); returns this body's
        largest |a| over its moving particles."""
        a = C.c_float()
        self._chk(lib().fppg_relax_forces(self._h, C.byref(a)))
        return a.value

    def relax_step(self, amax: float):
        """Second half of the iteration: the step with the given amax, then
        the projections."""
        self._chk(lib().fppg_relax_step(self._h, C.c_float(amax)))

    def relax_energy(self, n_iter: int):
        self._chk(lib().fppg_relax_energy(self._h, int(n_iter)))

    def stats(self) -> dict:
        s = _Stats()
        self._chk(lib().fppg_stats(self._h, C.byref(s)))
        return {"mean_S": s.mean_rho[0], "mean_V": s.mean_rho[1], "mean_F": s.mean_rho[2],
                "std_S": s.std_rho[0], "std_V": s.std_rho[1], "std_F": s.std_rho[2],
                "min_pair_over_dx": s.min_pair_over_dx, "max_disp_over_dx": s.max_disp_over_dx,
                "n_S": s.count[0], "n_V": s.count[1], "n_F": s.count[2]}

    def grid_lattice(self):
        """(origin, dx) of the body's generation lattice (fppg_grid_lattice)."""
        o, d = np.zeros(3, np.float32), C.c_float()
        self._chk(lib().fppg_grid_lattice(self._h, _ptr(o, C.c_float), C.byref(d)))
        return o, float(d.value)

    def debug_grid(self):
        n = self.n
        key, perm = np.zeros(max(n, 1), np.uint32), np.zeros(max(n, 1), np.uint32)
        nc = C.c_int64()
        self._chk(lib().fppg_debug_grid(self._h, None, None, None, None, None, 0, C.byref(nc)))
        cells, st, en = (np.zeros(max(nc.value, 1), np.uint32) for _ in range(3))
        self._chk(lib().fppg_debug_grid(self._h, _ptr(key, C.c_uint32), _ptr(perm, C.c_uint32),
                                        _ptr(cells, C.c_uint32), _ptr(st, C.c_uint32), _ptr(en, C.c_uint32),
                                        nc.value, C.byref(nc)))
        m = nc.value
        return key[:n], perm[:n], cells[:m], st[:m], en[:m]

    def debug_forces(self):
        n = self.n
        acc, cnt = np.zeros((max(n, 1), 3), np.float32), np.zeros(max(n, 1), np.int32)
        amax = np.zeros(1, np.float32)
        self._chk(lib().fppg_debug_forces(self._h, _ptr(acc, C.c_float), _ptr(cnt, C.c_int32),
                                          _ptr(amax, C.c_float)))
        return acc[:n], cnt[:n], float(amax[0])

    def project_points(self, y, cls, cons=None):
        y = _f32(y, (-1, 3))
        cls = _i32(cls)
        m = y.shape[0]
        cons = None if cons is None else _i32(cons)
        x, co, ok = np.zeros((max(m, 1), 3), np.float32), np.zeros(max(m, 1), np.int32), np.zeros(max(m, 1), np.int32)
        self._chk(lib().fppg_project_points(self._h, _ptr(y, C.c_float), _ptr(cls, C.c_int32),
                                            _ptr(cons, C.c_int32), m, _ptr(x, C.c_float), _ptr(co, C.c_int32),
                                            _ptr(ok, C.c_int32)))
        return x[:m], co[:m], ok[:m].astype(bool)

    def debug_search(self):
        """(particles sent to the triangle search in the last iteration,
        whether the mesh is closed so that inside certificates apply)."""
        q, c = C.c_int64(), C.c_int32()
        self._chk(lib().fppg_debug_search(self._h, C.byref(q), C.byref(c)))
        return q.value, bool(c.value)

    def debug_cell_lists(self):
        """(cells with a candidate list, list entries, cells whose list was
        too long and that are probed instead)."""
        a, b, c = C.c_int64(), C.c_int64(), C.c_int64()
        self._chk(lib().fppg_debug_cell_lists(self._h, C.byref(a), C.byref(b), C.byref(c)))
        return a.value, b.value, c.value

    def work_counts(self):
        """(candidates in the 27 cells, pairs within 2h, candidates actually
        tested by the force kernel) of one force pass on the current state."""
        c, p, t = C.c_int64(), C.c_int64(), C.c_int64()
        self._chk(lib().fppg_work_counts(self._h, C.byref(c), C.byref(p), C.byref(t)))
        return c.value, p.value, t.value

    def energy_ptr(self, y_ptr: int, verts_ptr: int = 0, gy_ptr: int = 0, gv_ptr: int = 0) -> float:
        """Energy (and gradients into device buffers) from device pointers."""
        E = C.c_double()
        self._chk(lib().fppg_energy(self._h, C.c_void_p(y_ptr), C.c_void_p(verts_ptr or None), C.byref(E),
                                    C.c_void_p(gy_ptr or None), C.c_void_p(gv_ptr or None)))
        return E.value

    def copy_positions_dev(self, ptr: int):
        self._chk(lib().fppg_copy_positions_dev(self._h, C.c_void_p(ptr)))


def check_status() -> tuple[int, bool]:
    """(codes of the failed bounds checks since the last call, whether the
    loaded library is the checked build); fppg_check_status."""
    w, c = C.c_uint32(), C.c_int32()
    r = lib().fppg_check_status(C.byref(w), C.byref(c))
    if r != OK:
        raise FPPGError(r, "fppg_check_status")
    return w.value, bool(c.value)


def device_sm_count() -> int:
    """SMs of the current CUDA device, as the library sees it."""
    v = C.c_int32()
    r = lib().fppg_device_sm_count(C.byref(v))
    if r != OK:
        raise FPPGError(r, lib().fppg_last_error(None).decode())
    return v.value


UNION, DIFFERENCE, INTERSECTION = 0, 1, 2
ORDER_ROWS, ORDER_MORTON_ROWS = 0, 1


def boolean(a: "Body", b: "Body", op: int) -> tuple[int, int]:
    """Boolean operation `op` (UNION, DIFFERENCE a - b, INTERSECTION) on
    bodies a and b (fppg_boolean): drops the particles the operation
    removes; the two then relax together in one Batch.  Returns the counts
    left."""
    na, nb_ = C.c_int64(), C.c_int64()
    r = lib().fppg_boolean(a.handle, b.handle, int(op), C.byref(na), C.byref(nb_))
    if r != OK:
        msg = lib().fppg_last_error(a.handle) or lib().fppg_last_error(None)
        raise FPPGError(r, msg.decode() if isinstance(msg, bytes) else str(msg))
    a.n, b.n = na.value, nb_.value
    return na.value, nb_.value


def boolean_curve(a: "Body", b: "Body") -> int:
    """Feature lines along the curve where a's surface crosses b's Boolean
    partner b, with their feature particles appended to a
    (fppg_boolean_curve); returns the particles added."""
    n = C.c_int64()
    r = lib().fppg_boolean_curve(a.handle, b.handle, C.byref(n))
    if r != OK:
        msg = lib().fppg_last_error(a.handle) or lib().fppg_last_error(None)
        raise FPPGError(r, msg.decode() if isinstance(msg, bytes) else str(msg))
    a.n += n.value
    return n.value


def _sized_call(fn, out_alloc):
    """Run an interval call once for its count (capacity 0), allocate the
    result with out_alloc(count) -> (pointers, tensors) and run it again."""
    n = C.c_int64()
    r = fn(None, 0, C.byref(n))
    if r != OK and not (r == ERR_ARG and n.value > 0):
        raise FPPGError(r, lib().fppg_last_error(None).decode())
    ptrs, out = out_alloc(n.value)
    if n.value > 0:
        r = fn(ptrs, n.value, C.byref(n))
        if r != OK:
            raise FPPGError(r, lib().fppg_last_error(None).decode())
    return out


def _runs_alloc(m):
    import torch
    b = torch.empty(max(m, 1), dtype=torch.int64, device="cuda")
    ln = torch.empty(max(m, 1), dtype=torch.int64, device="cuda")
    return (b.data_ptr(), ln.data_ptr()), (b[:m], ln[:m])


def lattice_intervals(xyz, origin, d, stream=None):
    """C_compact of the lattice cells holding the points (fppg_lattice_intervals):
    xyz a CUDA float32 tensor [n, 3]; returns (begin, len) as CUDA int64
    tensors (Morton codes of Eq. 9, below 2^63)."""
    x = xyz.contiguous()
    o = np.ascontiguousarray(np.asarray(origin, np.float32).reshape(3))
    sp = _stream_ptr(stream)

    def fn(ptrs, cap, n_out):
        b, ln = ptrs if ptrs else (None, None)
        return lib().fppg_lattice_intervals(x.data_ptr(), x.shape[0], _ptr(o, C.c_float), float(d), b, ln, cap,
                                            n_out, sp)
    return _sized_call(fn, _runs_alloc)


def interval_boolean(a, b, op, stream=None):
    """op(A, B) (UNION, DIFFERENCE A - B, INTERSECTION) of two run lists
    ((begin, len) CUDA int64 tensors) as maximal runs (fppg_interval_boolean)."""
    ab, al, bb, bl = (t.contiguous() for t in (a[0], a[1], b[0], b[1]))
    sp = _stream_ptr(stream)

    def fn(ptrs, cap, n_out):
        ob, ol = ptrs if ptrs else (None, None)
        return lib().fppg_interval_boolean(ab.data_ptr(), al.data_ptr(), ab.numel(), bb.data_ptr(), bl.data_ptr(),
                                           bb.numel(), int(op), ob, ol, cap, n_out, sp)
    return _sized_call(fn, _runs_alloc)


def interval_cells(runs, origin, d, stream=None):
    """The centres of the cells of a run list (fppg_interval_cells), a CUDA
    float32 tensor [cells, 3]."""
    import torch
    b, ln = (t.contiguous() for t in runs)
    o = np.ascontiguousarray(np.asarray(origin, np.float32).reshape(3))
    sp = _stream_ptr(stream)

    def alloc(m):
        x = torch.empty((max(m, 1), 3), dtype=torch.float32, device="cuda")
        return x.data_ptr(), x[:m]

    def fn(ptr, cap, n_out):
        return lib().fppg_interval_cells(b.data_ptr(), ln.data_ptr(), b.numel(), _ptr(o, C.c_float), float(d), ptr,
                                         cap, n_out, sp)
    return _sized_call(fn, alloc)


def union(a: "Body", b: "Body") -> tuple[int, int]:
    """Boolean union of bodies a and b (see boolean)."""
    return boolean(a, b, UNION)


class Batch:
    """Many bodies relaxed by one launch per phase (``fppg_batch_*``)."""

    def __init__(self, bodies, stream=None):
        L = lib()
        self.bodies = list(bodies)
        arr = (C.c_void_p * len(self.bodies))(*[b.handle for b in self.bodies])
        h_ = C.c_void_p()
        r = L.fppg_batch_create(arr, len(self.bodies), C.byref(h_))
        if r != OK:
            raise FPPGError(r, L.fppg_batch_last_error(None).decode())
        self._h = h_
        if stream is not None:
            self.set_stream(stream)

    def _chk(self, r):
        if r != OK:
            raise FPPGError(r, lib().fppg_batch_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            lib().fppg_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def n(self) -> int:
        return int(lib().fppg_batch_size(self._h))

    @property
    def kernels_per_iter(self) -> int:
        return int(lib().fppg_batch_kernels_per_iter(self._h))

    def set_stream(self, stream):
        self._chk(lib().fppg_batch_set_stream(self._h, _stream_ptr(stream)))

    def set_graph_iters(self, k: int):
        self._chk(lib().fppg_batch_set_graph_iters(self._h, int(k)))

    def relax(self, n_iter: int, use_graph: bool = True):
        self._chk(lib().fppg_batch_relax(self._h, int(n_iter), int(bool(use_graph))))

    def store(self):
        self._chk(lib().fppg_batch_store(self._h))

    def load(self):
        self._chk(lib().fppg_batch_load(self._h))

    def time_force(self, enable: bool = True):
        self._chk(lib().fppg_batch_time_force(self._h, int(bool(enable))))

    def autotune(self, iters: int = 5) -> dict:
        """Pick force variant, block size and search grid by timing; the state
        is restored afterwards."""
        v, tb, sc, inc, co, ms = C.c_int32(), C.c_int32(), C.c_int32(), C.c_int32(), C.c_int32(), C.c_double()
        self._chk(lib().fppg_batch_autotune(self._h, int(iters), C.byref(v), C.byref(tb), C.byref(sc),
                                            C.byref(inc), C.byref(co), C.byref(ms)))
        return {"force_variant": v.value, "force_block": tb.value, "search_ctas_per_sm": sc.value,
                "incremental_order": inc.value, "cell_order": co.value, "ms_per_iter": ms.value}

    def set_cell_order(self, order: int):
        """Order of the grid rows in the cell key: ORDER_ROWS (row-major) or
        ORDER_MORTON_ROWS (Eq. 9 over y, z); the same neighbours in the same
        order either way (forces equal up to FP32 rounding)."""
        self._chk(lib().fppg_batch_set_cell_order(self._h, int(order)))

    def set_incremental(self, on: bool):
        """Order the keys by repairing the previous order (True) or by a full
        stable sort (False); both give the same bits."""
        self._chk(lib().fppg_batch_set_incremental(self._h, int(bool(on))))

    def set_mobile_classes(self, classes):
        """Only these classes move, in every body of the batch."""
        self._chk(lib().fppg_batch_set_mobile_classes(self._h, sum(1 << int(c) for c in classes)))

    def configure(self, force_variant: int = 0, force_block: int = 256, search_ctas_per_sm: int = 16):
        """Set the kernel configuration by hand (the autotuner's choices)."""
        self._chk(lib().fppg_batch_configure(self._h, int(force_variant), int(force_block), int(search_ctas_per_sm)))

    def phase_ms(self) -> dict:
        """Device ms per iteration of grid build, force pass, step and
        triangle search, from the last graph replay with timing enabled."""
        ms = np.zeros(4, np.float64)
        self._chk(lib().fppg_batch_phase_ms(self._h, ms.ctypes.data_as(C.POINTER(C.c_double))))
        return {"grid": float(ms[0]), "force": float(ms[1]), "step": float(ms[2]), "search": float(ms[3])}

    def force_ms(self) -> float:
        ms = C.c_double()
        self._chk(lib().fppg_batch_force_ms(self._h, C.byref(ms)))
        return ms.value
