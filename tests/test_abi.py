"""The C ABI library builds for sm_103a, loads without a GPU and exports
every entry point that include/*.h declares."""
import ctypes
import glob
import os
import re

import pytest

import paper_2501_03056_gb300 as pkg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \*]*?\b(fppg_\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def library():
    from paper_2501_03056_gb300 import _build
    path = _build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_path():
    names = declared_symbols()
    for required in ("fppg_create", "fppg_extract_features", "fppg_set_particles", "fppg_relax",
                     "fppg_get_particles", "fppg_batch_relax", "fppg_energy", "fppg_destroy"):
        assert required in names


def test_every_declared_symbol_is_exported(library):
    missing = [n for n in declared_symbols() if not hasattr(library, n)]
    assert not missing, f"declared but not exported: {missing}"


def test_bad_arguments_are_rejected_without_a_gpu(library):
    # argument checks run on the host before any device call
    L = pkg.lib()
    out = ctypes.c_void_p()
    r = L.fppg_create(None, 0, None, 0, ctypes.c_float(0.1), ctypes.c_float(0.13), ctypes.byref(out))
    assert r == pkg.ERR_ARG and not out.value
    assert b"mesh" in L.fppg_last_error(None)
    assert L.fppg_relax(None, 1) == pkg.ERR_ARG
    assert L.fppg_batch_relax(None, 1, 1) == pkg.ERR_ARG


def test_package_fails_loudly_without_the_library(monkeypatch, tmp_path):
    monkeypatch.setattr(pkg, "_LIBPATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(pkg, "_lib", None)
    with pytest.raises(pkg.FPPGError):
        pkg.lib()


def test_tiny_cell_sizes_are_rejected_before_any_launch(library):
    # a cell far below the mesh extent would need more than 2^20 cells per
    # axis: rejected on the host (no cast to int of an overflowing count)
    import numpy as np
    from paper_2501_03056_gb300 import workloads as W
    L = pkg.lib()
    v, t = W.cube_mesh()
    v = np.ascontiguousarray(v, np.float32)
    t = np.ascontiguousarray(t, np.int32)
    fp, ip = ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_int32)
    for dx, h in ((0.05, 1e-9), (0.05, 1e-7), (1e-7, 0.065), (1e-30, 1e-30)):
        out = ctypes.c_void_p()
        r = L.fppg_create(v.ctypes.data_as(fp), len(v), t.ctypes.data_as(ip), len(t), ctypes.c_float(dx),
                          ctypes.c_float(h), ctypes.byref(out))
        assert r == pkg.ERR_ARG and not out.value, (dx, h)
    # the allocation-free force pass: the per-axis bound comes before the
    # cell product, so neither a wrapped nor a negative product passes
    L.fppg_forces_static.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, fp, fp, ctypes.c_float,
                                     ctypes.c_int32, ctypes.c_void_p, fp, ctypes.c_void_p]
    lo = np.full(3, -1.0, np.float32)
    hi = np.full(3, 1.0, np.float32)
    for h in (1e-7, 1e-20, 0.02):
        r = L.fppg_forces_static(None, None, 0, lo.ctypes.data_as(fp), hi.ctypes.data_as(fp), ctypes.c_float(h), 0,
                                 None, None, None)
        assert r == pkg.ERR_ARG, h
        assert b"131072" in L.fppg_last_error(None)


def test_negative_capacities_are_rejected(library):
    L = pkg.lib()
    n = ctypes.c_int64()
    # no handle: the null check comes first
    assert L.fppg_get_feature_edges(None, None, -1, ctypes.byref(n)) == pkg.ERR_ARG


def test_triangle_cell_hash_uses_the_primes_as_printed():
    # Eq. 10's primes, from the fixture transcribed from the paper (p1 is
    # used as printed, 738560931), against the constants the triangle-cell
    # lookup of the library hashes with
    gold = {}
    for line in open(os.path.join(ROOT, "tests", "golden", "hash_eq10.txt")):
        parts = line.split()
        if len(parts) == 2 and parts[0] in ("p1", "p2", "p3"):
            gold[parts[0]] = int(parts[1])
    src = open(os.path.join(ROOT, "paper_2501_03056_gb300", "csrc", "fppg_internal.cuh")).read()
    m = re.search(r"kHashP1\s*=\s*(\d+)u,\s*kHashP2\s*=\s*(\d+)u,\s*kHashP3\s*=\s*(\d+)u", src)
    assert m and gold == {"p1": int(m.group(1)), "p2": int(m.group(2)), "p3": int(m.group(3))}


def test_interval_calls_reject_bad_arguments_before_any_launch(library):
    # the C_compact interval calls check their arguments on the host first
    L = pkg.lib()
    n = ctypes.c_int64(-5)
    o = (ctypes.c_float * 3)(0.0, 0.0, 0.0)
    nan = (ctypes.c_float * 3)(float("nan"), 0.0, 0.0)
    # unknown op, negative sizes, a missing count pointer
    assert L.fppg_interval_boolean(None, None, 0, None, None, 0, 3, None, None, 0, ctypes.byref(n), None) == pkg.ERR_ARG
    assert b"op" in L.fppg_last_error(None)
    assert L.fppg_interval_boolean(None, None, -1, None, None, 0, pkg.UNION, None, None, 0, ctypes.byref(n),
                                   None) == pkg.ERR_ARG
    assert L.fppg_interval_boolean(None, None, 0, None, None, 0, pkg.UNION, None, None, 0, None, None) == pkg.ERR_ARG
    # runs given without their arrays, a capacity without output arrays
    assert L.fppg_interval_boolean(None, None, 4, None, None, 0, pkg.UNION, None, None, 0, ctypes.byref(n),
                                   None) == pkg.ERR_ARG
    assert L.fppg_interval_cells(None, None, 0, o, ctypes.c_float(1.0), None, 8, ctypes.byref(n), None) == pkg.ERR_ARG
    # a lattice spacing that is not finite and positive, a non-finite origin
    for d in (0.0, -1.0, float("inf"), float("nan")):
        assert L.fppg_lattice_intervals(None, 0, o, ctypes.c_float(d), None, None, 0, ctypes.byref(n),
                                        None) == pkg.ERR_ARG, d
        assert L.fppg_interval_cells(None, None, 0, o, ctypes.c_float(d), None, 0, ctypes.byref(n),
                                     None) == pkg.ERR_ARG, d
    assert L.fppg_lattice_intervals(None, 0, nan, ctypes.c_float(1.0), None, None, 0, ctypes.byref(n),
                                    None) == pkg.ERR_ARG
    # empty inputs need no device: an empty result
    n.value = -5
    assert L.fppg_interval_boolean(None, None, 0, None, None, 0, pkg.DIFFERENCE, None, None, 0, ctypes.byref(n),
                                   None) == pkg.OK and n.value == 0
    n.value = -5
    assert L.fppg_lattice_intervals(None, 0, o, ctypes.c_float(0.5), None, None, 0, ctypes.byref(n),
                                    None) == pkg.OK and n.value == 0
    d = ctypes.c_float()
    assert L.fppg_grid_lattice(None, o, ctypes.byref(d)) == pkg.ERR_ARG
