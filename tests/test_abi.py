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
