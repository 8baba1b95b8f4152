"""The allocation-free force pass (fppg_forces_static) against the regular
entry point (fppg_debug_forces) through the C ABI, on two calls in a row.

It serves callers that cannot call cudaMalloc (device memory owned by their
own pool allocator, or time-critical loops that must not allocate); its
temporaries live in one static device array shared by every call.  This file
is collected last so that a run stopping at its first failure has already
run every other test."""
import ctypes as C

import numpy as np
import pytest

import paper_2501_03056_gb300 as pkg
from paper_2501_03056_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2501_03056_gb300 import _build
    _build.build()
    L = pkg.lib()
    f = L.fppg_forces_static
    f.restype = C.c_int
    f.argtypes = [C.c_void_p, C.c_void_p, C.c_int64, C.POINTER(C.c_float), C.POINTER(C.c_float), C.c_float,
                  C.c_int32, C.c_void_p, C.POINTER(C.c_float), C.c_void_p]
    return L


def _call(L, x, c, n, bbmin, bbmax, h, out, stream):
    amax = C.c_float()
    r = L.fppg_forces_static(x.data_ptr(), c.data_ptr(), n, bbmin.ctypes.data_as(C.POINTER(C.c_float)),
                             bbmax.ctypes.data_as(C.POINTER(C.c_float)), C.c_float(h), 0, out.data_ptr(),
                             C.byref(amax), C.c_void_p(stream))
    return r, amax.value


@pytest.mark.parametrize("which", ["cube", "small_sphere"])
def test_static_force_pass_matches_the_regular_entry_point(lib, which):
    import torch
    if which == "cube":
        a = W.cube_workload()[0]
    else:
        a = W.sphere_torus_workload(seed=4, dx=0.06, level=3, torus_nu=64, torus_nv=24)[0]
    body = pkg.Body.from_assembly(a)
    ref, _, ref_amax = body.debug_forces()
    x = torch.from_numpy(np.ascontiguousarray(a.xyz)).cuda()
    c = torch.from_numpy(np.ascontiguousarray(a.cls)).cuda()
    bbmin = np.ascontiguousarray(a.verts.min(axis=0), dtype=np.float32)
    bbmax = np.ascontiguousarray(a.verts.max(axis=0), dtype=np.float32)
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):                       # the shared scratch is reused
        out = torch.full_like(x, float("nan"))
        r, amax = _call(lib, x, c, a.n, bbmin, bbmax, a.h, out, stream)
        assert r == pkg.OK, lib.fppg_last_error(None)
        got = out.cpu().numpy()
        assert np.isfinite(got).all()
        assert np.abs(got.astype(np.float64) - ref).max() <= 2e-5 * ref_amax
        assert amax == pytest.approx(ref_amax, rel=1e-6)


def test_static_force_pass_rejects_sizes_beyond_its_limit(lib):
    import torch
    n = 65537
    x = torch.zeros((n, 3), dtype=torch.float32, device="cuda")
    c = torch.ones(n, dtype=torch.int32, device="cuda")
    out = torch.empty_like(x)
    box = np.array([-1, -1, -1], np.float32), np.array([1, 1, 1], np.float32)
    r, _ = _call(lib, x, c, n, box[0], box[1], 0.05, out, 0)
    assert r == pkg.ERR_ARG and b"65536" in lib.fppg_last_error(None)
    # a box needing more grid cells than the scratch holds
    big = np.array([-50, -50, -50], np.float32), np.array([50, 50, 50], np.float32)
    r, _ = _call(lib, x[:10], c[:10], 10, big[0], big[1], 0.05, out, 0)
    assert r == pkg.ERR_ARG and b"131072" in lib.fppg_last_error(None)
