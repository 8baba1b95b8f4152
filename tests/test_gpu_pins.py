"""GPU parity on the cases the oracle is pinned on, and on what the timed
path does that the counting path does not.

- fixed feature lines (the paper treats feature particles as boundaries,
  Sec. 2.2): both sides keep them in place, the rest relaxes alike;
- the uniformity statistics on the closed-form sets of the oracle's pins
  (single particle W(0), population deviation, masked mobile-only smallest
  pair, exact lattice);
- the force kernel instantiation that the relaxation times (clamped
  weights, no exact r^2 < (2h)^2 test) against the oracle's forces on the
  clouds that stress the x-slab reach cut, through the allocation-free entry
  point, which runs that instantiation;
- the icosphere + torus workload at full size over 100 iterations of the
  batched graph form: positions against the oracle within the tolerance
  and the oracle's own conditioning, uniformity statistics within 1 %."""
import ctypes as C
import math

import numpy as np
import pytest

import oracle as O
import paper_2501_03056_gb300 as pkg
from paper_2501_03056_gb300 import workloads as W

pytestmark = pytest.mark.gpu
S, V, F, I, P = W.CLS_S, W.CLS_V, W.CLS_F, W.CLS_I, W.CLS_P


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2501_03056_gb300 import _build
    _build.build()


# ---- fixed feature lines ------------------------------------------------------------
def test_fixed_feature_lines_stay_and_the_rest_matches_the_oracle():
    a = W.cube_workload()[0]
    b = pkg.Body.from_assembly(a)
    o = O.from_assembly(a)
    b.set_fixed_features(True)
    o.set_fixed_features(True)
    x0, cls, _ = b.get_particles()
    b.relax(20)
    o.relax(20)
    x, _, _ = b.get_particles()
    ox, _, _ = o.get_particles()
    feat = np.isin(cls, [F, P])
    assert feat.sum() == 12 * 19 + 8
    assert np.array_equal(x[feat], x0[feat])                          # GPU: unmoved, bit for bit
    assert np.array_equal(ox[feat], x0[feat].astype(np.float64))      # oracle: unmoved
    err = np.abs(x.astype(np.float64) - ox).max(axis=1) / a.dx
    assert err.max() < 1e-4, err.max()
    # they still push: the surface particles next to the edges moved
    assert np.abs(x[~feat] - x0[~feat]).max() > 1e-3 * a.dx
    # the counting pass sees fixed feature particles with no force
    acc, _, _ = b.debug_forces()
    assert np.all(acc[feat] == 0)


# ---- statistics on the closed-form sets of the oracle pins -----------------------------
DX = 0.0625
H = float(np.float32(1.3 * DX))


def _stats_both(xyz, cls):
    v, t = W.cube_mesh(1.0)
    xyz = np.asarray(xyz, np.float32)
    cls = np.asarray(cls, np.int32)
    b = pkg.Body(v, t, DX, H)
    b.set_particles(xyz, cls)
    o = O.Oracle(v, t, DX, H)
    o.set_particles(xyz, cls)
    return b.stats(), o.stats()


def test_statistics_of_one_particle_and_of_three():
    s, so = _stats_both([[0.1, 0.2, -0.3]], [V])
    a = 21.0 / (16.0 * math.pi * H ** 3)
    assert s["mean_V"] == pytest.approx(a, rel=1e-6) and s["std_V"] == 0.0
    assert math.isinf(s["min_pair_over_dx"])
    r = 1.7 * DX
    s, so = _stats_both([[-0.6, -0.6, -0.6], [0.2, 0.0, 0.0], [0.2 + r, 0.0, 0.0]], [V, V, V])
    assert s["mean_V"] == pytest.approx(so["mean_V"], rel=1e-6)
    assert s["std_V"] == pytest.approx((s["mean_V"] - a) / math.sqrt(2.0), rel=1e-5)
    assert s["min_pair_over_dx"] == pytest.approx(so["min_pair_over_dx"], rel=1e-6)


def test_smallest_pair_is_masked_and_mobile_only():
    xyz = [[0.0, 0.0, 0.0], [DX, 0.0, 0.0], [0.0, 0.25 * DX, 0.0], [0.5, 0.5, 0.5],
           [0.5 + 0.125 * DX, 0.5, 0.5], [-0.5, 0.5, -0.5], [-0.5, 0.5 + 0.0625 * DX, -0.5],
           [-0.5, -0.5, 0.0], [-0.5 + 1.5 * DX, -0.5, 0.0]]
    cls = [S, S, I, I, I, P, P, S, V]
    s, so = _stats_both(xyz, cls)
    assert s["min_pair_over_dx"] == 1.0 == so["min_pair_over_dx"]
    s, so = _stats_both(xyz + [[-0.5 + 1.5 * DX, -0.5 + 0.5 * DX, 0.0]], cls + [I])
    assert s["min_pair_over_dx"] == 0.5 == so["min_pair_over_dx"]


def test_statistics_of_a_perfect_lattice():
    k = np.arange(12) - 5.5
    g = np.stack(np.meshgrid(k, k, k, indexing="ij"), -1).reshape(-1, 3)
    cls = np.where(np.all(np.abs(g) < 3, axis=1), V, I)
    s, so = _stats_both(g * DX, cls)
    assert s["n_V"] == 216 and s["min_pair_over_dx"] == 1.0
    assert s["std_V"] <= 1e-6 * s["mean_V"]                  # FP32 sums of one neighbourhood
    assert s["mean_V"] == pytest.approx(so["mean_V"], rel=1e-6)


# ---- the timed force instantiation -------------------------------------------------------
def _cloud(case, rng, org, cell):
    if case == "dense":                      # > 255 particles per cell: whole-cell ranges
        xyz = np.concatenate([rng.uniform(0.0, 0.05, (2500, 3)), rng.uniform(-0.3, 0.3, (3000, 3))])
    elif case == "uniform":
        xyz = rng.uniform(-0.3, 0.3, (8000, 3))
    else:                                    # exactly on slab boundaries in x, y and z
        k = rng.integers(0, 8 * 8, (6000, 3))
        xyz = org[None, :].astype(np.float64) + 6 * cell + k * (cell / 8)
    return xyz.astype(np.float32)


@pytest.mark.parametrize("case", ["slab_planes", "dense", "uniform"])
def test_timed_force_kernel_against_the_oracle(case):
    import torch
    v, t = W.cube_mesh(1.0)
    dx, h = 0.02, 0.026
    o = O.Oracle(v, t, dx, h)
    org, _, cell, _, _ = o.nbr_grid()
    rng = np.random.default_rng(11)
    xyz = _cloud(case, rng, org, cell)
    cls = rng.integers(0, 5, len(xyz)).astype(np.int32)
    o.set_particles(xyz, cls)
    oacc, _, oamax = o.forces()
    L = pkg.lib()
    f = L.fppg_forces_static
    f.restype = C.c_int
    f.argtypes = [C.c_void_p, C.c_void_p, C.c_int64, C.POINTER(C.c_float), C.POINTER(C.c_float), C.c_float,
                  C.c_int32, C.c_void_p, C.POINTER(C.c_float), C.c_void_p]
    x_d = torch.from_numpy(xyz).cuda()
    c_d = torch.from_numpy(cls).cuda()
    out = torch.full_like(x_d, float("nan"))
    lo = np.ascontiguousarray(v.min(axis=0), np.float32)
    hi = np.ascontiguousarray(v.max(axis=0), np.float32)
    amax = C.c_float()
    r = f(x_d.data_ptr(), c_d.data_ptr(), len(xyz), lo.ctypes.data_as(C.POINTER(C.c_float)),
          hi.ctypes.data_as(C.POINTER(C.c_float)), C.c_float(h), 0, out.data_ptr(), C.byref(amax),
          C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert r == pkg.OK, L.fppg_last_error(None)
    acc = out.cpu().numpy().astype(np.float64)
    assert np.isfinite(acc).all()
    assert np.abs(acc - oacc).max() <= 2e-5 * oamax, (case, np.abs(acc - oacc).max() / oamax)
    assert amax.value == pytest.approx(oamax, rel=1e-5)


def test_negative_capacity_is_an_argument_error():
    v, t = W.cube_mesh()
    b = pkg.Body(v, t, 0.05, 0.065)
    b.extract_features(30.0)
    n = C.c_int64()
    buf = np.zeros((24, 2), np.int32)
    r = pkg.lib().fppg_get_feature_edges(b.handle, buf.ctypes.data_as(C.POINTER(C.c_int32)), -1, C.byref(n))
    assert r == pkg.ERR_ARG
    r = pkg.lib().fppg_get_feature_lines(b.handle, None, None, -3, None, 0, C.byref(n), C.byref(n))
    assert r == pkg.ERR_ARG


# ---- the icosphere + torus workload over 100 iterations ----------------------------------
def _conditioning(a, iters):
    """Drift (in dx) of the FP64 oracle after `iters` iterations when its
    positions are rounded to FP32 after every iteration, as an FP32
    implementation stores them, against the plain FP64 run: the
    conditioning of the relaxation, which bounds what any FP32
    implementation can reproduce."""
    o1, o2 = O.from_assembly(a), O.from_assembly(a)
    o1.relax(iters)
    for _ in range(iters):
        o2.relax(1)
        x, _, _ = o2.get_particles()
        o2.set_state(x.astype(np.float32).astype(np.float64))
    return np.abs(o1.get_particles()[0] - o2.get_particles()[0]).max(axis=1) / a.dx


def test_full_size_icosphere_torus_over_100_iterations():
    asm = W.sphere_torus_workload()                      # 777,215 particles, dx = 0.02
    bodies = [pkg.Body.from_assembly(a) for a in asm]
    batch = pkg.Batch(bodies)
    batch.autotune(2)
    batch.set_graph_iters(50)
    batch.relax(100, use_graph=True)
    batch.store()
    for a, b in zip(asm, bodies):
        o = O.from_assembly(a)
        o.relax(100)
        x, cls, _ = b.get_particles()
        ox, _, _ = o.get_particles()
        err = np.abs(x.astype(np.float64) - ox).max(axis=1) / a.dx
        cond = _conditioning(a, 100)
        # the GPU may drift from the FP64 oracle as far as the oracle itself
        # drifts when its positions are stored in FP32, and no further: at
        # most twice as many particles beyond 1e-4 dx, a 99.9 % quantile and
        # a largest drift within twice the oracle's (measured: the torus has
        # 3,400 particles beyond against the oracle's own 3,358, and the same
        # largest drift, 0.057 dx -- the same decision flips on both)
        n_gpu, n_cond = int((err >= 1e-4).sum()), int((cond >= 1e-4).sum())
        q_gpu, q_cond = np.quantile(err, 0.999), np.quantile(cond, 0.999)
        info = (a.name, n_gpu, n_cond, len(err), err.max(), cond.max(), q_gpu, q_cond)
        assert n_gpu <= max(2 * n_cond, 0.002 * len(err)), info
        assert q_gpu <= max(1e-4, 2.0 * q_cond), info
        assert err.max() <= max(1e-4, 2.0 * cond.max()), info
        s, so = b.stats(), o.stats()
        for k in ("mean_S", "mean_V", "std_S", "std_V", "min_pair_over_dx"):
            assert s[k] == pytest.approx(so[k], rel=1e-2), (a.name, k, s[k], so[k])
