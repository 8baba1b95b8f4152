"""The bounds-checked build (-DFPPG_CHECKED): every hot-path kernel checks
the indices it computes before it uses them.  Run on the paths of the
method (plain and batched forms, both orderings of the keys, Morton rows,
a Boolean chain with its intersection curves, the energy-descent
relaxation, generation), no check fails, and the checked library gives the
same bits as the normal one."""
import os
import subprocess
import sys

import numpy as np
import pytest

import paper_2501_03056_gb300 as pkg
from paper_2501_03056_gb300 import workloads as W

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r'''
import sys, numpy as np
sys.path.insert(0, ROOT)
import paper_2501_03056_gb300 as pkg
from paper_2501_03056_gb300 import workloads as W
out = {}
a = W.cube_workload()[0]
b = pkg.Body.from_assembly(a)
b.relax(8)
out["cube"] = b.get_particles()[0]
asm = W.sphere_torus_workload(seed=1, dx=0.06, level=3, torus_nu=64, torus_nv=24)
for inc in (0, 1):
    bodies = [pkg.Body.from_assembly(x) for x in asm]
    bt = pkg.Batch(bodies)
    bt.set_incremental(bool(inc))
    bt.set_cell_order(inc)
    bt.set_graph_iters(4)
    bt.relax(8, use_graph=True)
    bt.store()
    out["st%d" % inc] = np.concatenate([g.get_particles()[0] for g in bodies])
# a union chain of three spheres with its curves
dx = 0.06
h = float(np.float32(1.3 * dx))
cs = [np.array([0.0, 0.0, 0.0]), np.array([0.7, 0.0131, 0.0217]), np.array([1.4, 0.0297, -0.0113])]
sp = []
for c in cs:
    v, t = W.icosphere_mesh(3, 0.5)
    g = pkg.Body((v.astype(np.float64) + c).astype(np.float32), t, dx, h)
    g.map_particles()
    sp.append(g)
pkg.union(sp[0], sp[1])
pkg.union(sp[1], sp[2])
pkg.boolean_curve(sp[0], sp[1])
pkg.boolean_curve(sp[1], sp[2])
bt = pkg.Batch(sp)
bt.relax(6, use_graph=False)
bt.store()
out["chain"] = np.concatenate([g.get_particles()[0] for g in sp])
g = pkg.Body.from_assembly(a)
g.relax_energy(4)
out["energy"] = g.get_particles()[0]
word, checked = pkg.check_status()
np.savez(OUT, word=word, checked=checked, **out)
'''


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2501_03056_gb300 import _build
    _build.build()
    _build.build(checked=True)


def run(checked, tmp_path):
    out = tmp_path / ("checked.npz" if checked else "normal.npz")
    env = dict(os.environ, FPPG_CHECKED="1" if checked else "0")
    code = "ROOT = %r\nOUT = %r\n" % (ROOT, str(out)) + SCRIPT
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    return np.load(out)


def test_no_bounds_check_fails_and_the_bits_are_the_same(tmp_path):
    chk = run(True, tmp_path)
    assert bool(chk["checked"]) and int(chk["word"]) == 0
    ref = run(False, tmp_path)
    assert not bool(ref["checked"]) and int(ref["word"]) == 0
    for k in ("cube", "st0", "st1", "chain", "energy"):
        assert np.array_equal(chk[k], ref[k]), k
