"""The bounds-checked debug build (-DITM_CHECK_BOUNDS).

That build checks the indices into the hash table (chain links, returned block
pointers), the depth image and the per-frame lists before each access and
reports a failed check as the sticky status ITM_ERR_BOUNDS, standing in for a
memory checker.  This test builds it and runs the tiny sequence through it in
a separate process — allocation, integration and raycast into a normal volume
and into one with 2^8 buckets (long excess chains), then the mesh and a
combined raycast, and a swapping run (swap-in, swap-out with a tight bound) —
and requires clean statuses and the oracle's volumes and host store bit for
bit.
"""

import os
import subprocess
import sys

import pytest

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import numpy as np, torch
import oracle
import paper_1708_00783_gb300 as itm
from synth import tiny_workload
from tests.parity_util import compare_volumes
assert itm.LIB_PATH.endswith("libitm_checked.so"), itm.LIB_PATH
w = tiny_workload()
ia = w.intr.as_array()
ci = itm.make_intrinsics(w.intr.width, w.intr.height, w.intr.fx, w.intr.fy, w.intr.cx, w.intr.cy)
g = itm.Scene(**w.params)
small = itm.Scene(**dict(w.params, num_buckets=1 << 8, num_excess=1 << 13))
o = oracle.Scene(**w.params)
sw = itm.Scene(**dict(w.params, num_buckets=1 << 8, num_excess=1 << 13))
so = oracle.Scene(**dict(w.params, num_buckets=1 << 8, num_excess=1 << 13))
sw.swap_enable(24, 1)
so.swap_enable(24, 1)
V = torch.zeros((w.intr.height, w.intr.width, 4), dtype=torch.float32, device="cuda")
N = torch.zeros_like(V)
for k in range(w.n_frames):
    f = w.frame(k)
    d = torch.from_numpy(f.depth).cuda()
    g.process(d, ci, f.T_wc, V, N)
    small.process(d, ci, f.T_wc, V, N)
    o.allocate(f.depth, ia, f.T_wc)
    o.integrate(f.depth, ia, f.T_wc)
    sw.allocate(d, ci, f.T_wc); sw.swap_in(); sw.integrate(d, ci, f.T_wc); sw.swap_out()
    so.allocate(f.depth, ia, f.T_wc); so.swap_in(); so.integrate(f.depth, ia, f.T_wc); so.swap_out()
n = itm.itm_mesh(g.handle)
buf = torch.empty((max(n, 1), 9), dtype=torch.float32, device="cuda")
itm.itm_mesh(g.handle, buf, n)
eye = np.stack([np.eye(4, dtype=np.float32)] * 2)
itm.itm_raycast_combined([g.handle, small.handle], eye, ci, w.frame(5).T_wc, V, N)
torch.cuda.synchronize()
assert g.status() == 0 and small.status() == 0 and sw.status() == 0, (g.status(), small.status(), sw.status())
rep = compare_volumes(g.export(), o.export())
assert rep["sdf_bitexact_frac"] == 1.0, rep
rep = compare_volumes(sw.export(), so.export())
assert rep["sdf_bitexact_frac"] == 1.0, rep
hg, ho = sw.swap_export_host(), so.swap_export_host()
ig, io = np.lexsort(hg[0].T[::-1]), np.lexsort(ho[0].T[::-1])
assert np.array_equal(hg[0][ig], ho[0][io]) and np.array_equal(hg[1][ig], ho[1][io]) and np.array_equal(hg[2][ig], ho[2][io])
assert sw.swap_counters()["moved_out"] > 0
print("checked build clean:", n, "triangles")
"""


def test_bounds_checked_build_runs_clean():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "paper_1708_00783_gb300", "build.py"), "--checked"],
                       cwd=ROOT, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    env = dict(os.environ, ITM_CHECK_BOUNDS="1", PYTHONPATH=ROOT + os.pathsep + os.environ.get("PYTHONPATH", ""))
    r = subprocess.run([sys.executable, "-c", SCRIPT], cwd=ROOT, env=env, capture_output=True, text=True)
    assert r.returncode == 0, (r.stdout[-2000:], r.stderr[-2000:])
    assert "checked build clean" in r.stdout
