"""The bounds-checking debug build (libtrajam_debug.so, selected with
TRAJAM_LIBRARY=libtrajam_debug.so).

Its fused, grouped and warp-pair kernels check their state and shared-memory indices
and report an index outside its array in the problem's status word (bit 2,
AM_ERR_STATE on the host) instead of trapping; the access is skipped.  On
valid shapes -- the tiny and paper-shaped workloads, an odd horizon whose
last pair of steps has one step, a grouped launch and the warp-pair
kernel on the paper shape, the odd horizon and the three- and four-warp
horizons (q = 151 and q = 256 with 64 obstacles) -- no check may fire,
and the checks must not change a single result: each build runs in its own
process and the states are compared bit for bit.
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import json, sys
import numpy as np
sys.path.insert(0, sys.argv[1])
from paper_2109_13030_b300 import trajam as T, workload as W
assert T.LIB_PATH.endswith(sys.argv[2]), T.LIB_PATH
out = {}
cases = {"tiny": W.make_problem("tiny", 0), "paper": W.make_problem("paper", 0, B=40),
         "odd_q": W.make_shape(11, B=9, q=51, n=5, m=3)}
wcases = {"paper": cases["paper"], "odd_q": cases["odd_q"], "q151": W.make_shape(12, B=11, q=151, n=12, m=2),
          "q256": W.make_shape(13, B=6, q=256, n=64, m=4)}
for name, pb in cases.items():
    P = T.Problem(pb)
    P.solve(pb["init"].astype(np.float32), 20)   # raises TrajamError on a nonzero status word
    out[name] = P.state().tolist()
    P.close()
for name, pb in wcases.items():                 # the warp-pair kernel
    P = T.Problem(pb, kernel=T.AM_KERNEL_WARP)
    P.solve(pb["init"].astype(np.float32), 20)
    out["warp_" + name] = P.state().tolist()
    P.close()
pbs = W.make_uneven(4, count=3, scale=1 / 128)
probs = [T.Problem(pb).init_state(pb["init"].astype(np.float32)) for pb in pbs]
G = T.Group(probs)
G.solve(10)
T.am_group_get_best(G.g, len(probs))            # reads the group's status words
out["group"] = [P.state().tolist() for P in probs]   # each state read checks its status word
G.close()
for P in probs:
    P.close()
# the warp-pair group kernels (AUTO handles: two and three warps per trajectory)
probs = [T.Problem(pb, kernel=T.AM_KERNEL_AUTO).init_state(pb["init"].astype(np.float32)) for pb in pbs]
G = T.Group(probs)
G.solve(10)
T.am_group_get_best(G.g, len(probs))
out["group_auto"] = [P.state().tolist() for P in probs]
G.close()
for P in probs:
    P.close()
print(json.dumps(out))
'''


def run(lib):
    env = dict(os.environ, TRAJAM_LIBRARY=lib)
    o = subprocess.run([sys.executable, "-c", CHILD, ROOT, lib], capture_output=True, text=True, env=env,
                       timeout=900)
    assert o.returncode == 0, o.stderr[-3000:]
    return json.loads(o.stdout.strip().splitlines()[-1])


def test_debug_build_runs_clean_and_matches_release():
    assert os.path.exists(os.path.join(ROOT, "paper_2109_13030_b300", "libtrajam_debug.so")), \
        "debug build missing: python paper_2109_13030_b300/build.py --debug"
    dbg, rel = run("libtrajam_debug.so"), run("libtrajam.so")
    assert dbg.keys() == rel.keys()
    for key in rel:
        a, b = (dbg[key], rel[key]) if key.startswith("group") else ([dbg[key]], [rel[key]])
        assert len(a) == len(b), key
        for x, y in zip(a, b):
            np.testing.assert_array_equal(np.asarray(x), np.asarray(y), err_msg=key)
