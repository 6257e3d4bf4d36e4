"""The GIC_DEBUG build (device-side index checks on field samples, shared-
memory tiles and Verlet rows, flagging GIC_STATUS_DEBUG_INDEX instead of
trapping) runs the plain 8,000-granule configuration and the wet block
(capillary bridges) with a clear status word and the release build's
parity against the oracle.  Run in a child process: a process loads one
build of the library."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, sys
import numpy as np, torch
sys.path.insert(0, ROOT)
import gic_inputs as gi, oracle
from paper_2504_00745_gb300 import gic, build
from paper_2504_00745_gb300.window import Simulator
assert gic.lib_path() == build.DEBUG_LIB
out = {}
for name, K in (("plain_fp64_8k", 10), ("wet_block", 3)):
    prob = gi.make(name)
    ref = oracle.run(prob, K=K)
    for prec in (gic.GIC_FP32, gic.GIC_FP64):
        sim = Simulator.from_problem(prob, prec)
        gic.gic_check_status(clear=True)
        sim.run(K)
        x, v = sim.positions()
        torch.cuda.synchronize()
        st = gic.gic_check_status(clear=True)
        ex = float(np.abs(x.cpu().numpy() - ref["x"]).max()) / prob.grid.dx
        out[f"{name}_{prec}"] = {"status": st, "dx_err": ex}
print(json.dumps(out))
"""


def test_debug_build_runs_clean():
    env = dict(os.environ, GIC_LIBRARY="debug")
    r = subprocess.run([sys.executable, "-c", CHILD.replace("ROOT", repr(ROOT))], capture_output=True, text=True,
                       env=env, cwd=ROOT, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    res = json.loads(r.stdout.strip().splitlines()[-1])
    for key, v in res.items():
        assert v["status"] == 0, (key, v)
        assert v["dx_err"] <= 1e-5, (key, v)
