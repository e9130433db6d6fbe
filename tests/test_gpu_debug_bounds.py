"""The bounds-checked build (libwl_debug.so, WL_DEBUG_BOUNDS): every global store of the
step and the computed global loads test their index, a bad one flags a bit and is skipped,
and canaries sit between the workspace's arrays.  Steps of grids that exercise every
kernel path (walls, periodic sides, a convective exit, ragged and odd sides, the smallest
legal grids, analytic and sampled bodies, 16-bit levels, every level split in 64 x 16
tiles, batched steps) run through it in
a child process and must leave no flag and intact canaries, with the same results as the
release library."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CASES = [
    dict(dims=(64, 32), nu=0.064, U=(1.0, 0.0), periodic=0, body=dict(kind=1, center=(16.0, 16.0), radius=5.0)),
    dict(dims=(37, 29), nu=0.03, U=(0.8, 0.1), periodic=0, body=dict(kind=1, center=(15.3, 13.7), radius=4.2)),
    dict(dims=(96, 40), nu=0.05, U=(1.0, 0.0), periodic=1, body=dict(kind=1, center=(30.5, 20.0), radius=6.0)),
    dict(dims=(64, 32, 32), nu=0.02, U=(1.0, 0.0, 0.0), periodic=0, body=dict(kind=1, center=(20.0, 16.0, 16.0),
                                                                              radius=6.0)),
    dict(dims=(35, 21, 19), nu=0.015, U=(0.6, 0.2, -0.1), periodic=2, body=dict(kind=1, center=(12.7, 10.1, 9.4),
                                                                                radius=3.6)),
    dict(dims=(48, 32, 32), nu=0.02, U=(1.0, 0.0, 0.0), periodic=0, body=dict(kind=2, center=(14.0, 16.3, 15.8),
                                                                              radius=8.0, radius2=3.0)),
    dict(dims=(64, 64, 64), nu=0.01, U=(0.0, 0.0, 0.0), periodic=7, body=None, ic=1),
    dict(dims=(128, 48, 24), nu=0.02, U=(0.3, 0.0, 0.0), periodic=3, body=None),
    dict(dims=(96, 40, 32), nu=0.02, U=(1.0, 0.0, 0.0), periodic=0, body=dict(kind=1, center=(30.0, 20.3, 15.8),
                                                                              radius=5.0), exit_bc=True),
    dict(dims=(9, 7, 5), nu=0.05, U=(1.0, 0.0, 0.0), periodic=0, body=dict(kind=1, center=(4.3, 3.2, 2.6), radius=1.7)),
    dict(dims=(2, 2), nu=0.1, U=(0.0, 0.0), periodic=3, body=None),
    dict(dims=(192, 96, 96), nu=0.01, U=(1.0, 0.0, 0.0), periodic=0, body=dict(kind=1, center=(60.3, 47.2, 49.7),
                                                                               radius=9.0), coarse_precision="bf16"),
    # every level split into band and uniform tiles, in 64 x 16 tiles where allowed
    dict(dims=(128, 64, 48), nu=0.02, U=(1.0, 0.0, 0.0), periodic=0, body=dict(kind=1, center=(40.3, 31.6, 24.2),
                                                                              radius=6.0),
         env={"WL_UNIFORM_ALL": "1", "WL_TY16_MIN_CELLS": "0"}),
    dict(dims=(96, 64, 40), nu=0.02, U=(1.0, 0.2, 0.0), periodic=4, body=None,
         env={"WL_UNIFORM_ALL": "1", "WL_TY16_MIN_CELLS": "0"}),
]

SCRIPT = r"""
import json, sys
import numpy as np
sys.path.insert(0, ROOT)
from paper_2304_08159_gb300 import wl
cases = json.loads(sys.argv[1])
out = []
import os
for c in cases:
    kw = {k: c[k] for k in ("exit_bc", "coarse_precision") if k in c}
    for k, v in c.get("env", {}).items():
        os.environ[k] = v
    sim = wl.Sim(c["dims"], c["nu"], c["U"], body=c["body"], periodic=c["periodic"], **kw)
    for k in c.get("env", {}):
        del os.environ[k]
    if c.get("ic"):
        sim.set_ic(c["ic"], 1.0)
    sim.step(3)
    rc, flags = wl.wl_debug_bounds(sim.h)
    out.append(dict(rc=rc, flags=flags, u=float(np.abs(sim.get(0).astype(np.float64)).sum()),
                    p=float(np.abs(sim.get(1).astype(np.float64)).sum())))
    sim.close()
import torch
sims = [wl.Sim(c["dims"], c["nu"], c["U"], body=c["body"], periodic=c["periodic"]) for c in cases[:6]]
batch = wl.Batch(1 << 17)
for _ in range(3):
    batch.step([s.h for s in sims], torch.cuda.current_stream().cuda_stream)
torch.cuda.synchronize()
for s in sims:
    rc, flags = wl.wl_debug_bounds(s.h)
    out.append(dict(rc=rc, flags=flags, u=float(np.abs(s.get(0).astype(np.float64)).sum()),
                    p=float(np.abs(s.get(1).astype(np.float64)).sum())))
print("RESULT " + json.dumps(out))
""".replace("ROOT", repr(ROOT))


def _run(lib):
    env = dict(os.environ, WL_LIB=lib)
    r = subprocess.run([sys.executable, "-c", SCRIPT, json.dumps(CASES)], capture_output=True, text=True, env=env,
                       cwd=ROOT, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    line = [x for x in r.stdout.splitlines() if x.startswith("RESULT ")][-1]
    return json.loads(line[len("RESULT "):])


def test_bounds_checked_build_flags_nothing():
    from paper_2304_08159_gb300 import wl

    assert os.path.exists(wl.DEBUG_LIB_PATH)
    dbg = _run("debug")
    rel = _run("release")
    for i, (d, r) in enumerate(zip(dbg, rel)):
        assert d["rc"] == wl.WL_OK and d["flags"] == 0, (i, d)
        assert r["rc"] == wl.WL_NODEBUG and r["flags"] == 0, (i, r)
        assert d["u"] == r["u"] and d["p"] == r["p"], (i, d, r)
