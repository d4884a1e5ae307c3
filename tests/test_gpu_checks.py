"""The debug library (libperch_checks.so: every scorer index checked before
use, a violation reported through the device error word instead of an
access) reports nothing on the parity workloads and gives the same costs.

It runs in a child process with PERCH_LIB=checks, so the normal library of
this process is untouched.
"""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import numpy as np
from oracle import oracle as O
from paper_2008_00326_gb300 import perch as P, scenes
assert P.load()._name.endswith("libperch_checks.so")
with P.Context(0) as ctx:
    cases = [(scenes.tabletop_small(), {}, None),
             (scenes.tabletop_3obj(W=320, H=240, grid_half=2, n_yaw=4, tri_scale=0.25), {"color_check": 0},
              (128, 2048, 2048)),
             (scenes.tabletop_3obj(W=320, H=240, grid_half=2, n_yaw=4, tri_scale=0.25),
              {"color_check": 0, "jo_mode": 1}, (128, 2048, 4096)),
             (scenes.sixdof_5obj(n_hyp=24, W=320, H=240, tri_scale=0.1), {"color_check": 0}, None)]
    for sc, over, shape in cases:
        for k, v in over.items():
            setattr(sc.params, k, v)
        ctx.set_launch_config(*(shape or (256, 8192)))
        sid = ctx.set_observation(sc)
        mids = [ctx.load_mesh(m) for m in sc.meshes]
        osc = O.OracleScene.from_scene(sc)
        for req in sc.requests:
            got = ctx.score(sid, mids[req.mesh_index], req.label, req.roi, req.poses)
            want, _ = O.score(osc, O.OracleMesh.from_mesh(sc.meshes[req.mesh_index]), req.poses,
                              label=req.label, roi=req.roi, nn="grid")
            assert np.array_equal(got, want), (sc.name, over, req.mesh_index)
        if sc.name == "tabletop_small":
            ref, info = ctx.refine(sid, mids[0], -1, None, sc.requests[0].poses[:8])
        P.perch_sync(ctx.ctx)
print("checks ok")
'''


def test_debug_build_reports_no_violation():
    from paper_2008_00326_gb300 import build
    build.build(checks=True)
    env = dict(os.environ, PERCH_LIB="checks", PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, "-c", CHILD], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-3000:]
    assert "checks ok" in r.stdout
