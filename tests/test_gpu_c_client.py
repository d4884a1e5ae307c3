"""The plain C client (tests/c_client/score_client.c) scores through the C ABI
alone and gets the same costs and argmin as the Python binding and the
oracle."""
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_2008_00326_gb300 import scenes

pytestmark = pytest.mark.gpu


def test_c_client_matches_binding_and_oracle(tmp_path, oracle):
    from paper_2008_00326_gb300 import build, perch as P
    sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
    import test_abi
    build.build()
    P.load()
    sc = scenes.tabletop_small(seed=3)
    poses = sc.requests[0].poses
    inp, out = str(tmp_path / "in.bin"), str(tmp_path / "out.bin")
    test_abi._write_client_input(inp, sc, poses)
    exe = test_abi.build_c_client(tmp_path)
    subprocess.check_call([exe, inp, out])
    raw = open(out, "rb").read()
    n = len(poses)
    costs = np.frombuffer(raw[:8 * n], np.int32).reshape(n, 2)
    best_index = int(np.frombuffer(raw[8 * n:8 * n + 8], np.int64)[0])
    best_cost = int(np.frombuffer(raw[8 * n + 8:8 * n + 12], np.int32)[0])
    with P.Context(0) as ctx:
        sid = ctx.set_observation(sc)
        mid = ctx.load_mesh(sc.meshes[0])
        want = ctx.score(sid, mid, -1, None, poses)
    assert np.array_equal(costs, want)
    ocosts, _ = oracle.score(oracle.OracleScene.from_scene(sc), oracle.OracleMesh.from_mesh(sc.meshes[0]), poses)
    assert np.array_equal(costs, ocosts)
    assert (best_index, best_cost) == oracle.best(ocosts)
