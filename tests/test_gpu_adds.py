"""ADD / ADD-S on the GPU against the float64 oracle (binary32 transforms and
distances on the device: agreement to 2 micrometres), and the AUC helper
against the oracle's step-function integral."""
import numpy as np
import pytest

from paper_2008_00326_gb300 import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    from paper_2008_00326_gb300 import build, perch
    build.build()
    perch.load()
    return perch


@pytest.mark.parametrize("symmetric", [True, False])
def test_add_s_matches_oracle(P, oracle, symmetric):
    rng = np.random.default_rng(31)
    meshes = [scenes.box_mesh(0.06, 0.08, 0.12, 5, 6, 9),
              scenes.ellipsoid_mesh(0.04, 0.03, 0.05, 41, 40)]
    with P.Context(0) as ctx:
        for m in meshes:
            mid = ctx.load_mesh(m)
            n = 12
            gt = np.stack([np.concatenate([scenes.rodrigues(rng.normal(size=3), rng.uniform(0, 3)),
                                           (rng.normal(size=3) * 0.05 + [0, 0, 0.8])[:, None]], 1)
                           for _ in range(n)]).astype(np.float32).reshape(n, 12)
            est = gt.copy().reshape(n, 3, 4).astype(np.float64)
            for i in range(n):
                est[i, :, :3] = scenes.rodrigues(rng.normal(size=3), rng.uniform(0, 0.3)) @ est[i, :, :3]
                est[i, :, 3] += rng.normal(size=3) * 0.01
            est = est.astype(np.float32).reshape(n, 12)
            got = P.perch_add_s(ctx.ctx, mid, est, gt, symmetric)
            want = np.array([oracle.add_s(m.verts, est[i], gt[i], symmetric) for i in range(n)])
            assert np.max(np.abs(got - want)) < 2e-6, np.max(np.abs(got - want))
            assert abs(P.perch_add_s_auc(got) - oracle.add_auc(got)) < 1e-12
