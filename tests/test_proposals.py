"""6-DoF pose proposals (Sec. V-B, Eq. 5-6): oracle pins (CPU) and GPU parity."""
import math

import numpy as np
import pytest

from oracle import proposals as OP
from paper_2008_00326_gb300 import scenes


def test_viewpoints_cover_the_sphere_evenly():
    M = 200
    v = np.stack([OP.viewpoint(i, M) for i in range(M)])
    assert np.allclose(np.linalg.norm(v, axis=1), 1.0, atol=1e-12)
    assert np.linalg.norm(v.mean(0)) < 0.02                   # balanced around the sphere
    d = np.arccos(np.clip(v @ v.T, -1, 1)) + np.eye(M) * 10
    nn = d.min(1)
    # near-equidistant: nearest-neighbour spacing within a factor 1.6 of sqrt(4 pi / M)
    assert nn.min() > 0.6 * math.sqrt(4 * math.pi / M) and nn.max() < 1.6 * math.sqrt(4 * math.pi / M)


def test_proposal_geometry_closed_forms():
    sc = scenes.sixdof_5obj(n_hyp=4, W=320, H=240, tri_scale=0.05)
    req = sc.requests[1]
    mesh = sc.meshes[req.mesh_index]
    lo, hi = mesh.verts.min(0), mesh.verts.max(0)
    M, N, K = 12, 6, 3
    poses, (z0, z1) = OP.proposals(sc.depth, sc.labels, req.label, req.roi, sc.fx, sc.fy, sc.cx, sc.cy,
                                   lo, hi, M, N, K)
    u0, v0, u1, v1 = req.roi
    sel = (sc.labels[v0:v1, u0:u1] == req.label) & (sc.depth[v0:v1, u0:u1] > 0)
    assert (z0, z1) == (int(sc.depth[v0:v1, u0:u1][sel].min()), int(sc.depth[v0:v1, u0:u1][sel].max()))
    m = 0.5 * (lo.astype(np.float64) + hi)
    for idx in range(M * N * K):
        P = poses[idx].reshape(3, 4)
        R, t = P[:, :3], P[:, 3]
        assert np.allclose(R @ R.T, np.eye(3), atol=1e-12) and abs(np.linalg.det(R) - 1) < 1e-12
        i, k, j = idx // (N * K), (idx // K) % N, idx % K
        assert np.allclose(R @ OP.viewpoint(i, M), [0, 0, -1], atol=1e-12)    # camera looks at the object
        c = R @ m + t                                                         # the mesh centre in the camera
        z = z0 / 1e4 + (z1 - z0) / 1e4 * j / (K - 1)
        assert abs(c[2] - z) < 1e-12
        assert abs(sc.fx * c[0] / c[2] + sc.cx - 0.5 * (u0 + u1 - 1)) < 1e-9
        assert abs(sc.fy * c[1] / c[2] + sc.cy - 0.5 * (v0 + v1 - 1)) < 1e-9
        # in-plane angle: relative to k = 0, a rotation by 2 pi k / N about the optical axis
        R0 = poses[(i * N) * K + j].reshape(3, 4)[:, :3]
        th = 2 * math.pi * k / N
        Rz = np.array([[math.cos(th), -math.sin(th), 0], [math.sin(th), math.cos(th), 0], [0, 0, 1]])
        assert np.allclose(R, Rz @ R0, atol=1e-12)


@pytest.mark.gpu
def test_proposals_gpu_parity():
    import torch
    from paper_2008_00326_gb300 import build, perch as P
    build.build()
    sc = scenes.sixdof_5obj(n_hyp=4, W=320, H=240, tri_scale=0.1)
    with P.Context(0) as ctx:
        sid = ctx.set_observation(sc)
        for req in sc.requests:
            mesh = sc.meshes[req.mesh_index]
            mid = ctx.load_mesh(mesh)
            for (M, N, K) in ((1, 1, 1), (42, 8, 5), (7, 3, 2)):
                got, zr = P.perch_pose_proposals(ctx.ctx, sid, mid, req.label, req.roi, M, N, K)
                want, zw = OP.proposals(sc.depth, sc.labels, req.label, req.roi, sc.fx, sc.fy, sc.cx,
                                        sc.cy, mesh.verts.min(0), mesh.verts.max(0), M, N, K)
                assert zr == zw
                assert np.max(np.abs(got - want)) < 2e-5, (req.mesh_index, M, N, K)
            dp = torch.empty((42 * 8 * 5, 12), dtype=torch.float32, device="cuda")
            dz = torch.empty(2, dtype=torch.int32, device="cuda")
            s = torch.cuda.Stream()
            P.perch_pose_proposals(ctx.ctx, sid, mid, req.label, req.roi, 42, 8, 5, dp, dz, stream=s)
            s.synchronize()
            host, zh = P.perch_pose_proposals(ctx.ctx, sid, mid, req.label, req.roi, 42, 8, 5)
            assert np.array_equal(dp.cpu().numpy(), host) and tuple(dz.cpu().tolist()) == zh
            # the proposals are valid scorer input
            costs = ctx.score(sid, mid, req.label, req.roi, host)
            assert costs.shape == (len(host), 2) and np.all(costs >= 0)
        # a label with no pixel in the box gives an empty depth range
        _, zr = P.perch_pose_proposals(ctx.ctx, sid, mid, 99, sc.requests[0].roi, 2, 2, 2)
        assert zr == (0, 0)
