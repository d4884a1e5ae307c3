"""GPU parity of the M2M GICP refinement (Sec. IV-A) against the oracle.

The refined poses and the per-hypothesis (updates, correspondences) must be
bit-identical to the oracle's: both sides evaluate the per-correspondence
terms in binary32 in the same order, round them to multiples of 2^-24 and sum
them exactly in int64, and solve in binary64 with the same operations.
Refined poses are then scored (rendered again) and compared like any other
pose.
"""
import numpy as np
import pytest

from paper_2008_00326_gb300 import scenes

pytestmark = pytest.mark.gpu

EMPTY = np.uint64(0xFFFFFFFFFFFFFFFF)


@pytest.fixture(scope="module")
def P():
    from paper_2008_00326_gb300 import build, perch
    build.build()
    perch.load()
    return perch


@pytest.fixture(scope="module")
def ctx(P):
    c = P.Context(0)
    yield c
    c.close()


def _rot(rng, deg):
    from scipy.spatial.transform import Rotation
    a = rng.normal(size=3)
    return Rotation.from_rotvec(a / np.linalg.norm(a) * np.radians(deg)).as_matrix()


def _perturb(P0, rng, n, deg, metres):
    out = []
    base = P0.reshape(3, 4).astype(np.float64)
    for _ in range(n):
        R = _rot(rng, rng.uniform(0, deg)) @ base[:, :3]
        d = rng.normal(size=3)
        t = base[:, 3] + d / np.linalg.norm(d) * rng.uniform(0, metres)
        out.append(np.concatenate([R, t[:, None]], 1))
    return np.asarray(out, np.float32).reshape(n, 12)


@pytest.fixture(scope="module")
def box_world(P, ctx, oracle):
    """A box rendered by the oracle itself (noise free) at the true pose."""
    mesh = scenes.box_mesh(0.06, 0.08, 0.12, 5, 6, 9)
    r_wc, t_wc = scenes.look_at(0.5, 45.0)
    P0 = scenes.tabletop_pose(r_wc, t_wc, 0.01, -0.02, 0.6).astype(np.float32).reshape(12)
    W, H, f = 160, 120, 150.0
    om = oracle.OracleMesh.from_mesh(mesh)
    tmp = oracle.OracleScene(np.zeros((H, W), np.uint16), np.zeros((H, W, 3), np.uint8), None, f, f,
                             W / 2, H / 2)
    keys, _ = oracle.render_keys(tmp, om, P0)
    depth = np.where(keys == EMPTY, 0, keys >> np.uint64(32)).astype(np.uint16)
    rgb = np.zeros((H, W, 3), np.uint8)
    params = P.perch_default_params(delta_m=0.01, color_check=0)
    sid = P.perch_set_observation(ctx.ctx, depth, rgb, None, f, f, W / 2, H / 2, params)
    mid = ctx.load_mesh(mesh)
    osc = oracle.OracleScene(depth, rgb, None, f, f, W / 2, H / 2, delta=0.01, color_check=0)
    return sid, mid, osc, om, P0


def test_true_pose_is_a_fixed_point(P, ctx, oracle, box_world):
    sid, mid, osc, om, P0 = box_world
    got, info = ctx.refine(sid, mid, -1, None, P0[None])
    want, winfo = oracle.gicp(osc, om, P0[None])
    assert np.array_equal(got, want) and np.array_equal(got[0], P0)
    assert np.array_equal(info, winfo)


@pytest.mark.parametrize("iters", [1, 10, 30])
def test_perturbed_poses_bitexact(P, ctx, oracle, box_world, iters):
    sid, mid, osc, om, P0 = box_world
    rng = np.random.default_rng(40 + iters)
    starts = _perturb(P0, rng, 24, 3.0, 0.006)
    gp = P.perch_default_gicp_params(max_iterations=iters)
    got, info = ctx.refine(sid, mid, -1, None, starts, gp)
    want, winfo = oracle.gicp(osc, om, starts, max_iters=iters)
    assert np.array_equal(info, winfo)
    assert np.array_equal(got.view(np.uint32), want.view(np.uint32))


def test_tabletop_small_refine_then_score(P, ctx, oracle):
    """The paper's order: render, refine, render again and score (noisy raycast
    observation, 968 grid hypotheses, sampled against the oracle)."""
    sc = scenes.tabletop_small(seed=5)
    sid = ctx.set_observation(sc)
    mid = ctx.load_mesh(sc.meshes[0])
    req = sc.requests[0]
    got, info = ctx.refine(sid, mid, req.label, req.roi, req.poses)
    osc = oracle.OracleScene.from_scene(sc)
    om = oracle.OracleMesh.from_mesh(sc.meshes[0])
    pick = np.random.default_rng(6).choice(len(req.poses), 40, replace=False)
    want, winfo = oracle.gicp(osc, om, req.poses[pick], label=req.label, roi=req.roi)
    assert np.array_equal(info[pick], winfo)
    assert np.array_equal(got[pick].view(np.uint32), want.view(np.uint32))
    assert np.any(info[:, 0] > 1)                       # the refinement did move poses
    costs = ctx.score(sid, mid, req.label, req.roi, got)
    wc, band = oracle.score(osc, om, want, label=req.label, roi=req.roi)
    assert np.array_equal(costs[pick], wc)              # colour off: exact


def test_full_size_stride2_sample(P, ctx, oracle):
    """640x480 with the observation (and source) on a stride-2 lattice."""
    sc = scenes.tabletop_3obj(grid_half=2)
    sc.params.stride = 2
    sid = ctx.set_observation(sc)
    osc = oracle.OracleScene.from_scene(sc)
    rng = np.random.default_rng(9)
    for k in (0, 2):
        req = sc.requests[k]
        mid = ctx.load_mesh(sc.meshes[req.mesh_index])
        got, info = ctx.refine(sid, mid, req.label, req.roi, req.poses)
        pick = rng.choice(len(req.poses), 2, replace=False)
        om = oracle.OracleMesh.from_mesh(sc.meshes[req.mesh_index])
        want, winfo = oracle.gicp(osc, om, req.poses[pick], label=req.label, roi=req.roi, max_iters=10)
        assert np.array_equal(info[pick], winfo), k
        assert np.array_equal(got[pick].view(np.uint32), want.view(np.uint32)), k


def test_wide_image_without_vertex_cache(P, ctx, oracle):
    """W > 1023: the refinement renders without the vertex cache."""
    sc = scenes.tabletop_small(seed=34, W=1200, H=388)
    sc.params.stride = 4
    sid = ctx.set_observation(sc)
    mid = ctx.load_mesh(sc.meshes[0])
    req = sc.requests[0]
    poses = req.poses[::97]
    got, info = ctx.refine(sid, mid, req.label, req.roi, poses)
    want, winfo = oracle.gicp(oracle.OracleScene.from_scene(sc), oracle.OracleMesh.from_mesh(sc.meshes[0]),
                              poses, label=req.label, roi=req.roi)
    assert np.array_equal(info, winfo)
    assert np.array_equal(got.view(np.uint32), want.view(np.uint32))


def test_labels_and_roi_6dof(P, ctx, oracle):
    sc = scenes.sixdof_5obj(n_hyp=48, W=320, H=240, tri_scale=0.1)
    sid = ctx.set_observation(sc)
    osc = oracle.OracleScene.from_scene(sc)
    for k in (1, 2):
        req = sc.requests[k]
        mid = ctx.load_mesh(sc.meshes[req.mesh_index])
        got, info = ctx.refine(sid, mid, req.label, req.roi, req.poses)
        om = oracle.OracleMesh.from_mesh(sc.meshes[req.mesh_index])
        want, winfo = oracle.gicp(osc, om, req.poses[:4], label=req.label, roi=req.roi)
        assert np.array_equal(info[:4], winfo), k
        assert np.array_equal(got[:4].view(np.uint32), want.view(np.uint32)), k


def test_device_mode_in_place_and_deterministic(P, ctx, box_world):
    import torch
    sid, mid, osc, om, P0 = box_world
    starts = _perturb(P0, np.random.default_rng(3), 300, 3.0, 0.006)
    host, hinfo = ctx.refine(sid, mid, -1, None, starts)
    s = torch.cuda.Stream()
    d = torch.from_numpy(starts).cuda()
    dinfo = torch.zeros((300, 2), dtype=torch.int32, device="cuda")
    P.perch_refine_hypotheses(ctx.ctx, sid, mid, -1, None, d, None, poses_out=d, info=dinfo, stream=s)
    s.synchronize()
    assert np.array_equal(d.cpu().numpy(), host) and np.array_equal(dinfo.cpu().numpy(), hinfo)
    again, ainfo = ctx.refine(sid, mid, -1, None, starts)
    assert np.array_equal(again, host) and np.array_equal(ainfo, hinfo)


def test_zero_iterations_and_errors(P, ctx, box_world):
    sid, mid, osc, om, P0 = box_world
    starts = _perturb(P0, np.random.default_rng(4), 8, 2.0, 0.004)
    got, info = ctx.refine(sid, mid, -1, None, starts, P.perch_default_gicp_params(max_iterations=0))
    assert np.array_equal(got, starts) and np.array_equal(info, np.zeros((8, 2), np.int32))
    with pytest.raises(P.PerchError) as e:
        ctx.refine(sid, mid, -1, None, starts, P.perch_default_gicp_params(max_source_points=10))
    assert e.value.status == -1
    got, info = P.perch_refine_hypotheses(ctx.ctx, sid, mid, -1, None, starts,
                                          P.perch_default_gicp_params(max_source_points=1 << 20))
    for bad in (dict(epsilon=0.0), dict(epsilon=1.0), dict(min_correspondences=0),
                dict(max_iterations=-1), dict(stop_rotation_rad=float("nan"))):
        with pytest.raises(P.PerchError):
            ctx.refine(sid, mid, -1, None, starts, P.perch_default_gicp_params(**bad))
    with pytest.raises(P.PerchError):
        ctx.refine(9999, mid, -1, None, starts)
