"""Pins of the oracle's cost (Eq. 1-4, Sec. IV-A/B, V-C) to things other than itself.

* nearest neighbours and the J_r / J_o bookkeeping against scipy's k-d tree;
* a ground-truth pose on a noise-free scene scores J = 0 and is the minimum;
* hypothesis-order invariance of costs and of the best id;
* closed-form occluder, admissible-cylinder, stride and back-projection cases.
"""
import math

import numpy as np
import pytest

from paper_2008_00326_gb300 import scenes

EMPTY = np.uint64(0xFFFFFFFFFFFFFFFF)


def _pose(R, t):
    return np.concatenate([np.asarray(R, np.float64), np.asarray(t, np.float64)[:, None]], 1).astype(
        np.float32).reshape(12)


def _tiny_mesh(oracle):
    """One small triangle (for scenes where only the observed side matters)."""
    v = np.array([[0, 0, 0], [0.001, 0, 0], [0, 0.001, 0]], np.float32)
    return v


@pytest.fixture(scope="module")
def small(oracle):
    sc = scenes.tabletop_small(seed=11, noise_m=0.002)
    sc.params.color_check = 1
    return sc


def _kdtree_costs(oracle, osc, om, pose, label, roi, delta, tau, colour, vol):
    from scipy.spatial import cKDTree
    keys, _ = oracle.render_keys(osc, om, pose, roi)
    q, qrgb, _ = oracle.rendered_points(osc, om, pose, keys, label)
    I, Ilab, Ipix = oracle.observed_points(osc)
    tree = cKDTree(I.astype(np.float64))
    dist, idx = tree.query(q.astype(np.float64), k=2)
    ambiguous = 0
    marks = np.zeros(len(I), bool)
    Jr = 0
    for k in range(len(q)):
        d0, j = dist[k, 0], idx[k, 0]
        if abs(dist[k, 1] - d0) < 1e-9:
            j = min(idx[k, 0], idx[k, 1])
            ambiguous += 1
        if abs(d0 - delta) < 1e-6:
            ambiguous += 1
        ok = d0 <= delta
        if ok and colour:
            dE, gap = oracle.ciede2000(oracle.srgb_to_lab(qrgb[k]), Ilab[j])
            if abs(dE - tau) < 1e-3 or gap < 1e-3:
                ambiguous += 1
            ok = dE <= tau
        if ok:
            marks[j] = True
        else:
            Jr += 1
    R = pose.reshape(3, 4)[:, :3].astype(np.float64)
    t = pose.reshape(3, 4)[:, 3].astype(np.float64)
    pl = (I.astype(np.float64) - t) @ R           # R^T (p - t), row-wise
    r, h = vol
    rad2 = pl[:, 0] ** 2 + pl[:, 1] ** 2
    inside = (rad2 <= r * r) & (pl[:, 2] >= 0) & (pl[:, 2] <= h)
    ambiguous += int(np.sum(np.abs(np.sqrt(rad2) - r) < 1e-6) + np.sum(np.abs(pl[:, 2]) < 1e-7)
                     + np.sum(np.abs(pl[:, 2] - h) < 1e-6))
    Jo = int(np.sum(inside & ~marks))
    return (Jo, Jr), ambiguous


@pytest.mark.parametrize("colour", [0, 1])
def test_costs_match_kdtree(oracle, small, colour):
    sc = small
    osc = oracle.OracleScene.from_scene(sc, color_check=colour)
    mesh = sc.meshes[0]
    om = oracle.OracleMesh.from_mesh(mesh)
    req = sc.requests[0]
    rng = np.random.default_rng(3)
    pick = np.unique(np.concatenate([[req.gt_index], rng.choice(len(req.poses), 7, replace=False)]))
    costs, band = oracle.score(osc, om, req.poses[pick])
    for n, h in enumerate(pick):
        want, amb = _kdtree_costs(oracle, osc, om, req.poses[h], -1, (0, 0, sc.W, sc.H),
                                  sc.params.delta_m, sc.params.tau_c, colour,
                                  (mesh.vol_radius, mesh.vol_height))
        got = tuple(int(c) for c in costs[n])
        if amb == 0:
            assert got == want, (h, got, want)
        else:
            assert abs(got[0] - want[0]) <= amb and abs(got[1] - want[1]) <= amb


def test_eq3_jo_matches_kdtree(oracle, small):
    """jo_mode 1 (Eq. 3 as written, Eq. 2 test): J_o = points of I cap V with
    no rendered point within delta, checked with scipy's k-d tree."""
    from scipy.spatial import cKDTree
    sc = small
    osc = oracle.OracleScene.from_scene(sc, jo_mode=1, color_check=0)
    mesh = sc.meshes[0]
    om = oracle.OracleMesh.from_mesh(mesh)
    req = sc.requests[0]
    pick = np.unique(np.concatenate([[req.gt_index], np.arange(0, len(req.poses), 97)]))
    costs, _ = oracle.score(osc, om, req.poses[pick])
    costs0, _ = oracle.score(oracle.OracleScene.from_scene(sc, color_check=0), om, req.poses[pick])
    assert np.array_equal(costs[:, 1], costs0[:, 1])            # J_r does not depend on the mode
    I, _, _ = oracle.observed_points(osc)
    for n, h in enumerate(pick):
        pose = req.poses[h]
        keys, _ = oracle.render_keys(osc, om, pose)
        q, _, _ = oracle.rendered_points(osc, om, pose, keys)
        R = pose.reshape(3, 4)[:, :3].astype(np.float64)
        t = pose.reshape(3, 4)[:, 3].astype(np.float64)
        pl = (I.astype(np.float64) - t) @ R
        inside = ((pl[:, 0] ** 2 + pl[:, 1] ** 2) <= mesh.vol_radius ** 2) & (pl[:, 2] >= 0) & \
                 (pl[:, 2] <= mesh.vol_height)
        if len(q):
            d, _ = cKDTree(q.astype(np.float64)).query(I[inside].astype(np.float64), k=1)
        else:
            d = np.full(int(inside.sum()), np.inf)
        assert np.min(np.abs(d - sc.params.delta_m)) > 1e-6
        assert costs[n, 0] == int(np.sum(d > sc.params.delta_m)), h


def test_eq3_jo_with_colour_matches_kdtree(oracle, small):
    """jo_mode 1 with the colour check (Eq. 3 with Eq. 4 applied from the
    observed side): p in I cap V is an inlier iff its nearest rendered point
    (scipy's k-d tree, ties to the lower index) lies within delta and their
    CIEDE2000 difference is at most tau_c.  Hypotheses near the ground truth,
    where many observed points pass the distance test and the colour decides."""
    from scipy.spatial import cKDTree
    sc = small
    tau = 12.5
    osc = oracle.OracleScene.from_scene(sc, jo_mode=1, color_check=1, tau_c=tau)
    mesh = sc.meshes[0]
    om = oracle.OracleMesh.from_mesh(mesh)
    req = sc.requests[0]
    g = req.gt_index
    pick = np.unique(np.clip(np.array([g, g - 1, g + 1, g - 8, g + 8, g - 88, g + 88, g + 3]), 0, len(req.poses) - 1))
    costs, band = oracle.score(osc, om, req.poses[pick])
    I, Ilab, _ = oracle.observed_points(osc)
    colour_decided = 0
    for n, h in enumerate(pick):
        pose = req.poses[h]
        keys, _ = oracle.render_keys(osc, om, pose)
        q, qrgb, _ = oracle.rendered_points(osc, om, pose, keys)
        R = pose.reshape(3, 4)[:, :3].astype(np.float64)
        t = pose.reshape(3, 4)[:, 3].astype(np.float64)
        pl = (I.astype(np.float64) - t) @ R
        inside = np.nonzero(((pl[:, 0] ** 2 + pl[:, 1] ** 2) <= mesh.vol_radius ** 2) & (pl[:, 2] >= 0) &
                            (pl[:, 2] <= mesh.vol_height))[0]
        jo, amb = 0, 0
        tree = cKDTree(q.astype(np.float64)) if len(q) else None
        for j in inside:
            if tree is None:
                jo += 1
                continue
            d, k = tree.query(I[j].astype(np.float64), k=2)
            kk = int(k[0])
            if abs(d[1] - d[0]) < 1e-9:
                kk = int(min(k[0], k[1]))
                amb += 1
            if abs(d[0] - sc.params.delta_m) < 1e-6:
                amb += 1
            ok = d[0] <= sc.params.delta_m
            if ok:
                dE, gap = oracle.ciede2000(oracle.srgb_to_lab(qrgb[kk]), Ilab[j])
                if abs(dE - tau) < 1e-3 or gap < 1e-3:
                    amb += 1
                colour_decided += dE > tau
                ok = dE <= tau
            jo += not ok
        assert abs(int(costs[n, 0]) - jo) <= amb, (h, costs[n, 0], jo, amb)
    assert colour_decided > 0          # the colour term changed some decisions


def _observation_from_render(oracle, sc, pose):
    """Noise-free observation made by the oracle's own renderer at `pose`."""
    blank = oracle.OracleScene(np.zeros((sc.H, sc.W), np.uint16), np.zeros((sc.H, sc.W, 3), np.uint8),
                               None, sc.fx, sc.fy, sc.cx, sc.cy, stride=1)
    om = oracle.OracleMesh.from_mesh(sc.meshes[0])
    keys, _ = oracle.render_keys(blank, om, pose)
    _, rgb, pix = oracle.rendered_points(blank, om, pose, keys)
    depth = np.zeros(sc.H * sc.W, np.uint16)
    col = np.zeros((sc.H * sc.W, 3), np.uint8)
    depth[pix] = (keys.reshape(-1)[pix] >> np.uint64(32)).astype(np.uint16)
    col[pix] = rgb
    return depth.reshape(sc.H, sc.W), col.reshape(sc.H, sc.W, 3)


def test_ground_truth_pose_is_minimal(oracle):
    sc = scenes.tabletop_small(seed=5, noise_m=0.0)
    req = sc.requests[0]
    depth, rgb = _observation_from_render(oracle, sc, req.poses[req.gt_index])
    osc = oracle.OracleScene(depth, rgb, None, sc.fx, sc.fy, sc.cx, sc.cy, delta=0.01,
                             color_check=1, tau_c=12.5)
    om = oracle.OracleMesh.from_mesh(sc.meshes[0])
    costs, band = oracle.score(osc, om, req.poses)
    J = costs.sum(1)
    assert tuple(costs[req.gt_index]) == (0, 0)
    osc1 = oracle.OracleScene(depth, rgb, None, sc.fx, sc.fy, sc.cx, sc.cy, delta=0.01,
                              color_check=1, tau_c=12.5, jo_mode=1)
    assert tuple(oracle.score(osc1, om, req.poses[req.gt_index][None])[0][0]) == (0, 0)
    # with the colour check on, the box's 180-degree twin no longer ties
    assert np.sum(J == 0) == 1
    assert oracle.best(costs) == (req.gt_index, 0)


def test_order_invariance(oracle, small):
    osc = oracle.OracleScene.from_scene(small)
    om = oracle.OracleMesh.from_mesh(small.meshes[0])
    poses = small.requests[0].poses[:200]
    costs, _ = oracle.score(osc, om, poses)
    perm = np.random.default_rng(9).permutation(len(poses))
    costs_p, _ = oracle.score(osc, om, poses[perm])
    assert np.array_equal(costs_p, costs[perm])
    bi, bc = oracle.best(costs)
    bi_p, bc_p = oracle.best(costs_p, ids=perm.astype(np.uint64))
    assert bc == bc_p and perm[bi_p] == bi


def test_best_ties_to_lowest_id(oracle):
    costs = np.array([[3, 4], [1, 2], [2, 1], [0, 9]], np.int32)
    assert oracle.best(costs) == (1, 3)
    assert oracle.best(costs, ids=np.array([9, 7, 5, 1], np.uint64)) == (2, 3)


def _wall_scene(oracle, z_units, W=64, H=48, f=60.0, labels=None, **kw):
    depth = np.full((H, W), z_units, np.uint16)
    rgb = np.full((H, W, 3), 100, np.uint8)
    return oracle.OracleScene(depth, rgb, labels, f, f, W / 2, H / 2, **kw)


def test_occluders_remove_hidden_points(oracle):
    box = scenes.box_mesh(0.06, 0.08, 0.12, 2, 2, 2)
    om = oracle.OracleMesh.from_mesh(box)
    pose = _pose(np.eye(3), (0.0, 0.0, 0.5))
    sc = _wall_scene(oracle, 3000, delta=0.01, occ_margin=100)      # wall at 0.3 m, in front
    costs, _ = oracle.score(sc, om, pose[None])
    assert tuple(costs[0]) == (0, 0)            # everything hidden, V holds no wall point
    # a margin beyond the gap keeps every rendered point: all unexplained
    sc_far = _wall_scene(oracle, 3000, delta=0.01, occ_margin=60000)
    keys, _ = oracle.render_keys(sc_far, om, pose)
    n_vis = int(np.sum(keys != EMPTY))
    costs, _ = oracle.score(sc_far, om, pose[None])
    assert tuple(costs[0]) == (0, n_vis)
    # labels: occluders that carry the object's own label do not hide it (Sec. V-C)
    lab = np.full((48, 64), 4, np.int32)
    sc_lab = _wall_scene(oracle, 3000, labels=lab, delta=0.01, occ_margin=100)
    costs, _ = oracle.score(sc_lab, om, pose[None], label=4, roi=(0, 0, 64, 48))
    assert costs[0, 1] == n_vis
    costs, _ = oracle.score(sc_lab, om, pose[None], label=3, roi=(0, 0, 64, 48))
    assert tuple(costs[0]) == (0, 0)            # label 3 owns no pixel: V empty, all hidden


def test_variant_without_occluder_marking(oracle):
    """PERCH 2.0-A (Sec. VI-A): with occluder marking off nothing is hidden."""
    box = scenes.box_mesh(0.06, 0.08, 0.12, 2, 2, 2)
    om = oracle.OracleMesh.from_mesh(box)
    pose = _pose(np.eye(3), (0.0, 0.0, 0.5))
    sc_on = _wall_scene(oracle, 3000, delta=0.01, occ_margin=100)
    sc_off = _wall_scene(oracle, 3000, delta=0.01, occ_margin=-1)
    keys, _ = oracle.render_keys(sc_off, om, pose)
    n_vis = int(np.sum(keys != EMPTY))
    assert tuple(oracle.score(sc_on, om, pose[None])[0][0]) == (0, 0)
    assert tuple(oracle.score(sc_off, om, pose[None])[0][0]) == (0, n_vis)


def test_admissible_cylinder_count(oracle):
    W, H, f = 64, 48, 60.0
    sc = _wall_scene(oracle, 5000, W=W, H=H, f=f, delta=0.01)
    r, h = 0.0523, 0.1
    v = _tiny_mesh(oracle)
    om = oracle.OracleMesh(v, np.zeros((3, 3), np.uint8), np.array([[0, 1, 2]], np.int32), r, h)
    tx, ty = 0.013, -0.021
    pose = _pose(np.eye(3), (tx, ty, 0.5 - h / 2))
    pose_far = pose.copy()
    # the tiny triangle itself sits far to the side so that nothing is rendered
    om_far = oracle.OracleMesh(v + np.float32([5.0, 0, 0]), np.zeros((3, 3), np.uint8),
                               np.array([[0, 1, 2]], np.int32), r, h)
    costs, _ = oracle.score(sc, om_far, pose_far[None])
    us, vs = np.meshgrid(np.arange(W), np.arange(H))
    x = (us - W / 2) * 0.5 / f - tx
    y = (vs - H / 2) * 0.5 / f - ty
    rho = np.sqrt(x * x + y * y)
    assert np.min(np.abs(rho - r)) > 1e-5          # no boundary ambiguity
    assert tuple(costs[0]) == (int(np.sum(rho <= r)), 0)


def test_stride_and_backprojection_roundtrip(oracle):
    W, H, f = 64, 48, 60.0
    s = 0.15
    verts = np.array([[-s, -s, 0], [s, -s, 0], [s, s, 0], [-s, s, 0]], np.float32)
    tris = np.array([[0, 1, 2], [0, 2, 3]], np.int32)
    om = oracle.OracleMesh(verts, np.zeros((4, 3), np.uint8), tris, 0.05, 0.1)
    ang = math.radians(25.0)
    R = np.array([[math.cos(ang), 0, math.sin(ang)], [0, 1, 0], [-math.sin(ang), 0, math.cos(ang)]])
    pose = _pose(R, (0.0, 0.0, 0.4))
    for stride in (1, 2, 3):
        sc = oracle.OracleScene(np.zeros((H, W), np.uint16), np.zeros((H, W, 3), np.uint8), None,
                                f, f, W / 2, H / 2, stride=stride)
        keys, _ = oracle.render_keys(sc, om, pose)
        q, _, pix = oracle.rendered_points(sc, om, pose, keys)
        cov = keys.reshape(-1) != EMPTY
        u, v = np.arange(W * H) % W, np.arange(W * H) // W
        assert len(q) == int(np.sum(cov & (u % stride == 0) & (v % stride == 0)))
        n = R[:, 2]
        c = float(n @ np.array([0.0, 0.0, 0.4]))
        assert np.max(np.abs(q.astype(np.float64) @ n - c)) < 2e-4
        # back-projection lands on the pixel's own ray
        pu = q[:, 0] / q[:, 2] * f + W / 2
        pv = q[:, 1] / q[:, 2] * f + H / 2
        assert np.max(np.abs(pu - pix % W)) < 1e-3 and np.max(np.abs(pv - pix // W)) < 1e-3
    full = oracle.OracleScene(np.full((H, W), 777, np.uint16), np.zeros((H, W, 3), np.uint8), None,
                              f, f, W / 2, H / 2, stride=2)
    assert len(oracle.observed_points(full)[0]) == (W // 2) * (H // 2)
