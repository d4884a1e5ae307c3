"""Pins of the oracle's M2M GICP refinement (Sec. IV-A "Parallel M2M GICP",
Sec. III-A's per-successor ICP) to things other than itself.

* the per-correspondence Gauss-Newton terms against a float64 finite-difference
  Jacobian of the GICP residual and numpy's matrix inverse;
* the 6x6 solve against numpy.linalg.solve, the rotation update against
  scipy's rotation of the closed-form angle 2 atan(|w| / 2);
* quantisation ties, triangle normals by their defining properties, observed
  normals of an analytic plane, and the rules that zero them;
* end to end: a pose that renders exactly the observation is a fixed point
  (bit for bit), and perturbed poses move back towards the truth.
"""
import math

import numpy as np
import pytest

from paper_2008_00326_gb300 import scenes

EMPTY = np.uint64(0xFFFFFFFFFFFFFFFF)


def _skew(p):
    return np.array([[0, -p[2], p[1]], [p[2], 0, -p[0]], [-p[1], p[0], 0]], np.float64)


def _unit(rng):
    x = rng.normal(size=3)
    return x / np.linalg.norm(x)


def _reference_terms(Rf, tf, a, na, b, nb, eps):
    """GN terms from the definition: r(xi) = b - ((I + [w]x) p + v), p = Rf a + tf,
    Jacobian by central differences, M = (C_b + C_a')^-1 with C(n) = I - (1-eps) n n^T."""
    Rf = np.asarray(Rf, np.float64).reshape(3, 3)
    p = Rf @ np.asarray(a, np.float64) + np.asarray(tf, np.float64)
    m = Rf @ np.asarray(na, np.float64)
    nb = np.asarray(nb, np.float64)
    e = 1.0 - eps
    C = (np.eye(3) - e * np.outer(nb, nb)) + (np.eye(3) - e * np.outer(m, m))
    M = np.linalg.inv(C)

    def r(xi):
        return np.asarray(b, np.float64) - ((np.eye(3) + _skew(xi[:3])) @ p + xi[3:])

    J = np.zeros((3, 6))
    h = 1e-3
    for k in range(6):
        d = np.zeros(6)
        d[k] = h
        J[:, k] = (r(d) - r(-d)) / (2 * h)
    r0 = r(np.zeros(6))
    H = J.T @ M @ J
    g = J.T @ M @ r0
    iu = np.triu_indices(6)
    return np.concatenate([H[iu], g, [r0 @ M @ r0]])


@pytest.mark.parametrize("seed", range(6))
def test_terms_match_finite_difference_gauss_newton(oracle, seed):
    from scipy.spatial.transform import Rotation
    rng = np.random.default_rng(seed)
    Rf = Rotation.from_rotvec(rng.normal(size=3) * (0.0 if seed == 0 else 0.2)).as_matrix()
    tf = np.zeros(3) if seed == 0 else rng.normal(size=3) * 0.01
    a = np.array([0.05, -0.03, 0.6]) + rng.normal(size=3) * 0.05
    na, nb = _unit(rng), _unit(rng)
    if seed == 1:
        nb = np.zeros(3)                       # observed point without a normal: C_b = I
    b = Rf @ a + tf + rng.normal(size=3) * 0.004
    Rf32, tf32 = Rf.astype(np.float32), tf.astype(np.float32)
    ok, got = oracle.gicp_terms(Rf32, tf32, a.astype(np.float32), na.astype(np.float32),
                                b.astype(np.float32), nb.astype(np.float32), 1e-3)
    assert ok
    ref = _reference_terms(Rf32.astype(np.float64), tf32.astype(np.float64), a.astype(np.float32),
                           na.astype(np.float32), b.astype(np.float32), nb.astype(np.float32), 1e-3)
    scale = np.max(np.abs(ref))
    np.testing.assert_allclose(got, ref, rtol=2e-3, atol=2e-4 * scale)


def test_terms_skip_oversized(oracle):
    # a point 1e4 m away makes the rotation terms exceed the bound: no terms
    ok, _ = oracle.gicp_terms(np.eye(3), np.zeros(3), [1e4, 0, 0], [0, 0, 1], [1e4, 0, 0.001],
                              [0, 0, 1], 1e-3)
    assert not ok


def test_quantise_ties_to_even(oracle):
    u = 2.0 ** -24
    assert oracle.gicp_quantise(1.0) == 2 ** 24
    assert oracle.gicp_quantise(0.5 * u) == 0
    assert oracle.gicp_quantise(1.5 * u) == 2
    assert oracle.gicp_quantise(2.5 * u) == 2
    assert oracle.gicp_quantise(-1.5 * u) == -2
    assert oracle.gicp_quantise(-3.0) == -3 * 2 ** 24


def _pack(H, g):
    iu = np.triu_indices(6)
    vals = np.concatenate([H[iu], g, [0.0]])
    return np.rint(vals * 2.0 ** 24).astype(np.int64)


@pytest.mark.parametrize("seed", range(4))
def test_solve_matches_numpy(oracle, seed):
    rng = np.random.default_rng(100 + seed)
    A = rng.normal(size=(9, 6)) * rng.uniform(0.1, 30.0)
    H = A.T @ A + np.eye(6) * 0.01
    g = rng.normal(size=6) * 5.0
    S = _pack(H, g)
    Hq = np.zeros((6, 6))
    iu = np.triu_indices(6)
    Hq[iu] = S[:21] / 2.0 ** 24
    Hq = Hq + np.triu(Hq, 1).T
    gq = S[21:27] / 2.0 ** 24
    ok, xi = oracle.gicp_solve(S)
    assert ok
    np.testing.assert_allclose(xi, np.linalg.solve(Hq, -gq), rtol=1e-8, atol=1e-12)


def test_solve_rejects_indefinite(oracle):
    H = np.diag([1.0, 2.0, -0.5, 1.0, 1.0, 1.0])
    ok, _ = oracle.gicp_solve(_pack(H, np.ones(6)))
    assert not ok
    ok, _ = oracle.gicp_solve(np.zeros(28, np.int64))
    assert not ok


@pytest.mark.parametrize("norm", [0.0, 1e-4, 0.01, 0.3, 1.0, 3.0])
def test_rotation_update_closed_form(oracle, norm):
    from scipy.spatial.transform import Rotation
    rng = np.random.default_rng(int(norm * 1000) + 7)
    w = _unit(rng) * norm
    R = oracle.gicp_rotation(w)
    if norm == 0.0:
        assert np.array_equal(R, np.eye(3))
        return
    ref = Rotation.from_rotvec(w / norm * 2.0 * math.atan(norm / 2.0)).as_matrix()
    np.testing.assert_allclose(R, ref, atol=1e-14)
    np.testing.assert_allclose(R @ R.T, np.eye(3), atol=1e-14)


def test_triangle_normals_are_unit_orthogonal_right_handed(oracle):
    rng = np.random.default_rng(3)
    v = rng.normal(size=(30, 3)).astype(np.float32)
    t = rng.integers(0, 30, size=(40, 3)).astype(np.int32)
    t = t[(t[:, 0] != t[:, 1]) & (t[:, 1] != t[:, 2]) & (t[:, 0] != t[:, 2])]
    om = oracle.OracleMesh(v, np.zeros((30, 3), np.uint8), t, 0.1, 0.1)
    for k in range(len(t)):
        n = oracle.triangle_normal(om, k).astype(np.float64)
        e1 = (v[t[k, 1]] - v[t[k, 0]]).astype(np.float64)
        e2 = (v[t[k, 2]] - v[t[k, 0]]).astype(np.float64)
        assert abs(np.linalg.norm(n) - 1.0) < 1e-6
        assert abs(n @ e1) < 1e-5 * np.linalg.norm(e1) and abs(n @ e2) < 1e-5 * np.linalg.norm(e2)
        assert np.linalg.det(np.stack([e1, e2, n])) > 0
    # degenerate (collinear) triangle: zero normal
    vd = np.array([[0, 0, 0], [1, 0, 0], [2, 0, 0]], np.float32)
    om = oracle.OracleMesh(vd, np.zeros((3, 3), np.uint8), np.array([[0, 1, 2]], np.int32), 0.1, 0.1)
    assert np.array_equal(oracle.triangle_normal(om, 0), np.zeros(3, np.float32))


def _plane_scene(oracle, n, c, W=160, H=120, f=150.0):
    """Depth image of the plane n . X = c (0.1 mm, rounded)."""
    u, v = np.meshgrid(np.arange(W), np.arange(H))
    ray = np.stack([(u - W / 2) / f, (v - H / 2) / f, np.ones_like(u, dtype=np.float64)], -1)
    Z = c / (ray @ n)
    depth = np.rint(Z * 1e4).astype(np.uint16)
    return depth, oracle.OracleScene(depth, np.zeros((H, W, 3), np.uint8), None, f, f, W / 2, H / 2)


def test_observed_normal_of_a_plane(oracle):
    n = np.array([0.3, -0.2, -1.0])
    n /= np.linalg.norm(n)
    depth, osc = _plane_scene(oracle, n, n @ np.array([0.0, 0.0, 0.4]))   # passes through Z = 0.4 m
    for (u, v) in [(80, 60), (10, 10), (150, 110), (33, 97)]:
        got = oracle.observed_normal(osc, u, v).astype(np.float64)
        assert abs(np.linalg.norm(got) - 1) < 1e-5
        ang = math.degrees(math.acos(min(1.0, abs(got @ n))))
        assert ang < 3.0, (u, v, ang)


def test_observed_normal_zero_cases(oracle):
    n = np.array([0.0, 0.0, -1.0])
    depth, osc = _plane_scene(oracle, n, -0.5)
    assert np.any(oracle.observed_normal(osc, 50, 50) != 0)
    for (u, v) in [(0, 50), (159, 50), (50, 0), (50, 119)]:      # image border
        assert np.array_equal(oracle.observed_normal(osc, u, v), np.zeros(3, np.float32))
    d2 = depth.copy()
    d2[50, 51] = 0                                                # a missing neighbour
    osc2 = oracle.OracleScene(d2, np.zeros((120, 160, 3), np.uint8), None, 150, 150, 80, 60)
    assert np.array_equal(oracle.observed_normal(osc2, 50, 50), np.zeros(3, np.float32))
    d3 = depth.copy()
    d3[:, 51:] += 300                                             # a 3 cm step right of u = 50
    osc3 = oracle.OracleScene(d3, np.zeros((120, 160, 3), np.uint8), None, 150, 150, 80, 60)
    assert np.array_equal(oracle.observed_normal(osc3, 50, 50, normal_jump=200), np.zeros(3, np.float32))
    assert np.any(oracle.observed_normal(osc3, 50, 50, normal_jump=400) != 0)


def _box_world(oracle):
    """A 6x8x12 cm box seen by the tabletop camera; the observation is the
    oracle's own render at the true pose (noise free), so the true pose
    renders exactly the observed cloud."""
    mesh = scenes.box_mesh(0.06, 0.08, 0.12, 5, 6, 9)
    r_wc, t_wc = scenes.look_at(0.5, 45.0)
    P = scenes.tabletop_pose(r_wc, t_wc, 0.01, -0.02, 0.6).astype(np.float32).reshape(12)
    W, H, f = 160, 120, 150.0
    om = oracle.OracleMesh.from_mesh(mesh)
    tmp = oracle.OracleScene(np.zeros((H, W), np.uint16), np.zeros((H, W, 3), np.uint8), None, f, f,
                             W / 2, H / 2)
    keys, _ = oracle.render_keys(tmp, om, P)
    depth = np.where(keys == EMPTY, 0, keys >> np.uint64(32)).astype(np.uint16)
    osc = oracle.OracleScene(depth, np.zeros((H, W, 3), np.uint8), None, f, f, W / 2, H / 2,
                             delta=0.01, color_check=0)
    return osc, om, P


def test_true_pose_is_a_fixed_point(oracle):
    osc, om, P = _box_world(oracle)
    out, info = oracle.gicp(osc, om, P[None])
    assert np.array_equal(out[0], P)
    assert info[0, 0] == 1                      # one (zero) update, then converged
    keys, _ = oracle.render_keys(osc, om, P)
    assert info[0, 1] == int(np.sum(keys != EMPTY))


def _pose_error(A, B):
    A = A.reshape(3, 4).astype(np.float64)
    B = B.reshape(3, 4).astype(np.float64)
    dR = A[:, :3] @ B[:, :3].T
    ang = math.degrees(math.acos(max(-1.0, min(1.0, (np.trace(dR) - 1) / 2))))
    return np.linalg.norm(A[:, 3] - B[:, 3]), ang


def test_perturbed_poses_move_back(oracle):
    from scipy.spatial.transform import Rotation
    osc, om, P = _box_world(oracle)
    rng = np.random.default_rng(21)
    starts = []
    for k in range(4):
        R = Rotation.from_rotvec(_unit(rng) * math.radians(1.0)).as_matrix() @ P.reshape(3, 4)[:, :3]
        t = P.reshape(3, 4)[:, 3] + _unit(rng) * 0.003
        starts.append(np.concatenate([R, t[:, None]], 1).astype(np.float32).reshape(12))
    starts = np.stack(starts)
    out, info = oracle.gicp(osc, om, starts, max_iters=30)
    for k in range(len(starts)):
        t0, a0 = _pose_error(starts[k], P)
        t1, a1 = _pose_error(out[k], P)
        assert t1 < 0.25 * t0 and a1 < 0.25 * a0, (k, t0, a0, t1, a1)
        assert info[k, 0] >= 2 and info[k, 1] > 100
