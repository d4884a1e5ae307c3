"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Tolerance: depth/key buffers and, with the colour check off, the (J_o, J_r)
counts are bit-exact -- every step that decides them is a fixed sequence of
binary32 operations on both sides.  With the colour check on, each count may
differ from the oracle's by at most the oracle's band count for that
hypothesis (points whose CIEDE2000 difference lies within 1e-3 of tau_c, or
within 1e-3 degree of the hue wrap: there the last-bit differences of the
transcendental functions between glibc and CUDA can flip the decision), and
the best pose must be identical.
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


def assert_within_band(got, want, band, tag=""):
    diff = np.abs(got.astype(np.int64) - want.astype(np.int64))
    ok = (diff[:, 0] <= band) & (diff[:, 1] <= band)
    bad = np.nonzero(~ok)[0]
    assert len(bad) == 0, f"{tag}: {len(bad)} hypotheses outside the band, e.g. {bad[:5]} " \
                          f"got {got[bad[:3]].tolist()} want {want[bad[:3]].tolist()} band {band[bad[:3]].tolist()}"


def _oracle(oracle, sc, req, **over):
    osc = oracle.OracleScene.from_scene(sc, **over)
    om = oracle.OracleMesh.from_mesh(sc.meshes[req.mesh_index])
    return osc, om


def _load(ctx, sc, **over):
    sid = ctx.set_observation(sc, **over)
    mids = [ctx.load_mesh(m) for m in sc.meshes]
    return sid, mids


# ---------------------------------------------------------------------------
# rasteriser: bit-exact key buffers
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("zbuf_words", [16384, 1024])
def test_key_buffers_bitexact(P, ctx, oracle, zbuf_words):
    ctx.set_launch_config(256, zbuf_words)
    cases = [scenes.tabletop_small(),
             scenes.tabletop_3obj(W=320, H=240, grid_half=2, n_yaw=4, tri_scale=0.25),
             scenes.sixdof_5obj(n_hyp=4, W=320, H=240, tri_scale=0.1)]
    try:
        for sc in cases:
            sid, mids = _load(ctx, sc)
            for req in sc.requests:
                osc, om = _oracle(oracle, sc, req)
                for pose in req.poses[:: max(1, len(req.poses) // 3)][:3]:
                    got = ctx.render_keys(sid, mids[req.mesh_index], req.roi, pose, sc.W, sc.H)
                    want, _ = oracle.render_keys(osc, om, pose, req.roi)
                    assert np.array_equal(got, want), (sc.name, int(np.sum(got != want)))
    finally:
        ctx.set_launch_config(256, 8192)


# ---------------------------------------------------------------------------
# costs
# ---------------------------------------------------------------------------

def test_small_colour_off_bitexact(ctx, oracle):
    sc = scenes.tabletop_small()
    sid, mids = _load(ctx, sc)
    req = sc.requests[0]
    got = ctx.score(sid, mids[0], req.label, req.roi, req.poses)
    want, band = oracle.score(*_oracle(oracle, sc, req), req.poses, label=req.label, roi=req.roi)
    assert np.array_equal(got, want)
    assert ctx.best(got) == oracle.best(want)


def test_small_colour_on_band(ctx, oracle):
    sc = scenes.tabletop_small(colour=True)
    sc.params.color_check = 1
    sid, mids = _load(ctx, sc)
    req = sc.requests[0]
    got = ctx.score(sid, mids[0], req.label, req.roi, req.poses)
    want, band = oracle.score(*_oracle(oracle, sc, req), req.poses, label=req.label, roi=req.roi)
    assert_within_band(got, want, band, "small colour")
    assert ctx.best(got) == oracle.best(want)


@pytest.mark.parametrize("delta", [0.0005, 0.03])
def test_cell_bitmap_on_and_off(ctx, oracle, delta):
    """delta 0.5 mm: the observed cloud spans more than 2^27 hash cells, so the
    near-cell filter is off; 3 cm: few, large cells.  Both bit-exact."""
    sc = scenes.tabletop_small(seed=21)
    sc.params.delta_m = delta
    sid, mids = _load(ctx, sc)
    req = sc.requests[0]
    poses = req.poses[::24]
    got = ctx.score(sid, mids[0], req.label, req.roi, poses)
    want, _ = oracle.score(*_oracle(oracle, sc, req), poses, label=req.label, roi=req.roi)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("threads,zbuf_words,mark_bits",
                         [(256, 8192, 0), (128, 1024, 1024), (512, 2048, 2048), (256, 16384, 0)])
def test_three_objects_reduced(ctx, oracle, threads, zbuf_words, mark_bits):
    """3 objects, colour on, occluders; launch shapes that force z-buffer tiles
    and admissible-box bands."""
    sc = scenes.tabletop_3obj(W=320, H=240, grid_half=3, n_yaw=4, tri_scale=0.25)
    sid, mids = _load(ctx, sc)
    ctx.set_launch_config(threads, zbuf_words, mark_bits)
    try:
        for req in sc.requests:
            got = ctx.score(sid, mids[req.mesh_index], req.label, req.roi, req.poses)
            want, band = oracle.score(*_oracle(oracle, sc, req), req.poses, label=req.label,
                                      roi=req.roi)
            assert_within_band(got, want, band, f"3obj mesh {req.mesh_index}")
            assert ctx.best(got) == oracle.best(want)
    finally:
        ctx.set_launch_config(256, 8192)


@pytest.mark.parametrize("mark_bits", [0, 1024])
def test_sixdof_reduced_labels(ctx, oracle, mark_bits):
    sc = scenes.sixdof_5obj(n_hyp=24, W=320, H=240, tri_scale=0.1)
    sid, mids = _load(ctx, sc)
    ctx.set_launch_config(256, 8192, mark_bits)
    try:
        for req in sc.requests:
            got = ctx.score(sid, mids[req.mesh_index], req.label, req.roi, req.poses)
            want, band = oracle.score(*_oracle(oracle, sc, req), req.poses, label=req.label,
                                      roi=req.roi)
            assert_within_band(got, want, band, f"6dof mesh {req.mesh_index}")
            assert ctx.best(got) == oracle.best(want)
    finally:
        ctx.set_launch_config(256, 8192)


def test_variant_without_occluder_marking(ctx, oracle):
    """PERCH 2.0-A: occluder marking off (occ_margin_units = -1)."""
    sc = scenes.tabletop_3obj(W=320, H=240, grid_half=3, n_yaw=4, tri_scale=0.25)
    sc.params.occ_margin_units = -1
    sid, mids = _load(ctx, sc)
    for req in sc.requests:
        got = ctx.score(sid, mids[req.mesh_index], req.label, req.roi, req.poses)
        want, band = oracle.score(*_oracle(oracle, sc, req), req.poses, label=req.label, roi=req.roi)
        assert_within_band(got, want, band, f"2.0-A mesh {req.mesh_index}")


@pytest.mark.parametrize("colour", [0, 1])
@pytest.mark.parametrize("shape", [(256, 8192, 0), (128, 2048, 4096)])
def test_eq3_exact_jo(ctx, oracle, colour, shape):
    """jo_mode 1: J_o as Eq. 3 writes it -- each observed point of V against
    its own nearest rendered point, with the distance test of Eq. 2 and, with
    the colour check on, Eq. 4 applied from the observed side.  Colour off:
    bit-exact; colour on: within the band.  The second launch shape forces
    several z-buffer tiles (the colour pass renders them again) and several
    bands of the admissible box."""
    ctx.set_launch_config(*shape)
    try:
        sc = scenes.tabletop_3obj(W=320, H=240, grid_half=3, n_yaw=4, tri_scale=0.25)
        sc.params.jo_mode = 1
        sc.params.color_check = colour
        sid, mids = _load(ctx, sc)
        for req in sc.requests:
            got = ctx.score(sid, mids[req.mesh_index], req.label, req.roi, req.poses)
            want, band = oracle.score(*_oracle(oracle, sc, req), req.poses, label=req.label, roi=req.roi)
            if colour == 0:
                assert np.array_equal(got, want)
            assert_within_band(got, want, band, f"jo_mode 1 mesh {req.mesh_index}")
        sc6 = scenes.sixdof_5obj(n_hyp=16, W=320, H=240, tri_scale=0.1)
        sc6.params.jo_mode = 1
        sc6.params.color_check = colour
        sid, mids = _load(ctx, sc6)
        for req in sc6.requests:
            got = ctx.score(sid, mids[req.mesh_index], req.label, req.roi, req.poses)
            want, band = oracle.score(*_oracle(oracle, sc6, req), req.poses, label=req.label, roi=req.roi)
            if colour == 0:
                assert np.array_equal(got, want)
            assert_within_band(got, want, band, f"jo_mode 1 6-DoF mesh {req.mesh_index}")
    finally:
        ctx.set_launch_config(256, 8192)


@pytest.mark.parametrize("stride", [2, 3])
def test_stride(ctx, oracle, stride):
    sc = scenes.tabletop_small()
    sc.params.stride = stride
    sid, mids = _load(ctx, sc)
    req = sc.requests[0]
    poses = req.poses[::7]
    got = ctx.score(sid, mids[0], req.label, req.roi, poses)
    want, _ = oracle.score(*_oracle(oracle, sc, req), poses, label=req.label, roi=req.roi)
    assert np.array_equal(got, want)


def test_full_size_three_objects_sampled(ctx, oracle):
    """640x480, 3 x 29,584 hypotheses, bench launch shape; oracle on samples."""
    sc = scenes.tabletop_3obj()
    sid, mids = _load(ctx, sc)
    rng = np.random.default_rng(0)
    for req in sc.requests:
        got = ctx.score(sid, mids[req.mesh_index], req.label, req.roi, req.poses)
        assert got.shape == (len(req.poses), 2) and np.all(got >= 0)
        bi, bc = ctx.best(got)
        J = got.astype(np.int64).sum(1)
        assert bc == J.min() and bi == int(np.nonzero(J == J.min())[0][0])
        pick = np.unique(np.concatenate([[bi], rng.choice(len(req.poses), 3, replace=False)]))
        want, band = oracle.score(*_oracle(oracle, sc, req), req.poses[pick], label=req.label,
                                  roi=req.roi)
        assert_within_band(got[pick], want, band, f"full 3obj mesh {req.mesh_index}")


def test_full_size_sixdof_sampled(ctx, oracle):
    sc = scenes.sixdof_5obj()
    sid, mids = _load(ctx, sc)
    rng = np.random.default_rng(1)
    for req in sc.requests:
        got = ctx.score(sid, mids[req.mesh_index], req.label, req.roi, req.poses)
        pick = np.sort(rng.choice(len(req.poses), 2, replace=False))
        want, band = oracle.score(*_oracle(oracle, sc, req), req.poses[pick], label=req.label,
                                  roi=req.roi)
        assert_within_band(got[pick], want, band, f"full 6dof mesh {req.mesh_index}")


# ---------------------------------------------------------------------------
# invariances, modes, edge cases
# ---------------------------------------------------------------------------

def test_order_invariance_and_determinism(ctx):
    sc = scenes.tabletop_3obj(W=320, H=240, grid_half=4, n_yaw=4, tri_scale=0.25)
    sid, mids = _load(ctx, sc)
    req = sc.requests[1]
    a = ctx.score(sid, mids[1], -1, None, req.poses)
    b = ctx.score(sid, mids[1], -1, None, req.poses)
    assert np.array_equal(a, b)
    perm = np.random.default_rng(4).permutation(len(req.poses))
    c = ctx.score(sid, mids[1], -1, None, req.poses[perm])
    assert np.array_equal(c, a[perm])
    assert ctx.best(c, ids=perm.astype(np.uint64))[1] == ctx.best(a)[1]
    assert perm[ctx.best(c, ids=perm.astype(np.uint64))[0]] == ctx.best(a)[0]


def test_async_device_mode_matches_host_mode(ctx):
    import torch
    sc = scenes.tabletop_small()
    sid, mids = _load(ctx, sc)
    req = sc.requests[0]
    host = ctx.score(sid, mids[0], -1, None, req.poses)
    dev_poses = torch.from_numpy(req.poses).cuda()
    dev_costs = torch.empty((len(req.poses), 2), dtype=torch.int32, device="cuda")
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        ctx.score(sid, mids[0], -1, None, dev_poses, dev_costs, stream=s)
        bi = torch.empty(1, dtype=torch.int64, device="cuda")
        bc = torch.empty(1, dtype=torch.int32, device="cuda")
        ctx.best(dev_costs, stream=s, out_index=bi, out_cost=bc)
    s.synchronize()
    assert np.array_equal(dev_costs.cpu().numpy(), host)
    assert (int(bi.item()), int(bc.item())) == ctx.best(host)


def test_best_matches_oracle(ctx, oracle):
    rng = np.random.default_rng(2)
    for n in (1, 7, 1000, 300_001):
        costs = rng.integers(0, 5, size=(n, 2)).astype(np.int32)
        ids = rng.permutation(n).astype(np.uint64)
        assert ctx.best(costs) == oracle.best(costs)
        assert ctx.best(costs, ids=ids) == oracle.best(costs, ids=ids)


def test_edge_cases(ctx, oracle, P):
    sc = scenes.tabletop_small()
    sid, mids = _load(ctx, sc)
    req = sc.requests[0]
    osc, om = _oracle(oracle, sc, req)
    # n = 0 is a no-op
    assert ctx.score(sid, mids[0], -1, None, np.zeros((0, 12), np.float32)).shape == (0, 2)
    # empty and ragged ROIs
    for roi in [(10, 10, 10, 50), (0, 0, 1, 1), (37, 11, 101, 77), (-5, -5, 500, 500)]:
        got = ctx.score(sid, mids[0], -1, roi, req.poses[:50])
        want, _ = oracle.score(osc, om, req.poses[:50], roi=roi)
        assert np.array_equal(got, want), roi
    # object behind the camera: nothing rendered
    behind = req.poses[:4].copy()
    behind[:, 11] = -1.0
    got = ctx.score(sid, mids[0], -1, None, behind)
    want, _ = oracle.score(osc, om, behind)
    assert np.array_equal(got, want) and np.all(got[:, 1] == 0)
    # an observation with no valid depth: every kept point unexplained, V empty
    sc0 = scenes.tabletop_small()
    sc0.depth[:] = 0
    sid0 = ctx.set_observation(sc0)
    got = ctx.score(sid0, mids[0], -1, None, req.poses[:20])
    want, _ = oracle.score(oracle.OracleScene.from_scene(sc0), om, req.poses[:20])
    assert np.array_equal(got, want) and np.all(got[:, 0] == 0)


def test_wide_image_and_64bit_keys(ctx, oracle):
    """W > 1023 (no vertex cache: triangles set up from the pose directly) at
    the largest image the int32 edge functions allow, and poses beyond 6.5 m
    (64-bit depth keys)."""
    sc = scenes.tabletop_small(seed=33, W=1200, H=388)
    sc.params.stride = 4                      # keeps the brute-force oracle quick
    assert sc.W * sc.H <= 466033
    sid, mids = _load(ctx, sc)
    req = sc.requests[0]
    osc, om = _oracle(oracle, sc, req)
    poses = req.poses[::61]
    got = ctx.score(sid, mids[0], req.label, req.roi, poses)
    want, _ = oracle.score(osc, om, poses, label=req.label, roi=req.roi)
    assert np.array_equal(got, want)
    far = poses.copy().reshape(-1, 3, 4)
    far[:, 2, 3] = 7.0                        # 7 m ahead: depths above 65,535 units
    far = far.reshape(-1, 12)
    sid_all = ctx.set_observation(sc, occ_margin_units=-1)   # keep the far points (no occluders)
    got = ctx.score(sid_all, mids[0], req.label, req.roi, far)
    want, _ = oracle.score(oracle.OracleScene.from_scene(sc, occ_margin=-1), om, far, label=req.label, roi=req.roi)
    assert np.array_equal(got, want) and np.all(want[:, 1] > 0)
    keys = ctx.render_keys(sid, mids[0], req.roi, far[0], sc.W, sc.H)
    wkeys, _ = oracle.render_keys(osc, om, far[0], req.roi)
    assert np.array_equal(keys, wkeys) and np.any((wkeys != EMPTY) & ((wkeys >> np.uint64(32)) > 65535))


def test_errors_and_budget(P):
    sc = scenes.tabletop_small()
    with P.Context(0, hbm_budget_bytes=1 << 16) as small:
        with pytest.raises(P.PerchError) as e:
            small.set_observation(sc)
        assert e.value.status == -3
    with P.Context(0) as c:
        sid = c.set_observation(sc)
        mid = c.load_mesh(sc.meshes[0])
        with pytest.raises(P.PerchError) as e:
            c.score(sid + 100, mid, -1, None, sc.requests[0].poses[:2])
        assert e.value.status == -4
        with pytest.raises(P.PerchError) as e:
            c.score(sid, mid, 3, None, sc.requests[0].poses[:2])      # no labels in this scene
        assert e.value.status == -1
        bad = sc.meshes[0].tris.copy()
        bad[0, 0] = 10 ** 6
        with pytest.raises(P.PerchError):
            P.perch_load_mesh(c.ctx, sc.meshes[0].verts, sc.meshes[0].rgb, bad, 0.03, 0.12)
        used = c.hbm_used
        c.set_observation(sc)
        assert c.hbm_used > used
