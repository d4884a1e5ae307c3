"""GPU parity of the rasteriser's tile bins (perch_set_raster_bins).

A hypothesis whose pixel box needs several z-buffer tiles lists each tile's
triangles first and rasterises the tile from that list.  A triangle covers
samples only inside its own sample box, so the z-buffer -- and every count
after it -- must be identical to the unbinned path, bit for bit: with bins
that hold every triangle, with bins that overflow (the tile falls back to
the whole mesh), in the batched form, and against the oracle.
"""
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


@pytest.fixture(scope="module")
def ctx(P):
    c = P.Context(0)
    yield c
    c.close()


def _score_all(ctx, sid, mids, sc, shape, bins):
    ctx.set_launch_config(*shape, bin_cap=bins)
    try:
        return [ctx.score(sid, mids[r.mesh_index], r.label, r.roi, r.poses) for r in sc.requests]
    finally:
        ctx.set_launch_config(256, 8192)


@pytest.mark.parametrize("shape", [(256, 1024, 0), (128, 2048, 2048), (512, 1024, 0)])
def test_bins_equal_unbinned_three_objects(ctx, oracle, shape):
    """Small z-buffers force 2-20 tiles per hypothesis; bins of 64 triangles
    overflow on the 2,500-triangle ellipsoid, bins of 4,096 never do."""
    sc = scenes.tabletop_3obj(W=320, H=240, grid_half=3, n_yaw=4, tri_scale=0.25)
    sid = ctx.set_observation(sc)
    mids = [ctx.load_mesh(m) for m in sc.meshes]
    plain = _score_all(ctx, sid, mids, sc, shape, 0)
    for bins in (64, 4096):
        got = _score_all(ctx, sid, mids, sc, shape, bins)
        for k, (g, p) in enumerate(zip(got, plain)):
            assert np.array_equal(g, p), (shape, bins, k)
    # and the binned costs against the oracle, within the colour band
    for r, g in zip(sc.requests, got):
        osc = oracle.OracleScene.from_scene(sc)
        om = oracle.OracleMesh.from_mesh(sc.meshes[r.mesh_index])
        want, band = oracle.score(osc, om, r.poses, label=r.label, roi=r.roi)
        diff = np.abs(g.astype(np.int64) - want)
        assert np.all(diff[:, 0] <= band) and np.all(diff[:, 1] <= band)
        assert ctx.best(g) == oracle.best(want)


def test_bins_equal_unbinned_labels_and_colour_off(ctx, oracle):
    """6-DoF poses, labels and ROIs; colour off, so bit-exact against the oracle too."""
    sc = scenes.sixdof_5obj(n_hyp=24, W=320, H=240, tri_scale=0.1)
    sc.params.color_check = 0
    sid = ctx.set_observation(sc)
    mids = [ctx.load_mesh(m) for m in sc.meshes]
    plain = _score_all(ctx, sid, mids, sc, (256, 1024, 0), 0)
    got = _score_all(ctx, sid, mids, sc, (256, 1024, 0), 1024)
    for r, g, p in zip(sc.requests, got, plain):
        assert np.array_equal(g, p), r.mesh_index
        osc = oracle.OracleScene.from_scene(sc)
        om = oracle.OracleMesh.from_mesh(sc.meshes[r.mesh_index])
        want, _ = oracle.score(osc, om, r.poses, label=r.label, roi=r.roi)
        assert np.array_equal(g, want), r.mesh_index


def test_bins_in_the_batched_form(ctx, P):
    """One batched call with bins equals the items scored alone without them."""
    batch = scenes.batched_scenes(n_scenes=4, hyp_range=(200, 600))
    specs, poses, alone, off = [], [], [], 0
    mesh_ids = {}
    for sc in batch:
        sid = ctx.set_observation(sc)
        for r in sc.requests:
            m = sc.meshes[r.mesh_index]
            if id(m) not in mesh_ids:
                mesh_ids[id(m)] = ctx.load_mesh(m)
            specs.append((sid, mesh_ids[id(m)], r.label, r.roi, off, len(r.poses)))
            poses.append(r.poses)
            alone.append(ctx.score(sid, mesh_ids[id(m)], r.label, r.roi, r.poses))
            off += len(r.poses)
    poses = np.concatenate(poses)
    ctx.set_launch_config(256, 1024, bin_cap=512)
    try:
        got = P.perch_score_batch(ctx.ctx, P.work_items(specs), poses)
    finally:
        ctx.set_launch_config(256, 8192)
    for k, (_, _, _, _, o, n) in enumerate(specs):
        assert np.array_equal(got[o:o + n], alone[k]), k


def test_bin_capacity_range(ctx, P):
    for bad in (-1, 1, 63, 65537):
        with pytest.raises(P.PerchError):
            P.perch_set_raster_bins(ctx.ctx, bad)
    P.perch_set_raster_bins(ctx.ctx, 64)
    P.perch_set_raster_bins(ctx.ctx, 0)
