"""Batched form: many scenes' searches in one call or one replayed graph.

Every item's costs must be identical whether it is scored alone
(perch_score_hypotheses) or inside a batch with other scenes, meshes, label
modes and ROIs, in any item order, and through a replayed CUDA graph; a
sample is also checked against the oracle.
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
def loaded(P):
    ctx = P.Context(0)
    pool = scenes.mesh_pool(tri_counts=(500, 2000, 5000, 10000))
    batch = scenes.batched_scenes(n_scenes=8, hyp_range=(100, 1500), pool=pool)
    batch.append(scenes.tabletop_small())
    mesh_ids = {}
    specs, poses, alone = [], [], []
    off = 0
    for sc in batch:
        sid = ctx.set_observation(sc)
        for req in sc.requests:
            m = sc.meshes[req.mesh_index]
            if id(m) not in mesh_ids:
                mesh_ids[id(m)] = ctx.load_mesh(m)
            mid = mesh_ids[id(m)]
            n = len(req.poses)
            specs.append((sid, mid, req.label, req.roi, off, n))
            poses.append(req.poses)
            alone.append(ctx.score(sid, mid, req.label, req.roi, req.poses))
            off += n
    yield ctx, batch, specs, np.concatenate(poses), alone
    ctx.close()


def _split(costs, specs):
    return [costs[off:off + n] for (_, _, _, _, off, n) in specs]


def test_batch_equals_alone_host_and_device(P, loaded):
    import torch
    ctx, batch, specs, poses, alone = loaded
    items = P.work_items(specs)
    got = P.perch_score_batch(ctx.ctx, items, poses)
    for k, (g, a) in enumerate(zip(_split(got, specs), alone)):
        assert np.array_equal(g, a), k
    dp = torch.from_numpy(poses).cuda()
    dc = torch.full((len(poses), 2), -1, dtype=torch.int32, device="cuda")
    s = torch.cuda.Stream()
    P.perch_score_batch(ctx.ctx, items, dp, dc, stream=s)
    s.synchronize()
    assert np.array_equal(dc.cpu().numpy(), got)


def test_batch_item_order_does_not_matter(P, loaded):
    ctx, batch, specs, poses, alone = loaded
    rng = np.random.default_rng(5)
    order = rng.permutation(len(specs))
    new_specs, new_poses, off = [], [], 0
    for k in order:
        sid, mid, label, roi, o, n = specs[k]
        new_specs.append((sid, mid, label, roi, off, n))
        new_poses.append(poses[o:o + n])
        off += n
    got = P.perch_score_batch(ctx.ctx, P.work_items(new_specs), np.concatenate(new_poses))
    for j, k in enumerate(order):
        o, n = new_specs[j][4], new_specs[j][5]
        assert np.array_equal(got[o:o + n], alone[k])


def test_graph_replay(P, loaded):
    import torch
    ctx, batch, specs, poses, alone = loaded
    items = P.work_items(specs)
    dp = torch.from_numpy(poses).cuda()
    dc = torch.zeros((len(poses), 2), dtype=torch.int32, device="cuda")
    g = P.perch_batch_graph_create(ctx.ctx, items, dp, dc)
    try:
        s = torch.cuda.Stream()
        for rep in range(2):
            dc.fill_(-1)
            P.perch_batch_graph_launch(ctx.ctx, g, s)
            s.synchronize()
            got = dc.cpu().numpy()
            for k, (gk, a) in enumerate(zip(_split(got, specs), alone)):
                assert np.array_equal(gk, a), (rep, k)
        # new poses in the same arrays: reversed order within every item
        rev = np.concatenate([poses[o:o + n][::-1] for (_, _, _, _, o, n) in specs])
        dp.copy_(torch.from_numpy(rev))
        P.perch_batch_graph_launch(ctx.ctx, g, s)
        s.synchronize()
        got = dc.cpu().numpy()
        for k, (gk, a) in enumerate(zip(_split(got, specs), alone)):
            assert np.array_equal(gk, a[::-1]), k
    finally:
        P.perch_batch_graph_destroy(g)


def test_autotune_keeps_results(P, loaded):
    import torch
    ctx, batch, specs, poses, alone = loaded
    items = P.work_items(specs)
    dp = torch.from_numpy(poses).cuda()
    dc = torch.zeros((len(poses), 2), dtype=torch.int32, device="cuda")
    t, z, b = P.perch_autotune(ctx.ctx, items, dp, dc)
    assert t in (128, 256, 512) and z in (2048, 4096, 7064, 8192, 16384) and b in (0, 1024, 4096)
    assert P.perch_autotune(ctx.ctx, items, dp, dc) == (t, z, b)    # remembered for the class
    got = P.perch_score_batch(ctx.ctx, items, poses)
    for k, (g, a) in enumerate(zip(_split(got, specs), alone)):
        assert np.array_equal(g, a), k
    ctx.set_launch_config(256, 8192)


def test_batch_sample_against_oracle(P, loaded, oracle):
    ctx, batch, specs, poses, alone = loaded
    rng = np.random.default_rng(8)
    k = 0
    for sc in batch[:4]:
        osc = oracle.OracleScene.from_scene(sc)
        for req in sc.requests:
            om = oracle.OracleMesh.from_mesh(sc.meshes[req.mesh_index])
            pick = np.sort(rng.choice(len(req.poses), min(3, len(req.poses)), replace=False))
            want, band = oracle.score(osc, om, req.poses[pick], label=req.label, roi=req.roi)
            diff = np.abs(alone[k][pick].astype(np.int64) - want)
            assert np.all(diff[:, 0] <= band) and np.all(diff[:, 1] <= band), (sc.name, req.mesh_index)
            k += 1


def test_batch_rejects_overlap_and_bad_ids(P, loaded):
    ctx, batch, specs, poses, alone = loaded
    bad = list(specs[:2])
    bad[1] = bad[1][:4] + (bad[0][4], bad[1][5])          # second item overlaps the first
    with pytest.raises(P.PerchError):
        P.perch_score_batch(ctx.ctx, P.work_items(bad), poses)
    bad = [(999, specs[0][1], -1, None, 0, 4)]
    with pytest.raises(P.PerchError) as e:
        P.perch_score_batch(ctx.ctx, P.work_items(bad), poses)
    assert e.value.status == -4
