"""Monotone Scene Generation tree search (variant 2.0-B) on the GPU against
the oracle's beam search: with the colour check off the chosen order, poses
and path costs are identical; with it on, the path the GPU returns is priced
by the oracle within the colour band of its points."""
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


def _setup(ctx, oracle, sc, ks, every=1, **over):
    sid = ctx.set_observation(sc, **over)
    osc = oracle.OracleScene.from_scene(sc, **{k: v for k, v in over.items() if k == "color_check"})
    gpu_objs, ora_objs = [], []
    for k in ks:
        req = sc.requests[k]
        m = sc.meshes[req.mesh_index]
        poses = req.poses[::every]
        gpu_objs.append((ctx.load_mesh(m), req.label, req.roi, poses))
        ora_objs.append((oracle.OracleMesh.from_mesh(m), req.label, req.roi, poses))
    return sid, osc, gpu_objs, ora_objs


@pytest.mark.parametrize("beam", [1, 3, 12])
def test_tree_search_matches_oracle(P, ctx, oracle, beam):
    from oracle import tree
    sc = scenes.tabletop_3obj(W=160, H=120, tri_scale=0.05, grid_half=1, n_yaw=2)
    sid, osc, gobj, oobj = _setup(ctx, oracle, sc, (0, 1, 2), color_check=0)
    order, pidx, lc, edges = P.perch_tree_search(ctx.ctx, sid, gobj, beam)
    want = tree.beam_search(osc, oobj, beam)
    assert (order, pidx, lc) == (want[0], want[1], want[2])
    n = [len(o[3]) for o in gobj]
    assert edges >= sum(n)


def test_tree_search_labels_6dof(P, ctx, oracle):
    from oracle import tree
    sc = scenes.sixdof_5obj(n_hyp=6, W=320, H=240, tri_scale=0.1)
    sid, osc, gobj, oobj = _setup(ctx, oracle, sc, (0, 2, 3), color_check=0)
    got = P.perch_tree_search(ctx.ctx, sid, gobj, 2)
    want = tree.beam_search(osc, oobj, 2)
    assert got[:3] == (want[0], want[1], want[2])


def test_tree_search_colour_priced_by_oracle(P, ctx, oracle):
    sc = scenes.tabletop_3obj(W=160, H=120, tri_scale=0.05, grid_half=1, n_yaw=2)
    sid, osc, gobj, oobj = _setup(ctx, oracle, sc, (0, 1, 2))
    order, pidx, lc, _ = P.perch_tree_search(ctx.ctx, sid, gobj, 4)
    state = oracle.empty_state(osc)
    g, slack = 0, 0
    for l, (j, h) in enumerate(zip(order, pidx)):
        mesh, label, roi, poses = oobj[j]
        c, band, state = oracle.score_tree(osc, mesh, poses[h:h + 1], state, label=label, roi=roi, child=True)
        assert c[0, 0] >= 0
        g += int(c[0].sum())
        slack += 2 * int(band[0])
        assert abs(lc[l] - g) <= slack, (l, lc[l], g, slack)
    assert sorted(order) == [0, 1, 2]


def test_tree_search_errors(P, ctx, oracle):
    sc = scenes.tabletop_3obj(W=160, H=120, tri_scale=0.05, grid_half=1, n_yaw=2)
    sid, osc, gobj, oobj = _setup(ctx, oracle, sc, (0, 1), color_check=0)
    with pytest.raises(P.PerchError):
        P.perch_tree_search(ctx.ctx, sid, gobj, 0)
    with pytest.raises(P.PerchError):
        P.perch_tree_search(ctx.ctx, sid, [], 1)
    with pytest.raises(P.PerchError) as e:
        P.perch_tree_search(ctx.ctx, 4242, gobj, 1)
    assert e.value.status == -4
    sid1 = ctx.set_observation(sc, jo_mode=1)
    with pytest.raises(P.PerchError):
        P.perch_tree_search(ctx.ctx, sid1, gobj, 1)
    bad = [(9999,) + gobj[0][1:]]
    with pytest.raises(P.PerchError):
        P.perch_tree_search(ctx.ctx, sid, bad, 1)
