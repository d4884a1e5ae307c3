"""Pins of the oracle's Monotone Scene Generation tree (Sec. III, Fig. 2;
variant 2.0-B) to things other than itself.

* from the empty state an edge costs exactly the plain score (Eq. 1 for one
  object);
* a state nearer everywhere hides the object (dJ_r = 0, dJ_o = |I cap V|,
  counted by the plain scorer), a state farther everywhere refuses it;
* placing the same object at the same pose twice costs nothing the second time;
* objects apart in the image and in space add up, in either order;
* an object that would cover a placed one is refused, the reverse order is not;
* beam search with a wide beam finds the exhaustive optimum.
"""
import numpy as np
import pytest

from paper_2008_00326_gb300 import scenes

EMPTY = np.uint64(0xFFFFFFFFFFFFFFFF)


@pytest.fixture(scope="module")
def small(oracle):
    sc = scenes.tabletop_small(seed=12, colour=True)
    osc = oracle.OracleScene.from_scene(sc)
    om = oracle.OracleMesh.from_mesh(sc.meshes[0])
    pick = np.random.default_rng(1).choice(len(sc.requests[0].poses), 30, replace=False)
    return sc, osc, om, sc.requests[0].poses[pick]


def test_root_edge_is_the_plain_score(oracle, small):
    sc, osc, om, poses = small
    want, wband = oracle.score(osc, om, poses)
    got, band = oracle.score_tree(osc, om, poses, oracle.empty_state(osc))
    assert np.array_equal(got, want) and np.array_equal(band, wband)


def test_state_in_front_hides_and_state_behind_refuses(oracle, small):
    sc, osc, om, poses = small
    _, _, work = oracle.score(osc, om, poses, with_work=True)
    d, m, v = oracle.empty_state(osc)
    near = (np.ones_like(d), m, v)
    got, _ = oracle.score_tree(osc, om, poses, near)
    assert np.array_equal(got[:, 1], np.zeros(len(poses), np.int32))
    assert np.array_equal(got[:, 0], work[:, 6].astype(np.int32))      # |I cap V|, none explained
    marked = (d, np.ones_like(m), v)                 # every observed point already explained
    got, _ = oracle.score_tree(osc, om, poses, marked)
    plain, _ = oracle.score(osc, om, poses)
    assert np.array_equal(got[:, 0], np.zeros(len(poses), np.int32))
    assert np.array_equal(got[:, 1], plain[:, 1])
    far = (np.full_like(d, 60000), m, v)
    got, _ = oracle.score_tree(osc, om, poses, far)
    renders = work[:, 3] > 0
    assert renders.all()
    assert np.array_equal(got, np.full((len(poses), 2), -1, np.int32))


def test_same_object_twice_costs_nothing(oracle, small):
    sc, osc, om, poses = small
    gt = sc.requests[0].poses[sc.requests[0].gt_index]
    for h, pose in enumerate(list(poses[:3]) + [gt]):
        c1, _, child = oracle.score_tree(osc, om, pose[None], oracle.empty_state(osc), child=True)
        c2, _ = oracle.score_tree(osc, om, pose[None], child)
        assert np.array_equal(c2, np.zeros((1, 2), np.int32)), h
        d, mk, vol = child
        keys, _ = oracle.render_keys(osc, om, pose)
        lattice = keys != EMPTY
        assert np.array_equal(d[lattice], (keys[lattice] >> np.uint64(32)).astype(np.uint32))
        assert not d[~lattice].any()
        assert vol.sum() >= 1
    # at the true pose the object explains observed points: marks are set
    assert mk.sum() >= 0.5 * (lattice.sum() - c1[0, 1])


def _render_mask(oracle, osc, om, pose):
    keys, _ = oracle.render_keys(osc, om, pose)
    return keys != EMPTY


@pytest.fixture(scope="module")
def three(oracle):
    sc = scenes.tabletop_3obj(W=160, H=120, tri_scale=0.05, grid_half=1, n_yaw=2)
    osc = oracle.OracleScene.from_scene(sc)
    oms = [oracle.OracleMesh.from_mesh(m) for m in sc.meshes]
    return sc, osc, oms


def test_apart_objects_add_up_in_either_order(oracle, three):
    sc, osc, oms = three
    gts = [np.asarray(g, np.float32).reshape(12) for g in sc.gt_poses]
    masks = [_render_mask(oracle, osc, oms[k], gts[k]) for k in range(3)]
    pairs = [(a, b) for a in range(3) for b in range(a + 1, 3) if not np.any(masks[a] & masks[b])]
    assert pairs, "no pair of objects apart in the image"
    for a, b in pairs:
        plain = [int(oracle.score(osc, oms[k], gts[k][None])[0].sum()) for k in (a, b)]
        for first, second in ((a, b), (b, a)):
            c1, _, st = oracle.score_tree(osc, oms[first], gts[first][None], oracle.empty_state(osc),
                                          child=True)
            c2, _ = oracle.score_tree(osc, oms[second], gts[second][None], st)
            assert int(c1.sum()) + int(c2.sum()) == sum(plain), (first, second)


def test_covering_a_placed_object_is_refused(oracle, small):
    sc, osc, om, poses = small
    back = poses[0].reshape(3, 4).astype(np.float64)
    c = back[:, 3]
    front = back.copy()
    front[:, 3] = c * 0.8                      # same object 20 % nearer along the line of sight
    back, front = back.astype(np.float32).reshape(12), front.astype(np.float32).reshape(12)
    assert np.any(_render_mask(oracle, osc, om, back) & _render_mask(oracle, osc, om, front))
    _, _, st_back = oracle.score_tree(osc, om, back[None], oracle.empty_state(osc), child=True)
    refused, _ = oracle.score_tree(osc, om, front[None], st_back)
    assert np.array_equal(refused, [[-1, -1]])
    _, _, st_front = oracle.score_tree(osc, om, front[None], oracle.empty_state(osc), child=True)
    ok, _ = oracle.score_tree(osc, om, back[None], st_front)
    alone, _ = oracle.score_tree(osc, om, back[None], oracle.empty_state(osc))
    assert ok[0, 0] >= 0 and ok[0, 1] <= alone[0, 1]    # partly hidden: fewer rendered points
    # the child composes the nearer surface: the front object's depth where both render
    _, _, both = oracle.score_tree(osc, om, back[None], st_front, child=True)
    df = st_front[0]
    kb, _ = oracle.render_keys(osc, om, back)
    dback = np.where(kb == EMPTY, 0, kb >> np.uint64(32)).astype(np.uint32)
    want = np.where(df == 0, dback, np.where(dback == 0, df, np.minimum(df, dback)))
    assert np.array_equal(both[0], want)


def test_beam_search_matches_exhaustive(oracle, three):
    from oracle import tree
    sc, osc, oms = three
    objs = []
    for k in (0, 1):
        req = sc.requests[k]
        objs.append((oms[k], req.label, req.roi, req.poses[::3][:4]))
    cost, order, pidx = tree.exhaustive(osc, objs)
    got = tree.beam_search(osc, objs, beam=10 ** 6)
    assert got[2][-1] == cost
    assert (got[0], got[1]) == (order, pidx)
    narrow = tree.beam_search(osc, objs, beam=1)
    assert narrow[2][-1] >= cost
