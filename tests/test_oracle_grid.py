"""The oracle's grid nearest-neighbour mode against its brute-force mode.

The grid mode (cells of edge delta (1 + 1/32), the 27 cells around a query)
exists so that whole configurations can be compared with the GPU; it must
give exactly what the brute-force scan of Eq. 2 gives: the same costs, the
same band counts and the same work counters (but the candidate count, which
only the brute force keeps), on tiny scenes in full and on
random hypotheses of every configuration, for both J_o readings, with the
colour check on and off, and for radii that put many points near delta.
"""
import numpy as np
import pytest

from paper_2008_00326_gb300 import scenes


def _both(O, sc, req, poses, **over):
    osc = O.OracleScene.from_scene(sc, **over)
    om = O.OracleMesh.from_mesh(sc.meshes[req.mesh_index])
    a = O.score(osc, om, poses, label=req.label, roi=req.roi, with_work=True, nn="brute")
    b = O.score(osc, om, poses, label=req.label, roi=req.roi, with_work=True, nn="grid")
    return a, b


def _assert_same(a, b, tag):
    for x, y, what in zip(a[:2], b[:2], ("costs", "band")):
        assert np.array_equal(x, y), f"{tag}: {what} differ"
    # every work counter but the delta-cell candidate count (brute force only)
    keep = [i for i in range(a[2].shape[1]) if i != 5]
    assert np.array_equal(a[2][:, keep], b[2][:, keep]), f"{tag}: work counters differ"


@pytest.mark.parametrize("jo_mode", [0, 1])
@pytest.mark.parametrize("colour", [0, 1])
@pytest.mark.parametrize("delta", [0.01, 0.004, 0.0013])
def test_tiny_scene_in_full(oracle, jo_mode, colour, delta):
    sc = scenes.tabletop_small(W=40, H=30, seed=21)
    req = sc.requests[0]
    a, b = _both(oracle, sc, req, req.poses, jo_mode=jo_mode, color_check=colour, delta=delta)
    _assert_same(a, b, f"tiny jo{jo_mode} colour{colour} delta{delta}")
    assert a[0][:, 1].max() > 0


def test_small_scene_in_full(oracle):
    sc = scenes.tabletop_small()
    req = sc.requests[0]
    a, b = _both(oracle, sc, req, req.poses[::3], color_check=1)
    _assert_same(a, b, "tabletop_small")


def test_radius_below_the_coordinate_bound_falls_back(oracle):
    """delta so small that |x / delta| exceeds the grid's coordinate bound:
    the grid mode falls back to the brute force and still agrees."""
    sc = scenes.tabletop_small(W=40, H=30, seed=3)
    req = sc.requests[0]
    a, b = _both(oracle, sc, req, req.poses[::50], delta=2e-7)
    _assert_same(a, b, "fallback")


@pytest.mark.parametrize("name", ["tabletop_3obj", "sixdof_5obj", "batched"])
def test_random_hypotheses_of_every_configuration(oracle, name):
    rng = np.random.default_rng(5)
    if name == "tabletop_3obj":
        sc = scenes.tabletop_3obj()
    elif name == "sixdof_5obj":
        sc = scenes.sixdof_5obj(n_hyp=64)
    else:
        sc = scenes.batched_scenes(n_scenes=3)[2]
    for req in sc.requests[:3]:
        pick = rng.choice(len(req.poses), 2, replace=False)
        for jo in (0, 1):
            a, b = _both(oracle, sc, req, req.poses[pick], jo_mode=jo)
            _assert_same(a, b, f"{name} mesh {req.mesh_index} jo{jo}")
