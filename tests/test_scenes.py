"""The seeded input generator is deterministic and produces the stated shapes."""
import numpy as np

from paper_2008_00326_gb300 import scenes


def test_deterministic_and_shapes():
    a = scenes.tabletop_small()
    b = scenes.tabletop_small()
    assert np.array_equal(a.depth, b.depth) and np.array_equal(a.rgb, b.rgb)
    assert np.array_equal(a.requests[0].poses, b.requests[0].poses)
    assert a.meshes[0].n_tris == 516 and a.requests[0].poses.shape == (968, 12)
    assert a.depth.dtype == np.uint16 and a.requests[0].poses.dtype == np.float32


def test_reduced_variants_keep_structure():
    s = scenes.tabletop_3obj(W=160, H=120, grid_half=2, n_yaw=4, tri_scale=0.05)
    assert len(s.meshes) == 3 and s.requests[0].poses.shape == (25 * 4, 12)
    # the two cylinders share geometry but not colour
    assert np.array_equal(s.meshes[1].verts, s.meshes[2].verts)
    assert not np.array_equal(s.meshes[1].rgb, s.meshes[2].rgb)
    d = scenes.sixdof_5obj(n_hyp=8, W=160, H=120, tri_scale=0.02)
    assert d.labels is not None and len(d.requests) == 5
    for r in d.requests:
        u0, v0, u1, v1 = r.roi
        assert 0 <= u0 < u1 <= 160 and 0 <= v0 < v1 <= 120
