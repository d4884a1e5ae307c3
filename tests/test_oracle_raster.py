"""Pins of the oracle's rasteriser (C1-C4) to hand counts and closed forms.

Hand-counted fixtures live in tests/golden/raster_hand_counts.txt.  Geometry:
fx = fy = 128, Z = 0.5 m, so a vertex at object X maps to pixel 256 X + cx;
quarter-pixel positions are exact in binary32 and on the 1/16 snapping grid.
"""
import math
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "raster_hand_counts.txt")
W, H, F, CX, CY, Z0 = 24, 16, 128.0, 12.0, 8.0, 0.5
EMPTY = np.uint64(0xFFFFFFFFFFFFFFFF)


def _fixtures():
    out = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        name, verts, count, _why = [s.strip() for s in line.split("|")]
        pts = [tuple(float(c) for c in v.split(",")) for v in verts.split()]
        out.append((name, pts, int(count)))
    return out


def _scene(O, depth=None, W_=W, H_=H, f=F, cx=CX, cy=CY, **kw):
    depth = np.zeros((H_, W_), np.uint16) if depth is None else depth
    rgb = np.zeros((H_, W_, 3), np.uint8)
    return O.OracleScene(depth, rgb, None, f, f, cx, cy, **kw)


def _polygon_mesh(O, pts, z=0.0):
    """Fan-triangulated planar polygon given in pixel coordinates at Z0."""
    verts = np.array([[(x - CX) / (2 * F) * (2 * Z0), (y - CY) / (2 * F) * (2 * Z0), z] for x, y in pts],
                     np.float32)
    tris = np.array([[0, i, i + 1] for i in range(1, len(pts) - 1)], np.int32)
    rgb = np.full((len(pts), 3), 200, np.uint8)
    return O.OracleMesh(verts, rgb, tris, 0.05, 0.1)


IDENT = np.array([1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, Z0], np.float32)


@pytest.mark.parametrize("name,pts,count", _fixtures())
def test_hand_counted_coverage(oracle, name, pts, count):
    sc = _scene(oracle)
    mesh = _polygon_mesh(oracle, pts)
    keys, work = oracle.render_keys(sc, mesh, IDENT)
    covered = keys != EMPTY
    assert int(covered.sum()) == count, name
    # every covered sample is produced by exactly one triangle: no double
    # counting along shared edges (fragments == covered pixels)
    assert int(work[2]) == count, name
    # fronto-parallel at Z = 0.5 m: depth is exactly 5000 units everywhere
    assert np.all((keys[covered] >> np.uint64(32)) == 5000)


def test_vertex_order_and_triangle_order(oracle):
    sc = _scene(oracle)
    pts = [(2.5, 1.5), (8.5, 1.5), (8.5, 7.5), (2.5, 7.5)]
    m1 = _polygon_mesh(oracle, pts)
    k1, _ = oracle.render_keys(sc, m1, IDENT)
    # reversed winding of every triangle: rendered two-sided, identical buffer
    m2 = oracle.OracleMesh(m1.verts, m1.rgb, m1.tris[:, ::-1].copy(), 0.05, 0.1)
    k2, _ = oracle.render_keys(sc, m2, IDENT)
    assert np.array_equal(k1, k2)
    # reversed triangle order: depths identical, only triangle ids renumbered
    m3 = oracle.OracleMesh(m1.verts, m1.rgb, m1.tris[::-1].copy(), 0.05, 0.1)
    k3, _ = oracle.render_keys(sc, m3, IDENT)
    assert np.array_equal(k1 == EMPTY, k3 == EMPTY)
    assert np.array_equal(k1 >> np.uint64(32), k3 >> np.uint64(32))


def test_nearest_depth_wins(oracle):
    sc = _scene(oracle)
    pts = [(3.25, 2.25), (9.75, 2.25), (9.75, 6.75), (3.25, 6.75)]
    near = _polygon_mesh(oracle, pts)
    # same quad 1 cm further away, listed first in the triangle list
    far_v = near.verts.copy()
    far_v[:, 2] = 0.01
    verts = np.concatenate([far_v, near.verts])
    tris = np.concatenate([near.tris, near.tris + 4]).astype(np.int32)
    mesh = oracle.OracleMesh(verts, np.full((8, 3), 9, np.uint8), tris, 0.05, 0.1)
    keys, _ = oracle.render_keys(sc, mesh, IDENT)
    cov = keys != EMPTY
    # object z = +0.01 moves the first copy 1 cm away from the camera
    d = keys[cov] >> np.uint64(32)
    # the winning surface is the near quad (depth 5000) and its triangles are 2, 3
    assert np.all(d == 5000)
    assert set(np.unique(keys[cov] & np.uint64(0xFFFFFFFF)).tolist()) <= {2, 3}


def test_tilted_plane_depth_matches_ray_plane(oracle):
    """Depth of a tilted square = analytic ray-plane intersection (+-1 unit)."""
    Wt, Ht, f, cx, cy = 64, 48, 60.0, 32.0, 24.0
    sc = _scene(oracle, W_=Wt, H_=Ht, f=f, cx=cx, cy=cy)
    s = 0.15
    verts = np.array([[-s, -s, 0], [s, -s, 0], [s, s, 0], [-s, s, 0]], np.float32)
    tris = np.array([[0, 1, 2], [0, 2, 3]], np.int32)
    mesh = oracle.OracleMesh(verts, np.zeros((4, 3), np.uint8), tris, 0.05, 0.1)
    ang = math.radians(35.0)
    R = np.array([[1, 0, 0], [0, math.cos(ang), -math.sin(ang)], [0, math.sin(ang), math.cos(ang)]])
    t = np.array([0.01, -0.02, 0.6])
    pose = np.concatenate([R, t[:, None]], 1).astype(np.float32)
    keys, _ = oracle.render_keys(sc, mesh, pose.reshape(12))
    cov = keys != EMPTY
    assert cov.sum() > 200
    Rf = pose[:, :3].astype(np.float64)
    tf = pose[:, 3].astype(np.float64)
    n = Rf[:, 2]                      # plane normal in the camera frame
    c = float(n @ tf)                 # plane: n . X = c
    vs, us = np.nonzero(cov)
    dirs = np.stack([(us - cx) / f, (vs - cy) / f, np.ones_like(us, np.float64)], 1)
    z = c / (dirs @ n)
    d = (keys[cov] >> np.uint64(32)).astype(np.int64)
    assert np.max(np.abs(d - np.rint(z * 10000))) <= 1


def test_near_plane_and_guard_band_cull(oracle):
    sc = _scene(oracle)
    pts = [(3.25, 2.25), (9.75, 2.25), (9.75, 6.75)]
    mesh = _polygon_mesh(oracle, pts)
    behind = IDENT.copy()
    behind[11] = 0.04                    # Z = 0.04 < z_near = 0.05
    keys, work = oracle.render_keys(sc, mesh, behind)
    assert np.all(keys == EMPTY) and work[1] == 1
    far_side = IDENT.copy()
    far_side[3] = 0.5                    # 0.5 m to the right: x = 268 px >= 2W
    keys, work = oracle.render_keys(sc, mesh, far_side)
    assert np.all(keys == EMPTY) and work[1] == 1


def test_roi_restricts_coverage(oracle):
    sc = _scene(oracle)
    mesh = _polygon_mesh(oracle, [(2.5, 1.5), (8.5, 1.5), (8.5, 7.5), (2.5, 7.5)])
    keys, _ = oracle.render_keys(sc, mesh, IDENT, roi=(4, 3, 6, 100))
    vs, us = np.nonzero(keys != EMPTY)
    assert set(us.tolist()) == {4, 5} and set(vs.tolist()) == set(range(3, 8))
