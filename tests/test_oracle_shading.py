"""Pins of the oracle's colour interpolation (C5: screen-space affine
interpolation of per-vertex uint8 colour, integer arithmetic, rounded half up).

The pins are closed forms of barycentric interpolation, independent of how
the oracle evaluates it:
  * a colour that is an affine function f(u, v) of the pixel position at the
    vertices is reproduced exactly at every covered pixel (the weights of a
    sample sum to the doubled area A and reproduce its position), so the
    oracle must return floor(f + 1/2): with f = ... + u/2 every odd column
    lies exactly half-way between two codes, which tells half-up rounding
    apart from floor and from ties-to-even;
  * the same holds for a triangle tilted in depth whose vertices project
    onto integer pixels -- the interpolation is affine in the image, not
    perspective-correct;
  * at a vertex, the weights are (A, 0, 0): the pixel takes that vertex's
    colour exactly, whatever the other vertices carry.
A permutation of the weights against the vertex colours, a floor instead of
the half-up rounding, or a perspective-correct interpolation each fails one.
"""
from fractions import Fraction

import numpy as np
import pytest

W, H, F, CX, CY = 64, 48, 128.0, 32.0, 24.0
EMPTY = np.uint64(0xFFFFFFFFFFFFFFFF)
IDENT = np.array([1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0], np.float32)   # camera frame = object frame


def _scene(O):
    return O.OracleScene(np.zeros((H, W), np.uint16), np.zeros((H, W, 3), np.uint8), None, F, F, CX, CY)


def _vertex(u, v, z):
    """Camera-frame point at depth z that projects exactly onto pixel (u, v):
    x = (u - cx) z / f, exact in binary32 for the dyadic z used here."""
    return [(u - CX) * z / F, (v - CY) * z / F, z]


# per channel: c(u, v) = k0 + ku u + kv v, with ku or kv = 1/2 so that half the
# columns (or rows) fall exactly between two codes
FIELDS = ((Fraction(10), Fraction(1, 2), Fraction(3)),        # R
          (Fraction(200), Fraction(-2), Fraction(1, 2)),      # G
          (Fraction(7), Fraction(3, 2), Fraction(2)))         # B


def _field(u, v):
    return [k0 + ku * u + kv * v for (k0, ku, kv) in FIELDS]


def _render(O, verts_uvz, rgb):
    sc = _scene(O)
    verts = np.array([_vertex(*p) for p in verts_uvz], np.float32)
    tris = np.arange(len(verts_uvz), dtype=np.int32).reshape(-1, 3)
    mesh = O.OracleMesh(verts, np.asarray(rgb, np.uint8), tris, 0.05, 0.1)
    keys, _ = O.render_keys(sc, mesh, IDENT)
    xyz, out_rgb, pix = O.rendered_points(sc, mesh, IDENT, keys)
    return keys, out_rgb, pix


@pytest.mark.parametrize("zs", [(0.5, 0.5, 0.5), (0.5, 0.625, 0.75), (0.75, 0.5, 0.625)])
def test_affine_colour_field_is_reproduced_with_half_up_rounding(oracle, zs):
    uv = [(2, 2), (40, 4), (6, 30)]
    rgb = []
    for (u, v) in uv:
        c = _field(u, v)
        assert all(x.denominator == 1 and 0 <= x <= 255 for x in c)
        rgb.append([int(x) for x in c])
    keys, out, pix = _render(oracle, [(u, v, z) for (u, v), z in zip(uv, zs)], rgb)
    assert len(pix) > 300
    halves = 0
    for k, p in enumerate(pix):
        u, v = int(p) % W, int(p) // W
        want = []
        for x in _field(u, v):
            assert 0 <= x <= 255
            halves += x.denominator == 2
            want.append(int((x + Fraction(1, 2)) // 1))      # floor(f + 1/2): half up
        assert out[k].tolist() == want, (u, v, out[k].tolist(), want, zs)
    assert halves > 200          # the half-way cases were exercised


def test_vertex_pixel_takes_the_vertex_colour(oracle):
    """A fan around a centre vertex on pixel (20, 20): the centre pixel is
    covered by exactly one triangle of the fan, where the weights are (A, 0, 0)
    for the centre: its colour is the centre's, not a rim vertex's."""
    centre = (20, 20)
    rim = [(30, 20), (26, 29), (14, 28), (10, 19), (15, 11), (27, 12)]
    uvz, rgb = [], []
    for i in range(len(rim)):
        for p, c in ((centre, (11, 22, 33)), (rim[i], (250, 5, 140)), (rim[(i + 1) % len(rim)], (90, 240, 1))):
            uvz.append((p[0], p[1], 0.5))
            rgb.append(c)
    keys, out, pix = _render(oracle, uvz, rgb)
    at = np.nonzero(pix == centre[1] * W + centre[0])[0]
    assert len(at) == 1
    assert out[at[0]].tolist() == [11, 22, 33]
    # and every rim vertex pixel that is covered carries one of the two rim colours
    for (u, v) in rim:
        k = np.nonzero(pix == v * W + u)[0]
        if len(k):
            assert out[k[0]].tolist() in ([250, 5, 140], [90, 240, 1])
