"""Pins of the oracle's CIELAB conversion and CIEDE2000 difference (Eq. 4).

The CIEDE2000 special cases below reduce the published formula to short closed
forms (evaluated here in float64): the neutral axis, pure chroma differences
on the a* axis, and hue pairs mirrored about the a* and b* axes.  Identities
(zero distance, symmetry, hue-wrap continuity) complete the set.
"""
import math

import numpy as np
import pytest


def test_lab_reference_points(oracle):
    white = oracle.srgb_to_lab([255, 255, 255])
    assert abs(white[0] - 100.0) < 1e-3 and abs(white[1]) < 1e-2 and abs(white[2]) < 1e-2
    black = oracle.srgb_to_lab([0, 0, 0])
    assert np.allclose(black, 0.0, atol=1e-5)
    # primaries of sRGB under D65 (standard values to two decimals)
    for rgb, lab in (([255, 0, 0], (53.24, 80.09, 67.20)),
                     ([0, 255, 0], (87.73, -86.18, 83.18)),
                     ([0, 0, 255], (32.30, 79.19, -107.86))):
        assert np.allclose(oracle.srgb_to_lab(rgb), lab, atol=0.02), rgb


@pytest.mark.parametrize("g", [1, 5, 10, 30, 60, 119, 128, 200, 254])
def test_lab_grey_axis_closed_form(oracle, g):
    c = g / 255.0
    y = c / 12.92 if c <= 0.04045 else ((c + 0.055) / 1.055) ** 2.4
    L = 116.0 * y ** (1 / 3) - 16.0 if y > (6 / 29) ** 3 else (29 / 3) ** 3 * y
    lab = oracle.srgb_to_lab([g, g, g])
    assert abs(lab[0] - L) < 2e-3
    assert abs(lab[1]) < 2e-2 and abs(lab[2]) < 2e-2


def _de(oracle, a, b):
    return oracle.ciede2000(np.array(a, np.float32), np.array(b, np.float32))[0]


def test_identity_and_symmetry(oracle):
    rng = np.random.default_rng(7)
    for _ in range(200):
        a = np.array([rng.uniform(0, 100), rng.uniform(-100, 100), rng.uniform(-100, 100)])
        b = np.array([rng.uniform(0, 100), rng.uniform(-100, 100), rng.uniform(-100, 100)])
        assert _de(oracle, a, a) == 0.0
        assert abs(_de(oracle, a, b) - _de(oracle, b, a)) <= 1e-4 * max(1.0, _de(oracle, a, b))
        assert _de(oracle, a, b) >= 0.0


def _SL(Lb):
    return 1 + 0.015 * (Lb - 50) ** 2 / math.sqrt(20 + (Lb - 50) ** 2)


def _G(Cb):
    return 0.5 * (1 - math.sqrt(Cb ** 7 / (Cb ** 7 + 25.0 ** 7)))


@pytest.mark.parametrize("L1,L2", [(10, 20), (50, 55), (70, 30), (95, 99.5)])
def test_neutral_axis(oracle, L1, L2):
    want = abs(L2 - L1) / _SL((L1 + L2) / 2)
    assert abs(_de(oracle, (L1, 0, 0), (L2, 0, 0)) - want) < 1e-4


@pytest.mark.parametrize("a1,a2", [(5, 8), (20, 35), (60, 61)])
def test_pure_chroma_on_a_axis(oracle, a1, a2):
    g = _G((a1 + a2) / 2)
    c1, c2 = (1 + g) * a1, (1 + g) * a2
    want = abs(c2 - c1) / (1 + 0.045 * (c1 + c2) / 2)
    assert abs(_de(oracle, (50, a1, 0), (50, a2, 0)) - want) < 1e-4


def _T(h):
    r = math.radians
    return (1 - 0.17 * math.cos(r(h - 30)) + 0.24 * math.cos(r(2 * h)) + 0.32 * math.cos(r(3 * h + 6))
            - 0.20 * math.cos(r(4 * h - 63)))


@pytest.mark.parametrize("a,b", [(30, 4), (12, 9), (40, 25)])
def test_hue_pair_mirrored_about_a_axis(oracle, a, b):
    # (a, b) and (a, -b): equal chroma, mean hue 0 deg, dH = 2 C' sin(phi)
    C = math.hypot(a, b)
    ap = (1 + _G(C)) * a
    Cp = math.hypot(ap, b)
    phi = math.atan2(b, ap)
    want = 2 * Cp * math.sin(phi) / (1 + 0.015 * Cp * _T(0.0))
    assert abs(_de(oracle, (60, a, b), (60, a, -b)) - want) < 1e-4


@pytest.mark.parametrize("a,b", [(4, 30), (9, 12), (25, 40)])
def test_hue_pair_mirrored_about_b_axis(oracle, a, b):
    # (a, b) and (-a, b): equal chroma, mean hue 90 deg
    C = math.hypot(a, b)
    ap = (1 + _G(C)) * a
    Cp = math.hypot(ap, b)
    psi = math.atan2(ap, b)
    want = 2 * Cp * math.sin(psi) / (1 + 0.015 * Cp * _T(90.0))
    assert abs(_de(oracle, (40, a, b), (40, -a, b)) - want) < 1e-4


def test_hue_wrap_mean_angle(oracle):
    # hues 350 and 10 deg average to 0 deg (not 180): same value as -10/+10
    C = 30.0
    r = math.radians
    x = _de(oracle, (50, C * math.cos(r(350)), C * math.sin(r(350))), (50, C * math.cos(r(10)), C * math.sin(r(10))))
    y = _de(oracle, (50, C * math.cos(r(-10)), C * math.sin(r(-10))), (50, C * math.cos(r(10)), C * math.sin(r(10))))
    assert abs(x - y) < 1e-4
    # a pair 180 deg apart reports a zero wrap gap (band case)
    _, gap = oracle.ciede2000(np.array([50, 20, 0], np.float32), np.array([50, -20, 0], np.float32))
    assert gap < 1e-3


def _lch(L, C, h_deg):
    h = math.radians(h_deg)
    return (L, C * math.cos(h), C * math.sin(h))


@pytest.mark.parametrize("centre,expect_rotation", [(270.0, True), (90.0, False), (180.0, False)])
def test_rotation_term_by_swapped_chromas(oracle, centre, expect_rotation):
    """The rotation term R_T (dC'/S_C)(dH'/S_H) is the only part of CIEDE2000
    that changes sign when two colours at hues centre -+ phi swap chromas:
    with hues mirrored about the a* or b* axis (centres 90, 180 and 270 deg),
    C', h'-bar, S_C, S_H and |dC' dH'| are the same for both pairs.  So the
    two distances differ only where the rotation acts -- in the blue region
    around 275 deg -- and there the pair with dC' dH' > 0 is the closer one
    (R_T < 0)."""
    phi, C1, C2, L = 10.0, 20.0, 40.0, 50.0
    pair1 = _de(oracle, _lch(L, C1, centre - phi), _lch(L, C2, centre + phi))   # dC' > 0, dh' > 0
    pair2 = _de(oracle, _lch(L, C2, centre - phi), _lch(L, C1, centre + phi))   # dC' < 0, dh' > 0
    if expect_rotation:
        assert pair1 < pair2 - 0.05, (pair1, pair2)
    else:
        assert abs(pair1 - pair2) < 1e-4, (pair1, pair2)


def _lab_from_primed(L, Cp1, hp1, Cp2, hp2):
    """Two Lab colours whose primed chromas and hues (after CIEDE2000's a*
    rescaling by 1 + G, G from the mean unprimed chroma) are (Cp1, hp1) and
    (Cp2, hp2) degrees: the fixed point a = a' / (1 + G(C-bar)), float64."""
    r = math.radians
    ap1, b1 = Cp1 * math.cos(r(hp1)), Cp1 * math.sin(r(hp1))
    ap2, b2 = Cp2 * math.cos(r(hp2)), Cp2 * math.sin(r(hp2))
    g = 0.0
    for _ in range(60):
        a1, a2 = ap1 / (1 + g), ap2 / (1 + g)
        g = _G((math.hypot(a1, b1) + math.hypot(a2, b2)) / 2)
    return (L, ap1 / (1 + g), b1), (L, ap2 / (1 + g), b2)


def _primed(lab):
    """Primed chroma and hue (degrees) of a float32-rounded pair, float64."""
    l1, l2 = (np.asarray(x, np.float32).astype(np.float64) for x in lab)
    g = _G((math.hypot(l1[1], l1[2]) + math.hypot(l2[1], l2[2])) / 2)
    out = []
    for l in (l1, l2):
        ap = (1 + g) * l[1]
        out.append((math.hypot(ap, l[2]), math.degrees(math.atan2(l[2], ap)) % 360.0))
    return out


@pytest.mark.parametrize("hm", [275.0, 250.0, 300.0, 262.0])
def test_rotation_term_magnitude_in_closed_form(oracle, hm):
    """R_T = -sin(2 dtheta) R_C with dtheta = 30 deg exp(-((h'-bar - 275 deg) / 25 deg)^2)
    and R_C = 2 sqrt(C'-bar^7 / (C'-bar^7 + 25^7)).  With equal lightness,
    dE00^2 = x^2 + y^2 + R_T x y for x = dC'/S_C and y = dH'/S_H (S_C, S_H, G
    and T are pinned by the tests above), so one pair isolates R_T.  The
    primed chromas are chosen with mean 25, where R_C = sqrt(2): at the centre
    hue 275 deg R_T = -sqrt(6)/2 exactly; at 250 and 300 deg (one Gaussian
    width either side) dtheta = 30 deg / e, equal on both sides; 262 deg
    pins the width again off the inflection."""
    phi, Cp1, Cp2 = 9.0, 15.0, 35.0
    lab1, lab2 = _lab_from_primed(50.0, Cp1, hm - phi, Cp2, hm + phi)
    (c1, h1), (c2, h2) = _primed((lab1, lab2))
    cbar, hbar = (c1 + c2) / 2, (h1 + h2) / 2
    x = (c2 - c1) / (1 + 0.045 * cbar)
    y = 2 * math.sqrt(c1 * c2) * math.sin(math.radians(h2 - h1) / 2) / (1 + 0.015 * cbar * _T(hbar))
    de = _de(oracle, lab1, lab2)
    rt_measured = (de * de - x * x - y * y) / (x * y)
    dtheta = 30.0 * math.exp(-((hm - 275.0) / 25.0) ** 2)
    rc = 2 * math.sqrt(25.0 ** 7 / (25.0 ** 7 + 25.0 ** 7))          # = sqrt(2) at C'-bar = 25
    want = -math.sin(math.radians(2 * dtheta)) * rc
    if hm == 275.0:
        assert abs(want + math.sqrt(6) / 2) < 1e-12
    assert abs(cbar - 25.0) < 1e-4 and abs(hbar - hm) < 1e-4
    assert abs(rt_measured - want) < 2e-3, (hm, rt_measured, want)
