"""Pins of the oracle's ADD / ADD-S pose errors and their AUC (the accuracy
measures of Sec. VI) to closed forms and invariants."""
import math

import numpy as np
import pytest

from paper_2008_00326_gb300 import scenes


def _pose(R, t):
    return np.concatenate([np.asarray(R, np.float64), np.asarray(t, np.float64)[:, None]], 1).astype(
        np.float32).reshape(12)


@pytest.fixture(scope="module")
def can():
    return scenes.cylinder_mesh(0.03, 0.1, 24, 3)


def test_identical_poses_score_zero(oracle, can):
    P = _pose(scenes.rot_z(0.3), [0.1, 0.0, 0.8])
    assert oracle.add_s(can.verts, P, P, True) == 0.0
    assert oracle.add_s(can.verts, P, P, False) == 0.0


def test_translation_is_its_length_for_add(oracle, can):
    A = _pose(np.eye(3), [0.01, -0.02, 0.5])
    B = _pose(np.eye(3), [0.013, -0.016, 0.5])
    assert abs(oracle.add_s(can.verts, A, B, False) - 0.005) < 1e-7
    assert oracle.add_s(can.verts, A, B, True) <= 0.005 + 1e-9


def test_symmetry_rotation_is_free_for_add_s_only(oracle, can):
    # a turn by one segment of the 24-gon maps the vertex set onto itself
    A = _pose(scenes.rot_z(2 * math.pi / 24), [0.0, 0.0, 0.7])
    B = _pose(np.eye(3), [0.0, 0.0, 0.7])
    assert oracle.add_s(can.verts, A, B, True) < 1e-6
    ring = 2 * 0.03 * math.sin(math.pi / 24)             # chord of one segment
    add = oracle.add_s(can.verts, A, B, False)
    assert add > 0.5 * ring and add <= ring + 1e-6


def test_add_s_never_exceeds_add(oracle, can):
    rng = np.random.default_rng(2)
    for _ in range(5):
        A = _pose(scenes.rodrigues(rng.normal(size=3), rng.uniform(0, 1)), rng.normal(size=3) * 0.02)
        B = _pose(scenes.rodrigues(rng.normal(size=3), rng.uniform(0, 1)), rng.normal(size=3) * 0.02)
        assert oracle.add_s(can.verts, A, B, True) <= oracle.add_s(can.verts, A, B, False) + 1e-12


def test_auc_closed_forms(oracle):
    assert oracle.add_auc([0.0, 0.0]) == 1.0
    assert oracle.add_auc([0.2, 0.1]) == 0.0
    assert abs(oracle.add_auc([0.05]) - 0.5) < 1e-15
    assert abs(oracle.add_auc([0.0, 0.05, 0.2]) - (1.0 + 0.5 + 0.0) / 3) < 1e-15
    # against a trapezoid of the accuracy curve on a fine grid
    e = np.random.default_rng(3).uniform(0, 0.15, size=50)
    t = np.linspace(0, 0.1, 200001)
    acc = (e[None, :] < t[:, None]).mean(1)
    assert abs(oracle.add_auc(e) - np.trapezoid(acc, t) / 0.1) < 1e-4
