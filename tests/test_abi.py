"""The C-ABI library loads and exports every function include/perch.h declares.

No compute calls: this runs on machines without a GPU.
"""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "perch.h")).read()
    return sorted(set(re.findall(r"PERCH_API\s+[\w\s\*]+?\b(perch_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2008_00326_gb300 import build, perch
    build.build()
    return perch.load()


def test_header_declares_the_api():
    names = _declared()
    for required in ("perch_load_mesh", "perch_set_observation", "perch_score_hypotheses",
                     "perch_best"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    from paper_2008_00326_gb300 import perch
    names = _declared()
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(perch.EXPORTS) == names


def test_no_device_means_no_context(lib):
    """Without a CUDA device the library refuses to create a context (no CPU fallback)."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2008_00326_gb300 import perch
    with pytest.raises(perch.PerchError):
        perch.perch_create(0)


def test_default_params(lib):
    from paper_2008_00326_gb300 import perch
    p = perch.perch_default_params()
    assert abs(p.delta_m - 0.01) < 1e-9 and abs(p.tau_c - 12.5) < 1e-6 and p.stride == 1


def _write_client_input(path, sc, poses):
    import numpy as np
    m = sc.meshes[0]
    with open(path, "wb") as f:
        np.array([sc.W, sc.H, len(m.verts), len(m.tris), len(poses)], np.int32).tofile(f)
        np.array([sc.fx, sc.fy, sc.cx, sc.cy, sc.params.delta_m, sc.params.tau_c, m.vol_radius, m.vol_height],
                 np.float32).tofile(f)
        np.array([sc.params.color_check], np.int32).tofile(f)
        np.ascontiguousarray(sc.depth, np.uint16).tofile(f)
        np.ascontiguousarray(sc.rgb, np.uint8).tofile(f)
        np.ascontiguousarray(m.verts, np.float32).tofile(f)
        np.ascontiguousarray(m.rgb, np.uint8).tofile(f)
        np.ascontiguousarray(m.tris, np.int32).tofile(f)
        np.ascontiguousarray(poses, np.float32).tofile(f)


def build_c_client(tmp_path):
    """Compile the plain C client against include/perch.h and libperch.so."""
    import subprocess
    pkg = os.path.join(ROOT, "paper_2008_00326_gb300")
    exe = str(tmp_path / "score_client")
    subprocess.check_call(["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
                           os.path.join(ROOT, "tests", "c_client", "score_client.c"), "-L", pkg, "-lperch",
                           "-Wl,-rpath," + pkg, "-o", exe])
    return exe


def test_c_client_links_and_refuses_without_a_device(lib, tmp_path):
    """The ABI is usable from plain C; without a GPU the context is refused."""
    import subprocess
    import torch
    from paper_2008_00326_gb300 import scenes
    exe = build_c_client(tmp_path)
    if torch.cuda.is_available():
        pytest.skip("a GPU is present (the GPU test runs the client)")
    sc = scenes.tabletop_small()
    inp = str(tmp_path / "in.bin")
    _write_client_input(inp, sc, sc.requests[0].poses[:8])
    r = subprocess.run([exe, inp, str(tmp_path / "out.bin")])
    assert r.returncode == 7            # perch_create failed: no device, no fallback
