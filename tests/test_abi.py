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
