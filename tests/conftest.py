import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built librst.so")
    config.addinivalue_line("markers", "slow: full-size parity cases")


def _ensure_built():
    need = [os.path.join(ROOT, "oracle", "liboracle.so"),
            os.path.join(ROOT, "paper_2603_11645_gb300", "gen", "libgraphgen.so"),
            os.path.join(ROOT, "paper_2603_11645_gb300", "librst.so")]
    if not all(os.path.exists(p) for p in need):
        import __graft_entry__
        __graft_entry__.build()


_ensure_built()


def pytest_collection_modifyitems(config, items):
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except Exception:  # pragma: no cover
        has_gpu = False
    if has_gpu:
        return
    skip = pytest.mark.skip(reason="no CUDA device")
    for it in items:
        if "gpu" in it.keywords:
            it.add_marker(skip)


def load_golden(name):
    """Parse a tests/golden file into {section: [[ints...], ...]}."""
    path = os.path.join(ROOT, "tests", "golden", name)
    out, cur = {}, None
    with open(path) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if line[0].isalpha():
                cur = line.split()[0]
                out[cur] = []
                continue
            out[cur].append([int(x) for x in line.split()])
    return out
