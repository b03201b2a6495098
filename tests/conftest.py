import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built CUDA library")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def pytest_collection_modifyitems(config, items):
    try:
        import torch
        have_gpu = torch.cuda.is_available()
    except Exception:
        have_gpu = False
    if have_gpu:
        return
    skip = pytest.mark.skip(reason="no CUDA device")
    for it in items:
        if "gpu" in it.keywords:
            it.add_marker(skip)


@pytest.fixture(scope="session")
def oracle_mod():
    import oracle
    oracle.build()
    return oracle


def read_golden(path):
    """Parse a tests/golden/*.txt fixture."""
    n = None; motif = None; medges = []; edges = []; count = None
    with open(path) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            tok = line.split()
            if tok[0] == "n":
                n = int(tok[1])
            elif tok[0] == "motif":
                motif = (int(tok[1]), int(tok[2]))
            elif tok[0] == "medge":
                medges.append((int(tok[1]), int(tok[2]), int(tok[3])))
            elif tok[0] == "edge":
                edges.append((int(tok[1]), int(tok[2]), int(tok[3])))
            elif tok[0] == "count":
                count = int(tok[1])
    return dict(n=n, nv=motif[0], delta=motif[1], medges=medges, edges=edges, count=count)
