import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "fullsize: runs a workload at its full measured size")


def pytest_collection_modifyitems(config, items):
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except Exception:  # pragma: no cover
        has_gpu = False
    if has_gpu:
        return
    skip = pytest.mark.skip(reason="no CUDA GPU in this environment")
    for item in items:
        if "gpu" in item.keywords:
            item.add_marker(skip)


@pytest.fixture(scope="session")
def golden_worked():
    """Parse tests/golden/worked_3x2x2.txt (hand-worked MTTKRP/loss example)."""
    import numpy as np
    path = os.path.join(ROOT, "tests", "golden", "worked_3x2x2.txt")
    data = {}
    entries = []
    in_entries = False
    with open(path) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if ":" in line:
                key, rest = line.split(":", 1)
                key = key.strip()
                rest = rest.strip()
                in_entries = key == "entries"
                if in_entries:
                    continue
                if ";" in rest:
                    data[key] = np.array([[float(x) for x in row.split()] for row in rest.split(";")])
                else:
                    data[key] = np.array([float(x) for x in rest.split()])
            elif in_entries:
                entries.append([float(x) for x in line.split()])
    ent = np.array(entries)
    order = len(data["dims"])
    data["dims"] = [int(d) for d in data["dims"]]
    data["R"] = int(data["R"][0])
    data["idx"] = [ent[:, k].astype(np.uint32) for k in range(order)]
    data["val"] = ent[:, order]
    data["U"] = [data[f"U{k}"] for k in range(order)]
    return data
