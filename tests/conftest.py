import json
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

GOLDEN = os.path.join(ROOT, "tests", "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs an sm_103 GPU and the CUDA library")


def csr_of(edges):
    """Hyperedge list -> (e_ptr int64, e_idx int32) with rows sorted."""
    rows = [sorted(set(e)) for e in edges]
    ptr = np.zeros(len(rows) + 1, dtype=np.int64)
    ptr[1:] = np.cumsum([len(r) for r in rows])
    idx = np.array([v for r in rows for v in r], dtype=np.int32)
    return ptr, idx


def load_json(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


@pytest.fixture(scope="session")
def native_cpu():
    """Generator and oracle built (plain gcc/g++, no GPU needed)."""
    import hgen
    import oracle

    hgen.build()
    oracle.build()
    return True


@pytest.fixture(scope="session")
def hglib(native_cpu):
    """The CUDA library, built in-tree, with the torch allocator installed."""
    import importlib.util

    spec = importlib.util.spec_from_file_location(
        "_hg_build", os.path.join(ROOT, "paper_2504_02271_gb300", "build.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    mod.build()
    import torch

    import paper_2504_02271_gb300 as hg

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    hg.use_torch_allocator()
    return hg
