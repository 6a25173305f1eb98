import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")


def pytest_collection_modifyitems(config, items):
    # GPU tests without a GPU are skipped only when explicitly deselected by -m;
    # if someone runs them on a CPU machine they fail loudly in the fixture below.
    pass


@pytest.fixture(scope="session")
def arol():
    """The CUDA library binding.  Fails (never falls back) when it is missing."""
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU test selected but no CUDA device is visible")
    import paper_1105_4424_gb300 as A
    return A
