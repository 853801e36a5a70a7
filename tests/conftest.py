import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

MODEL_DIR = os.path.join(ROOT, "paper_1702_06735_gb300", "amplitude_models")
GOLDEN_DIR = os.path.join(ROOT, "tests", "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built library")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on CPU")


def model_path(name: str) -> str:
    return os.path.join(MODEL_DIR, name + ".json")


@pytest.fixture(scope="session")
def two_chain_path():
    return model_path("d0_k3pi_2chain")


@pytest.fixture(scope="session")
def full_path():
    return model_path("d0_k3pi_full")
