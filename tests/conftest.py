import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built library")
    config.addinivalue_line("markers", "slow: longer CPU runs of the oracle")


GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def printed(name: str) -> dict:
    """A value set the paper prints, from tests/golden/paper_printed_values.json."""
    with open(os.path.join(GOLDEN, "paper_printed_values.json")) as fh:
        return json.load(fh)[name]
