"""Shared pytest configuration.

Markers:
  gpu  -- needs a CUDA GPU and the compiled libbbp; the parity tests proper.
"""

import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU and the compiled libbbp")


def load_pins():
    with open(os.path.join(ROOT, "tests", "golden", "paper_pins.json")) as fh:
        return {p["name"]: p for p in json.load(fh)["pins"]}


@pytest.fixture(scope="session")
def pins():
    return load_pins()
