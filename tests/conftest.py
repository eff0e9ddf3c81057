import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line(
        "markers", "gpu: needs a CUDA GPU (run with -m gpu on a GB300)")


GOLDEN = os.path.join(ROOT, "tests", "golden")


def read_golden(name):
    rows = {}
    lines = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for ln in fh:
            ln = ln.strip()
            if not ln or ln.startswith("#"):
                continue
            lines.append(ln.split())
            rows[ln.split()[0]] = ln.split()[1:]
    return rows, lines
