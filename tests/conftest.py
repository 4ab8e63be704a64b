"""Shared pytest configuration.

Markers: `gpu` marks tests that need a CUDA device (the parity tests proper,
which call the CUDA path through the C ABI); everything else runs on a CPU-only
host.
"""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (run with -m gpu)")
    config.addinivalue_line("markers", "slow: long-running CPU test")
