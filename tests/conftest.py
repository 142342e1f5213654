import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (B300) and the built librgx")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def pytest_terminal_summary(terminalreporter):
    """Rounding-divergent segment decisions seen by the GPU parity comparisons."""
    try:
        from helpers import DIVERGENCE_LOG, PARITY_LOG
    except Exception:
        return
    if DIVERGENCE_LOG:
        terminalreporter.write_sep("-", "pixels with a rounding-divergent decision (accepted by schedule replay)")
        for name, nd, n in DIVERGENCE_LOG:
            terminalreporter.write_line(f"{name}: {nd} of {n}")
    if PARITY_LOG:
        terminalreporter.write_sep("-", "parity against the FP64 oracle (tolerances: RGBA 1e-4, gradients 1e-3)")
        for name, q, v in PARITY_LOG:
            terminalreporter.write_line(f"{name}: {q} {v:.3g}")
