import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: takes more than a few seconds")


@pytest.fixture(scope="session")
def root_dir():
    return ROOT


def pytest_terminal_summary(terminalreporter):
    """How many forward parity points were judged under the relaxed bar
    (max(1e-5, 8 u |E_max|), above 1e-5 only where every weight at the point
    is below about e^-21) rather than the flat 1e-5."""
    try:
        from gpu_helpers import RELAXED_LOG, RELAXED_FROM
    except ImportError:
        return
    if not RELAXED_LOG:
        return
    tr = terminalreporter
    tr.section("forward parity: points under the relaxed tolerance")
    tot = sum(r[1] for r in RELAXED_LOG)
    rel = sum(r[2] for r in RELAXED_LOG)
    tr.write_line(f"{len(RELAXED_LOG)} comparisons, {tot} points compared, {rel} judged under "
                  f"the relaxed bar (|E_max| > {RELAXED_FROM:.2f}), the rest at the flat 1e-5")
    for name, n, k, worst in RELAXED_LOG:
        if k:
            tr.write_line(f"  {name}: {k} of {n} points relaxed; their largest raw error "
                          f"{worst:.2f} x 1e-5")
