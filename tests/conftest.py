import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built libgsb.so")
    config.addinivalue_line("markers", "slow: long CPU oracle runs")


def pytest_terminal_summary(terminalreporter, exitstatus, config):
    """How many replicas each parity check excused or judged under a widened
    bar (tests/_parity.py WIDENED)."""
    try:
        from tests._parity import WIDENED
    except Exception:
        return
    if not WIDENED:
        return
    terminalreporter.write_sep("-", "replicas excused or judged under a widened bar")
    for what, k, n, how in WIDENED:
        terminalreporter.write_line(f"{what}: {k} of {n} ({how})")
