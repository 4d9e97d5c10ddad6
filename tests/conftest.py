import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU check")


# Errors against the exact sums measured by the GPU parity tests, printed in
# the terminal summary: (test, eps, E_gpu, E_oracle_pipeline, bar).
EXACT_ERRORS = []


def record_exact_error(name, eps, e_gpu, e_oracle, bar):
    EXACT_ERRORS.append((name, eps, e_gpu, e_oracle, bar))


def pytest_terminal_summary(terminalreporter):
    if not EXACT_ERRORS:
        return
    tr = terminalreporter
    tr.write_sep("-", "relative l2 error against the exact sums (GPU, oracle pipeline, bar)")
    for name, eps, eg, eo, bar in EXACT_ERRORS:
        tr.write_line("%-70s eps=%-7.0e E_gpu=%.3e (%.2f eps)  E_oracle=%.3e  bar=%.3e"
                      % (name[:70], eps, eg, eg / eps, eo, bar))
