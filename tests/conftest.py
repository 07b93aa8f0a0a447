import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# Iteration-count records of the GPU parity tests: (test, rhs, form, gpu count, clean oracle count,
# oracle range under rounding noise, allowed range); printed in the terminal summary.
COUNT_LOG = []


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU and the built libhkgeneo.so")
    config.addinivalue_line("markers", "slow: full-size cases (minutes of oracle time)")


def pytest_terminal_summary(terminalreporter):
    if not COUNT_LOG:
        return
    tr = terminalreporter
    tr.write_sep("-", "FGMRES iteration counts: GPU vs oracle")
    tr.write_line(f"{'case':<44} {'rhs':>3} {'form':<5} {'gpu':>5} {'oracle':>6} {'noise range':>12} {'allowed':>10}")
    for name, r, form, got, clean, lo, hi, alo, ahi in COUNT_LOG:
        allowed = f"{alo}..{ahi}" if ahi != "" else str(alo)
        tr.write_line(f"{name:<44} {r:>3} {form:<5} {got:>5} {clean:>6} {f'{lo}..{hi}':>12} {allowed:>10}")
