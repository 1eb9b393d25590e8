import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


def pytest_terminal_summary(terminalreporter):
    """Print the FP32-form errors the parity tests measured (worst
    error/bound ratio per checked force result, largest position deviation)."""
    h = sys.modules.get("tests.harness")
    rec = getattr(h, "RECORD", None) if h is not None else None
    if not rec:
        return
    tr = terminalreporter
    tr.section("FP32-form errors against the FP64 oracle")
    for r in rec:
        if r["kind"] == "force":
            t = r["worst_ratio_terms_base"]
            tr.write_line("%-60s n=%-9d worst err/bound %.3g (terms base %s)  max |dF| %.3g" % (
                r["what"][:60], r["n"], r["worst_ratio"], "-" if t is None else "%.3g" % t, r["max_err"]))
        else:
            tr.write_line("%-60s n=%-9d max |dx| %.3g um" % (r["what"][:60], r["n"], r["max_err"]))
