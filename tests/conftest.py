"""Shared pytest setup: the `gpu` marker and the repository root on sys.path."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built libp2s")


def pytest_terminal_summary(terminalreporter):
    """Print every parity comparison's relative-L2 and max-abs error (GPU runs only)."""
    mod = sys.modules.get("gpu_common")
    recs = getattr(mod, "RECORDS", None) if mod else None
    if not recs:
        return
    tr = terminalreporter
    tr.write_sep("-", f"parity figures ({len(recs)} comparisons): rel_l2 < tol, max_abs <= bound")
    for test, what, r, mx, bound, tol in recs:
        tr.write_line(f"{test[:58]:58s} {what[:18]:18s} rel={r:.2e} tol={tol:.0e} max={mx:.2e} bound={bound:.1e}")
