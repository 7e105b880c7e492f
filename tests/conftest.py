import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")


def pytest_collection_modifyitems(config, items):
    # GPU tests are skipped (not failed) where no GPU is present, so that
    # `-m "not gpu"` and plain runs behave on CPU-only machines.
    try:
        import torch

        has_gpu = torch.cuda.is_available()
    except Exception:  # pragma: no cover
        has_gpu = False
    if has_gpu:
        return
    skip = pytest.mark.skip(reason="no CUDA device")
    for it in items:
        if "gpu" in it.keywords:
            it.add_marker(skip)


def pytest_terminal_summary(terminalreporter, exitstatus, config):
    """Print every recorded parity comparison (label, size, relative errors
    and their tolerances), whichever way pytest was invoked."""
    try:
        import parity_log
    except ImportError:  # pragma: no cover
        return
    if not parity_log.RECORDS:
        return
    terminalreporter.write_sep("-", f"parity: {len(parity_log.RECORDS)} comparisons against the FP64 oracle")
    worst = {}
    for label, n, errs, tols in parity_log.RECORDS:
        parts = " ".join(f"{k}={v:.2e}/{tols.get(k, float('nan')):.0e}" for k, v in errs.items())
        terminalreporter.write_line(f"[parity] {label} (n={n}): {parts}")
        for k, v in errs.items():
            t = tols.get(k)
            if t:
                worst[k] = max(worst.get(k, 0.0), v / t)
    terminalreporter.write_line("[parity] largest error / tolerance: "
                                + " ".join(f"{k} {r:.3f}" for k, r in sorted(worst.items())))
