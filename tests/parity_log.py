"""Per-case parity errors of the GPU tests, collected for the session
summary (tests/conftest.py prints them at the end of the run, so that a run
with -q still shows every measured error next to its tolerance)."""

RECORDS = []


def record(label, n, errors, tolerances):
    """Record one comparison: `errors` and `tolerances` are dicts keyed by
    the compared quantity (e.g. "v", "C"), relative errors and bounds."""
    RECORDS.append((str(label), int(n), dict(errors), dict(tolerances)))
    parts = " ".join(f"{k} err {v:.2e} (tol {tolerances.get(k, float('nan')):.0e})" for k, v in errors.items())
    print(f"[parity] {label}: n={n} {parts}")
