"""The oracle reproduces its recorded outputs (tests/golden/oracle_regression.txt, written by the
script beside it from the oracle alone): exact bucket sums and the bits of the finalized
estimates and standard errors of three small seeded runs.  A change to the oracle's arithmetic
fails here until the record is rewritten, with the passage of the paper that justifies it."""
import importlib.util
import os
import platform

import pytest

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _writer():
    spec = importlib.util.spec_from_file_location(
        "write_oracle_regression", os.path.join(GOLDEN, "write_oracle_regression.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_oracle_matches_its_record():
    with open(os.path.join(GOLDEN, "oracle_regression.txt")) as f:
        lines = [line.rstrip("\n") for line in f]
    machine = next(line.split()[2] for line in lines if line.startswith("# machine "))
    if machine != platform.machine():
        pytest.skip(f"recorded on {machine}: libm's exp may round differently on {platform.machine()}")
    stored = [line for line in lines if not line.startswith("#")]
    now = _writer().records()
    assert len(now) == len(stored) == 18
    for a, b in zip(now, stored):
        assert a == b, a.split()[:2]
