"""Writes tests/golden/oracle_regression.txt: the oracle's exact integer bucket sums for a few
small seeded runs (coupled, capped with lag 3, uncoupled score-weighted), and their finalized
estimates printed as IEEE-754 hex.  It calls only `oracle/` and `synth/`.  The file is a regression
record of the oracle, not an independent pin: it makes any later change to the oracle's arithmetic
show as a diff, which the change must then justify against the paper.

  python tests/golden/write_oracle_regression.py
"""
import os
import platform
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import synth  # noqa: E402

# name: (run, slots, window length L of the estimator: l - k + 1 coupled, the length uncoupled)
CASES = {
    "coupled": (lambda: oracle.coupled_run(3, 20, 90, seed=4), 48, 18),
    "capped_lag3": (lambda: oracle.coupled_run(3, 20, 90, seed=4, meeting_cap=40, lag=3), 48, 18),
    "uncoupled": (lambda: oracle.uncoupled_run(2, 18, 90, seed=9), 48, 18),
}


def records():
    """Lines `case key v0 v1 ...` for every case, deterministic."""
    import numpy as np
    M = oracle.Model(synth.tiny_config(2))
    out = []
    for name, (make, P, L) in CASES.items():
        r = M.run_slots(make(), 0, P, 1)
        for key in ("S1", "S2_lo", "S2_hi", "count"):
            out.append(f"{name} {key} " + " ".join(str(int(v)) for v in np.asarray(r[key]).ravel()))
        est, se = M.finalize(r, P, L)
        for key, vals in (("est", est), ("se", se)):
            out.append(f"{name} {key} " + " ".join(float(v).hex() for v in vals))
    return out


if __name__ == "__main__":
    with open(os.path.join(HERE, "oracle_regression.txt"), "w") as f:
        f.write("# written by tests/golden/write_oracle_regression.py (oracle only); tiny 20x8 k=3 design,\n")
        f.write("# seed 2, 48 slots per case; bucket sums as integers, estimates and SEs as IEEE-754 hex\n")
        f.write(f"# machine {platform.machine()} (the oracle calls libm exp, whose last bit may differ by architecture)\n")
        for line in records():
            f.write(line + "\n")
