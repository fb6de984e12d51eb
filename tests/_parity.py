"""Deviation record of the GPU parity tests.

The parity bars of the method are fixed numbers: per-iteration scalars within 1e-12 relative,
iteration counts within +-2, x within 1e-9 relative at the same iteration count.  Where a
case's gate is wider (the oracle's own one-ulp rounding spread is larger than the fixed bar;
see the readings on BiCGStab, GMRES and irregular CG), the test still reports the deviation it
measured next to the fixed bar: record() appends one JSON line per quantity to the file named
by the environment variable PK_PARITY_LOG (nothing is written when it is unset).
"""
from __future__ import annotations

import json
import os


def record(test: str, case: str, quantity: str, measured: float, fixed_bar: float, gate: float,
           **extra) -> None:
    path = os.environ.get("PK_PARITY_LOG")
    if not path:
        return
    line = {"test": test, "case": case, "quantity": quantity, "measured": float(measured),
            "fixed_bar": float(fixed_bar), "gate": float(gate),
            "within_fixed_bar": bool(measured <= fixed_bar), **extra}
    with open(path, "a") as f:
        f.write(json.dumps(line) + "\n")


def rel_dev(got, ref):
    """Largest elementwise relative deviation |got - ref| / |ref| (entries with ref = 0 skipped)."""
    import numpy as np

    got = np.asarray(got, dtype=float)
    ref = np.asarray(ref, dtype=float)
    m = ref != 0
    return float(np.max(np.abs(got[m] - ref[m]) / np.abs(ref[m]))) if m.any() else 0.0


def perturbed_b(W, b, k):
    """b with a one-ulp-sized relative perturbation (2^-52 uniform_pm1(100 + k)), the same in
    the oracle's sensitivity runs and on the GPU."""
    return b * (1 + 2.0 ** -52 * W.uniform_pm1(100 + k, b.size))


def count_gate(oracle_counts):
    """Gate for comparing iteration-count distributions: the medians of the GPU's and the
    oracle's counts over the same right-hand sides (b and its one-ulp perturbations) may differ
    by half the oracle's sample range + 2.  BiCGStab's count is a heavy-tailed function of
    rounding: on the power-law matrix with 10^6 rows one-ulp changes of b move the oracle's
    count over 753..888 and the GPU's over 763..1035 (medians 812 and 812), so one run against
    one run says nothing about agreement."""
    import numpy as np

    o = np.asarray(oracle_counts)
    return 2 + (o.max() - o.min()) / 2.0


def median(v):
    import numpy as np

    return float(np.median(np.asarray(v, dtype=float)))
