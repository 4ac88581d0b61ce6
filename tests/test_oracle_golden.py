"""The rate-averaging rule of Tables 4-5 (drop the highest and the lowest rate, average the
rest), pinned against the averages the paper prints (tests/golden/paper_rates.txt).

The printed MFD Gamma = 0 average 3.87 is 3.863 by this rule (a rounding slip in the
paper); every other printed average agrees to the printed two decimals.
"""
import os

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_rates.txt")


def _load():
    rows = {}
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        m, n, *vals = line.split()
        rows.setdefault(m, []).append((n, [float(v) for v in vals]))
    return rows


def test_trimmed_mean_reproduces_printed_averages():
    rows = _load()
    for method, data in rows.items():
        table = [v for n, v in data if n != "avg"]
        printed = [v for n, v in data if n == "avg"][0]
        for col in range(3):
            got = oracle.trimmed_mean([r[col] for r in table])
            if method == "MFD" and col == 0:
                assert abs(got - printed[col]) < 0.008, (got, printed[col])  # printed slip
            else:
                assert round(got, 2) == printed[col], (method, col, got, printed[col])


def test_rates_helper_matches_definition():
    # e ~ C h^4  ->  rate exactly 4
    Ns = [16, 32, 64]
    errs = [3.0 * (1.0 / n) ** 4 for n in Ns]
    assert all(abs(r - 4.0) < 1e-12 for r in oracle.rates(errs, Ns))
