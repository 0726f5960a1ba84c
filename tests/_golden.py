"""Readers for the text fixtures under tests/golden/."""
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def exact_qr_cases():
    """[(name, A, R)] from exact_qr_cases.txt (hand-built A = Q R)."""
    rows = []
    with open(os.path.join(GOLDEN, "exact_qr_cases.txt")) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    out = []
    t = 0
    while t < len(rows):
        assert rows[t][0] == "case"
        name, m, n = rows[t][1], int(rows[t][2]), int(rows[t][3])
        A = np.array([[float(v) for v in r] for r in rows[t + 1:t + 1 + m]])
        R = np.array([[float(v) for v in r] for r in rows[t + 1 + m:t + 1 + m + n]])
        out.append((name, A, R))
        t += 1 + m + n
    return out
