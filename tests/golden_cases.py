"""Reader for tests/golden/trsm_integer.txt (integer-valued solves A X = alpha B)."""
import os

import numpy as np

PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "trsm_integer.txt")


def load():
    """List of (dtype, A, B, alpha, X): column-major numpy arrays."""
    cases, cur = [], None
    for line in open(PATH):
        if line.startswith("#") or not line.strip():
            continue
        f = line.split()
        if f[0] == "case":
            dtype, m, n, alpha = f[1], int(f[2]), int(f[3]), float(f[4])
            t = np.complex128 if dtype == "c128" else np.float64
            cur = {"dtype": dtype, "alpha": alpha, "A": np.zeros((m, m), t, order="F"),
                   "B": np.zeros((m, n), t, order="F"), "X": np.zeros((m, n), t, order="F")}
            cases.append(cur)
            continue
        i, j, re, im = int(f[1]), int(f[2]), float(f[3]), float(f[4])
        cur[f[0]][i, j] = complex(re, im) if cur["dtype"] == "c128" else re
    return [(c["dtype"], c["A"], c["B"], c["alpha"], c["X"]) for c in cases]
