"""Reader for the hand-worked fixtures under tests/golden/ ("key: values"
lines; values may be fractions a/b; '|' separates groups and is ignored)."""
import os
from fractions import Fraction

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def read_golden(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, vals = line.split(":", 1)
            nums = [float(Fraction(t)) for t in vals.replace("|", " ").split()]
            out[key.strip()] = np.array(nums, dtype=np.float64)
    out["x"] = out["x"].astype(np.float32)
    return out
