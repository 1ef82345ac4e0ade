"""Reader for the small text fixtures in this folder (key followed by numbers)."""
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))


def read(name: str) -> dict:
    out = {}
    with open(os.path.join(HERE, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            key, *vals = line.split()
            out[key] = np.array([float(v) for v in vals])
    return out
