"""Reader for the hand-derived fixtures in tests/golden/."""
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load(name):
    n = None
    src, dst, core = [], [], None
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            tag, *rest = line.split()
            if tag == "n":
                n = int(rest[0])
            elif tag == "e":
                src.append(int(rest[0]))
                dst.append(int(rest[1]))
            elif tag == "core":
                core = np.array([int(x) for x in rest], np.int32)
    return n, np.array(src, np.int32), np.array(dst, np.int32), core


def names():
    return sorted(f for f in os.listdir(GOLDEN) if f.endswith(".txt"))
