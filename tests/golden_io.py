"""Reader for the hand-solved graph fixtures under tests/golden/."""
import math
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _num(t: str) -> float:
    return math.inf if t == "inf" else float(t)


def load(name: str) -> dict:
    out = dict(edges=[], init=None, iterations=None, goal=None, h=None)
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            key, *vals = line.split()
            if key == "edge":
                out["edges"].append((int(vals[0]), int(vals[1]), float(vals[2])))
            elif key in ("n", "root", "iterations", "goal"):
                out[key] = int(vals[0])
            elif key == "h":
                out["h"] = np.array([float(t) for t in vals])
            elif key == "g":
                out["g"] = np.array([_num(t) for t in vals])
            elif key in ("parent", "init"):
                out[key] = np.array([int(t) for t in vals], dtype=np.int32)
    e = out["edges"]
    out["u"] = np.array([a for a, _, _ in e], dtype=np.int32)
    out["v"] = np.array([b for _, b, _ in e], dtype=np.int32)
    out["c"] = np.array([c for _, _, c in e], dtype=np.float64)
    return out


def names() -> list:
    return sorted(f for f in os.listdir(GOLDEN) if f.endswith(".txt"))
