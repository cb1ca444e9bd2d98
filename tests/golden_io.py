"""Reader for the hand-derived golden trees under tests/golden/."""
from __future__ import annotations

import glob
import os

import numpy as np

GOLDEN_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
MODES = {"mod": 0, "contiguous": 1, "explicit": 2}
KEYS = {"cyclic": 0, "widest": 1}


def load(path: str) -> dict:
    fields = {}
    for line in open(path):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        k, *v = line.split()
        fields[k] = v
    d, n = int(fields["d"][0]), int(fields["n"][0])
    pts = np.array([[float(x) for x in fields[f"x{j}"]] for j in range(d)], dtype=np.float32)
    assert pts.shape == (d, n)
    case = {
        "name": os.path.basename(path),
        "points": pts,
        "r": int(fields["r"][0]),
        "subset_mode": MODES[fields["mode"][0]],
        "key_rule": KEYS[fields["key"][0]],
        "depth": int(fields["depth"][0]),
        "leaf_size": int(fields.get("leaf_size", ["1"])[0]),
        "max_levels": int(fields.get("max_levels", ["20"])[0]),
        "perm": np.array([int(x) for x in fields["perm"]], np.int64),
        "split_vals": np.array([float(x) for x in fields["split_vals"]], np.float32),
        "split_dims": np.array([int(x) for x in fields["split_dims"]], np.int64),
        "offsets": np.array([int(x) for x in fields["offsets"]], np.int64),
        "levels": int(fields["levels"][0]),
    }
    if "sid" in fields:
        case["sid"] = np.array([int(x) for x in fields["sid"]], np.uint8)
    return case


def all_cases() -> list[dict]:
    return [load(p) for p in sorted(glob.glob(os.path.join(GOLDEN_DIR, "*.txt")))]
