"""Readers for the hand-worked fixtures under tests/golden/."""
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def read_kv(name: str) -> dict:
    """``key v1 v2 ...`` lines; '#' starts a comment."""
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            key, *vals = line.split()
            out[key] = vals
    return out


def read_rows(name: str) -> list:
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                rows.append(line.split())
    return rows


def alg1_case(name: str):
    kv = read_kv(name)
    x = np.array([float(v) for v in kv["x"]], dtype=np.float32).reshape(-1, 1)
    return dict(x=x, eps=float(kv["eps"][0]), min_pts=int(kv["min_pts"][0]),
                min_pts_db=int(kv["min_pts_db"][0]),
                labels=np.array([int(v) for v in kv["labels"]], dtype=np.int32),
                core=np.array([int(v) for v in kv["core"]], dtype=np.uint8))
