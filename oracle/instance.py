"""Flatten an oracle-built H^2 instance into plain arrays (oracle; test
infrastructure).

The library's ``h2_import`` takes an H^2 instance as plain host arrays: the
points, the tree permutation and leaf offsets, per-level box dimensions D_l
and ranks K_l, the near and far pair lists, the ID bases X_l and the skeleton
point indices SK_l.  Factor and solve parity are then checked on the same
instance (two independent constructions agree only to the truncation error).
"""
from __future__ import annotations

import numpy as np


def flatten(H):
    L = H["L"]
    out = dict(
        N=int(H["N"]), L=int(L),
        points=np.ascontiguousarray(H["points"], dtype=np.float64),
        perm=np.ascontiguousarray(H["perm"], dtype=np.int64),
        leaf_offsets=np.ascontiguousarray(H["ranges"][L], dtype=np.int64),
        D=np.array(H["D"], dtype=np.int32),
        K=np.array(H["K"], dtype=np.int32),
        near=[np.ascontiguousarray(np.array(H["near"][l], dtype=np.int32).reshape(-1, 2)) for l in range(L + 1)],
        far=[np.ascontiguousarray(np.array(H["far"][l], dtype=np.int32).reshape(-1, 2)) for l in range(L + 1)],
        X=[None] + [np.ascontiguousarray(H["X"][l], dtype=np.float64) for l in range(1, L + 1)],
        SK=[None] + [np.ascontiguousarray(H["SK"][l], dtype=np.int64) for l in range(1, L + 1)],
    )
    return out


def save_npz(H, path):
    f = flatten(H)
    arrs = dict(N=f["N"], L=f["L"], points=f["points"], perm=f["perm"],
                leaf_offsets=f["leaf_offsets"], D=f["D"], K=f["K"])
    for l in range(f["L"] + 1):
        arrs[f"near{l}"] = f["near"][l]
        arrs[f"far{l}"] = f["far"][l]
        if l:
            arrs[f"X{l}"] = f["X"][l]
            arrs[f"SK{l}"] = f["SK"][l]
    np.savez(path, **arrs)
