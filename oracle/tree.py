"""Binary cluster tree, admissibility and near/far interaction lists (oracle).

Section 3.5 / Algorithm 1: the boxes of level l-1 are formed from
their two children 2i and 2i+1 at level l, so the tree is a complete binary
tree whose box i at level l has children 2i and 2i+1 at level l+1.  The root
is level 0; the leaves are level L.

Partition rule (the paper sorts points in a space-filling order but does not
fix the split): every box is cut at the median of its points along the longest
axis of the box's tight bounding box.  Points are ordered by (coordinate,
original index), the first floor(n/2) go to the left child 2i.  The depth is
L = ceil(log2(N / leaf)) (0 when N <= leaf), so every leaf holds
floor or ceil of N / 2^L points.

Admissibility (Section 6.2 defines it only as the acceptable ratio of the
maximum radius and the centre distance): boxes i != j are admissible
(well-separated, "far") when |c_i - c_j| > eta * (R_i + R_j), with c the
centre and R the half-diagonal of the tight bounding box.  eta = 0 makes every
pair of distinct boxes admissible, the HSS case of Section 6.3.

Lists: level 0 has the single near pair (0, 0).  At level l the candidates are
the child pairs of the near pairs of level l-1; admissible candidates are
"far" (coupling blocks S_ij), the rest are "near" (dense blocks).  Both lists
hold ordered pairs (i, j) and are symmetric.
"""
from __future__ import annotations

import math

import numpy as np


def depth(n: int, leaf: int) -> int:
    if n <= leaf:
        return 0
    return int(math.ceil(math.log2(n / leaf)))


def build_tree(points: np.ndarray, leaf: int):
    """Return (perm, ranges): perm[t] is the original index of tree position t;
    ranges[l] is an array of nb_l + 1 offsets, box i of level l covering tree
    positions ranges[l][i] : ranges[l][i+1]."""
    n = len(points)
    L = depth(n, leaf)
    boxes = [np.arange(n, dtype=np.int64)]
    sizes = [[n]]
    for _ in range(L):
        nxt = []
        for idx in boxes:
            X = points[idx]
            ext = X.max(axis=0) - X.min(axis=0) if len(idx) else np.zeros(3)
            ax = int(np.argmax(ext))
            order = np.lexsort((idx, X[:, ax]))  # by coordinate, then by original index
            h = len(idx) // 2
            nxt.append(idx[order[:h]])
            nxt.append(idx[order[h:]])
        boxes = nxt
        sizes.append([len(b) for b in boxes])
    perm = np.concatenate(boxes) if boxes else np.zeros(0, dtype=np.int64)
    # Offsets per level: the leaves are in order, and box i of level l is the
    # union of its descendants, which are contiguous.
    ranges = []
    for l in range(L + 1):
        nb = 1 << l
        span = 1 << (L - l)
        leaf_off = np.concatenate([[0], np.cumsum(sizes[L])])
        ranges.append(np.array([leaf_off[i * span] for i in range(nb + 1)], dtype=np.int64))
    return perm, ranges


def box_geometry(points: np.ndarray, perm: np.ndarray, rng_l: np.ndarray):
    """Centres and half-diagonals of the tight bounding boxes of one level."""
    nb = len(rng_l) - 1
    c = np.zeros((nb, 3))
    R = np.zeros(nb)
    for i in range(nb):
        X = points[perm[rng_l[i]:rng_l[i + 1]]]
        lo, hi = X.min(axis=0), X.max(axis=0)
        c[i] = (lo + hi) / 2.0
        R[i] = np.linalg.norm(hi - lo) / 2.0
    return c, R


def admissible(c, R, i: int, j: int, eta: float) -> bool:
    return i != j and float(np.linalg.norm(c[i] - c[j])) > eta * (R[i] + R[j])


def interaction_lists(points: np.ndarray, perm: np.ndarray, ranges, eta: float):
    """near[l], far[l]: sorted lists of ordered pairs (i, j) for each level."""
    L = len(ranges) - 1
    near = [[(0, 0)]]
    far = [[]]
    for l in range(1, L + 1):
        c, R = box_geometry(points, perm, ranges[l])
        nl, fl = [], []
        for (p, q) in near[l - 1]:
            for a in (2 * p, 2 * p + 1):
                for b in (2 * q, 2 * q + 1):
                    (fl if admissible(c, R, a, b, eta) else nl).append((a, b))
        near.append(sorted(nl))
        far.append(sorted(fl))
    return near, far
