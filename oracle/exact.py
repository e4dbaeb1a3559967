"""Exact host cardinalities, Definition 1 -- TEST INFRASTRUCTURE.

|OP(aip, t, k)| is the number of distinct bips that appear with aip in the
window W(t, k) of k successive slices (Sec. 1, Sec. 2.1, Definition 1).  This
is the plain set definition written with numpy: encode each pair as the 64-bit
key (aip << 32) | bip, take the distinct keys of the window's slices, and count
them per aip.  A pure-Python set version is kept for the tiniest inputs so
that the numpy version itself is checked against the definition.
"""
from __future__ import annotations

import numpy as np


def _keys(pairs: np.ndarray) -> np.ndarray:
    p = np.asarray(pairs, dtype=np.uint32).reshape(-1, 2)
    return (p[:, 0].astype(np.uint64) << np.uint64(32)) | p[:, 1].astype(np.uint64)


def window_cardinalities(slices: list[np.ndarray], t: int, k: int,
                         aips: np.ndarray) -> np.ndarray:
    """|OP(aip, t-k+1, k)| for every aip in ``aips``: the window of the last
    k slices that end with slice ``t`` (0-based; earlier slices than 0 do not
    exist, so the first windows are shorter)."""
    lo = max(0, t - k + 1)
    keys = np.unique(np.concatenate([_keys(s) for s in slices[lo:t + 1]]))
    hosts = (keys >> np.uint64(32)).astype(np.uint32)
    uh, counts = np.unique(hosts, return_counts=True)
    aips = np.asarray(aips, dtype=np.uint32)
    pos = np.searchsorted(uh, aips)
    pos_c = np.minimum(pos, max(len(uh) - 1, 0))
    found = (len(uh) > 0) & (uh[pos_c] == aips) if len(uh) else np.zeros(len(aips), bool)
    out = np.zeros(len(aips), dtype=np.int64)
    out[found] = counts[pos_c[found]]
    return out


def window_cardinalities_sets(slices: list[np.ndarray], t: int, k: int,
                              aips) -> list[int]:
    """The same quantity with Python sets, for tiny inputs only."""
    lo = max(0, t - k + 1)
    op: dict[int, set] = {}
    for s in slices[lo:t + 1]:
        for aip, bip in np.asarray(s, dtype=np.uint32).reshape(-1, 2).tolist():
            op.setdefault(aip, set()).add(bip)
    return [len(op.get(int(a), ())) for a in aips]
