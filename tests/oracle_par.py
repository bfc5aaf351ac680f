"""Test-side helper: an oracle estimate over N points computed as contiguous point ranges
on host threads.

The oracle's estimators take a point offset (the generators are counter-based), so
theta over points 0..N-1 of a replication is the count-weighted mean of the estimates over
disjoint ranges that cover them (the sharding identity, pinned by tests/test_sharding.py).
ctypes releases the GIL during each oracle call, so the ranges run in parallel; every call
runs single-threaded inside.  This reorders only the final sum over points."""
from __future__ import annotations

from concurrent.futures import ThreadPoolExecutor

import numpy as np

import oracle as O


def ranges(N: int, parts: int):
    cuts = np.linspace(0, N, max(1, min(parts, N)) + 1).astype(np.int64)
    return [(int(a), int(b - a)) for a, b in zip(cuts[:-1], cuts[1:]) if b > a]


def over_points(fn, N: int, threads: int = 0):
    """fn(offset, count) -> tuple of arrays (or one array), each a mean over its points;
    returns the same structure averaged over all N points."""
    threads = threads or min(O.max_threads(), 16)
    rs = ranges(N, threads)
    with ThreadPoolExecutor(len(rs)) as ex:
        parts = list(ex.map(lambda r: fn(r[0], r[1]), rs))
    w = [c for _, c in rs]
    if isinstance(parts[0], tuple):
        return tuple(sum(p[k] * c for p, c in zip(parts, w)) / N for k in range(len(parts[0])))
    return sum(p * c for p, c in zip(parts, w)) / N
