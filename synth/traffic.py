"""Seeded synthetic (aip, bip) traffic -- the shared input generator.

This module feeds both the CPU oracle (tests) and the CUDA library (tests,
bench).  It holds none of the VBDR method's arithmetic: no hashing, no LBP1,
no estimator -- only the shape of the workload.  The paper measures on no
trace or dataset, so every workload is synthetic:

* hosts  : H distinct uniform-random 32-bit aips; host of rank r = 1..H has
           target window cardinality c_r = max(1, floor(C_max * r^-s))
           (rank-size Zipf law);
* bips   : each host keeps a pool of ceil(c_r / (1 + churn (k-1))) uniform
           random 32-bit bips; each slice every pool entry is replaced by a
           fresh bip with probability ``churn``, so a window of k slices sees
           about c_r distinct bips and old bips expire;
* pairs  : per slice, the host is drawn with probability proportional to c_r
           (Walker alias table) and the bip uniformly from that host's pool;
           optionally a fraction of pairs is repeated inside the slice, half as
           adjacent duplicates (bursts), half as copies of a uniformly random
           earlier pair.

Random numbers come from numpy's PCG64 seeded with the workload seed.
"""
from __future__ import annotations

import math

import numpy as np

U32 = np.uint32


def distinct_u32(rng: np.random.Generator, n: int) -> np.ndarray:
    """n distinct uniform random 32-bit values, in random order."""
    out = np.empty(0, dtype=U32)
    while out.size < n:
        extra = rng.integers(0, 1 << 32, size=int((n - out.size) * 1.05) + 16,
                             dtype=np.uint64).astype(U32)
        out = np.unique(np.concatenate([out, extra]))
    rng.shuffle(out)
    return out[:n].copy()


def zipf_cardinalities(n_hosts: int, s: float, c_max: int) -> np.ndarray:
    r = np.arange(1, n_hosts + 1, dtype=np.float64)
    return np.maximum(1, np.floor(c_max * r ** (-s))).astype(np.int64)


class AliasTable:
    """Walker/Vose alias table: O(1) sampling proportional to ``weights``."""

    def __init__(self, weights: np.ndarray):
        w = np.asarray(weights, dtype=np.float64)
        n = w.size
        p = w * (n / w.sum())
        self.prob = np.ones(n, dtype=np.float64)
        self.alias = np.arange(n, dtype=np.int64)
        small = list(np.nonzero(p < 1.0)[0])
        large = list(np.nonzero(p >= 1.0)[0])
        p = p.copy()
        while small and large:
            s = small.pop()
            l = large[-1]
            self.prob[s] = p[s]
            self.alias[s] = l
            p[l] -= 1.0 - p[s]
            if p[l] < 1.0:
                large.pop()
                small.append(l)
        self.n = n

    def sample(self, rng: np.random.Generator, size: int) -> np.ndarray:
        u = rng.random(size) * self.n
        idx = u.astype(np.int64)
        np.minimum(idx, self.n - 1, out=idx)
        frac = u - idx
        return np.where(frac < self.prob[idx], idx, self.alias[idx])


class ZipfTraffic:
    """Slice-by-slice traffic generator for the plain-VBDR workloads.

    ``next_slice(n)`` returns an (n, 2) uint32 array of (aip, bip) pairs.
    """

    def __init__(self, n_hosts: int, zipf_s: float, c_max: int, k: int,
                 seed: int, churn: float = 0.05, repeat_frac: float = 0.0):
        self.rng = np.random.default_rng(seed)
        self.n_hosts, self.k = n_hosts, k
        self.churn, self.repeat_frac = churn, repeat_frac
        self.aips = distinct_u32(self.rng, n_hosts)
        self.card = zipf_cardinalities(n_hosts, zipf_s, c_max)
        denom = 1.0 + churn * (k - 1)
        self.pool_size = np.maximum(1, np.ceil(self.card / denom)).astype(np.int64)
        self.pool_off = np.concatenate([[0], np.cumsum(self.pool_size)[:-1]])
        total = int(self.pool_size.sum())
        self.pool = self.rng.integers(0, 1 << 32, size=total,
                                      dtype=np.uint64).astype(U32)
        self.alias = AliasTable(self.card.astype(np.float64))
        self.slices_made = 0

    def _churn(self) -> None:
        if self.churn <= 0 or self.slices_made == 0:
            return
        m = self.rng.random(self.pool.size) < self.churn
        cnt = int(m.sum())
        self.pool[m] = self.rng.integers(0, 1 << 32, size=cnt,
                                         dtype=np.uint64).astype(U32)

    def next_slice(self, n: int) -> np.ndarray:
        self._churn()
        self.slices_made += 1
        out = np.empty((n, 2), dtype=U32)
        if n == 0:
            return out
        host = self.alias.sample(self.rng, n)
        j = (self.rng.random(n) * self.pool_size[host]).astype(np.int64)
        np.minimum(j, self.pool_size[host] - 1, out=j)
        out[:, 0] = self.aips[host]
        out[:, 1] = self.pool[self.pool_off[host] + j]
        if self.repeat_frac > 0 and n > 1:
            # each position i >= 1 becomes a repeat with probability
            # repeat_frac, half of them of the previous pair (bursts), half
            # of a uniformly random earlier pair
            u = self.rng.random(n)
            u[0] = 1.0
            pos = np.nonzero(u < self.repeat_frac)[0]
            adj = pos[u[pos] < self.repeat_frac / 2]
            far = pos[u[pos] >= self.repeat_frac / 2]
            out[adj] = out[adj - 1]  # bursts: copy the previous pair
            src = (self.rng.random(far.size) * far).astype(np.int64)
            out[far] = out[src]      # copies of a random earlier pair
        return out


def uniform_pairs(rng: np.random.Generator, n: int, aips: np.ndarray) -> np.ndarray:
    """n pairs with the aip drawn uniformly from ``aips`` and bip uniform u32."""
    out = np.empty((n, 2), dtype=U32)
    out[:, 0] = aips[rng.integers(0, aips.size, size=n)]
    out[:, 1] = rng.integers(0, 1 << 32, size=n, dtype=np.uint64).astype(U32)
    return out


def log_uniform_sizes(rng: np.random.Generator, n_slices: int, lo: int,
                      hi: int) -> np.ndarray:
    """Slice sizes floor(2^U(log2 lo, log2 hi)), for the streaming workload."""
    e = rng.uniform(math.log2(lo), math.log2(hi), size=n_slices)
    return np.floor(2.0 ** e).astype(np.int64)


# Workload presets (sizes of the configurations the method is run on).
SMALL = dict(name="small k=10 N=1e5 H=1000 Z=2^16 g=128", k=10, n_pairs=100_000,
             n_hosts=1000, zipf_s=1.1, c_max=5000, Z=1 << 16, log2_g=7,
             repeat_frac=0.0)
TRACE = dict(name="trace k=30 N=64M H=1M Z=2^24 g=256", k=30, n_pairs=64 << 20,
             n_hosts=1_000_000, zipf_s=1.05, c_max=2_000_000, Z=1 << 24, log2_g=8,
             repeat_frac=0.10)


class StreamingTraffic:
    """Traffic of the streaming-service workload: host ranks Zipf(s) over
    n_hosts active hosts (drawn by inverting the continuous rank-size law,
    O(1) per pair), bips uniform 32-bit, plus bursty superspreaders -- a
    fraction `spreader_frac` of the hosts, each active in bursts of 1..5
    slices with probability `burst_p` per slice, emitting about
    `spreader_pairs` fresh bips per active slice.

    make_pool(n) returns one (n, 2) uint32 block; a slice of size N is a
    window of a pool block.
    """

    def __init__(self, n_hosts: int, zipf_s: float, seed: int, spreader_frac: float = 1e-4,
                 burst_p: float = 0.05, spreader_pairs: int = 100_000):
        self.rng = np.random.default_rng(seed)
        self.n_hosts, self.s = n_hosts, zipf_s
        self.aips = distinct_u32(self.rng, n_hosts)
        n_sp = max(1, int(round(n_hosts * spreader_frac)))
        self.spreaders = self.aips[self.rng.choice(n_hosts, n_sp, replace=False)]
        self.burst_p, self.spreader_pairs = burst_p, spreader_pairs
        self.burst_left = np.zeros(n_sp, dtype=np.int64)

    def _ranks(self, n: int) -> np.ndarray:
        a = 1.0 - self.s
        u = self.rng.random(n)
        r = np.floor((u * (self.n_hosts ** a - 1.0) + 1.0) ** (1.0 / a)).astype(np.int64)
        return np.clip(r, 1, self.n_hosts) - 1

    def make_pool(self, n: int) -> np.ndarray:
        out = np.empty((n, 2), dtype=U32)
        # superspreader bursts: start with probability burst_p, last 1..5 slices
        start = (self.burst_left == 0) & (self.rng.random(self.spreaders.size) < self.burst_p)
        self.burst_left[start] = self.rng.integers(1, 6, size=int(start.sum()))
        active = self.spreaders[self.burst_left > 0]
        self.burst_left = np.maximum(self.burst_left - 1, 0)
        n_sp = min(n // 2, active.size * self.spreader_pairs)
        n_bg = n - n_sp
        out[:n_bg, 0] = self.aips[self._ranks(n_bg)]
        if n_sp:
            out[n_bg:, 0] = np.repeat(active, self.spreader_pairs)[:n_sp]
        out[:, 1] = self.rng.integers(0, 1 << 32, size=n, dtype=np.uint64).astype(U32)
        out[:] = out[self.rng.permutation(n)] if n <= (1 << 22) else out
        return out


STREAM = dict(name="stream N~logU[1M,128M] H=8M Z=2^26 g=256 k=30", k=30, n_lo=1 << 20,
              n_hi=128 << 20, n_hosts=8_000_000, zipf_s=1.1, Z=1 << 26, log2_g=8)
