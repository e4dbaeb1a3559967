"""Seeded register-level synthetic state for the batched-estimation workload.

4M hosts whose true cardinalities span 1..1e7 log-uniformly cannot be built
by scanning pairs (about 2.5e12 distinct pairs), so the workload is generated
one level down, at the hosts' virtual registers.  This module holds none of
the VBDR method's arithmetic (no hashing, no BDR update): it only draws, for
every host and every one of its g virtual registers, the value a register
takes when c distinct hashed items are spread uniformly over g registers.

* hosts : distinct uniform-random 32-bit aips; host aip uses g = 2^b with
          b = b_min + (aip >> 30) (the mixed-g workload convention: four
          groups by the top two address bits);
* c     : floor(10^U(0, log10 c_max)) per host, the ground truth;
* value : Poissonised -- the number of items landing in one register is
          Poisson(c / g), each item's leftmost-1 position is geometric
          (P(r) = 2^-r) and capped at 32 - b, so the register's maximum r
          satisfies P(max <= r) = exp(-(c/g) 2^-r) for r < 32 - b; it is
          drawn by inverting that distribution with one uniform per register.

The output is host-major: vregs[off[h] : off[h] + g_h] are host h's values.
"""
from __future__ import annotations

import numpy as np

from .traffic import distinct_u32


class BatchedRegisters:
    def __init__(self, n_hosts: int, b_min: int, c_max: float, seed: int,
                 chunk: int = 1 << 16):
        rng = np.random.default_rng(seed)
        self.aips = distinct_u32(rng, n_hosts)
        self.b = (b_min + (self.aips >> np.uint32(30))).astype(np.int64)
        self.g = np.left_shift(1, self.b)
        self.card = np.floor(10.0 ** rng.uniform(0.0, np.log10(c_max), size=n_hosts)).astype(np.int64)
        self.offsets = np.concatenate([[0], np.cumsum(self.g)]).astype(np.uint64)
        total = int(self.offsets[-1])
        self.vregs = np.empty(total, dtype=np.uint8)
        for h0 in range(0, n_hosts, chunk):
            h1 = min(n_hosts, h0 + chunk)
            o0, o1 = int(self.offsets[h0]), int(self.offsets[h1])
            reps = self.g[h0:h1]
            lam = np.repeat(self.card[h0:h1] / reps, reps)
            cap = np.repeat(32 - self.b[h0:h1], reps)
            u = rng.random(o1 - o0)
            # max <= r  <=>  exp(-lam 2^-r) >= u  <=>  2^r >= lam / (-ln u)
            t = -np.log(np.maximum(u, 1e-300))
            with np.errstate(divide="ignore"):
                r = np.ceil(np.log2(lam / t))
            r = np.where(t >= lam, 0.0, r)  # no item in the register
            r = np.clip(r, 0, cap)
            self.vregs[o0:o1] = r.astype(np.uint8)
        self.offsets = self.offsets[:-1].copy()

    @property
    def n_hosts(self) -> int:
        return self.aips.size
