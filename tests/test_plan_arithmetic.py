"""The planned estimate's exact-sum decomposition, checked on the CPU.

Each register value M adds 2^(32-M) to its host's harmonic sum S.  The
kernel keeps three 32-bit fields per host -- V (M = 0), Shi (1 <= M <= 16,
units of 2^16) and Slo (M > 16) -- selecting the field with (M + 15) >> 4 and
the increment with 1 << ((16 - M) & 15), and rebuilds S = V 2^32 + Shi 2^16
+ Slo.  This checks the identity for every register value and that no field
overflows for g up to 2^16 virtual registers per host."""
import numpy as np


def _decompose(M):
    which = min((M + 15) >> 4, 2)
    inc = 1 << ((16 - M) & 15)
    return which, inc


def test_every_register_value_rebuilds_its_term():
    for M in range(0, 33):
        which, inc = _decompose(M)
        fields = [0, 0, 0]
        fields[which] += inc
        S = (fields[0] << 32) + (fields[1] << 16) + fields[2]
        assert S == 1 << (32 - M), M
        assert which == (0 if M == 0 else 1 if M <= 16 else 2)


def test_random_hosts_sum_exactly_and_fit_32_bits():
    rng = np.random.default_rng(1)
    for g in (16, 256, 4096, 1 << 16):
        for _ in range(20):
            Ms = rng.integers(0, 33, size=g)
            fields = [0, 0, 0]
            for M in Ms.tolist():
                which, inc = _decompose(M)
                fields[which] += inc
            assert all(f < 1 << 32 for f in fields)
            assert (fields[0] << 32) + (fields[1] << 16) + fields[2] == sum(1 << (32 - int(M)) for M in Ms)
    # worst cases: every register 1 (largest Shi) or 17 (largest Slo)
    for M in (1, 17):
        which, inc = _decompose(M)
        assert inc * (1 << 16) < 1 << 32
