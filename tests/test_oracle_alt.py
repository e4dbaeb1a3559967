"""Pins of the oracle's LogLog and PCSA estimators (Sec. 4.1: the BDR pool
can serve PCSA and LogLog counting as well as HyperLogLog).

LogLog: Durand & Flajolet, "Loglog counting of large cardinalities" (2003):
n = alpha_m m 2^(mean register), alpha_m -> alpha_inf = e^-gamma sqrt(2)/2
~ 0.39701, standard error ~ 1.30 / sqrt(m).  PCSA: Flajolet & Martin,
"Probabilistic counting algorithms for data base applications" (1985):
n = (m / 0.77351) 2^(mean lowest-unset position), standard error ~ 0.78 /
sqrt(m).  The statistical pins draw registers and bitmaps straight from the
definitions with numpy, independent of the oracle's hashing.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import Oracle
from synth import traffic

SEED = 0x9E3779B97F4A7C15
EULER_GAMMA = 0.5772156649015329


def test_loglog_alpha_limit_and_published_value():
    a_inf = math.exp(-EULER_GAMMA) * math.sqrt(2) / 2
    assert abs(oracle.loglog_alpha(2.0 ** 28) - a_inf) < 1e-8
    assert abs(oracle.loglog_alpha(2.0 ** 20) - 0.39701) < 1e-5  # the paper's 5 digits
    ms = [16, 32, 64, 128, 1024, 2 ** 16]
    al = [oracle.loglog_alpha(m) for m in ms]
    assert all(x < y for x, y in zip(al, al[1:]))  # increasing towards alpha_inf
    # first-order convergence: (alpha_inf - alpha_m) m tends to a constant
    c = [(a_inf - oracle.loglog_alpha(m)) * m for m in (2 ** 12, 2 ** 14, 2 ** 16)]
    assert max(c) - min(c) < 1e-4 and 0.2 < c[0] < 0.5


def _registers_and_bitmaps(rng, m, n):
    """n elements into m buckets: bucket uniform, rho geometric (P = 2^-r)."""
    j = rng.integers(0, m, n)
    rho = np.minimum(rng.geometric(0.5, n), 32)
    M = np.zeros(m, dtype=np.int64)
    np.maximum.at(M, j, rho)
    bits = np.zeros(m, dtype=np.uint64)
    np.bitwise_or.at(bits, j, (np.uint64(1) << (rho - 1).astype(np.uint64)))
    # lowest unset position of each bitmap
    R = np.array([int((~int(b)) & (int(b) + 1)).bit_length() - 1 for b in bits])
    return M, R


@pytest.mark.parametrize("m", [64, 256])
def test_loglog_and_pcsa_unbiased_with_their_standard_errors(m):
    rng = np.random.default_rng(40 + m)
    n, trials = 40 * m * 8, 300
    ll, pc = [], []
    for _ in range(trials):
        M, R = _registers_and_bitmaps(rng, m, n)
        ll.append(oracle.loglog(m, int(M.sum())) / n - 1)
        pc.append(oracle.pcsa(m, int(R.sum())) / n - 1)
    ll, pc = np.array(ll), np.array(pc)
    for rel, se in ((ll, 1.30), (pc, 0.78)):
        sigma = se / math.sqrt(m)
        assert abs(rel.mean()) < 4 * sigma / math.sqrt(trials) + 0.01
        assert 0.8 * sigma < rel.std() < 1.25 * sigma


def _pair_history_pcsa(o, slices, t, k):
    """Brute force: the window bitmap of every pidx (bit rho-1 set iff a pair
    of LBP1 rho hit it in the last min(k, t+1) slices) and its lowest unset
    position, capped at R."""
    bits = np.zeros(o.Z, dtype=np.uint64)
    for s in slices[max(0, t - k + 1):t + 1]:
        for aip, bip in s.tolist():
            pidx, rho, _ = o.hash_pair(aip, bip)
            bits[pidx] |= np.uint64(1) << np.uint64(rho - 1)
    out = np.empty(o.Z, dtype=np.uint8)
    for j, b in enumerate(bits.tolist()):
        out[j] = min(((~b) & (b + 1)).bit_length() - 1, o.R)
    return out


@pytest.mark.parametrize("k", [1, 3])
def test_pcsa_statistic_is_lowest_unset_position_of_window_bitmap(k):
    """gsmall's DRV records every LBP1 (Alg. 9), so its window bitmap holds
    every position seen in the last k slices."""
    rng = np.random.default_rng(50 + k)
    aips = traffic.distinct_u32(rng, 12)
    o = Oracle("gsmall", k=k, Z=257, b=4, seed=SEED)
    slices = []
    for t in range(9):
        s = traffic.uniform_pairs(rng, int(rng.integers(0, 300)), aips)
        slices.append(s)
        o.scan(s)
        o.slide()
        want = _pair_history_pcsa(o, slices, t, k)
        np.testing.assert_array_equal(o.pcsa_statistics(), want)
        L_Z, P_Z = o.pool_sums_alt()
        assert P_Z == int(want.astype(np.int64).sum())
        assert L_Z == int(o.registers().astype(np.int64).sum())


def test_alt_estimates_closed_form_one_host_in_empty_pool():
    """Only one host's g virtual registers are set, all to r: the host sum
    is g r, the pool sum r times the number of distinct BDRs the host maps
    to; the estimate is the noise-removal formula of the two."""
    g, b, Z, r = 64, 6, 1 << 16, 9
    o = Oracle("gfast", k=2, Z=Z, b=b, seed=SEED)
    aip = 0x0A000001
    pidx = {o.phy_idx(aip, i) for i in range(g)}
    reg = np.zeros(Z, dtype=np.uint8)
    reg[list(pidx)] = r
    o.set_registers(reg)
    L_Z = r * len(pidx)
    n_g = oracle.loglog_alpha(g) * g * 2.0 ** r
    n_Z = oracle.loglog_alpha(Z) * Z * 2.0 ** (L_Z / Z)
    want = max(0.0, Z * g / (Z - g) * (n_g / g - n_Z / Z))
    got = o.estimate_alt(np.array([aip], dtype=np.uint32), "loglog")[0]
    assert want > 1000 and abs(got - want) <= 1e-9 * want
    with pytest.raises(ValueError):
        o.estimate_alt(np.array([aip], dtype=np.uint32), "pcsa")  # gfast has no bitmap


@pytest.mark.parametrize("estimator,se,variant", [("loglog", 1.30, "gfast"),
                                                  ("pcsa", 0.78, "gsmall")])
def test_alt_estimates_single_host_envelope(estimator, se, variant):
    """End to end through the scan: with a pool far larger than the load,
    hosts of true cardinality n are estimated within the estimator's
    standard error and without visible bias."""
    g, b = 128, 7
    rng = np.random.default_rng(60)
    aips = traffic.distinct_u32(rng, 40)
    o = Oracle(variant, k=2, Z=1 << 20, b=b, seed=SEED)
    cards = rng.integers(10000, 60000, size=aips.size)
    pairs = np.concatenate([
        np.stack([np.full(c, a, dtype=np.uint32), traffic.distinct_u32(rng, int(c))], 1)
        for a, c in zip(aips, cards)])
    o.scan(pairs)
    o.slide()
    rel = (o.estimate_alt(aips, estimator) - cards) / cards
    sigma = se / math.sqrt(g)
    assert np.mean(np.abs(rel)) < 1.3 * sigma
    assert abs(np.mean(rel)) < 3 * sigma / math.sqrt(aips.size) + 0.01
