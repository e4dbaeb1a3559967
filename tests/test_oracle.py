"""Pins of the CPU oracle against what the paper and mathematics fix.

None of these tests compares the oracle with itself: each one checks it
against a published value, a closed form, an invariant the paper states, a
statistical law, or brute force on tiny inputs.
"""
import math
import os

import numpy as np
import pytest

import oracle
from oracle import Oracle, exact
from synth import traffic

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
SEED = 0x9E3779B97F4A7C15


def _golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


# ------------------------------------------------------------------ hashing

def test_mix64_matches_published_splitmix64_sequence():
    """H is built on the SplitMix64 mix; its generator's published
    known-answer sequence pins the constants and shifts."""
    want = [int(r[0]) for r in _golden("splitmix64_seed1234567.txt")]
    assert oracle.splitmix64_sequence(1234567, len(want)) == want


def test_H_full_range_is_high_half_of_published_outputs():
    """mix64(0) = 0, so H(x, 2^32, 0) = hi32(mix64(x)); at x = the SplitMix64
    generator state after i steps from 1234567, mix64(x) is the generator's
    published i-th output.  This pins the choice of the HIGH 32 bits."""
    want = [int(r[0]) for r in _golden("splitmix64_seed1234567.txt")]
    gamma = 0x9E3779B97F4A7C15
    for i, out in enumerate(want, start=1):
        state = (1234567 + i * gamma) % (1 << 64)
        assert oracle.H(state, 1 << 32, 0) == out >> 32


def test_H_range_reduction_properties():
    """H(x, N, A) is in [0, N), H(x, 2^32, A) is the full 32-bit hash and the
    multiply-shift reduction is monotone in the full hash (Sec. 4.1)."""
    rng = np.random.default_rng(1)
    for _ in range(300):
        x = int(rng.integers(0, 1 << 32))
        A = int(rng.integers(0, 1 << 63))
        N = int(rng.integers(1, 1 << 32))
        full = oracle.H(x, 1 << 32, A)
        assert 0 <= full < (1 << 32)
        h = oracle.H(x, N, A)
        assert 0 <= h < N
        # floor(full * N / 2^32), computed here with exact rational arithmetic
        assert h == (full * N) // (1 << 32)
        assert oracle.H(x, 1, A) == 0


def test_H_is_uniform_chi_square():
    rng = np.random.default_rng(2)
    N = 97
    cnt = np.zeros(N)
    for x in rng.integers(0, 1 << 32, size=20000):
        cnt[oracle.H(int(x), N, 12345)] += 1
    exp = 20000 / N
    chi2 = ((cnt - exp) ** 2 / exp).sum()
    # 96 degrees of freedom: mean 96, sd ~13.9; 5 sd bound
    assert chi2 < 96 + 5 * 13.9


def test_seed_changes_hash():
    xs = range(1000)
    a = [oracle.H(x, 1 << 32, 1) for x in xs]
    b = [oracle.H(x, 1 << 32, 2) for x in xs]
    assert sum(int(p == q) for p, q in zip(a, b)) <= 2


# --------------------------------------------------------- LBP1 and vidx

@pytest.mark.parametrize("b", [4, 7, 8])
def test_rho_and_vidx_distribution(b):
    """LBP1 of a uniform hashed word is geometric: P(rho = r) = 2^-r for
    r < 32-b, the cap 32-b collecting the tail 2^-(31-b); the virtual index
    (left b bits) is uniform on [0, 2^b)  (Sec. 3, Alg. 4)."""
    o = Oracle("gfast", k=4, Z=1 << 12, b=b, seed=SEED)
    rng = np.random.default_rng(3)
    n = 60000
    rhos = np.zeros(40, dtype=np.int64)
    vid = np.zeros(1 << b, dtype=np.int64)
    for bip in rng.integers(0, 1 << 32, size=n):
        pidx, rho, vidx = o.hash_pair(77, int(bip))
        assert 1 <= rho <= 32 - b
        assert 0 <= pidx < o.Z
        rhos[rho] += 1
        vid[vidx] += 1
    # first 8 bins against 2^-r: each within 5 binomial sd
    for r in range(1, 9):
        p = 2.0 ** -r
        assert abs(rhos[r] - n * p) < 5 * math.sqrt(n * p * (1 - p)) + 1, r
    exp = n / (1 << b)
    chi2 = ((vid - exp) ** 2 / exp).sum()
    dof = (1 << b) - 1
    assert chi2 < dof + 6 * math.sqrt(2 * dof)


def test_rho_is_leftmost_one_of_shifted_hash():
    """For pairs whose A1 hash is known, LBP1 counted from the left of
    (bip' << b) by brute-force bit inspection, capped at 32-b."""
    b = 7
    o = Oracle("gfast", k=4, Z=1 << 12, b=b, seed=SEED)
    A1 = oracle.lib().orc_A1(o._h)
    rng = np.random.default_rng(4)
    for bip in rng.integers(0, 1 << 32, size=3000):
        bip = int(bip)
        bipp = oracle.H(bip, 1 << 32, A1)
        shifted = (bipp << b) & 0xFFFFFFFF
        bits = format(shifted, "032b")
        r = bits.index("1") + 1 if "1" in bits else 33
        r = min(r, 32 - b)
        pidx, rho, vidx = o.hash_pair(5, bip)
        assert rho == r
        assert vidx == int(format(bipp, "032b")[:b], 2)
        assert pidx == o.phy_idx(5, vidx)


def test_rho_cap_on_all_zero_shifted_word():
    """A hashed bip whose 32-b low bits are all zero has no 1 bit left after
    the shift; its LBP1 is capped at 32-b (the last DR of the DRV).  The bip
    is found by brute-force search over the hash."""
    b = 16
    o = Oracle("gfast", k=4, Z=(1 << 16) + 7, b=b, seed=SEED)
    A1 = oracle.lib().orc_A1(o._h)
    found = None
    for bip in range(1 << 22):
        if (oracle.H(bip, 1 << 32, A1) & 0xFFFF) == 0:
            found = bip
            break
    assert found is not None
    pidx, rho, vidx = o.hash_pair(9, found)
    assert rho == 32 - b


def test_phy_idx_follows_alg3_two_hashes():
    """Alg. 3: s1 = H(i, 2^32, A0), j = H(aip, Z, s1); collisions allowed."""
    o = Oracle("gfast", k=4, Z=1000, b=5, seed=SEED)
    for aip in (0, 1, 0xFFFFFFFF, 123456789):
        for i in range(32):
            s1 = oracle.H(i, 1 << 32, SEED)
            assert o.phy_idx(aip, i) == oracle.H(aip, 1000, s1)


def test_mixed_group_rule():
    o = Oracle("gfast", k=4, Z=1 << 14, b=6, seed=SEED, b_min=6, group_rule=1)
    for aip in (0, 0x3FFFFFFF, 0x40000000, 0x80000000, 0xC0000000, 0xFFFFFFFF):
        assert o.host_b(aip) == 6 + (aip >> 30)


# -------------------------------------------------- DR / BDR machinery

def _pair_history_registers(o, slices, t, k):
    """Brute force: register of every pidx = max LBP1 among the pairs that
    hit it in the last min(k, t+1) slices (Sec. 3: a DR is active iff its
    LBP1 value was seen within the window)."""
    reg = np.zeros(o.Z, dtype=np.uint8)
    for s in slices[max(0, t - k + 1):t + 1]:
        for aip, bip in s.tolist():
            pidx, rho, _ = o.hash_pair(aip, bip)
            reg[pidx] = max(reg[pidx], rho)
    return reg


@pytest.mark.parametrize("variant", ["gfast", "gsmall", "serial"])
@pytest.mark.parametrize("k", [1, 3])
def test_register_equals_max_rho_over_window(variant, k):
    """BDR invariant: after closing slice t the register of each BDR is the
    largest LBP1 of the pairs mapped to it within W(t-k+1, k); k = 1 is the
    discrete window (plain per-slice HyperLogLog)."""
    rng = np.random.default_rng(10 + k)
    aips = traffic.distinct_u32(rng, 12)
    o = Oracle(variant, k=k, Z=257, b=4, seed=SEED)
    slices = []
    for t in range(9):
        n = int(rng.integers(0, 120))
        s = traffic.uniform_pairs(rng, n, aips)
        slices.append(s)
        o.scan(s)
        o.slide()
        reg = o.state()["reg"]
        np.testing.assert_array_equal(reg, _pair_history_registers(o, slices, t, k))


def test_dr_values_are_ages_gfast():
    """gfast state after a slide: DR[r] = number of slices since LBP1 value r
    was last the slice maximum of the BDR, saturating at 2^w - 1 (Sec. 3)."""
    k = 5
    o = Oracle("gfast", k=k, Z=64, b=4, seed=SEED)
    assert o.dr_max == 7  # w = ceil(log2(6)) = 3
    rng = np.random.default_rng(21)
    aips = traffic.distinct_u32(rng, 4)
    last_max = {}  # (pidx, r) -> slice where r was the slice max of pidx
    for t in range(14):
        s = traffic.uniform_pairs(rng, int(rng.integers(0, 40)), aips)
        smax = {}
        for aip, bip in s.tolist():
            pidx, rho, _ = o.hash_pair(aip, bip)
            smax[pidx] = max(smax.get(pidx, 0), rho)
        for pidx, r in smax.items():
            last_max[(pidx, r)] = t
        o.scan(s)
        o.slide()
        dr = o.state()["dr"]
        want = np.full_like(dr, o.dr_max)
        for (pidx, r), ts in last_max.items():
            want[pidx, r - 1] = min(t - ts, o.dr_max)
        np.testing.assert_array_equal(dr, want)
        assert (o.state()["bs"] == 0).all()


def test_serial_and_gfast_have_identical_drv():
    """nowLBP1 (Alg. 1/4) and bsLBP1 (Alg. 6/7) record the same slice
    maximum, so the DRVs agree after every slice."""
    rng = np.random.default_rng(22)
    aips = traffic.distinct_u32(rng, 50)
    a = Oracle("serial", k=6, Z=999, b=5, seed=SEED)
    b = Oracle("gfast", k=6, Z=999, b=5, seed=SEED)
    for t in range(12):
        s = traffic.uniform_pairs(rng, 3000, aips)
        for o in (a, b):
            o.scan(s)
            o.slide()
        sa, sb = a.state(), b.state()
        np.testing.assert_array_equal(sa["dr"], sb["dr"])
        np.testing.assert_array_equal(sa["reg"], sb["reg"])


def test_gsmall_registers_equal_gfast_registers():
    """Sec. 4.2: both GPU variants yield the same LBP1 through Alg. 2."""
    rng = np.random.default_rng(23)
    aips = traffic.distinct_u32(rng, 40)
    a = Oracle("gsmall", k=4, Z=4099, b=6, seed=SEED)
    b = Oracle("gfast", k=4, Z=4099, b=6, seed=SEED)
    for t in range(10):
        s = traffic.uniform_pairs(rng, int(rng.integers(0, 5000)), aips)
        for o in (a, b):
            o.scan(s)
            o.slide()
        np.testing.assert_array_equal(a.state()["reg"], b.state()["reg"])
        assert a.pool_sums() == b.pool_sums()


def test_gsmall_drv_is_aged_last_seen():
    """gsmall state after a slide: every LBP1 value ever seen at a BDR has
    DR = slices since it was last seen, plus one (the aging for the next
    slice has been applied), saturating at DR_MAX."""
    k = 3
    o = Oracle("gsmall", k=k, Z=31, b=4, seed=SEED)
    rng = np.random.default_rng(24)
    aips = traffic.distinct_u32(rng, 3)
    seen = {}
    for t in range(9):
        s = traffic.uniform_pairs(rng, int(rng.integers(0, 30)), aips)
        for aip, bip in s.tolist():
            pidx, rho, _ = o.hash_pair(aip, bip)
            seen[(pidx, rho)] = t
        o.scan(s)
        o.slide()
        dr = o.state()["dr"]
        want = np.full_like(dr, o.dr_max)
        for (pidx, r), ts in seen.items():
            want[pidx, r - 1] = min(t - ts + 1, o.dr_max)
        np.testing.assert_array_equal(dr, want)


def test_saturation_and_expiry():
    """A pair seen only in slice t counts in windows t .. t+k-1 and in no
    later one; untouched DRs stay at DR_MAX."""
    k = 4
    for variant in ("gfast", "gsmall", "serial"):
        o = Oracle(variant, k=k, Z=101, b=4, seed=SEED)
        pair = np.array([[1234, 98765]], dtype=np.uint32)
        pidx, rho, _ = o.hash_pair(1234, 98765)
        o.scan(pair)
        for t in range(3 * k):
            o.slide()
            st = o.state()
            assert st["reg"][pidx] == (rho if t < k else 0), (variant, t)
            assert (st["dr"] <= o.dr_max).all()
            others = np.delete(np.arange(o.Z), pidx)
            assert (st["reg"][others] == 0).all()
        assert (o.state()["dr"] == o.dr_max).all()


def test_scan_is_order_independent():
    rng = np.random.default_rng(25)
    aips = traffic.distinct_u32(rng, 30)
    for variant in ("gfast", "gsmall", "serial"):
        a = Oracle(variant, k=5, Z=2048, b=5, seed=SEED)
        b = Oracle(variant, k=5, Z=2048, b=5, seed=SEED)
        for t in range(6):
            s = traffic.uniform_pairs(rng, 4000, aips)
            a.scan(s)
            b.scan(s[rng.permutation(len(s))])
            sa, sb = a.state(), b.state()
            np.testing.assert_array_equal(sa["bs"], sb["bs"])
            np.testing.assert_array_equal(sa["dr"], sb["dr"])
            np.testing.assert_array_equal(sa["now"], sb["now"])
            a.slide()
            b.slide()


def test_race_example_highest_lbp1_wins():
    """Sec. 4.2's conflict: two pairs r1 < r2 on one BDR must leave r2 as the
    slice maximum, in either order."""
    o = Oracle("gfast", k=3, Z=1 << 10, b=4, seed=SEED)
    rng = np.random.default_rng(26)
    by_pidx = {}
    for bip in rng.integers(0, 1 << 32, size=20000):
        pidx, rho, _ = o.hash_pair(42, int(bip))
        by_pidx.setdefault(pidx, {}).setdefault(rho, int(bip))
    pidx, rs = next((p, r) for p, r in by_pidx.items() if len(r) >= 3)
    r_small, r_big = sorted(rs)[1], sorted(rs)[-1]
    for order in ((r_small, r_big), (r_big, r_small)):
        for variant in ("gfast", "serial", "gsmall"):
            o2 = Oracle(variant, k=3, Z=1 << 10, b=4, seed=SEED)
            o2.scan(np.array([[42, rs[order[0]]], [42, rs[order[1]]]], dtype=np.uint32))
            o2.slide()
            assert o2.state()["reg"][pidx] == r_big


def test_pool_sums_definition():
    rng = np.random.default_rng(27)
    aips = traffic.distinct_u32(rng, 30)
    o = Oracle("gfast", k=5, Z=3000, b=5, seed=SEED)
    o.scan(traffic.uniform_pairs(rng, 5000, aips))
    o.slide()
    reg = o.state()["reg"].astype(np.int64)
    S = sum(2 ** (32 - int(r)) for r in reg)
    assert o.pool_sums() == (S, int((reg == 0).sum()))


# ------------------------------------------------------------- estimator

def test_hll_alpha_constants():
    for m, a in _golden("hll_constants.txt"):
        assert oracle.hll_alpha(float(m)) == pytest.approx(float(a), rel=1e-12)


@pytest.mark.parametrize("g", [16, 64, 256])
def test_hll_closed_form_equal_registers(g):
    """All g registers equal r: the harmonic mean gives alpha_g * g * 2^r."""
    for r in range(3, 20):
        S = g * (1 << (32 - r))
        assert oracle.hll(g, S, 0) == pytest.approx(oracle.hll_alpha(g) * g * 2.0 ** r,
                                                    rel=1e-12)


def test_hll_linear_counting_closed_form():
    """Small range: with V empty registers out of m and the raw estimate at
    most 2.5 m, the estimate is m ln(m / V)."""
    m = 128
    for V in (1, 10, 64, 127):
        S = V * (1 << 32) + (m - V) * (1 << 31)  # others hold 1
        assert oracle.hll(m, S, V) == pytest.approx(m * math.log(m / V), rel=1e-12)
    assert oracle.hll(m, m * (1 << 32), m) == 0.0  # all empty


def test_vhll_noise_removal_closed_forms():
    """vHLL: n = Zg/(Z-g) (n_g/g - n_Z/Z).  A host whose registers look like
    the pool's average gets 0; with an empty pool (no noise) and large Z the
    estimate tends to the host's plain HLL estimate."""
    Z, g = 1 << 20, 128
    # host registers all 5, pool registers all 5: same per-register load
    S_host, S_pool = g * (1 << 27), Z * (1 << 27)
    assert oracle.vhll(Z, g, S_host, 0, S_pool, 0) == pytest.approx(0.0, abs=1e-6)
    # pool empty but the host's own registers: n -> n_g * Z/(Z-g)
    S_pool = (Z - g) * (1 << 32) + g * (1 << 27)
    n_g = oracle.hll(g, S_host, 0)
    n_Z = oracle.hll(Z, S_pool, Z - g)
    want = Z * g / (Z - g) * (n_g / g - n_Z / Z)
    got = oracle.vhll(Z, g, S_host, 0, S_pool, Z - g)
    assert got == pytest.approx(want, rel=1e-12)
    assert got == pytest.approx(n_g, rel=2e-3)
    # host less loaded than the pool -> clamped at zero
    assert oracle.vhll(Z, g, g * (1 << 30), 0, Z * (1 << 27), 0) == 0.0


def test_exact_numpy_matches_sets():
    rng = np.random.default_rng(30)
    aips = traffic.distinct_u32(rng, 7)
    slices = []
    for t in range(6):
        s = traffic.uniform_pairs(rng, 40, aips)
        s[:, 1] %= 50  # force repeats across slices
        slices.append(s)
    for t in range(6):
        for k in (1, 2, 4):
            a = exact.window_cardinalities(slices, t, k, aips)
            b = exact.window_cardinalities_sets(slices, t, k, aips)
            assert list(a) == b


def test_estimator_accuracy_single_host_envelope():
    """Statistical pin: with a pool far larger than the load, the estimate of
    a host of true cardinality n has relative standard error near HLL's
    1.04/sqrt(g) (Sec. 2.2's HyperLogLog); the mean relative error over many
    independent hosts stays inside that envelope and the bias is small."""
    g, b = 128, 7
    rng = np.random.default_rng(31)
    rel = []
    aips = traffic.distinct_u32(rng, 40)
    o = Oracle("gfast", k=2, Z=1 << 20, b=b, seed=SEED)
    cards = rng.integers(2000, 60000, size=aips.size)
    pairs = np.concatenate([
        np.stack([np.full(c, a, dtype=np.uint32), traffic.distinct_u32(rng, int(c))], 1)
        for a, c in zip(aips, cards)])
    o.scan(pairs)
    o.slide()
    est = o.estimate(aips)
    rel = (est - cards) / cards
    sigma = 1.04 / math.sqrt(g)
    assert np.mean(np.abs(rel)) < 1.3 * sigma
    assert abs(np.mean(rel)) < 3 * sigma / math.sqrt(aips.size) + 0.01


def test_estimator_removes_sharing_noise():
    """Many hosts share a small pool: without the noise term a small host
    would be over-estimated by about g * (pool load per register)."""
    g, b, Z = 64, 6, 1 << 14
    rng = np.random.default_rng(32)
    # many background hosts, so that every physical BDR is shared by many
    # virtual ones (the regime the sharing model assumes)
    big = traffic.distinct_u32(rng, 5000)
    o = Oracle("gfast", k=1, Z=Z, b=b, seed=SEED)
    bulk = np.stack([np.repeat(big, 20), rng.integers(0, 1 << 32, 100000, dtype=np.uint64).astype(np.uint32)], 1)
    small_hosts = traffic.distinct_u32(np.random.default_rng(33), 60)
    small = np.stack([np.repeat(small_hosts, 300),
                      rng.integers(0, 1 << 32, 60 * 300, dtype=np.uint64).astype(np.uint32)], 1)
    o.scan(np.concatenate([bulk, small]))
    o.slide()
    est = o.estimate(small_hosts)
    # pool load 118000 / 16384 ~ 7.2 per register: uncorrected bias ~ +460
    assert abs(np.mean(est) - 300) < 60
    S_Z, V_Z = o.pool_sums()
    noisy = [oracle.hll(g, *o.host_registers(int(a))[:2]) for a in small_hosts]
    assert np.mean(noisy) > 600


def test_small_workload_mre_vs_exact():
    """End to end on the small workload shape (downsized: 4 slices of 20k
    pairs): hosts whose window cardinality is large against the pool noise
    are estimated within the HLL envelope."""
    cfg = traffic.SMALL
    gen = traffic.ZipfTraffic(cfg["n_hosts"], cfg["zipf_s"], cfg["c_max"], cfg["k"], seed=7)
    o = Oracle("gfast", k=cfg["k"], Z=cfg["Z"], b=cfg["log2_g"], seed=SEED)
    slices = []
    for t in range(4):
        s = gen.next_slice(20000)
        slices.append(s)
        o.scan(s)
        o.slide()
    truth = exact.window_cardinalities(slices, 3, cfg["k"], gen.aips)
    est = o.estimate(gen.aips)
    big = truth >= 1000
    assert big.sum() >= 3
    rel = np.abs(est[big] - truth[big]) / truth[big]
    assert rel.mean() < 2.5 * 1.04 / math.sqrt(128)


def test_table1_bits():
    """Table 1 with log2(n/g) read as R = 32-b DRs and log2(k+1) as w."""
    o = Oracle("gfast", k=10, Z=1 << 10, b=7, seed=SEED)  # R=25, w=4
    assert o.table1_bits("gsmall") == 100
    assert o.table1_bits("gfast") == 125
    assert o.table1_bits("serial") == 105
    o = Oracle("gfast", k=30, Z=1 << 10, b=8, seed=SEED)  # R=24, w=5
    assert (o.table1_bits("gsmall"), o.table1_bits("gfast"),
            o.table1_bits("serial")) == (120, 144, 125)


def test_invalid_parameters_rejected():
    with pytest.raises(ValueError):
        Oracle("gfast", k=0, Z=100, b=4, seed=1)
    with pytest.raises(ValueError):
        Oracle("gfast", k=3, Z=16, b=4, seed=1)  # Z must exceed g
    with pytest.raises(ValueError):
        Oracle("gfast", k=3, Z=1 << 32, b=4, seed=1)  # the pool sum must fit 64 bits
    o = Oracle("gfast", k=3, Z=100, b=4, seed=1)
    with pytest.raises(RuntimeError):
        o.estimate(np.array([1], dtype=np.uint32))


# ------------------------------------------ register-level state loading

def _virtual_registers_of(o, reg, aips):
    """Host-major virtual registers reg[pidx(aip, i)], i < g(aip), with pidx
    from Alg. 3 (o.phy_idx, pinned above), and their offsets."""
    gs = [1 << o.host_b(int(a)) for a in aips]
    offsets = np.concatenate([[0], np.cumsum(gs)[:-1]]).astype(np.uint64)
    vregs = np.empty(int(sum(gs)), dtype=np.uint8)
    for h, a in enumerate(aips):
        for i in range(gs[h]):
            vregs[int(offsets[h]) + i] = reg[o.phy_idx(int(a), i)]
    return offsets, vregs


def test_load_virtual_registers_rebuilds_scanned_state():
    """Invariant: after a scan, every physical register is the largest of
    the virtual registers that Alg. 3 maps onto it (a BDR no pair reached is
    0).  So loading the virtual registers a scanned state implies, for the
    hosts that made the traffic, rebuilds that state's registers exactly --
    into an instance whose registers were dirty before (untouched BDRs must
    come out 0), with mixed g (host-major offsets of uneven length)."""
    k, Z, b_min = 3, 1 << 14, 5
    gen = traffic.ZipfTraffic(60, 1.1, 3000, k, seed=41)
    o = Oracle("gfast", k=k, Z=Z, b=b_min + 3, seed=SEED, b_min=b_min, group_rule=1)
    for _ in range(3):
        o.scan(gen.next_slice(20000))
        o.slide()
    reg = o.registers()
    assert (reg == 0).sum() > Z // 4  # BDRs no host maps to stay 0
    assert len({o.host_b(int(a)) for a in gen.aips}) >= 3
    offsets, vregs = _virtual_registers_of(o, reg, gen.aips)
    dirty = Oracle("gfast", k=k, Z=Z, b=b_min + 3, seed=SEED, b_min=b_min, group_rule=1)
    other = traffic.ZipfTraffic(2000, 1.1, 3000, k, seed=42)
    dirty.scan(other.next_slice(60000))
    dirty.slide()
    # stale values where the loaded hosts map nothing, and where they do
    assert ((dirty.registers() != 0) & (reg == 0)).sum() > 1000
    assert (dirty.registers() != reg).sum() > Z // 4
    dirty.load_virtual_registers(gen.aips, offsets, vregs)
    np.testing.assert_array_equal(dirty.registers(), reg)
    assert dirty.pool_sums() == o.pool_sums()
    np.testing.assert_allclose(dirty.estimate(gen.aips), o.estimate(gen.aips), rtol=0, atol=0)


def test_load_virtual_registers_collisions_fold_by_max():
    """Brute force on a tiny pool: two hosts whose virtual registers collide
    on physical BDRs; each physical register is the maximum over its
    colliding virtual registers, the rest 0."""
    Z, b = 97, 4
    o = Oracle("gfast", k=2, Z=Z, b=b, seed=SEED)
    rng = np.random.default_rng(43)
    aips = traffic.distinct_u32(rng, 12)
    vregs = rng.integers(0, 29, size=12 * 16).astype(np.uint8)
    offsets = (np.arange(12) * 16).astype(np.uint64)
    want = np.zeros(Z, dtype=np.uint8)
    hits = np.zeros(Z, dtype=np.int64)
    for h, a in enumerate(aips):
        for i in range(16):
            j = o.phy_idx(int(a), i)
            hits[j] += 1
            want[j] = max(want[j], vregs[h * 16 + i])
    assert (hits >= 2).sum() > 10  # collisions happen
    o.load_virtual_registers(aips, offsets, vregs)
    np.testing.assert_array_equal(o.registers(), want)
    S = sum(1 << (32 - int(m)) for m in want)
    assert o.pool_sums() == (S, int((want == 0).sum()))


def test_load_virtual_registers_accuracy_per_group():
    """Statistical pin of the register-level workload: registers drawn as
    the maximum of Poisson(c/g) geometric LBP1 values and loaded into a
    pool far larger than the load are HyperLogLog registers of c items, so
    each g group's estimates have relative standard error about 1.04/sqrt(g)
    (Flajolet et al. 2007) and little bias."""
    from synth.registers import BatchedRegisters
    b_min = 6
    br = BatchedRegisters(1200, b_min, 3e5, seed=44)
    keep = br.card >= 200  # above HLL's small-range regime
    o = Oracle("gfast", k=60, Z=1 << 22, b=b_min + 3, seed=SEED, b_min=b_min, group_rule=1)
    o.load_virtual_registers(br.aips, br.offsets, br.vregs)
    est = o.estimate(br.aips)
    for b in range(b_min, b_min + 4):
        sel = keep & (br.b == b)
        assert sel.sum() > 100
        rel = (est[sel] - br.card[sel]) / br.card[sel]
        sigma = 1.04 / math.sqrt(1 << b)
        assert math.sqrt(np.mean(rel ** 2)) < 1.5 * sigma, (b, math.sqrt(np.mean(rel ** 2)))
        assert abs(np.mean(rel)) < 4 * sigma / math.sqrt(sel.sum()) + 0.01, b
