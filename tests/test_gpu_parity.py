"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

State (DRV, bsLBP1, registers, pool sums) must match bit for bit after every
slice; estimates within 1e-6 relative (absolute 1e-6 below magnitude 1) of
the oracle's FP64 values -- the FP32 output rounding alone is 6e-8.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from synth import traffic  # noqa: E402

pytestmark = pytest.mark.gpu

SEED = 0x9E3779B97F4A7C15
EST_RTOL = 1e-6


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def _dev(a: np.ndarray):
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).cuda()


def _make(layout, k, Z, b, b_min=None, group_rule=0, seed=SEED, scan_mode="direct"):
    from paper_1810_13132_gb300 import Config, Vbdr
    v = Vbdr(Config(k=k, num_bdr=Z, log2_g=b, layout=layout, seed=seed,
                    log2_g_min=b_min or 0, group_rule=group_rule))
    v.set_scan_mode(scan_mode)
    o = oracle.Oracle(layout, k=k, Z=Z, b=b, seed=seed, b_min=b_min,
                      group_rule=group_rule)
    assert v.R == o.R
    return v, o


def _slice_max_state(os_, layout):
    # the per-slice state of the layout: bsLBP1 (gfast), nowLBP1 (serial)
    return os_["now"].astype(np.uint32) if layout == "serial" else os_["bs"]


def _compare_state(v, o, tag=""):
    gs, os_ = v.state(), o.state()
    np.testing.assert_array_equal(gs["reg"], os_["reg"], err_msg=f"reg {tag}")
    np.testing.assert_array_equal(gs["dr"], os_["dr"], err_msg=f"dr {tag}")
    np.testing.assert_array_equal(gs["bs"], _slice_max_state(os_, v.cfg.layout), err_msg=f"bs {tag}")
    assert v.pool_sums() == o.pool_sums(), tag


def _compare_estimates(v, o, aips):
    got = v.estimate(_dev(aips)).cpu().numpy().astype(np.float64)
    want = o.estimate(aips)
    err = np.abs(got - want) / np.maximum(np.abs(want), 1.0)
    assert err.max() <= EST_RTOL, (err.max(), int(err.argmax()))
    return got, want


def _run(layout, k, Z, b, slices, aips, b_min=None, group_rule=0, every=True,
         split=1, scan_mode="direct"):
    v, o = _make(layout, k, Z, b, b_min, group_rule, scan_mode=scan_mode)
    for t, s in enumerate(slices):
        if split == 1:
            v.scan(_dev(s))
        else:  # several scan calls per slice, 16-byte aligned pieces
            cuts = np.linspace(0, len(s), split + 1).astype(int) & ~1
            cuts[-1] = len(s)
            for a, c in zip(cuts[:-1], cuts[1:]):
                v.scan(_dev(s[a:c]))
        o.scan(s)
        if every:  # state after the scan, before the slide (bsLBP1 / DRV)
            _compare_state_scan(v, o, f"t={t} after scan")
        v.slide()
        o.slide()
        if every or t == len(slices) - 1:
            _compare_state(v, o, f"t={t}")
    _compare_estimates(v, o, aips)
    v.close()
    return o


def _compare_state_scan(v, o, tag):
    gs, os_ = v.state(), o.state()
    np.testing.assert_array_equal(gs["dr"], os_["dr"], err_msg=f"dr {tag}")
    np.testing.assert_array_equal(gs["bs"], _slice_max_state(os_, v.cfg.layout), err_msg=f"bs {tag}")


# ---------------------------------------------------------------- workloads

@pytest.mark.parametrize("layout", ["gfast", "gsmall", "serial"])
def test_small_workload_every_slice(layout):
    """The small configuration at full size: k=10, 1e5 pairs per slice,
    1000 Zipf(1.1) hosts capped at 5000, Z = 2^16, g = 128; 13 slices so
    that the window wraps and DRs saturate."""
    cfg = traffic.SMALL
    gen = traffic.ZipfTraffic(cfg["n_hosts"], cfg["zipf_s"], cfg["c_max"], cfg["k"], seed=101)
    slices = [gen.next_slice(cfg["n_pairs"]) for _ in range(13)]
    _run(layout, cfg["k"], cfg["Z"], cfg["log2_g"], slices, gen.aips)


@pytest.mark.parametrize("layout", ["gfast", "gsmall", "serial"])
def test_trace_shape_downscaled(layout):
    """Trace-shaped traffic (Zipf 1.05, 10% in-slice repeats, k=30, g=256)
    at 1/64 of the pairs and hosts, 1/64 of the pool; 33 slices."""
    gen = traffic.ZipfTraffic(16384, 1.05, 2_000_000 // 64, 30, seed=102, repeat_frac=0.10)
    slices = [gen.next_slice(1 << 20) for _ in range(33)]
    _run(layout, 30, 1 << 18, 8, slices, gen.aips, every=False)


@pytest.mark.parametrize("layout", ["gfast", "gsmall", "serial"])
def test_mixed_g_groups(layout):
    """Four host groups g = 64..512 in one pool (b_min = 6, R = 26, k = 60)."""
    rng = np.random.default_rng(103)
    aips = traffic.distinct_u32(rng, 4000)
    slices = [traffic.uniform_pairs(rng, 200_001, aips) for _ in range(4)]
    _run(layout, 60, (1 << 18) + 12345, 6, slices, aips, b_min=6, group_rule=1)


# --------------------------------------------------------------- edge cases

@pytest.mark.parametrize("layout", ["gfast", "gsmall", "serial"])
def test_empty_single_and_odd_slices(layout):
    rng = np.random.default_rng(104)
    aips = traffic.distinct_u32(rng, 50)
    sizes = [0, 1, 3, 0, 17, 1023, 1, 0, 65537, 2]
    slices = [traffic.uniform_pairs(rng, n, aips) for n in sizes]
    _run(layout, 4, 4099, 5, slices, aips)


@pytest.mark.parametrize("layout", ["gfast", "gsmall", "serial"])
@pytest.mark.parametrize("k", [1, 15])
def test_discrete_window_and_k_at_dr_max(layout, k):
    """k = 1 (discrete window) and k = 15 = DR_MAX with w = 4."""
    rng = np.random.default_rng(105 + k)
    aips = traffic.distinct_u32(rng, 300)
    slices = [traffic.uniform_pairs(rng, int(rng.integers(1000, 30000)), aips)
              for _ in range(20)]
    _run(layout, k, 10007, 7, slices, aips)


@pytest.mark.parametrize("layout", ["gfast", "gsmall", "serial"])
def test_max_contention_one_host(layout):
    """Every pair to one aip with g = 2: all updates hit two BDRs."""
    rng = np.random.default_rng(106)
    aip = np.array([0xDEADBEEF], dtype=np.uint32)
    slices = [traffic.uniform_pairs(rng, 300_000, aip) for _ in range(3)]
    _run(layout, 3, 1000, 1, slices, aip)


@pytest.mark.parametrize("layout", ["gfast", "gsmall", "serial"])
def test_lbp1_at_the_cap(layout):
    """Pairs whose shifted hash word is all zero below the virtual-index bits
    (LBP1 = R = 32 - b, the capped case), found by brute force over bips with
    the oracle's hash, mixed with ordinary pairs: the DR at the cap and the
    registers equal to R must match the oracle."""
    b, Z = 15, (1 << 17) + 5
    h = oracle.Oracle(layout, k=3, Z=Z, b=b, seed=SEED)
    aips = np.array([0x0A0B0C0D, 0x7F000001], dtype=np.uint32)
    capped = [(int(a), bip) for a in aips for bip in range(0, 400_000)
              if h.hash_pair(int(a), bip)[1] == 32 - b]
    assert len(capped) >= 4
    rng = np.random.default_rng(108)
    slices = []
    for t in range(4):
        s = np.concatenate([np.array(capped[t::2], dtype=np.uint32).reshape(-1, 2),
                            traffic.uniform_pairs(rng, 5000, aips)])
        slices.append(s)
    o = _run(layout, 3, Z, b, slices, aips)
    assert (o.state()["reg"] == 32 - b).any()


@pytest.mark.parametrize("layout", ["gfast", "gsmall", "serial"])
def test_duplicate_heavy_and_split_scans(layout):
    """Bursts of identical pairs inside a warp, and one slice scanned in
    several calls: same state as the single-call oracle."""
    rng = np.random.default_rng(107)
    aips = traffic.distinct_u32(rng, 40)
    slices = []
    for _ in range(5):
        s = traffic.uniform_pairs(rng, 50_000, aips)
        s = np.repeat(s, rng.integers(1, 6, size=len(s)), axis=0)[:120_000]
        slices.append(np.ascontiguousarray(s))
    _run(layout, 5, 8191, 6, slices, aips, split=7)


@pytest.mark.parametrize("layout", ["gfast", "gsmall", "serial"])
def test_order_independence_on_gpu(layout):
    from paper_1810_13132_gb300 import Config, Vbdr
    rng = np.random.default_rng(108)
    aips = traffic.distinct_u32(rng, 500)
    s = traffic.uniform_pairs(rng, 400_000, aips)
    a = Vbdr(Config(k=3, num_bdr=1 << 15, log2_g=7, layout=layout))
    b = Vbdr(Config(k=3, num_bdr=1 << 15, log2_g=7, layout=layout))
    a.scan(_dev(s))
    b.scan(_dev(s[rng.permutation(len(s))]))
    a.slide()
    b.slide()
    sa, sb = a.state(), b.state()
    for key in ("dr", "bs", "reg"):
        np.testing.assert_array_equal(sa[key], sb[key])


def test_all_layouts_agree_on_gpu():
    """Sec. 4.2: the GPU variants yield the same registers (and estimates);
    serial and gfast also hold the same DRV (Alg. 1 and Alg. 6 fold the same
    slice maximum)."""
    from paper_1810_13132_gb300 import Config, Vbdr
    gen = traffic.ZipfTraffic(2000, 1.1, 5000, 6, seed=109)
    a = Vbdr(Config(k=6, num_bdr=1 << 16, log2_g=7, layout="gfast"))
    b = Vbdr(Config(k=6, num_bdr=1 << 16, log2_g=7, layout="gsmall"))
    c = Vbdr(Config(k=6, num_bdr=1 << 16, log2_g=7, layout="serial"))
    for _ in range(9):
        s = _dev(gen.next_slice(100_000))
        for v in (a, b, c):
            v.scan(s)
            v.slide()
        np.testing.assert_array_equal(a.registers(), b.registers())
        np.testing.assert_array_equal(a.registers(), c.registers())
        np.testing.assert_array_equal(a.state()["dr"], c.state()["dr"])
    aips = _dev(gen.aips)
    assert torch.equal(a.estimate(aips), b.estimate(aips))
    assert torch.equal(a.estimate(aips), c.estimate(aips))


# ------------------------------------------------------ bucketed scan path
# With the bucketed scan selected, slices of at least 2^18 pairs (gfast,
# gsmall) become records in per-tile buckets that each pool tile applies in
# shared memory.  These cases stress what is specific to it.

@pytest.mark.parametrize("layout", ["gfast", "gsmall"])
def test_bucketed_scan_trace_shape_downscaled(layout):
    """The trace-shaped workload at 1/64 (1M pairs per slice, two passes'
    worth of records on a 2^18 pool), state after every slice."""
    gen = traffic.ZipfTraffic(16384, 1.05, 2_000_000 // 64, 30, seed=122, repeat_frac=0.10)
    slices = [gen.next_slice(1 << 20) for _ in range(6)]
    _run(layout, 30, 1 << 18, 8, slices, gen.aips, scan_mode="bucketed")


@pytest.mark.parametrize("layout", ["gfast", "gsmall"])
def test_bucketed_scan_bucket_overflow(layout):
    """One host with g = 16: all records fall into at most 16 of the 16 pool
    tiles, far above a bucket's share, so the overflowing records take the
    direct path; several passes per slice (2M pairs)."""
    rng = np.random.default_rng(120)
    aip = np.array([0x01020304], dtype=np.uint32)
    slices = [traffic.uniform_pairs(rng, 2_000_001, aip) for _ in range(3)]
    _run(layout, 3, 1 << 20, 4, slices, aip, scan_mode="bucketed")


@pytest.mark.parametrize("layout", ["gfast", "gsmall"])
def test_bucketed_scan_threshold_split_and_mixed_g(layout):
    """Slices just below and at the bucketed-scan threshold, a slice scanned
    in two calls that both take the bucketed path, mixed g, a pool that is
    not a whole number of tiles; state after every scan and slide."""
    rng = np.random.default_rng(121)
    aips = traffic.distinct_u32(rng, 6000)
    sizes = [(1 << 18) - 2, 1 << 18, 600_001, (1 << 18) + 1]
    slices = [traffic.uniform_pairs(rng, n, aips) for n in sizes]
    _run(layout, 7, (3 << 16) + 77, 6, slices[:2], aips, b_min=6, group_rule=1,
         scan_mode="bucketed")
    _run(layout, 7, (3 << 16) + 77, 6, slices[2:], aips, b_min=6, group_rule=1, split=2,
         scan_mode="bucketed")


# --------------------------------------------------------- host-buffer path

@pytest.mark.parametrize("layout", ["gfast", "gsmall", "serial"])
def test_host_buffer_entry_points(layout):
    """vbdr_scan_slice_host / vbdr_estimate_host (pinned and pageable) give
    the same state and estimates as the device-buffer calls."""
    from paper_1810_13132_gb300 import Config, Vbdr
    gen = traffic.ZipfTraffic(3000, 1.1, 5000, 4, seed=110)
    a = Vbdr(Config(k=4, num_bdr=1 << 16, log2_g=7, layout=layout))
    b = Vbdr(Config(k=4, num_bdr=1 << 16, log2_g=7, layout=layout))
    for t in range(5):
        s = gen.next_slice(9_000_001 if t == 2 else 200_001)  # > one staging chunk
        a.scan(_dev(s))
        if t % 2:
            b.scan_host(s)
        else:
            pinned = torch.from_numpy(s.view(np.int32)).pin_memory()
            b.scan_host(pinned)
        a.slide()
        b.slide()
        torch.cuda.synchronize()
    np.testing.assert_array_equal(a.registers(), b.registers())
    np.testing.assert_array_equal(a.state()["dr"], b.state()["dr"])
    out = np.empty(gen.aips.size, dtype=np.float32)
    b.estimate_host(gen.aips, out)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out, a.estimate(_dev(gen.aips)).cpu().numpy())


def test_estimate_before_slide_is_an_order_error():
    from paper_1810_13132_gb300 import Config, Vbdr, VbdrError
    v = Vbdr(Config(k=3, num_bdr=4096, log2_g=5))
    with pytest.raises(VbdrError) as e:
        v.estimate(_dev(np.arange(4, dtype=np.uint32)))
    assert e.value.code == -5


def test_scan_mode_selection():
    from paper_1810_13132_gb300 import Config, Vbdr, VbdrError
    v = Vbdr(Config(k=3, num_bdr=4096, log2_g=5, layout="serial"))
    with pytest.raises(VbdrError) as e:
        v.set_scan_mode("bucketed")  # the bucketed scan serves gfast and gsmall
    assert e.value.code == -1
    v.set_scan_mode("direct")


def test_misaligned_pairs_rejected():
    from paper_1810_13132_gb300 import Config, Vbdr, VbdrError
    v = Vbdr(Config(k=3, num_bdr=4096, log2_g=5))
    buf = _dev(np.arange(64, dtype=np.uint32))
    with pytest.raises(VbdrError) as e:
        v.scan(buf[2:])  # 8-byte offset
    assert e.value.code == -1


# ------------------------------------------------ full-size trace, sampled

@pytest.mark.parametrize("layout,scan_mode", [("gfast", "direct"), ("gsmall", "direct"),
                                              ("serial", "direct"), ("gfast", "bucketed"),
                                              ("gsmall", "bucketed")])
def test_trace_full_size_two_slices(layout, scan_mode):
    """The trace configuration at full size (N = 64M pairs per slice, 1M
    hosts, Z = 2^24, g = 256, k = 30, 10% repeats), two slices in the launch
    configuration the benchmark uses: state bit-exact after both slides and
    estimates of 20000 sampled hosts within tolerance."""
    cfg = traffic.TRACE
    gen = traffic.ZipfTraffic(cfg["n_hosts"], cfg["zipf_s"], cfg["c_max"], cfg["k"],
                              seed=111, repeat_frac=cfg["repeat_frac"])
    v, o = _make(layout, cfg["k"], cfg["Z"], cfg["log2_g"], scan_mode=scan_mode)
    for t in range(2):
        s = gen.next_slice(cfg["n_pairs"])
        v.scan(_dev(s))
        o.scan(s)
        v.slide()
        o.slide()
    gs, os_ = v.state(), o.state()
    np.testing.assert_array_equal(gs["reg"], os_["reg"])
    np.testing.assert_array_equal(gs["dr"], os_["dr"])
    assert v.pool_sums() == o.pool_sums()
    sample = np.random.default_rng(5).choice(gen.aips, 20000, replace=False)
    _compare_estimates(v, o, sample)
