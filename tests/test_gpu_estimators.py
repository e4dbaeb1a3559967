"""LogLog and PCSA estimates on the GPU against the oracle (Sec. 4.1: the
BDR pool serves PCSA and LogLog counting as well as HyperLogLog).

PCSA statistics and the pool sums must match bit for bit after every slide;
estimates within 1e-6 relative (absolute below magnitude 1) of the oracle's
FP64 values.
"""
import ctypes

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


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).cuda()


def _make(layout, k, Z, b, b_min=None, group_rule=0):
    from paper_1810_13132_gb300 import Config, Vbdr
    v = Vbdr(Config(k=k, num_bdr=Z, log2_g=b, layout=layout, seed=SEED,
                    log2_g_min=b_min or 0, group_rule=group_rule))
    o = oracle.Oracle(layout, k=k, Z=Z, b=b, seed=SEED, b_min=b_min, group_rule=group_rule)
    return v, o


def _close(got, want):
    err = np.abs(got.astype(np.float64) - want) / np.maximum(np.abs(want), 1.0)
    assert err.max() <= EST_RTOL, (err.max(), int(err.argmax()))


def _check(v, o, aips, layout):
    L_Z, P_Z = v.pool_sums_alt()
    assert (L_Z, P_Z if layout == "gsmall" else 0) == o.pool_sums_alt()
    d = _dev(aips)
    _close(v.estimate(d, estimator="loglog").cpu().numpy(), o.estimate_alt(aips, "loglog"))
    if layout == "gsmall":
        np.testing.assert_array_equal(v.pcsa_statistics(), o.pcsa_statistics())
        _close(v.estimate(d, estimator="pcsa").cpu().numpy(), o.estimate_alt(aips, "pcsa"))


def _run(layout, k, Z, b, slices, aips, **kw):
    v, o = _make(layout, k, Z, b, **kw)
    for s in slices:
        v.scan(_dev(s))
        o.scan(s)
        v.slide()
        o.slide()
        _check(v, o, aips, layout)
    return v, o


@pytest.mark.parametrize("layout", ["gfast", "gsmall", "serial"])
def test_small_workload_every_slice(layout):
    """The small configuration at full size (k=10, 1e5 pairs, 1000 hosts,
    Z = 2^16, g = 128), 12 slices so that the window wraps."""
    cfg = traffic.SMALL
    gen = traffic.ZipfTraffic(cfg["n_hosts"], cfg["zipf_s"], cfg["c_max"], cfg["k"], seed=301)
    slices = [gen.next_slice(cfg["n_pairs"]) for _ in range(12)]
    _run(layout, cfg["k"], cfg["Z"], cfg["log2_g"], slices, gen.aips)


@pytest.mark.parametrize("k", [1, 15])
def test_pcsa_discrete_window_and_saturated_drs(k):
    """k = 1 (plain per-slice PCSA) and k = 15 = DR_MAX (4-bit DRs: an aged
    DR can no longer tell 'seen k slices ago' from 'never')."""
    rng = np.random.default_rng(302 + k)
    aips = traffic.distinct_u32(rng, 200)
    slices = [traffic.uniform_pairs(rng, int(n), aips) for n in (30000, 0, 5, 70001, 30000, 1)]
    _run("gsmall", k, 20011, 6, slices, aips)


def test_mixed_g_groups():
    """Four host groups g = 64..512 (b_min = 6) in one pool."""
    rng = np.random.default_rng(304)
    aips = traffic.distinct_u32(rng, 3000)
    slices = [traffic.uniform_pairs(rng, 150_001, aips) for _ in range(3)]
    _run("gsmall", 60, (1 << 18) + 12345, 6, slices, aips, b_min=6, group_rule=1)
    _run("gfast", 60, (1 << 18) + 12345, 6, slices[:2], aips, b_min=6, group_rule=1)


def test_errors():
    from paper_1810_13132_gb300 import VbdrError, load
    rng = np.random.default_rng(305)
    aips = traffic.distinct_u32(rng, 10)
    v, _ = _make("gfast", 4, 4099, 5)
    d = _dev(aips)
    with pytest.raises(VbdrError):
        v.estimate(d, estimator="loglog")  # before the first slide
    v.scan(_dev(traffic.uniform_pairs(rng, 1000, aips)))
    v.slide()
    with pytest.raises(VbdrError):
        v.estimate(d, estimator="pcsa")  # gfast records no bitmap
    with pytest.raises(VbdrError):
        v.pcsa_statistics()
    out = torch.empty(aips.size, dtype=torch.float32, device="cuda")
    lib = load()
    assert lib.vbdr_estimate_alt(v._h, d.data_ptr(), aips.size, out.data_ptr(), 7, None) == -1


def test_checkpoint_keeps_pcsa():
    """A gsmall checkpoint carries the PCSA statistics and all pool sums: the
    resumed handle estimates like the saved one."""
    from paper_1810_13132_gb300 import Config, Vbdr
    rng = np.random.default_rng(306)
    aips = traffic.distinct_u32(rng, 500)
    cfg = Config(k=5, num_bdr=1 << 16, log2_g=7, layout="gsmall", seed=SEED)
    v = Vbdr(cfg)
    for _ in range(3):
        v.scan(_dev(traffic.uniform_pairs(rng, 100_000, aips)))
        v.slide()
    blob = v.save()
    w = Vbdr(cfg)
    w.load(blob)
    d = _dev(aips)
    for est in ("hll", "loglog", "pcsa"):
        a = v.estimate(d, estimator=est).cpu().numpy()
        b = w.estimate(d, estimator=est).cpu().numpy()
        np.testing.assert_array_equal(a.view(np.uint32), b.view(np.uint32))
    np.testing.assert_array_equal(v.pcsa_statistics(), w.pcsa_statistics())
    assert v.pool_sums_alt() == w.pool_sums_alt()


def test_trace_full_size_gsmall():
    """The trace configuration at full size (64M pairs, 1M hosts, Z = 2^24,
    g = 256, k = 30), gsmall: PCSA statistics of all 2^24 BDRs bit-exact and
    20000 sampled hosts' LogLog and PCSA estimates within tolerance."""
    cfg = traffic.TRACE
    gen = traffic.ZipfTraffic(cfg["n_hosts"], cfg["zipf_s"], cfg["c_max"], cfg["k"],
                              seed=307, repeat_frac=cfg["repeat_frac"])
    v, o = _make("gsmall", cfg["k"], cfg["Z"], cfg["log2_g"])
    s = gen.next_slice(cfg["n_pairs"])
    v.scan(_dev(s))
    o.scan(s)
    v.slide()
    o.slide()
    sample = np.random.default_rng(10).choice(gen.aips, 20000, replace=False)
    _check(v, o, sample, "gsmall")
