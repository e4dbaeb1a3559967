"""The compact learned correction fused into the planned estimate
(vbdr_estimate_planned_compact) against its FP64 reference.

Reference: the oracle's features of each host (oracle.Oracle.features), the
compact network in FP64 (oracle/learned.py: compact_features,
compact_forward) and learned.correct, with the plain estimate kept where it
is above nmax.  The kernel computes the plain estimate exactly as
vbdr_estimate does (same integer sums, same FP64 finish), then the ten
inputs and the network in FP32 with the fast exponential, logarithm and
division.  Tolerance: the inputs carry FP32 rounding (relative 2^-24 each;
the logarithms within 2^-21 absolute), the 32 dot products of at most 16
terms and the GELU of each unit (one exponential, one division, each within
a few ulp) add a few ulp each, so delta is off by at most about 1e-5 for
weights of order 1, and the estimate exp(ln(1 + n) + delta) - 1 by about
that relatively or 1e-6 absolutely: 2e-4 relative (absolute below magnitude
1) leaves a margin of 20.
"""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from oracle import learned  # noqa: E402
from synth import traffic  # noqa: E402

pytestmark = pytest.mark.gpu

SEED = 0x9E3779B97F4A7C15
RTOL = 2e-4
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
WEIGHTS = os.path.join(ROOT, "paper_1810_13132_gb300", "weights", "correction_compact_trace.npz")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def _dev(a, dtype=np.int32):
    return torch.from_numpy(np.ascontiguousarray(a).view(dtype)).cuda()


def _make(layout, k, Z, b, b_min=None, group_rule=0):
    from paper_1810_13132_gb300 import Config, Vbdr
    v = Vbdr(Config(k=k, num_bdr=Z, log2_g=b, layout=layout, seed=SEED,
                    log2_g_min=b_min or 0, group_rule=group_rule))
    o = oracle.Oracle(layout, k=k, Z=Z, b=b, seed=SEED, b_min=b_min, group_rule=group_rule)
    return v, o


def _nets():
    """The trained network and a random one (the arithmetic, not the
    training, is under test)."""
    from paper_1810_13132_gb300 import CompactNet
    rng = np.random.default_rng(40)
    out = [("random", CompactNet(rng.normal(0, 0.5, learned.C_N_PARAMS), 1e30))]
    if os.path.exists(WEIGHTS):
        out.append(("trained", CompactNet.load(WEIGHTS)))
    return out


def _check(v, o, aips, net, sample=None):
    plan = v.plan(_dev(aips))
    got = v.estimate_planned_compact(plan, net).cpu().numpy().astype(np.float64)
    plain = v.estimate_planned(plan).cpu().numpy()
    plan.status()
    plan.close()
    idx = np.arange(len(aips)) if sample is None else sample
    X, n_plain = o.features(aips[idx])
    theta = net.theta.astype(np.float64)
    d = learned.compact_forward(theta, learned.compact_features(X))
    keep = n_plain > net.nmax
    want = np.where(keep, n_plain, learned.correct(n_plain, d))
    err = np.abs(got[idx] - want) / np.maximum(np.abs(want), 1.0)
    assert err.max() <= RTOL, (err.max(), int(err.argmax()))
    # hosts above nmax keep the plain estimate, bit for bit
    np.testing.assert_array_equal(got[idx][keep].astype(np.float32), plain[idx][keep])
    return got, plain


@pytest.mark.parametrize("layout", ["gfast", "gsmall"])
def test_small_workload(layout):
    """The small configuration (1000 hosts, Z = 2^16, g = 128) after 12
    slices, both networks."""
    cfg = traffic.SMALL
    gen = traffic.ZipfTraffic(cfg["n_hosts"], cfg["zipf_s"], cfg["c_max"], cfg["k"], seed=301)
    v, o = _make(layout, cfg["k"], cfg["Z"], cfg["log2_g"])
    for _ in range(12):
        s = gen.next_slice(cfg["n_pairs"])
        v.scan(_dev(s))
        o.scan(s)
        v.slide()
        o.slide()
    for _, net in _nets():
        _check(v, o, gen.aips, net)


def test_mixed_g_nmax_split_and_ragged_chunk():
    """Hosts of g = 64..512 in a pool of nine chunks, the last one partial;
    nmax inside the range of the estimates, so that both branches run."""
    from paper_1810_13132_gb300 import CompactNet
    rng = np.random.default_rng(302)
    aips = traffic.distinct_u32(rng, 5000)
    v, o = _make("gfast", 20, (1 << 18) + 12345, 6, b_min=6, group_rule=1)
    for _ in range(3):
        s = traffic.uniform_pairs(rng, 400_000, aips)
        v.scan(_dev(s))
        o.scan(s)
        v.slide()
        o.slide()
    net = CompactNet(np.random.default_rng(41).normal(0, 0.5, learned.C_N_PARAMS), 1e30)
    _, plain = _check(v, o, aips, net)
    # nmax in a gap of the estimates near their median, so that no host sits
    # within rounding of it
    u = np.unique(plain.astype(np.float64))
    i = len(u) // 2
    while i + 1 < len(u) and u[i + 1] - u[i] <= 1e-3 * max(u[i], 1.0):
        i += 1
    split = CompactNet(net.theta, float(np.float32(0.5 * (u[i] + u[i + 1]))))
    got, plain = _check(v, o, aips, split)
    above = plain > split.nmax
    assert 0 < above.sum() < len(aips)


def test_empty_pool_and_edge_lists():
    """All registers 0 (the counts n_0 = g), an empty host list, one host."""
    rng = np.random.default_rng(303)
    aips = traffic.distinct_u32(rng, 300)
    v, o = _make("gfast", 5, 40_000, 9)
    v.slide()
    o.slide()
    for _, net in _nets():
        _check(v, o, aips, net)
        _check(v, o, aips[:1], net)
        empty = v.plan(torch.empty(0, dtype=torch.int32, device="cuda"))
        assert v.estimate_planned_compact(empty, net).numel() == 0
        empty.close()


def test_refusals():
    from paper_1810_13132_gb300 import CompactNet, VbdrError
    rng = np.random.default_rng(304)
    aips = traffic.distinct_u32(rng, 50)
    net = CompactNet(np.zeros(learned.C_N_PARAMS), 1e30)
    v, _ = _make("gfast", 3, 1 << 16, 10)  # g = 1024: beyond the packed counts
    v.slide()
    plan = v.plan(_dev(aips))
    with pytest.raises(VbdrError) as e:
        v.estimate_planned_compact(plan, net)
    assert e.value.code == -4
    plan.close()
    w, _ = _make("gfast", 3, 1 << 16, 8)
    plan = w.plan(_dev(aips))
    with pytest.raises(VbdrError) as e:  # before the first slide
        w.estimate_planned_compact(plan, net)
    assert e.value.code == -5
    plan.close()


def test_trace_full_size():
    """The trace configuration at full size (64M pairs per slice, 1M hosts,
    Z = 2^24, g = 256): 20000 sampled hosts against the reference, the
    trained network."""
    if not os.path.exists(WEIGHTS):
        pytest.skip("no trained compact network")
    from paper_1810_13132_gb300 import CompactNet
    cfg = traffic.TRACE
    gen = traffic.ZipfTraffic(cfg["n_hosts"], cfg["zipf_s"], cfg["c_max"], cfg["k"],
                              seed=305, repeat_frac=cfg["repeat_frac"])
    v, o = _make("gfast", cfg["k"], cfg["Z"], cfg["log2_g"])
    s = gen.next_slice(cfg["n_pairs"])
    v.scan(_dev(s))
    o.scan(s)
    v.slide()
    o.slide()
    sample = np.random.default_rng(11).choice(len(gen.aips), 20000, replace=False)
    _check(v, o, gen.aips, CompactNet.load(WEIGHTS), sample)
