"""Planned estimate (vbdr_plan_create / vbdr_estimate_planned) against the
oracle and against the gather estimate.

The plan only reorders the work of Alg. 5 (registers visited chunk by
chunk); the sums are the same integers and the finish the same FP64
function, so planned estimates must equal vbdr_estimate's bit for bit and
the oracle's FP64 values within 1e-6 relative (absolute below magnitude 1).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from synth import traffic  # noqa: E402
from synth.registers import BatchedRegisters  # noqa: E402

pytestmark = pytest.mark.gpu

SEED = 0x9E3779B97F4A7C15
EST_RTOL = 1e-6
CHUNK = 1 << 15  # BDRs per register chunk of a plan


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def _dev(a, dtype=np.int32):
    return torch.from_numpy(np.ascontiguousarray(a).view(dtype)).cuda()


def _make(layout, k, Z, b, b_min=None, group_rule=0, seed=SEED):
    from paper_1810_13132_gb300 import Config, Vbdr
    v = Vbdr(Config(k=k, num_bdr=Z, log2_g=b, layout=layout, seed=seed,
                    log2_g_min=b_min or 0, group_rule=group_rule))
    o = oracle.Oracle(layout, k=k, Z=Z, b=b, seed=seed, b_min=b_min, group_rule=group_rule)
    return v, o


def _close(got, want):
    err = np.abs(got.astype(np.float64) - want) / np.maximum(np.abs(want), 1.0)
    assert err.max() <= EST_RTOL, (err.max(), int(err.argmax()))


def _check_plan(v, plan, aips_np, o=None, sample=None):
    """planned == gather bit for bit; planned vs oracle (on a sample)."""
    aips = _dev(aips_np)
    got = v.estimate_planned(plan).cpu().numpy()
    ref = v.estimate(aips).cpu().numpy()
    np.testing.assert_array_equal(got.view(np.uint32), ref.view(np.uint32))
    if o is not None:
        idx = np.arange(len(aips_np)) if sample is None else sample
        _close(got[idx], o.estimate(aips_np[idx]))
    plan.status()
    return got


def _entries_bounds(plan, gsum, Z):
    info = plan.info()
    nchunks = -(-Z // CHUNK)
    assert info["hosts"] == plan.n_hosts
    assert gsum <= info["entries"]
    # padding: at most 3 per (block of hosts, chunk); at most n blocks
    assert info["entries"] <= gsum + 3 * nchunks * max(1, plan.n_hosts)


@pytest.mark.parametrize("layout", ["gfast", "gsmall"])
def test_small_workload_every_slice(layout):
    """The small configuration (k=10, 1e5 pairs, 1000 hosts, Z=2^16: two
    register chunks, g=128) for 13 slices; one plan serves every slide."""
    cfg = traffic.SMALL
    gen = traffic.ZipfTraffic(cfg["n_hosts"], cfg["zipf_s"], cfg["c_max"], cfg["k"], seed=201)
    v, o = _make(layout, cfg["k"], cfg["Z"], cfg["log2_g"])
    plan = v.plan(_dev(gen.aips))
    _entries_bounds(plan, len(gen.aips) << cfg["log2_g"], cfg["Z"])
    for t in range(13):
        s = gen.next_slice(cfg["n_pairs"])
        v.scan(_dev(s))
        o.scan(s)
        v.slide()
        o.slide()
        _check_plan(v, plan, gen.aips, o)


def test_mixed_g_and_ragged_last_chunk():
    """Four host groups g = 64..512 (b_min = 6) in a pool whose size is not
    a whole number of chunks (Z = 2^18 + 12345: nine chunks, the last one
    partial)."""
    rng = np.random.default_rng(202)
    aips = traffic.distinct_u32(rng, 4000)
    Z = (1 << 18) + 12345
    v, o = _make("gfast", 60, Z, 6, b_min=6, group_rule=1)
    plan = v.plan(_dev(aips))
    gsum = int(np.sum(1 << (6 + (aips >> 30).astype(np.int64))))
    _entries_bounds(plan, gsum, Z)
    for t in range(4):
        s = traffic.uniform_pairs(rng, 200_001, aips)
        v.scan(_dev(s))
        o.scan(s)
        v.slide()
        o.slide()
        _check_plan(v, plan, aips, o)


def test_edge_host_lists():
    """Empty list, one host, duplicated hosts, hosts never seen, a pool
    smaller than one chunk, and the first slide empty."""
    rng = np.random.default_rng(203)
    aips = traffic.distinct_u32(rng, 64)
    Z = 4099
    v, o = _make("gfast", 4, Z, 5)
    empty = v.plan(torch.empty(0, dtype=torch.int32, device="cuda"))
    one = v.plan(_dev(aips[:1]))
    dup = np.concatenate([aips[:7], aips[:7], aips[3:4]])
    dplan = v.plan(_dev(dup))
    unseen = traffic.distinct_u32(np.random.default_rng(9), 33)
    uplan = v.plan(_dev(unseen))
    for t, n in enumerate([0, 1, 3, 5000, 0, 17]):
        s = traffic.uniform_pairs(rng, n, aips)
        v.scan(_dev(s))
        o.scan(s)
        v.slide()
        o.slide()
        assert v.estimate_planned(empty).numel() == 0
        _check_plan(v, one, aips[:1], o)
        got = _check_plan(v, dplan, dup, o)
        np.testing.assert_array_equal(got[:7], got[7:14])
        _check_plan(v, uplan, unseen, o)


def test_plan_reuse_across_handles_and_misuse():
    """A plan is valid for any handle of the same configuration; another Z
    is refused, and so is an estimate before the first slide."""
    from paper_1810_13132_gb300 import VbdrError
    rng = np.random.default_rng(204)
    aips = traffic.distinct_u32(rng, 300)
    v1, o = _make("gfast", 8, 1 << 17, 7)
    v2, _ = _make("gsmall", 8, 1 << 17, 7)
    v3, _ = _make("gfast", 8, (1 << 17) + 1, 7)
    plan = v1.plan(_dev(aips))
    with pytest.raises(VbdrError):
        v1.estimate_planned(plan)  # no slide yet
    s = traffic.uniform_pairs(rng, 100_000, aips)
    for v in (v1, v2, v3):
        v.scan(_dev(s))
        v.slide()
    o.scan(s)
    o.slide()
    _check_plan(v1, plan, aips, o)
    _check_plan(v2, plan, aips, o)  # gsmall registers equal gfast's
    with pytest.raises(VbdrError):
        v3.estimate_planned(plan)


def test_host_output_entry_point():
    rng = np.random.default_rng(205)
    aips = traffic.distinct_u32(rng, 2500)
    v, o = _make("gfast", 6, 1 << 16, 7)
    plan = v.plan(_dev(aips))
    s = traffic.uniform_pairs(rng, 300_000, aips)
    v.scan(_dev(s))
    v.slide()
    o.scan(s)
    o.slide()
    out = torch.empty(len(aips), dtype=torch.float32).pin_memory()
    v.estimate_planned_host(plan, out)
    torch.cuda.synchronize()
    dev = v.estimate_planned(plan).cpu()
    np.testing.assert_array_equal(out.numpy().view(np.uint32), dev.numpy().view(np.uint32))
    _close(out.numpy(), o.estimate(aips))


def test_several_waves_of_blocks():
    """More hosts than one wave of blocks holds (152 SMs x 8000 hosts), g=16:
    blocks of two waves, the last one ragged."""
    rng = np.random.default_rng(206)
    aips = traffic.distinct_u32(rng, 1_300_001)
    v, o = _make("gfast", 3, 1 << 16, 4)
    plan = v.plan(_dev(aips))
    _entries_bounds(plan, len(aips) << 4, 1 << 16)
    for t in range(2):
        s = traffic.uniform_pairs(rng, 1 << 20, aips)
        v.scan(_dev(s))
        o.scan(s)
        v.slide()
        o.slide()
    sample = np.random.default_rng(7).choice(len(aips), 20000, replace=False)
    sample = np.concatenate([sample, [0, len(aips) - 1]])
    _check_plan(v, plan, aips, o, sample)


def test_trace_full_size():
    """The trace configuration at full size (64M pairs per slice, 1M hosts,
    Z = 2^24, g = 256, k = 30): all 1M planned estimates equal the gather
    estimate bit for bit; 20000 sampled hosts against the oracle."""
    cfg = traffic.TRACE
    gen = traffic.ZipfTraffic(cfg["n_hosts"], cfg["zipf_s"], cfg["c_max"], cfg["k"],
                              seed=207, repeat_frac=cfg["repeat_frac"])
    v, o = _make("gfast", cfg["k"], cfg["Z"], cfg["log2_g"])
    plan = v.plan(_dev(gen.aips))
    _entries_bounds(plan, len(gen.aips) << cfg["log2_g"], cfg["Z"])
    s = gen.next_slice(cfg["n_pairs"])
    v.scan(_dev(s))
    o.scan(s)
    v.slide()
    o.slide()
    sample = np.random.default_rng(8).choice(len(gen.aips), 20000, replace=False)
    _check_plan(v, plan, gen.aips, o, sample)


def test_batched_mixed_g_full_size():
    """The batched configuration: 4M hosts of mixed g (64..512) over
    Z = 2^26 registers (2048 chunks) loaded at register level; planned ==
    gather for every host; 20000 sampled against the oracle."""
    from paper_1810_13132_gb300 import Config, Vbdr
    br = BatchedRegisters(4_000_000, 6, 1e7, seed=208)
    Z = 1 << 26
    v = Vbdr(Config(k=60, num_bdr=Z, log2_g=6, log2_g_min=6, group_rule=1, seed=SEED))
    v.load_virtual_registers(_dev(br.aips), _dev(br.offsets, np.int64), _dev(br.vregs, np.uint8))
    plan = v.plan(_dev(br.aips))
    o = oracle.Oracle("gfast", k=60, Z=Z, b=6, seed=SEED, b_min=6, group_rule=1)
    o.load_virtual_registers(br.aips, br.offsets, br.vregs)
    sample = np.random.default_rng(9).choice(len(br.aips), 20000, replace=False)
    _check_plan(v, plan, br.aips, o, sample)


# ------------------------------------------- learned correction through a plan

def _mlp(seed=11):
    """A network with random parameters (the correction's arithmetic, not its
    training, is under test) that corrects every host."""
    from paper_1810_13132_gb300 import Mlp
    m = Mlp(seed=seed)
    params, _ = m.get_params()
    m.set_params(params, 3.0e38)
    return m


def _check_learned(v, aips_np, mlp):
    """planned learned == gather learned, bit for bit (features, plain
    estimates and the network are the same arithmetic)."""
    aips = _dev(aips_np)
    plan = v.plan(aips, learned=True)
    got = v.estimate_learned_planned(mlp, plan).cpu().numpy()
    ref = v.estimate_learned(mlp, aips).cpu().numpy()
    np.testing.assert_array_equal(got.view(np.uint32), ref.view(np.uint32))
    # the learned plan also serves the plain planned estimate
    np.testing.assert_array_equal(v.estimate_planned(plan).cpu().numpy().view(np.uint32),
                                  v.estimate(aips).cpu().numpy().view(np.uint32))
    plan.status()
    plan.close()


def test_learned_planned_equals_gather_trace_shape():
    """Trace-shaped traffic at 1/16 (4M pairs per slice, 62500 hosts, g = 256,
    Z = 2^20), several slices; the host list takes several blocks and a
    ragged last block."""
    gen = traffic.ZipfTraffic(62_500, 1.05, 2_000_000 // 16, 30, seed=230, repeat_frac=0.10)
    v, _ = _make("gfast", 30, 1 << 20, 8)
    for _ in range(4):
        v.scan(_dev(gen.next_slice(1 << 22)))
        v.slide()
    _check_learned(v, gen.aips, _mlp())


def test_learned_planned_overflowing_bins_and_mixed_g():
    """An empty pool: every register is 0, so every host's histogram has a
    single bin of g >= 256 counts -- more than a byte bin holds -- and the
    exact recount must take over; then the same hosts (g = 64..512) after
    traffic."""
    rng = np.random.default_rng(231)
    aips = traffic.distinct_u32(rng, 9000)
    v, _ = _make("gsmall", 6, (1 << 18) + 77, 9, b_min=6, group_rule=1)
    v.slide()  # one empty slice: all registers 0
    _check_learned(v, aips, _mlp(12))
    for _ in range(3):
        v.scan(_dev(traffic.uniform_pairs(rng, 300_000, aips)))
        v.slide()
    _check_learned(v, aips, _mlp(13))


def test_groups_larger_than_the_staging_slots():
    """Few register chunks and many hosts per block (150000 hosts, g = 256,
    Z = 2^16: two chunks, about 126k entries per group): most of every group
    is read from global memory past its staged part, in the plain and in the
    learned planned kernel."""
    rng = np.random.default_rng(233)
    aips = traffic.distinct_u32(rng, 150_000)
    v, o = _make("gfast", 5, 1 << 16, 8)
    for _ in range(2):
        s = traffic.uniform_pairs(rng, 1 << 20, aips)
        v.scan(_dev(s))
        o.scan(s)
        v.slide()
        o.slide()
    sample = np.random.default_rng(10).choice(len(aips), 3000, replace=False)
    _check_plan(v, v.plan(_dev(aips)), aips, o, sample)
    _check_learned(v, aips, _mlp(14))


def test_learned_planned_refuses_a_plain_plan():
    from paper_1810_13132_gb300 import VbdrError
    rng = np.random.default_rng(232)
    aips = traffic.distinct_u32(rng, 600_000)  # more than 3300 hosts per block of a wave
    v, _ = _make("gfast", 3, 1 << 16, 7)
    v.slide()
    plan = v.plan(_dev(aips))  # blocks of up to 7000 hosts: here about 3950
    with pytest.raises(VbdrError) as e:
        v.estimate_learned_planned(_mlp(), plan)
    assert e.value.code == -1
