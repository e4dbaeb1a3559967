"""Batched estimation: hosts of mixed g (64..512) in one persistent launch.

The register-level state (synth.registers) goes through the library's
vbdr_load_virtual_registers and the oracle's own fold; registers must match
bit for bit, estimates within 1e-6 of the oracle's FP64 values, and every
launch shape (lanes per host x threads per block, the autotuner's search
space) must give the identical result.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from synth.registers import BatchedRegisters  # noqa: E402

pytestmark = pytest.mark.gpu

SEED = 0x9E3779B97F4A7C15
EST_RTOL = 1e-6
SHAPES = [(32, 256), (16, 256), (8, 256), (32, 128), (16, 128), (8, 128), (32, 512),
          (16, 512), (8, 512)]


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def _dev(a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a).view(dtype)).cuda()


def _load(br, Z, k=60, b_min=6, layout="gfast"):
    from paper_1810_13132_gb300 import Config, Vbdr
    v = Vbdr(Config(k=k, num_bdr=Z, log2_g=b_min, log2_g_min=b_min, group_rule=1,
                    layout=layout, seed=SEED))
    v.load_virtual_registers(_dev(br.aips, np.int32), _dev(br.offsets, np.int64),
                             _dev(br.vregs, np.uint8))
    o = oracle.Oracle(layout, k=k, Z=Z, b=b_min, seed=SEED, b_min=b_min, group_rule=1)
    o.load_virtual_registers(br.aips, br.offsets, br.vregs)
    return v, o


def _close(got, want):
    err = np.abs(got.astype(np.float64) - want) / np.maximum(np.abs(want), 1.0)
    assert err.max() <= EST_RTOL, (err.max(), int(err.argmax()))


def test_mixed_g_registers_and_estimates_all_shapes():
    br = BatchedRegisters(60_000, 6, 1e7, seed=21)
    Z = (1 << 21) + 7
    v, o = _load(br, Z)
    np.testing.assert_array_equal(v.registers(), o.state()["reg"])
    assert v.pool_sums() == o.pool_sums()
    want = o.estimate(br.aips)
    aips = _dev(br.aips, np.int32)
    outs = []
    for lanes, threads in SHAPES:
        v.set_estimate_launch(lanes, threads)
        outs.append(v.estimate(aips).cpu().numpy())
    for got in outs:
        _close(got, want)
        np.testing.assert_array_equal(got, outs[0])
    lanes, threads = v.autotune_estimate(aips)
    assert (lanes, threads) in SHAPES
    np.testing.assert_array_equal(v.estimate(aips).cpu().numpy(), outs[0])


def test_ragged_batches_and_tiny_host_counts():
    """Host counts that leave partial warps and partial batches."""
    br = BatchedRegisters(1_000, 6, 1e5, seed=22)
    v, o = _load(br, 1 << 16)
    for n in (1, 2, 31, 33, 257, 999):
        a = br.aips[:n]
        want = o.estimate(a)
        for lanes, threads in ((8, 128), (32, 512)):
            v.set_estimate_launch(lanes, threads)
            _close(v.estimate(_dev(a, np.int32)).cpu().numpy(), want)


def test_light_load_accuracy_per_group():
    """Few hosts in a large pool: each g group is estimated within HLL's
    1.04/sqrt(g) envelope (ground truth is the generator's c)."""
    br = BatchedRegisters(2_000, 6, 1e5, seed=23)
    v, _ = _load(br, 1 << 24)
    est = v.estimate(_dev(br.aips, np.int32)).cpu().numpy().astype(np.float64)
    rel = (est - br.card) / br.card
    for b in (6, 7, 8, 9):
        m = (br.b == b) & (br.card >= 500)
        assert m.sum() > 50
        assert np.sqrt(np.mean(rel[m] ** 2)) < 1.5 * 1.04 / np.sqrt(2 ** b)


def test_batched_full_size_sampled():
    """The batched workload at full size: 4M hosts, cardinalities 1..1e7
    log-uniform, g in {64,128,256,512}, Z = 2^26, k = 60, one persistent
    launch; registers bit-exact and 20000 sampled estimates within 1e-6."""
    br = BatchedRegisters(4_000_000, 6, 1e7, seed=24)
    Z = 1 << 26
    v, o = _load(br, Z)
    np.testing.assert_array_equal(v.registers(), o.registers())
    aips = _dev(br.aips, np.int32)
    v.autotune_estimate(aips)
    got = v.estimate(aips).cpu().numpy()
    idx = np.random.default_rng(1).choice(br.aips.size, 20000, replace=False)
    _close(got[idx], o.estimate(br.aips[idx]))
