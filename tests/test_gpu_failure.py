"""Failure detection on the GPU without a fault: a bounded device-side wait
that runs out (an mbarrier nothing arrives on) reports VBDR_ETIMEOUT and
leaves the context usable."""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from synth import traffic  # noqa: E402

pytestmark = pytest.mark.gpu

VBDR_ETIMEOUT = -6


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


@pytest.mark.parametrize("limit_us", [1000, 50000])
def test_expired_wait_is_reported_and_context_survives(limit_us):
    from paper_1810_13132_gb300 import Config, Vbdr, load
    lib = load()
    t0 = time.perf_counter()
    rc = lib.vbdr_selftest_bounded_wait(limit_us, None)
    elapsed = time.perf_counter() - t0
    assert rc == VBDR_ETIMEOUT
    assert elapsed >= limit_us * 1e-6
    # the context still works: a small planned and plain estimate match the oracle
    rng = np.random.default_rng(7)
    aips = traffic.distinct_u32(rng, 100)
    v = Vbdr(Config(k=4, num_bdr=1 << 14, log2_g=6))
    o = oracle.Oracle("gfast", k=4, Z=1 << 14, b=6, seed=0x9E3779B97F4A7C15)
    s = traffic.uniform_pairs(rng, 50_000, aips)
    d = torch.from_numpy(s.view(np.int32)).cuda()
    v.scan(d)
    v.slide()
    o.scan(s)
    o.slide()
    da = torch.from_numpy(aips.view(np.int32)).cuda()
    plan = v.plan(da)
    got = v.estimate_planned(plan).cpu().numpy().astype(np.float64)
    plan.status()
    want = o.estimate(aips)
    assert np.max(np.abs(got - want) / np.maximum(np.abs(want), 1.0)) <= 1e-6
