"""Streaming service: tenants admitted under a device-memory budget, one CUDA
graph replay per slice, tenants overlapping on the device.  Each tenant's
results must be the same alone and in the mix (the state update is
order-independent and the estimate deterministic, so: bit for bit), equal to
the direct handle API and to the CPU oracle (estimates within 1e-6 of its
FP64 values after every slice, registers and pool sums bit for bit), and
admission must wait for memory to free up."""
import threading
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from synth import traffic  # noqa: E402

pytestmark = pytest.mark.gpu

SEED = 0x9E3779B97F4A7C15


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def _workload(seed, n_slices=10):
    gen = traffic.ZipfTraffic(3000, 1.1, 5000, 5, seed=seed)
    rng = np.random.default_rng(seed)
    sizes = traffic.log_uniform_sizes(rng, n_slices, 1000, 300_000)
    sizes[3] = 0  # an empty slice
    slices = [torch.from_numpy(gen.next_slice(int(n)).view(np.int32)).pin_memory() for n in sizes]
    return gen.aips, slices


def _cfg(layout="gfast"):
    from paper_1810_13132_gb300 import Config
    return Config(k=5, num_bdr=(1 << 16) + 3, log2_g=7, layout=layout, seed=SEED)


def _run_tenant(srv, cfg, aips, slices, mlp=None, results=None, key=None, events=None,
                states=None):
    t = srv.open(cfg, 300_000, aips, mlp=mlp)
    if events is not None:
        events.append(("open", key, time.monotonic()))
    outs, pending = [], []
    for s in slices:
        pending.append(srv.submit(t, s))
        if len(pending) == 2:
            o = np.empty(aips.size, dtype=np.float32)
            srv.wait(t, pending.pop(0), o)
            outs.append(o)
    for tk in pending:
        o = np.empty(aips.size, dtype=np.float32)
        srv.wait(t, tk, o)
        outs.append(o)
    if events is not None:
        events.append(("close", key, time.monotonic()))
    if states is not None:  # every slice has been waited for: the final state
        view = srv.tenant_view(t, cfg)
        states[key] = (view.registers(), view.pool_sums())
        view.close()
    srv.close_tenant(t)
    if results is not None:
        results[key] = outs
    return outs


@pytest.mark.parametrize("layout", ["gfast", "gsmall"])
def test_alone_equals_mix_equals_direct(layout):
    from paper_1810_13132_gb300 import Server, Vbdr
    works = {i: _workload(100 + i) for i in range(3)}
    srv = Server(budget_bytes=8 << 30)
    alone = {i: _run_tenant(srv, _cfg(layout), *works[i]) for i in works}
    mixed = {}
    th = [threading.Thread(target=_run_tenant, args=(srv, _cfg(layout), *works[i]),
                           kwargs=dict(results=mixed, key=i)) for i in works]
    for x in th:
        x.start()
    for x in th:
        x.join()
    for i in works:
        assert len(mixed[i]) == len(alone[i])
        for a, b in zip(alone[i], mixed[i]):
            np.testing.assert_array_equal(a, b)
    # direct handle API on tenant 0's traffic
    aips, slices = works[0]
    v = Vbdr(_cfg(layout))
    d_aips = torch.from_numpy(aips.view(np.int32)).cuda()
    for s, want in zip(slices, alone[0]):
        v.scan(s.cuda())
        v.slide()
        np.testing.assert_array_equal(v.estimate(d_aips).cpu().numpy(), want)
    srv.close()


def test_admission_waits_for_memory_and_times_out():
    from paper_1810_13132_gb300 import Server, VbdrError
    works = {i: _workload(200 + i, n_slices=6) for i in range(3)}
    probe = Server(budget_bytes=1 << 40)
    need = probe.tenant_bytes(_cfg(), 300_000, works[0][0].size)
    probe.close()
    srv = Server(budget_bytes=2 * need + need // 2)  # room for two tenants
    # a third tenant cannot get in while two hold their memory
    t0 = srv.open(_cfg(), 300_000, works[0][0])
    t1 = srv.open(_cfg(), 300_000, works[1][0])
    with pytest.raises(VbdrError) as e:
        srv.open(_cfg(), 300_000, works[2][0], timeout_ms=200)
    assert e.value.code == -6
    assert srv.in_use()[1] == 2
    srv.close_tenant(t0)
    srv.close_tenant(t1)
    # three concurrent tenants through a two-tenant budget: every result matches
    alone = {i: _run_tenant(srv, _cfg(), *works[i]) for i in works}
    events, mixed = [], {}
    th = [threading.Thread(target=_run_tenant, args=(srv, _cfg(), *works[i]),
                           kwargs=dict(results=mixed, key=i, events=events)) for i in works]
    for x in th:
        x.start()
    for x in th:
        x.join()
    for i in works:
        for a, b in zip(alone[i], mixed[i]):
            np.testing.assert_array_equal(a, b)
    # never more than two tenants admitted at once
    live, peak = 0, 0
    for kind, _, _ in sorted(events, key=lambda e: e[2]):
        live += 1 if kind == "open" else -1
        peak = max(peak, live)
    assert peak <= 2
    srv.close()


def test_learned_tenant_matches_direct_learned_estimate():
    from paper_1810_13132_gb300 import Mlp, Server, Vbdr
    aips, slices = _workload(300)
    mlp = Mlp(seed=5)
    srv = Server(budget_bytes=4 << 30)
    outs = _run_tenant(srv, _cfg(), aips, slices, mlp=mlp)
    v = Vbdr(_cfg())
    d_aips = torch.from_numpy(aips.view(np.int32)).cuda()
    for s, want in zip(slices, outs):
        v.scan(s.cuda())
        v.slide()
        np.testing.assert_array_equal(v.estimate_learned(mlp, d_aips).cpu().numpy(), want)
    srv.close()


def _oracle_run(cfg, aips, slices):
    o = oracle.Oracle(cfg.layout, k=cfg.k, Z=cfg.num_bdr, b=cfg.log2_g, seed=cfg.seed)
    outs = []
    for s in slices:
        o.scan(s.numpy().view(np.uint32).reshape(-1, 2))
        o.slide()
        outs.append(o.estimate(aips))
    return outs, o.registers(), o.pool_sums()


def _assert_close_to_oracle(got, want, tag):
    got = got.astype(np.float64)
    err = np.abs(got - want) / np.maximum(np.abs(want), 1.0)
    assert err.max() <= 1e-6, (tag, float(err.max()), int(err.argmax()))


@pytest.mark.parametrize("layout", ["gfast", "gsmall"])
def test_served_results_match_oracle_alone_and_in_mix(layout):
    """Each tenant's per-slice estimates, served alone and in a mix of three
    concurrent tenants, against the CPU oracle run on the same slices; the
    slice sizes are log-uniform with one empty slice and one at the
    tenant's capacity; the final registers and pool sums bit for bit."""
    from paper_1810_13132_gb300 import Server
    works = {i: _workload(400 + i) for i in range(3)}
    gen = traffic.ZipfTraffic(3000, 1.1, 5000, 5, seed=499)
    works[0][1][6] = torch.from_numpy(gen.next_slice(300_000).view(np.int32)).pin_memory()
    assert works[0][1][3].numel() == 0 and works[0][1][6].numel() == 2 * 300_000
    cfg = _cfg(layout)
    srv = Server(budget_bytes=8 << 30)
    alone, alone_state = {}, {}
    for i in works:
        alone[i] = _run_tenant(srv, cfg, *works[i], states=alone_state, key=i)
    mixed, mixed_state = {}, {}
    th = [threading.Thread(target=_run_tenant, args=(srv, cfg, *works[i]),
                           kwargs=dict(results=mixed, key=i, states=mixed_state)) for i in works]
    for x in th:
        x.start()
    for x in th:
        x.join()
    srv.close()
    for i in works:
        want, reg, sums = _oracle_run(cfg, *works[i])
        assert len(alone[i]) == len(mixed[i]) == len(want)
        for t, (a, m, w) in enumerate(zip(alone[i], mixed[i], want)):
            _assert_close_to_oracle(a, w, (i, t, "alone"))
            _assert_close_to_oracle(m, w, (i, t, "mix"))
        for st in (alone_state[i], mixed_state[i]):
            np.testing.assert_array_equal(st[0], reg)
            assert st[1] == sums
