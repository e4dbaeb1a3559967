"""The bounds-checked build (libvbdr_check.so, -DVBDR_CHECK) on the GPU:
every kernel tests its physical indices, LBP1 and register values and
records a violation instead of making the access.  A run through every
layout, the planned estimate, LogLog / PCSA, batched registers, the learned
correction (gathered and planned), the bucketed scan and the multi-rank
calls must match the oracle and leave no violation recorded.

Runs in a child process, because a process loads one of the two builds."""
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import numpy as np, torch
import oracle
from synth import traffic
from synth.registers import BatchedRegisters
from paper_1810_13132_gb300 import CompactNet, Config, Vbdr, Mlp, live_features
torch.cuda.set_device(0)
SEED = 0x9E3779B97F4A7C15

def close(got, want):
    err = np.abs(got.astype(np.float64) - want) / np.maximum(np.abs(want), 1.0)
    assert err.max() <= 1e-6, err.max()

rng = np.random.default_rng(901)
aips = traffic.distinct_u32(rng, 3000)
Z = (1 << 18) + 12345
for layout in ("gfast", "gsmall", "serial"):
    v = Vbdr(Config(k=6, num_bdr=Z, log2_g=6, log2_g_min=6, group_rule=1, layout=layout, seed=SEED))
    o = oracle.Oracle(layout, k=6, Z=Z, b=6, seed=SEED, b_min=6, group_rule=1)
    d_aips = torch.from_numpy(aips.view(np.int32)).cuda()
    plan = v.plan(d_aips)
    for t in range(4):
        s = traffic.uniform_pairs(rng, 200_001, aips)
        v.scan(torch.from_numpy(s.view(np.int32)).cuda())
        o.scan(s)
        v.slide()
        o.slide()
        np.testing.assert_array_equal(v.registers(), o.state()["reg"])
        want = o.estimate(aips)
        close(v.estimate(d_aips).cpu().numpy(), want)
        close(v.estimate_planned(plan).cpu().numpy(), want)
        close(v.estimate(d_aips, estimator="loglog").cpu().numpy(), o.estimate_alt(aips, "loglog"))
        if layout == "gsmall":
            close(v.estimate(d_aips, estimator="pcsa").cpu().numpy(), o.estimate_alt(aips, "pcsa"))
    m = Mlp(seed=3)
    v.estimate_learned(m, d_aips)
    flags, checked = v.check_flags()
    assert checked and flags == 0, (layout, flags)

br = BatchedRegisters(20_000, 6, 1e6, seed=902)
v = Vbdr(Config(k=60, num_bdr=1 << 20, log2_g=6, log2_g_min=6, group_rule=1, seed=SEED))
v.load_virtual_registers(torch.from_numpy(br.aips.view(np.int32)).cuda(),
                         torch.from_numpy(br.offsets.view(np.int64)).cuda(),
                         torch.from_numpy(br.vregs).cuda())
o = oracle.Oracle("gfast", k=60, Z=1 << 20, b=6, seed=SEED, b_min=6, group_rule=1)
o.load_virtual_registers(br.aips, br.offsets, br.vregs)
close(v.estimate(torch.from_numpy(br.aips.view(np.int32)).cuda()).cpu().numpy(), o.estimate(br.aips))
flags, checked = v.check_flags()
assert checked and flags == 0, flags

# the opt-in bucketed scan, the learned plan and the multi-rank calls
gen = traffic.ZipfTraffic(5000, 1.05, 60_000, 5, seed=903, repeat_frac=0.1)
d_aips = torch.from_numpy(gen.aips.view(np.int32)).cuda()
for layout in ("gfast", "gsmall"):
    v = Vbdr(Config(k=5, num_bdr=(1 << 18) + 77, log2_g=8, layout=layout, seed=SEED))
    v.set_scan_mode("bucketed")
    o = oracle.Oracle(layout, k=5, Z=(1 << 18) + 77, b=8, seed=SEED)
    w = Vbdr(Config(k=5, num_bdr=(1 << 18) + 77, log2_g=8, layout=layout, seed=SEED))
    for t in range(3):
        s = gen.next_slice(600_001)
        d_s = torch.from_numpy(s.view(np.int32)).cuda()
        v.scan(d_s)
        o.scan(s)
        recs, fill = w.route_records(d_s, 2)
        f = fill.cpu()
        w.apply_records(torch.cat([recs[r, :int(f[r])] for r in range(2)]))
        v.slide(); o.slide(); w.slide()
        np.testing.assert_array_equal(v.registers(), o.state()["reg"])
        np.testing.assert_array_equal(w.registers(), o.state()["reg"])
    lplan = v.plan(d_aips, learned=True)
    m = Mlp(seed=4)
    np.testing.assert_array_equal(v.estimate_learned_planned(m, lplan).cpu().numpy(),
                                  v.estimate_learned(m, d_aips).cpu().numpy())
    # the compact correction's counting variant of the planned kernel; with
    # nmax 0 every host keeps its plain estimate, bit for bit
    keep_plain = CompactNet(np.zeros(CompactNet.N_PARAMS), 0.0)
    np.testing.assert_array_equal(v.estimate_planned_compact(lplan, keep_plain).cpu().numpy(),
                                  v.estimate_planned(lplan).cpu().numpy())
    w.merge_slice_state(v.slice_state())
    w.set_registers(v.registers_device(), v.pcsa_device() if layout == "gsmall" else None)
    close(w.estimate(d_aips).cpu().numpy(), o.estimate(gen.aips))
    for h in (v, w):
        flags, checked = h.check_flags()
        assert checked and flags == 0, (layout, flags)
print("checked build: no violation")
'''


def test_checked_build_runs_clean():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    env = dict(os.environ, VBDR_CHECKED="1", PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, "-c", CHILD], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert "no violation" in r.stdout
