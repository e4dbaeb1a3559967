"""The library's multi-rank calls driven by two gloo ranks (world size 2).

Both ranks run on cuda:0 with a handle each; they exchange device buffers
through the host (gloo), so no kernel waits on another rank.  Two designs,
each checked after every slide against one CPU oracle that scans the whole
slice:

* pair-sharded replicas: every rank scans its half of each slice into a full
  replica; the ranks all-gather their slice states and merge them with
  vbdr_merge_slice_state before the slide -> DRV, registers and pool sums
  bit for bit, estimates within 1e-6;
* pool-partitioned: every rank routes its half of the pairs into records by
  owner with vbdr_route_records, the ranks exchange them (all-to-all), apply
  what they received with vbdr_apply_records, slide, and install the
  byte-wise maximum of their register arrays with vbdr_set_registers ->
  registers and pool sums bit for bit, estimates within 1e-6.

Not measured on several GPUs: every call here gets one GPU.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import oracle  # noqa: E402
from synth import traffic  # noqa: E402

pytestmark = pytest.mark.gpu

SEED = 0x9E3779B97F4A7C15
K, Z, B = 4, (1 << 17) + 3001, 6


def _slices():
    rng = np.random.default_rng(78)
    aips = traffic.distinct_u32(rng, 300)
    sizes = [0, 40_000, 1, 600_001, 25_000, 300_000, 7, 90_000]
    return aips, [traffic.uniform_pairs(rng, n, aips) for n in sizes]


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).cuda()


def _max_all(t):
    """Byte-wise maximum over the ranks of a uint8 CUDA tensor."""
    x = t.to(torch.int32).cpu()
    dist.all_reduce(x, op=dist.ReduceOp.MAX)
    return x.to(torch.uint8).cuda()


def _replica_worker(rank, world, port, layout, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    torch.cuda.set_device(0)
    from paper_1810_13132_gb300 import Config, Vbdr
    aips, slices = _slices()
    v = Vbdr(Config(k=K, num_bdr=Z, log2_g=B, layout=layout, seed=SEED))
    out = []
    for s in slices:
        mine = np.ascontiguousarray(s[rank::world])
        if len(mine):
            v.scan(_dev(mine))
        st = v.slice_state().cpu()
        parts = [torch.empty_like(st) for _ in range(world)]
        dist.all_gather(parts, st)
        for r in range(world):
            if r != rank:
                v.merge_slice_state(parts[r].cuda())
        v.slide()
        est = v.estimate(_dev(aips)).cpu().numpy()
        out.append((v.state()["dr"], v.registers(), v.pool_sums(), est))
    q.put((rank, out))
    dist.destroy_process_group()


def _owner_worker(rank, world, port, layout, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    torch.cuda.set_device(0)
    from paper_1810_13132_gb300 import Config, Vbdr
    aips, slices = _slices()
    v = Vbdr(Config(k=K, num_bdr=Z, log2_g=B, layout=layout, seed=SEED))
    zr = (Z + world - 1) // world
    out = []
    for s in slices:
        mine = np.ascontiguousarray(s[rank::world])
        recs, fill = v.route_records(_dev(mine) if len(mine) else _dev(np.zeros((0, 2), np.uint32)),
                                     world, cap=max(len(mine), 1))
        counts = fill.cpu()
        assert int(counts.sum()) == len(mine) and (counts <= max(len(mine), 1)).all()
        send = torch.cat([recs[r, :int(counts[r])].cpu() for r in range(world)])
        for r in range(world):  # every record lies in its owner's range
            p = recs[r, :int(counts[r])].cpu().numpy().view(np.uint32) >> 5
            assert ((p >= r * zr) & (p < (r + 1) * zr)).all()
        recv_counts = torch.empty_like(counts)
        dist.all_to_all_single(recv_counts, counts)
        recv = torch.empty(int(recv_counts.sum()), dtype=torch.int32)
        dist.all_to_all_single(recv, send, [int(c) for c in recv_counts], [int(c) for c in counts])
        v.apply_records(recv.cuda())
        v.slide()
        reg = _max_all(v.registers_device())
        pcsa = _max_all(v.pcsa_device()) if layout == "gsmall" else None
        v.set_registers(reg, pcsa)
        est = v.estimate(_dev(aips)).cpu().numpy()
        out.append((None, v.registers(), v.pool_sums(), est))
    q.put((rank, out))
    dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _single_rank(layout):
    aips, slices = _slices()
    o = oracle.Oracle(layout, k=K, Z=Z, b=B, seed=SEED)
    out = []
    for s in slices:
        o.scan(s)
        o.slide()
        out.append((o.state()["dr"], o.registers(), o.pool_sums(), o.estimate(aips)))
    return out


def _run(worker, layout):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    pc = mp.start_processes(worker, args=(2, _free_port(), layout, q), nprocs=2,
                            start_method="spawn", join=False)
    got = dict(q.get() for _ in range(2))  # read before joining
    while not pc.join(timeout=120):
        pass
    return got


def _check(got, want, drv):
    for rank in (0, 1):
        for t, ((dr_g, reg_g, sums_g, est_g), (dr_w, reg_w, sums_w, est_w)) in enumerate(
                zip(got[rank], want)):
            if drv:
                np.testing.assert_array_equal(dr_g, dr_w, err_msg=f"rank {rank} slice {t}")
            np.testing.assert_array_equal(reg_g, reg_w, err_msg=f"rank {rank} slice {t}")
            assert sums_g == sums_w, (rank, t)
            err = np.abs(est_g.astype(np.float64) - est_w) / np.maximum(np.abs(est_w), 1.0)
            assert err.max() <= 1e-6, (rank, t, float(err.max()))


@pytest.mark.parametrize("layout", ["gfast", "gsmall", "serial"])
def test_pair_sharded_replicas_through_the_library(layout):
    _check(_run(_replica_worker, layout), _single_rank(layout), drv=True)


@pytest.mark.parametrize("layout", ["gfast", "gsmall", "serial"])
def test_pool_partitioned_through_the_library(layout):
    _check(_run(_owner_worker, layout), _single_rank(layout), drv=False)
