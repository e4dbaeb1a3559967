"""Multi-rank logic of the sharded design, on CPU ranks (gloo, world size 2).

Pairs are independent and every update is an idempotent, commutative lattice
operation (OR of bsLBP1 bits for gfast, zeroing of DRs -- a MIN -- for
gsmall).  So a slice may be split across ranks that each scan their share
into a full replica of the pool; merging the replicas with bitwise OR (gfast)
or element-wise MIN of the DRs (gsmall) before the slide must give exactly
the single-rank state.  A second form owns pools by pidx range: each rank
routes its pairs' (pidx, LBP1) records to the owner (all_to_all) and the
owners' slides are local.  Both are checked against one oracle that scans
everything, slice after slice.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from synth import traffic

SEED = 0x9E3779B97F4A7C15
K, Z, B = 4, 3001, 6


def _slices():
    rng = np.random.default_rng(77)
    aips = traffic.distinct_u32(rng, 60)
    return aips, [traffic.uniform_pairs(rng, int(rng.integers(0, 6000)), aips) for _ in range(8)]


def _replica_worker(rank, world, port, layout, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    aips, slices = _slices()
    o = oracle.Oracle(layout, k=K, Z=Z, b=B, seed=SEED)
    states = []
    for s in slices:
        o.scan(s[rank::world])  # this rank's share of the slice
        st = o.state()
        if layout == "gfast":
            bs = torch.from_numpy(st["bs"].view(np.int32).copy())
            dist.all_reduce(bs, op=dist.ReduceOp.BOR)
            o.set_state(bs=bs.numpy().view(np.uint32))
        else:
            dr = torch.from_numpy(st["dr"].astype(np.int32))
            dist.all_reduce(dr, op=dist.ReduceOp.MIN)
            o.set_state(dr=dr.numpy().astype(np.uint8))
        o.slide()
        states.append((o.state()["dr"].copy(), o.registers().copy(), o.pool_sums()))
    if rank == 0:
        q.put(states)
    dist.destroy_process_group()


def _owner_worker(rank, world, port, q):
    """Pool partitioned by pidx range; records routed to their owner."""
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    aips, slices = _slices()
    o = oracle.Oracle("gfast", k=K, Z=Z, b=B, seed=SEED)
    lo, hi = rank * Z // world, (rank + 1) * Z // world
    regs = []
    for s in slices:
        mine = s[rank::world]
        rec = np.array([o.hash_pair(int(a), int(b))[:2] for a, b in mine], dtype=np.int64).reshape(-1, 2)
        # owner r holds pidx in [r Z / world, (r+1) Z / world)
        bounds = np.array([r * Z // world for r in range(world)])
        owner = np.searchsorted(bounds, rec[:, 0], side="right") - 1
        counts = torch.tensor([int((owner == r).sum()) for r in range(world)])
        recv_counts = torch.empty_like(counts)
        dist.all_to_all_single(recv_counts, counts)
        send = torch.from_numpy(rec[np.argsort(owner, kind="stable")].reshape(-1).copy())
        recv = torch.empty(int(recv_counts.sum()) * 2, dtype=torch.int64)
        dist.all_to_all_single(recv, send, [int(c) * 2 for c in recv_counts], [int(c) * 2 for c in counts])
        st = o.state()
        bs = st["bs"].copy()
        for p, r in recv.view(-1, 2).tolist():
            assert lo <= p < hi
            bs[p] |= np.uint32(1 << (r - 1))
        o.set_state(bs=bs)
        o.slide()
        regs.append(o.registers()[lo:hi].copy())
    gathered = [None] * world
    dist.all_gather_object(gathered, regs)
    if rank == 0:
        q.put([np.concatenate([gathered[r][t] for r in range(world)]) for t in range(len(slices))])
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
        out.append((o.state()["dr"].copy(), o.registers().copy(), o.pool_sums()))
    return out


@pytest.mark.parametrize("layout", ["gfast", "gsmall"])
def test_pair_sharded_replicas_merge_to_single_rank_state(layout):
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    pc = mp.start_processes(_replica_worker, args=(2, _free_port(), layout, q), nprocs=2,
                            start_method="spawn", join=False)
    got = q.get()  # read before joining: a large result blocks the writer
    while not pc.join(timeout=60):
        pass
    want = _single_rank(layout)
    for (dr_g, reg_g, sums_g), (dr_w, reg_w, sums_w) in zip(got, want):
        np.testing.assert_array_equal(dr_g, dr_w)
        np.testing.assert_array_equal(reg_g, reg_w)
        assert sums_g == sums_w


def test_pool_partitioned_owners_match_single_rank_registers():
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    pc = mp.start_processes(_owner_worker, args=(2, _free_port(), q), nprocs=2,
                            start_method="spawn", join=False)
    got = q.get()
    while not pc.join(timeout=60):
        pass
    want = _single_rank("gfast")
    for reg_g, (_, reg_w, _) in zip(got, want):
        np.testing.assert_array_equal(reg_g, reg_w)
