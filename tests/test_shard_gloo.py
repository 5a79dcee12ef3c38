"""The multi-rank path on CPU (world size 2, gloo): drop partition, the sharded operator
(target ownership + all-gather of densities, evaluated by the oracle) against the single-process
operator, and the bench's cross-rank timing reduction."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import inputs
from oracle import operators
from paper_1811_10270_gb300 import shard


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _drops():
    rng = np.random.default_rng(4)
    out = []
    for p, c in ((4, (0, 0, 0)), (5, (2.7, 0, 0)), (3, (0, 2.8, 0.2))):
        out.append(inputs.Drop(p, inputs.perturbed_coef(p, rng, 1.0, c, lmax=3), np.zeros((p + 1) ** 2), 2.0,
                               np.asarray(c, float), 1.0))
    return out


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    drops = _drops()
    parts = shard.partition_drops([shard.drop_cost(d.p) for d in drops], world)
    mine = parts[rank]
    rng = np.random.default_rng(10)
    sig_all = [inputs.random_density(d.p, rng)[0] for d in drops]
    # each rank starts with the densities of its own drops only, then all-gathers
    local = {i: sig_all[i] for i in mine}
    gathered = [None] * world
    dist.all_gather_object(gathered, local)
    sig = [None] * len(drops)
    for g in gathered:
        for i, v in g.items():
            sig[i] = v
    sysm = operators.System([operators.DropGeom(d.xcoef, d.p, d.lam) for d in drops])
    vals = {i: sysm.laplace_targets("ladl", sig, i) for i in mine}
    # a GMRES-style dot product over the owned coefficients, all-reduced
    dot = torch.tensor([sum(float(sig[i] @ sig[i]) for i in mine)], dtype=torch.float64)
    dist.all_reduce(dot)
    ms, units = shard.reduce_timing(10.0 + rank, 100.0, dist)
    out = [None] * world
    dist.all_gather_object(out, vals)
    if rank == 0:
        q.put((out, float(dot.item()), ms, units, parts))
    dist.barrier()
    dist.destroy_process_group()


def test_partition_is_balanced_and_complete():
    costs = [shard.drop_cost(p) for p in (16, 24, 32, 48, 16, 32, 48, 24)]
    parts = shard.partition_drops(costs, 3)
    assert sorted(i for p in parts for i in p) == list(range(8))
    loads = [sum(costs[i] for i in p) for p in parts]
    # greedy longest-first bound: no rank exceeds the average by more than one drop's cost
    assert max(loads) <= sum(costs) / 3 + max(costs)
    even = shard.partition_drops([1.0] * 9, 3)
    assert [len(p) for p in even] == [3, 3, 3]


def test_sharded_operator_and_reductions_on_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out, dot, ms, units, parts = q.get(timeout=300)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    drops = _drops()
    rng = np.random.default_rng(10)
    sig = [inputs.random_density(d.p, rng)[0] for d in drops]
    sysm = operators.System([operators.DropGeom(d.xcoef, d.p, d.lam) for d in drops])
    ref = [sysm.laplace_targets("ladl", sig, i) for i in range(len(drops))]
    got = {}
    for part in out:
        got.update(part)
    assert sorted(got) == [0, 1, 2] and all(len(p) > 0 for p in parts)
    for i in range(3):
        np.testing.assert_allclose(got[i], ref[i], rtol=0, atol=1e-13)
    assert abs(dot - sum(float(s @ s) for s in sig)) < 1e-12
    assert ms == 11.0 and units == 200.0
