"""Multi-rank host logic on CPU ranks (gloo, world size 2): whole-job throughput reduction,
instance sharding, and the gather / norm arithmetic of the row split of one instance's RHS
on the FP64 oracle (rows evaluated on separate ranks and all-gathered equal the full RHS;
the global WRMS norm is one scalar all-reduce).  The same split through librtbte's row-sliced
contexts is tests/test_gpu_row_shards.py."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import rtbte_inputs as ri
from paper_2412_13402_gb300 import ranks


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _run(rank, world, port, fn, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        q.put((rank, fn(rank, world)))
    finally:
        dist.destroy_process_group()


def spawn(fn, world=2):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_run, args=(r, world, port, fn, q)) for r in range(world)]
    for p in ps:
        p.start()
    out = dict(q.get(timeout=180) for _ in range(world))
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    return out


def _throughput(rank, world):
    units = [100.0, 250.0][rank]
    ms = [40.0, 55.0][rank]
    return ranks.job_throughput(units, ms, dist)


def test_job_throughput_sums_units_and_takes_the_slowest_rank():
    out = spawn(_throughput)
    assert out[0] == out[1] == (350.0, 55.0)
    assert ranks.job_throughput(7.0, 3.0) == (7.0, 3.0)


def test_balanced_slices_cover_all_rows_in_order():
    rng = np.random.default_rng(0)
    w = rng.integers(0, 100, 1000)
    for world in (1, 2, 3, 8):
        sl = ranks.balanced_slices(w, world)
        assert sl[0][0] == 0 and sl[-1][1] == len(w)
        assert all(a[1] == b[0] for a, b in zip(sl, sl[1:]))
        loads = [w[a:b].sum() for a, b in sl]
        assert max(loads) - min(loads) <= 2 * w.max()


def test_instance_shards_partition_the_ensemble():
    w = [(24 + 3 * i) ** 2 for i in range(10)]  # ensemble-like instance sizes
    sh = ranks.instance_shards(w, 3)
    flat = sorted(i for s in sh for i in s)
    assert flat == list(range(10))
    loads = [sum(w[i] for i in s) for s in sh]
    assert max(loads) - min(loads) <= max(w)


def _row_shard(rank, world):
    import oracle

    m = ri.graphene_small(24)
    o = oracle.Oracle(m)
    f, N = ri.random_populations(m, 5)
    y = np.concatenate([f, N])
    n_y = m.n_c + m.n_ph
    # rows balanced by a cost proxy (uniform here), each rank evaluates its slice only
    a, b = ranks.balanced_slices(np.ones(n_y), world)[rank]
    emask = np.zeros(m.n_c, np.uint8)
    pmask = np.zeros(m.n_ph, np.uint8)
    for r in range(a, b):
        if r < m.n_c:
            emask[r] = 1
        else:
            pmask[r - m.n_c] = 1
    part = o.rhs_literal(y, emask=emask, pmask=pmask)[a:b]
    gathered = [None] * world
    dist.all_gather_object(gathered, (a, b, part))
    full = np.zeros(n_y)
    for a2, b2, p2 in gathered:
        full[a2:b2] = p2
    # WRMS of a stand-in error vector: local sum of squares, one scalar all-reduce
    e = 1e-7 * full
    w = 1.0 / (1e-5 * np.abs(y) + 1e-12)
    ss = torch.tensor([float(np.sum((e[a:b] * w[a:b]) ** 2))], dtype=torch.float64)
    dist.all_reduce(ss)
    return full, float(np.sqrt(ss.item() / n_y)), o.rhs_literal(y), float(np.sqrt(np.mean((e * w) ** 2)))


def test_row_shards_all_gather_to_the_full_rhs():
    import oracle

    oracle.build()  # once, before the ranks load it
    out = spawn(_row_shard)
    for r in (0, 1):
        full, wrms, ref, wrms_ref = out[r]
        assert np.array_equal(full, ref)
        assert wrms == pytest.approx(wrms_ref, rel=1e-12)
