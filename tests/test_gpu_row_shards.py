"""The destination-row split of one instance, run through librtbte by several processes.

Each rank (gloo, world size 2, both ranks on cuda:0: their kernels never wait on each other)
counts every row's channels (RTBTE_CH_COUNT), takes a contiguous row slice balanced by those
counts, builds a context that stores and streams only its slice's channels (rtbte_desc
row_begin / row_end), evaluates rtbte_rhs, and all-gathers its rows over gloo.  The gathered
RHS equals the unsliced context's rtbte_rhs bit for bit and the FP64 oracle to 1e-5, and the
slices' stored entries add up to the unsliced context's.
"""
import os
import socket

import numpy as np
import pytest

import rtbte_inputs as ri

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MODELS = {"graphene36": lambda: ri.graphene_small(36), "silicon16": lambda: ri.silicon(16)}


@pytest.fixture(scope="module")
def rt():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_13402_gb300 import build

    build.build()
    import paper_2412_13402_gb300 as m

    return m


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, name, prec, q):
    import torch.distributed as dist

    import paper_2412_13402_gb300 as rt
    from paper_2412_13402_gb300 import ranks

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        m = MODELS[name]()
        counter = rt.Context(m, precision=prec)
        counter.upload_channels(count_only=True)
        w = counter.row_entries()
        counter.close()
        a, b = ranks.balanced_slices(w + 1, world)[rank]  # +1: a row's fixed cost
        ctx = rt.Context(m, precision=prec, row_range=(a, b))
        ctx.upload_channels()
        s = ctx.sizes(0)
        y = torch.tensor(np.concatenate(ri.random_populations(m, 12)), device="cuda")
        part = ctx.rhs(y).cpu().numpy()
        outside = np.concatenate([part[:a], part[b:]])
        ctx.close()
        got = [None] * world
        dist.all_gather_object(got, (a, b, part[a:b], s["eph_entries"] + s["phe_entries"] + s["pp_entries"],
                                     not outside.any(), int(w.sum())))
        q.put((rank, got))
    finally:
        dist.destroy_process_group()


def spawn(name, prec, world=2):
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, world, port, name, prec, q)) for r in range(world)]
    for p in ps:
        p.start()
    out = dict(q.get(timeout=300) for _ in range(world))
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    return out


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("name", list(MODELS))
def test_row_slices_gather_to_the_full_rhs(rt, oracle_lib, name, prec):
    out = spawn(name, prec)
    assert len(out) == 2
    m = MODELS[name]()
    full = np.zeros(m.n_y)
    covered = np.zeros(m.n_y, bool)
    entries = 0
    for a, b, rows, ent, zero_outside, counted in out[0]:
        full[a:b] = rows
        assert not covered[a:b].any()
        covered[a:b] = True
        entries += ent
        assert zero_outside
    assert covered.all()
    ctx = rt.Context(m, precision=prec)
    ctx.upload_channels()
    s = ctx.sizes(0)
    y = np.concatenate(ri.random_populations(m, 12))
    one = ctx.rhs(torch.tensor(y, device="cuda")).cpu().numpy()
    ctx.close()
    assert entries == s["eph_entries"] + s["phe_entries"] + s["pp_entries"] == out[0][0][5]
    assert np.array_equal(full, one)
    o = oracle_lib.Oracle(m)
    o.build_lists()
    ref = o.rhs(y)
    assert np.linalg.norm(full - ref) / np.linalg.norm(ref) <= (1e-5 if prec == "fp32" else 1e-12)


def test_sliced_context_refuses_integration_and_bad_slices(rt):
    m = ri.graphene_small(24)
    ctx = rt.Context(m, row_range=(0, m.n_c))
    ctx.upload_channels()
    y = torch.tensor(m.y0(), device="cuda")
    with pytest.raises(rt.RtbteError) as e:
        ctx.advance_to(0.01, y, method="zon43", t0=0.0)
    assert e.value.code == -9
    ctx.close()
    for bad in ((0, m.n_y + 1), (5, 5), (-1, 3)):
        with pytest.raises(rt.RtbteError) as e:
            rt.Context(m, row_range=bad)
        assert e.value.code == -1
