"""The 64-instance ensemble (sides 24-96, E_x 0.1-1 eV, T 100-500 K; 5.7e8 stored entries) in
the launch configuration the bench times: one persistent launch over every instance, with
8-, 16- and 32-lane items chosen per staging group.  Sampled rows of the smallest, the
largest and two middle instances within the RHS tolerance (relative L2 1e-5, FP32 compensated
sums) of the oracle's literal sums; one batched adaptive window ends with every instance at
t_out and a finite state."""
import numpy as np
import pytest

import rtbte_inputs as ri

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ens():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_13402_gb300 import build

    build.build()
    import paper_2412_13402_gb300 as rt

    ms = ri.ensemble()
    ctx = rt.Context(ms, precision="fp32")
    for i in range(len(ms)):
        ctx.upload_channels(i)
    ctx.autotune(rt.RTBTE_ALL)
    yield rt, ms, ctx
    ctx.close()


def relL2(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def test_ensemble_sampled_rows_match_literal_sums(ens, oracle_lib):
    rt, ms, ctx = ens
    ys = [np.concatenate(ri.random_populations(m, 30 + i)) for i, m in enumerate(ms)]
    got = ctx.rhs(torch.tensor(np.concatenate(ys), device="cuda")).cpu().numpy()
    sides = np.array([m.nk[0] for m in ms])
    picks = {int(np.argmin(sides)), int(np.argmax(sides)), 17, 42}
    rng = np.random.default_rng(8)
    for i in sorted(picks):
        m = ms[i]
        off = ctx.sizes(i)["y_offset"]
        o = oracle_lib.Oracle(m)
        full = o.pp_full_index()
        e_rows = rng.choice(m.n_c, min(12, m.n_c), replace=False)
        p_rows = np.unique(np.concatenate([rng.choice(m.n_ph, 12, replace=False),
                                           full[rng.choice(len(full), min(12, len(full)), replace=False)]]))
        em = np.zeros(m.n_c, np.uint8)
        pm = np.zeros(m.n_ph, np.uint8)
        em[e_rows] = 1
        pm[p_rows] = 1
        ref = o.rhs_literal(ys[i], 7, em, pm)
        g = got[off:off + m.n_c + m.n_ph]
        rows = np.concatenate([e_rows, m.n_c + p_rows])
        assert relL2(g[rows], ref[rows]) <= 1e-5, (i, m.nk)


def test_ensemble_window_reaches_t_out(ens):
    rt, ms, ctx = ens
    y = torch.tensor(np.concatenate([m.y0() for m in ms]), device="cuda")
    st = ctx.advance_to(0.005, y, method="zon43", t0=0.0, rtol=1e-5, atol_c=1e-9, atol_ph=1e-12)
    assert st["status"] == 0 and st["t"] == 0.005
    assert all(ctx.get_controller(i).t == 0.005 for i in range(len(ms)))
    assert torch.isfinite(y).all()
