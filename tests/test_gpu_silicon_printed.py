"""The silicon-like workload at the printed grids (80^3 k-grid, 40^3 q-grid, 36 321 electron
states, 384 000 phonons, ph-ph on the 20^3 sub-lattice; ~2.2e9 stored entries), built on the
device and evaluated in the launch configuration the bench times (FP32 compensated sums,
automatic e-ph q-blocks so that every group is staged in shared memory).  Parity on sampled
rows that the oracle computes one by one from the literal sums (Eq. e-ph, Eq. ph-ph): relative
L2 <= 1e-5 per family of rows (the RHS tolerance), for the initial state and a random one."""
import numpy as np
import pytest

import rtbte_inputs as ri

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def si80(oracle_lib):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_13402_gb300 import build

    build.build()
    import paper_2412_13402_gb300 as rt

    m = ri.silicon_printed()
    ctx = rt.Context(m, precision="fp32")
    ctx.upload_channels()
    yield m, ctx, oracle_lib.Oracle(m)
    ctx.close()


def relL2(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def test_printed_silicon_sizes(si80):
    m, ctx, o = si80
    s = ctx.sizes(0)
    assert (m.n_c, m.n_ph) == (36321, 384000)
    assert s["n_pp"] == 48000 == len(o.pp_full_index())
    assert 1.0e9 < s["eph_entries"] < 1.4e9 and 2.5e8 < s["pp_entries"] < 5e8
    assert s["eph_stored"] % 4 == 0 and s["phe_stored"] % 4 == 0 and s["pp_stored"] % 4 == 0
    # f (145 KB) and one mode's N on the 40^3 grid (256 KB) exceed shared memory: q-blocked
    assert s["eph_q_blocks"] >= 2


@pytest.mark.parametrize("state", ["y0", "random"])
def test_printed_silicon_sampled_rows_match_literal_sums(si80, state):
    m, ctx, o = si80
    y = m.y0() if state == "y0" else np.concatenate(ri.random_populations(m, 11))
    rng = np.random.default_rng(5)
    full = o.pp_full_index()
    e_rows = rng.choice(m.n_c, 12, replace=False)
    p_rows = rng.choice(m.n_ph, 12, replace=False)  # mostly ph-e only (off the ph-ph sub-lattice)
    s_rows = full[rng.choice(len(full), 12, replace=False)]  # ph-e + ph-ph
    em = np.zeros(m.n_c, np.uint8)
    pm = np.zeros(m.n_ph, np.uint8)
    em[e_rows] = 1
    pm[p_rows] = 1
    pm[s_rows] = 1
    ref = o.rhs_literal(y, emask=em, pmask=pm)
    got = ctx.rhs(torch.tensor(y, device="cuda")).cpu().numpy()
    for rows in (e_rows, m.n_c + p_rows, m.n_c + s_rows):
        assert np.linalg.norm(ref[rows]) > 0
        assert relL2(got[rows], ref[rows]) <= 1e-5
