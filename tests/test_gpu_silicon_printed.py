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


def test_printed_silicon_sampled_lists_match_oracle(si80):
    """Channel lists of sampled destinations of every family, read back segment by segment
    (rtbte_download_segments), bit-exact in their indices against the oracle's brute-force
    enumeration; weights within one FP32 ulp of the oracle's FP64 values."""
    import paper_2412_13402_gb300 as rt

    m, ctx, o = si80
    rng = np.random.default_rng(6)

    def w_close(got, want):
        assert np.all(np.abs(got - want) <= 2.0 ** -23 * np.abs(want))

    dests = np.sort(rng.choice(m.n_c, 6, replace=False)).astype(np.int32)
    Lo = o.eph_lists(dests=dests)
    for i, d in enumerate(dests):
        for nu in range(m.nmodes):
            g0 = (nu * m.n_c + int(d)) * 2
            got = ctx.download_segments(0, rt.RTBTE_EPH, g0, g0 + 2)
            for proc in (0, 1):
                sl = slice(Lo["off"][2 * i + proc], Lo["off"][2 * i + proc + 1])
                sel = (Lo["ph"][sl] // m.N_q) == nu
                gs = slice(got["off"][proc], got["off"][proc + 1])
                assert np.array_equal(got["a"][gs], Lo["src"][sl][sel])
                assert np.array_equal(got["b"][gs], Lo["ph"][sl][sel])
                w_close(got["W"][gs], Lo["W"][sl][sel])
    phon = np.sort(rng.choice(m.n_ph, 6, replace=False))
    Lp = o.phe_lists(phonons=phon)
    for i, p in enumerate(phon):
        got = ctx.download_segments(0, rt.RTBTE_PHE, int(p), int(p) + 1)
        ls = slice(Lp["off"][i], Lp["off"][i + 1])
        assert np.array_equal(got["a"], Lp["dst"][ls]) and np.array_equal(got["b"], Lp["src"][ls])
        w_close(got["W"], Lp["W"][ls])
    pd = np.sort(rng.choice(m.n_pp, 4, replace=False))
    Lq = o.pp_lists(dests=pd)
    for i, a in enumerate(pd):
        got = ctx.download_segments(0, rt.RTBTE_PHPH, 2 * int(a), 2 * int(a) + 2)
        ls = slice(Lq["off"][2 * i], Lq["off"][2 * i + 2])
        assert np.array_equal(got["a"], Lq["b"][ls]) and np.array_equal(got["b"], Lq["c"][ls])
        w_close(got["W"], Lq["W"][ls])


def test_printed_silicon_fp64_reads_populations_from_global_memory(oracle_lib):
    """FP64 at the printed grids: f alone (290 KB) exceeds shared memory, so no q-blocking
    helps and the collision kernel reads every population from global memory (the kernel
    instance no smaller workload takes).  Sampled rows of every family within the FP64 parity
    tolerance (1e-12) of the oracle's literal sums."""
    import paper_2412_13402_gb300 as rt

    m = ri.silicon_printed()
    ctx = rt.Context(m, precision="fp64")
    ctx.upload_channels()
    assert ctx.sizes(0)["eph_q_blocks"] == 1
    o = oracle_lib.Oracle(m)
    rng = np.random.default_rng(12)
    y = np.concatenate(ri.random_populations(m, 13))
    full = o.pp_full_index()
    e_rows = rng.choice(m.n_c, 8, replace=False)
    p_rows = np.unique(np.concatenate([rng.choice(m.n_ph, 8, replace=False), full[rng.choice(len(full), 8, replace=False)]]))
    em = np.zeros(m.n_c, np.uint8)
    pm = np.zeros(m.n_ph, np.uint8)
    em[e_rows] = 1
    pm[p_rows] = 1
    ref = o.rhs_literal(y, emask=em, pmask=pm)
    got = ctx.rhs(torch.tensor(y, device="cuda")).cpu().numpy()
    assert relL2(got[e_rows], ref[e_rows]) <= 1e-12
    assert relL2(got[m.n_c + p_rows], ref[m.n_c + p_rows]) <= 1e-12
    ctx.close()
