"""GPU parity of the q-blocked e-ph layout (rtbte_desc.eph_q_blocks): the built e-ph lists of
each mode split into contiguous phonon-wavevector blocks, one staging group per (mode, block),
so that the staged populations fit in shared memory on large grids.  Forced here on small
models: the stored lists, merged back by the download, bit-exact (indices) against the
oracle's; RHS against the oracle within the parity tolerances (1e-5 FP32 collision sums,
1e-12 FP64); FP64 RHS and integration equal to the unblocked layout's to rounding."""
import numpy as np
import pytest

import rtbte_inputs as ri

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EPH, PHE, PHPH, FAST, SLOW, ALL = 1, 2, 4, 3, 4, 7

MODELS = {
    "graphene36": (lambda: ri.graphene_small(36), 3),
    "silicon16": (lambda: ri.silicon(16), 3),
}


@pytest.fixture(scope="module")
def rt():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_13402_gb300 import build

    build.build()
    import paper_2412_13402_gb300 as m

    return m


def relL2(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def mode_blocked(m, L):
    """Oracle e-ph lists (segments (d, proc), entries by (mode, src)) regrouped into segments
    (mode, d, proc), sources ascending: the order rtbte_download_channels returns for any
    blocking."""
    off = L["off"]
    seg = np.repeat(np.arange(len(off) - 1), np.diff(off))
    nu = L["ph"] // m.N_q
    d, proc = seg // 2, seg % 2
    key = (nu * m.n_c + d) * 2 + proc
    order = np.argsort(key, kind="stable")
    cnt = np.bincount(key, minlength=2 * m.nmodes * m.n_c)
    o = np.zeros(cnt.size + 1, np.int64)
    np.cumsum(cnt, out=o[1:])
    return dict(off=o, a=L["src"][order], b=L["ph"][order], W=L["W"][order])


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("name", list(MODELS))
def test_q_blocked_lists_match_oracle(rt, oracle_lib, name, prec):
    mk, nqb = MODELS[name]
    m = mk()
    ctx = rt.Context(m, precision=prec, eph_q_blocks=nqb)
    ctx.upload_channels()
    L = oracle_lib.Oracle(m).build_lists()
    assert ctx.sizes(0)["eph_q_blocks"] == nqb  # stored in (mode, block, electron, process) segments
    want = mode_blocked(m, L["eph"])
    got = ctx.download_channels(0, rt.RTBTE_EPH)  # blocks merged back, sources ascending
    assert np.array_equal(got["off"], want["off"])
    assert np.array_equal(got["a"], want["a"]) and np.array_equal(got["b"], want["b"])
    if prec == "fp64":
        assert np.all(np.abs(got["W"] - want["W"]) <= 1e-14 * np.abs(want["W"]))
    else:
        assert np.all(np.abs(got["W"] - want["W"]) <= 2.0 ** -23 * np.abs(want["W"]))
    ctx.close()


@pytest.mark.parametrize("prec,tol", [("fp32", 1e-5), ("fp64", 1e-12)])
@pytest.mark.parametrize("name", list(MODELS))
def test_q_blocked_rhs_matches_oracle_and_the_unblocked_layout(rt, oracle_lib, name, prec, tol):
    mk, nqb = MODELS[name]
    m = mk()
    blocked = rt.Context(m, precision=prec, eph_q_blocks=nqb)
    blocked.upload_channels()
    plain = rt.Context(m, precision=prec)
    plain.upload_channels()
    o = oracle_lib.Oracle(m)
    o.build_lists()
    for seed in (3, 9):
        y = np.concatenate(ri.random_populations(m, seed))
        yt = torch.tensor(y, device="cuda")
        for parts in (ALL, EPH):
            got = blocked.rhs(yt, parts=parts).cpu().numpy()
            assert relL2(got, o.rhs(y, parts)) <= tol
            if prec == "fp64":  # only the order of the e-ph partial sums differs
                assert relL2(got, plain.rhs(yt, parts=parts).cpu().numpy()) <= 1e-13
    blocked.close()
    plain.close()


def test_q_blocked_integration_follows_the_unblocked_one(rt):
    m = ri.graphene_small(36)
    runs = []
    for nqb in (0, 4):
        ctx = rt.Context(m, precision="fp64", eph_q_blocks=nqb)
        ctx.upload_channels()
        y = torch.tensor(m.y0(), device="cuda")
        st = ctx.advance_to(0.03, y, method="zon43", t0=0.0, rtol=1e-6, atol_c=1e-9, atol_ph=1e-12)
        assert st["status"] == 0
        runs.append((y.cpu().numpy(), st["steps"], st["fails"]))
        ctx.close()
    (ya, sa, fa), (yb, sb, fb) = runs
    assert (sa, fa) == (sb, fb)
    assert relL2(yb, ya) < 1e-12


def test_fp64_graphene_180_takes_q_blocks_and_matches_literal_rows(rt, oracle_lib):
    """FP64 on the 180 x 180 graphene-like workload: f (102 KB) and one mode's N (259 KB) exceed
    shared memory, so the build takes two q-blocks per mode automatically; sampled rows of
    every family within the FP64 parity tolerance (1e-12) of the oracle's literal sums."""
    m = ri.graphene()
    ctx = rt.Context(m, precision="fp64")
    ctx.upload_channels()
    assert ctx.sizes(0)["eph_q_blocks"] == 2
    o = oracle_lib.Oracle(m)
    rng = np.random.default_rng(4)
    y = np.concatenate(ri.random_populations(m, 21))
    e_rows = rng.choice(m.n_c, 16, replace=False)
    full = o.pp_full_index()
    p_rows = np.unique(np.concatenate([rng.choice(m.n_ph, 16, replace=False), full[rng.choice(len(full), 16, replace=False)]]))
    em = np.zeros(m.n_c, np.uint8)
    pm = np.zeros(m.n_ph, np.uint8)
    em[e_rows] = 1
    pm[p_rows] = 1
    ref = o.rhs_literal(y, ALL, em, pm)
    got = ctx.rhs(torch.tensor(y, device="cuda")).cpu().numpy()
    assert relL2(got[e_rows], ref[e_rows]) <= 1e-12
    assert relL2(got[m.n_c + p_rows], ref[m.n_c + p_rows]) <= 1e-12
    ctx.close()
