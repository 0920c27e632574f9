"""GPU parity of librtbte against the FP64 CPU oracle, through the C ABI.

Channel lists: indices and offsets bit-exact, weights within one FP32 ulp (FP32 storage)
or 1e-14 relative (FP64 storage; the two sides' exp() may differ in the last bit).
RHS: relative L2 <= 1e-5 in FP32_COMP mode, <= 1e-12 in FP64 mode.
Integrated populations: relative L2 <= 1e-6 (FP32 collision sums) or tighter in FP64.
"""
import numpy as np
import pytest

import rtbte_inputs as ri

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EPH, PHE, PHPH, FAST, SLOW, ALL = 1, 2, 4, 3, 4, 7


@pytest.fixture(scope="module")
def rt():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_13402_gb300 import build

    build.build()
    import paper_2412_13402_gb300 as m

    return m


def relL2(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300))


def sym_state(m, seed):
    f, N = ri.random_populations(m, seed)
    nx, ny, nz = m.nq
    q = np.arange(m.N_q)
    x, y, z = q % nx, (q // nx) % ny, q // (nx * ny)
    qi = ((-z % nz) * ny + (-y % ny)) * nx + (-x % nx)
    inv = (np.arange(m.nmodes)[:, None] * m.N_q + qi[None, :]).ravel()
    N = 0.5 * (N + N[inv])
    return np.concatenate([f, N])


def mode_blocked(m, L):
    """Oracle e-ph lists (segments (d, proc), entries by (mode, src)) regrouped into segments
    (mode, d, proc)."""
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


def assert_w_close(got, want, fp64):
    if fp64:
        assert np.all(np.abs(got - want) <= 1e-14 * np.abs(want))
    else:
        # FP32 storage: within one ulp of the FP64 value (round-to-nearest plus exp's last bit)
        assert np.all(np.abs(got - want) <= 2.0 ** -23 * np.abs(want))


MODELS = {
    "tiny2d": lambda: ri.tiny((4, 4, 1)),
    "tiny3d_fold2": lambda: ri.tiny((4, 4, 4), fold=2, nbands=2, nmodes=2, pp_stride=1),
    "tiny2d_pp2": lambda: ri.tiny((6, 6, 1), pp_stride=2, sigma_pp=0.03),
    "toy2d": lambda: ri.toy2d(),
    "ladder": lambda: ri.ladder(n=6),
    "ladder3d_fold2": lambda: ri.ladder3d(n=8),
    "graphene36": lambda: ri.graphene_small(36),
    "silicon16": lambda: ri.silicon(16),
}


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("name", list(MODELS))
def test_channel_lists_match_oracle(rt, oracle_lib, name, prec):
    m = MODELS[name]()
    ctx = rt.Context(m, precision=prec)
    ctx.upload_channels()
    o = oracle_lib.Oracle(m)
    L = o.build_lists()
    want = mode_blocked(m, L["eph"])
    got = ctx.download_channels(0, rt.RTBTE_EPH)
    assert np.array_equal(got["off"], want["off"])
    assert np.array_equal(got["a"], want["a"]) and np.array_equal(got["b"], want["b"])
    assert_w_close(got["W"], want["W"], prec == "fp64")
    got = ctx.download_channels(0, rt.RTBTE_PHE)
    assert np.array_equal(got["off"], L["phe"]["off"])
    assert np.array_equal(got["a"], L["phe"]["dst"]) and np.array_equal(got["b"], L["phe"]["src"])
    assert_w_close(got["W"], L["phe"]["W"], prec == "fp64")
    if m.pp_stride > 0:
        got = ctx.download_channels(0, rt.RTBTE_PHPH)
        assert np.array_equal(got["off"], L["pp"]["off"])
        assert np.array_equal(got["a"], L["pp"]["b"]) and np.array_equal(got["b"], L["pp"]["c"])
        assert_w_close(got["W"], L["pp"]["W"], prec == "fp64")
    s = ctx.sizes(0)
    assert s["eph_entries"] == L["eph"]["off"][-1] and s["eph_stored"] % 4 == 0
    ctx.close()


@pytest.mark.parametrize("parts", [ALL, EPH, PHE, PHPH, FAST])
@pytest.mark.parametrize("prec,tol", [("fp32", 1e-5), ("fp64", 1e-12)])
@pytest.mark.parametrize("name", ["tiny3d_fold2", "tiny2d_pp2", "toy2d", "graphene36", "silicon16", "ladder3d_fold2"])
def test_rhs_matches_oracle(rt, oracle_lib, name, prec, tol, parts):
    m = MODELS[name]()
    ctx = rt.Context(m, precision=prec)
    ctx.upload_channels()
    o = oracle_lib.Oracle(m)
    o.build_lists()
    # scale of the rates away from equilibrium: the exact-resonance model's start is an
    # equilibrium whose oracle RHS is rounding only, so there the error is measured against it
    scale = np.linalg.norm(o.rhs(np.concatenate(ri.random_populations(m, 9)), parts))
    for y in (m.y0(), sym_state(m, 3), np.concatenate(ri.random_populations(m, 9))):
        ref = o.rhs(y, parts)
        got = ctx.rhs(torch.tensor(y, device="cuda"), parts=parts).cpu().numpy()
        if np.linalg.norm(ref) == 0:
            assert np.abs(got).max() == 0
        elif np.linalg.norm(ref) < 1e-9 * scale:
            assert np.linalg.norm(got - ref) <= tol * scale, (name, prec, parts)
        else:
            assert relL2(got, ref) <= tol, (name, prec, parts)
        # rows of parts not requested are exactly zero
        if not parts & EPH:
            assert not got[: m.n_c].any()
    ctx.close()


def test_prebuilt_upload_equals_device_build(rt, oracle_lib):
    m = ri.graphene_small(36)
    o = oracle_lib.Oracle(m)
    L = o.build_lists()
    a = rt.Context(m)
    a.upload_channels()
    b = rt.Context(m)
    b.upload_channels(prebuilt=L)
    y = torch.tensor(sym_state(m, 2), device="cuda")
    ra, rb = a.rhs(y).cpu().numpy(), b.rhs(y).cpu().numpy()
    assert relL2(rb, ra) < 1e-6
    assert relL2(rb, o.rhs(y.cpu().numpy())) < 1e-5
    a.close()
    b.close()


def test_rhs_host_pointers_and_determinism(rt):
    m = ri.graphene_small(36)
    ctx = rt.Context(m)
    ctx.upload_channels()
    y = sym_state(m, 5)
    dev = ctx.rhs(torch.tensor(y, device="cuda")).cpu().numpy()
    dev2 = ctx.rhs(torch.tensor(y, device="cuda")).cpu().numpy()
    host = ctx.rhs(torch.tensor(y)).numpy()
    assert np.array_equal(dev, dev2)
    assert np.array_equal(dev, host)
    ctx.close()


def test_autotune_keeps_results_bitwise(rt):
    m = ri.graphene_small(36)
    ctx = rt.Context(m)
    ctx.upload_channels()
    y = torch.tensor(sym_state(m, 8), device="cuda")
    before = ctx.rhs(y).cpu().numpy()
    w = ctx.autotune(ALL)
    assert w > 0
    after = ctx.rhs(y).cpu().numpy()
    assert np.array_equal(before, after)
    st = ctx.advance_to(0.01, y, method="zon43", t0=0.0)
    assert st["status"] == 0
    ctx.close()


def test_per_mask_tuning_is_kept_per_mask(rt):
    """Tuning the fast and slow masks of MRI leaves the full-RHS launch parameters as they were,
    and no tuning changes any result bit."""
    m = ri.graphene_small(36)
    ctx = rt.Context(m)
    ctx.upload_channels()
    y = torch.tensor(sym_state(m, 9), device="cuda")
    before = {p: ctx.rhs(y, parts=p).cpu().numpy() for p in (ALL, FAST, SLOW)}
    ctx.autotune(ALL)
    t_all = ctx.tuning()
    ctx.autotune(FAST)
    ctx.autotune(SLOW)
    assert ctx.tuning() == t_all
    for p, b in before.items():
        assert np.array_equal(ctx.rhs(y, parts=p).cpu().numpy(), b)
    ctx.close()


@pytest.mark.parametrize("which", ["wide", "sub-warp"])
def test_fp32_launch_forms_agree_bitwise(rt, which):
    """The two FP32 launch forms (two entry buffers per warp at 16 warps per SM; one buffer at
    24) compute every item partial with the same arithmetic.  By default a launch with e-ph work
    takes the 24-warp form and a ph-e-only launch the 16-warp form, so the phonon rows of
    parts = e-ph + ph-e (only ph-e items reach them) equal those of parts = ph-e bit for bit."""
    ms = [ri.graphene_small(36)] if which == "wide" else [ri.graphene_small(24), ri.graphene(n=30, window=0.6, seed=77)]
    ctx = rt.Context(ms)
    for i in range(len(ms)):
        ctx.upload_channels(i)
    y = torch.tensor(np.concatenate([sym_state(m, 21 + i) for i, m in enumerate(ms)]), device="cuda")
    both = ctx.rhs(y, parts=EPH | PHE).cpu().numpy()
    phe = ctx.rhs(y, parts=PHE).cpu().numpy()
    off = 0
    for m in ms:
        ph = slice(off + m.n_c, off + m.n_c + m.n_ph)
        assert np.array_equal(both[ph], phe[ph])
        assert np.any(phe[ph] != 0.0)
        off += m.n_c + m.n_ph
    ctx.close()


def test_batched_instances_equal_single_contexts(rt):
    ms = [ri.graphene_small(24), ri.graphene_small(36, seed=5), ri.graphene(n=30, window=0.6, seed=77)]
    ctx = rt.Context(ms)
    for i in range(len(ms)):
        ctx.upload_channels(i)
    ys = [sym_state(m, 10 + i) for i, m in enumerate(ms)]
    got = ctx.rhs(torch.tensor(np.concatenate(ys), device="cuda")).cpu().numpy()
    off = 0
    for i, m in enumerate(ms):
        c1 = rt.Context(m)
        c1.upload_channels()
        one = c1.rhs(torch.tensor(ys[i], device="cuda")).cpu().numpy()
        assert np.array_equal(got[off:off + m.n_y], one)
        assert ctx.sizes(i)["y_offset"] == off
        off += m.n_y
        c1.close()
    ctx.close()


@pytest.mark.parametrize("method", ["zon43", "mri"])
def test_batched_integration_has_independent_controllers(rt, method):
    """Instances of one context integrate with their own step-size controllers: the batched
    result equals each instance integrated alone, bit for bit, although the instances take
    different step sequences."""
    ms = [ri.graphene_small(24), ri.graphene_small(36, seed=5), ri.graphene(n=30, window=0.6, seed=77)]
    kw = dict(method=method, t0=0.0, rtol=1e-5, atol_c=1e-9, atol_ph=1e-12)
    if method == "mri":
        kw["h_s"] = 0.01
    ctx = rt.Context(ms)
    for i in range(len(ms)):
        ctx.upload_channels(i)
    y = torch.tensor(np.concatenate([m.y0() for m in ms]), device="cuda")
    st = ctx.advance_to(0.03, y, **kw)
    assert st["status"] == 0 and st["t"] == 0.03
    got = y.cpu().numpy()
    off, steps = 0, []
    for m in ms:
        c1 = rt.Context(m)
        c1.upload_channels()
        y1 = torch.tensor(m.y0(), device="cuda")
        s1 = c1.advance_to(0.03, y1, **kw)
        assert np.array_equal(got[off:off + m.n_y], y1.cpu().numpy())
        steps.append(s1["steps"])
        off += m.n_y
        c1.close()
    assert st["steps"] == sum(steps) and len(set(steps)) > 1
    ctx.close()


def test_batched_windows_equal_single_contexts(rt):
    """Three consecutive windows of a batched integration (controllers resumed, instances
    finishing each window at different attempts, so the device re-split of the active groups is
    recomputed, reused and recomputed again) equal the same windows of each instance alone."""
    ms = [ri.graphene_small(24), ri.graphene_small(36, seed=5), ri.graphene(n=30, window=0.6, seed=77)]
    kw = dict(method="zon43", rtol=1e-5, atol_c=1e-9, atol_ph=1e-12)
    ctx = rt.Context(ms)
    for i in range(len(ms)):
        ctx.upload_channels(i)
    y = torch.tensor(np.concatenate([m.y0() for m in ms]), device="cuda")
    singles = []
    for m in ms:
        c1 = rt.Context(m)
        c1.upload_channels()
        singles.append((c1, torch.tensor(m.y0(), device="cuda")))
    for w, (t0, t1) in enumerate(((0.0, 0.01), (0.01, 0.02), (0.02, 0.03))):
        st = ctx.advance_to(t1, y, t0=t0, resume=1 if w else 0, **kw)
        assert st["status"] == 0
        for c1, y1 in singles:
            assert c1.advance_to(t1, y1, t0=t0, resume=1 if w else 0, **kw)["status"] == 0
        got = y.cpu().numpy()
        off = 0
        for m, (c1, y1) in zip(ms, singles):
            assert np.array_equal(got[off:off + m.n_y], y1.cpu().numpy()), (w, m.name)
            off += m.n_y
    for c1, _ in singles:
        c1.close()
    ctx.close()


def test_full_graphene_workload_sampled(rt, oracle_lib):
    """The 180 x 180 graphene-like workload in the launch configuration the benchmark uses:
    sampled channel segments bit-exact and sampled RHS rows within 1e-5 of the literal sums."""
    m = ri.graphene()
    ctx = rt.Context(m, precision="fp32")
    ctx.upload_channels()
    o = oracle_lib.Oracle(m)
    rng = np.random.default_rng(0)
    s = ctx.sizes(0)
    assert 0.8e8 < s["eph_entries"] < 2e8 and s["pp_entries"] > 1e7
    # e-ph segments of sampled destinations (mode-blocked on the device)
    dests = np.sort(rng.choice(m.n_c, 24, replace=False)).astype(np.int32)
    got = ctx.download_channels(0, rt.RTBTE_EPH)
    Lo = o.eph_lists(dests=dests)
    for i, d in enumerate(dests):
        for proc in (0, 1):
            sl = slice(Lo["off"][2 * i + proc], Lo["off"][2 * i + proc + 1])
            src, ph, W = Lo["src"][sl], Lo["ph"][sl], Lo["W"][sl]
            for nu in range(m.nmodes):
                sel = (ph // m.N_q) == nu
                g = (nu * m.n_c + d) * 2 + proc
                gs = slice(got["off"][g], got["off"][g + 1])
                assert np.array_equal(got["a"][gs], src[sel]) and np.array_equal(got["b"][gs], ph[sel])
                assert_w_close(got["W"][gs], W[sel], False)
    del got
    phon = np.sort(rng.choice(m.n_ph, 48, replace=False))
    got = ctx.download_channels(0, rt.RTBTE_PHE)
    Lo = o.phe_lists(phonons=phon)
    for i, p in enumerate(phon):
        gs = slice(got["off"][p], got["off"][p + 1])
        ls = slice(Lo["off"][i], Lo["off"][i + 1])
        assert np.array_equal(got["a"][gs], Lo["dst"][ls]) and np.array_equal(got["b"][gs], Lo["src"][ls])
        assert_w_close(got["W"][gs], Lo["W"][ls], False)
    del got
    pd = np.sort(rng.choice(m.n_pp, 16, replace=False))
    got = ctx.download_channels(0, rt.RTBTE_PHPH)
    Lo = o.pp_lists(dests=pd)
    for i, a in enumerate(pd):
        gs = slice(got["off"][2 * a], got["off"][2 * a + 2])
        ls = slice(Lo["off"][2 * i], Lo["off"][2 * i + 2])
        assert np.array_equal(got["a"][gs], Lo["b"][ls]) and np.array_equal(got["b"][gs], Lo["c"][ls])
        assert_w_close(got["W"][gs], Lo["W"][ls], False)
    del got
    # sampled RHS rows vs the literal definition
    y = m.y0()
    gpu = ctx.rhs(torch.tensor(y, device="cuda")).cpu().numpy()
    emask = np.zeros(m.n_c, np.uint8)
    emask[dests] = 1
    full = o.pp_full_index()
    prow = np.unique(np.concatenate([phon, full[pd]]))
    pmask = np.zeros(m.n_ph, np.uint8)
    pmask[prow] = 1
    ref = o.rhs_literal(y, ALL, emask, pmask)
    rows = np.concatenate([dests, m.n_c + prow])
    assert relL2(gpu[rows], ref[rows]) <= 1e-5
    assert relL2(gpu[dests], ref[dests]) <= 1e-5
    ctx.close()


# ---------------------------------------------------------------------------
# integrators
# ---------------------------------------------------------------------------
def test_rk4_and_bs32_toy_fp64(rt, oracle_lib):
    m = ri.toy2d()
    o = oracle_lib.Oracle(m)
    o.build_lists()
    ctx = rt.Context(m, precision="fp64")
    ctx.upload_channels()
    y = torch.tensor(m.y0(), device="cuda")
    st = ctx.advance_to(0.1, y, method="rk4", t0=0.0, h=0.001)
    yo, sto = o.rk4(m.y0(), 0.0, 0.1, 0.001)
    assert st["status"] == 0 and st["steps"] == sto["steps"] == 100 and st["rhs_full"] == 400
    assert relL2(y.cpu().numpy(), yo) < 1e-12
    y = torch.tensor(m.y0(), device="cuda")
    st = ctx.advance_to(0.1, y, method="bs32", t0=0.0, rtol=1e-8, atol_c=1e-15, atol_ph=1e-15)
    yo, sto = o.erk(m.y0(), 0.0, 0.1, method=oracle_lib.BS32, rtol=1e-8, atol_c=1e-15, atol_ph=1e-15)
    assert st["status"] == 0 and abs(st["t"] - 0.1) == 0
    assert st["steps"] == sto["steps"] and st["fails"] == sto["fails"]
    assert st["rhs_full"] == sto["rhs_evals"]
    assert relL2(y.cpu().numpy(), yo) < 1e-11
    ctx.close()


@pytest.mark.parametrize("prec,tol", [("fp32", 1e-6), ("fp64", 1e-11)])
def test_zonneveld_and_mri_graphene(rt, oracle_lib, prec, tol):
    m = ri.graphene_small(36)
    o = oracle_lib.Oracle(m)
    o.build_lists()
    ctx = rt.Context(m, precision=prec)
    ctx.upload_channels()
    kw = dict(rtol=1e-5, atol_c=1e-9, atol_ph=1e-12)
    y = torch.tensor(m.y0(), device="cuda")
    st = ctx.advance_to(0.03, y, method="zon43", t0=0.0, **kw)
    yo, sto = o.erk(m.y0(), 0.0, 0.03, method=oracle_lib.ZON43, **kw)
    assert st["status"] == 0
    assert relL2(y.cpu().numpy(), yo) < tol
    if prec == "fp64":
        assert st["steps"] == sto["steps"] and st["rhs_full"] == sto["rhs_evals"]
    y = torch.tensor(m.y0(), device="cuda")
    st = ctx.advance_to(0.03, y, method="mri", t0=0.0, h_s=0.01, **kw)
    yo, sto = o.mri(m.y0(), 0.0, 0.03, 0.01, **kw)
    assert st["status"] == 0 and st["slow_steps"] == 3 and st["rhs_slow"] == 9 == sto["rhs_slow"]
    assert relL2(y.cpu().numpy(), yo) < tol
    if prec == "fp64":
        assert st["steps"] == sto["steps"] and st["rhs_fast"] == sto["rhs_evals"]
    ctx.close()


def test_rk4_beyond_its_stability_limit_reports_nonfinite(rt):
    """Fixed-step RK4 diverges when h is too long (Results: RK4 diverges for h > 5 fs on graphene);
    on the toy model 5 fs is past the limit and the device controller stops with NONFINITE,
    handing back the last finite state."""
    m = ri.toy2d()
    ctx = rt.Context(m, precision="fp64")
    ctx.upload_channels()
    y = torch.tensor(m.y0(), device="cuda")
    st = ctx.advance_to(0.1, y, method="rk4", t0=0.0, h=0.005)
    assert st["rc"] == -7 and 0 < st["t"] < 0.1
    assert torch.isfinite(y).all()
    ctx.close()


def test_split_rk4_graphene_fp64(rt, oracle_lib):
    m = ri.graphene_small(24)
    o = oracle_lib.Oracle(m)
    o.build_lists()
    ctx = rt.Context(m, precision="fp64")
    ctx.upload_channels()
    y = torch.tensor(m.y0(), device="cuda")
    st = ctx.advance_to(0.02, y, method="split_rk4", t0=0.0, h_s=0.005, h=0.001)
    yo, sto = o.split_rk4(m.y0(), 0.0, 0.02, 0.005, 0.001)
    assert st["status"] == 0 and st["slow_steps"] == 4
    assert relL2(y.cpu().numpy(), yo) < 1e-12
    ctx.close()


# ---------------------------------------------------------------------------
# edge cases and failure statuses (host-side and bounded; nothing faults the GPU)
# ---------------------------------------------------------------------------
def test_no_channels_gives_zero_rhs(rt):
    m = ri.tiny((4, 4, 1), sigma_eph=1e-9, sigma_pp=1e-9)
    ctx = rt.Context(m)
    ctx.upload_channels()
    s = ctx.sizes(0)
    assert s["eph_entries"] == 0 and s["pp_entries"] == 0
    got = ctx.rhs(torch.tensor(m.y0(), device="cuda")).cpu().numpy()
    assert not got.any()
    ctx.close()


def test_status_codes(rt):
    m = ri.graphene_small(24)
    ctx = rt.Context(m)
    y = torch.tensor(m.y0(), device="cuda")
    with pytest.raises(rt.RtbteError) as e:
        ctx.rhs(y)
    assert e.value.code == -9  # no channels yet
    ctx.upload_channels()
    with pytest.raises(rt.RtbteError) as e:
        ctx.rhs(y, parts=0)
    assert e.value.code == -1
    with pytest.raises(rt.RtbteError) as e:
        ctx.advance_to(0.0, y, method="zon43", t0=0.0)
    assert e.value.code == -1
    st = ctx.advance_to(1.0, y, method="zon43", t0=0.0, max_steps=2)
    assert st["rc"] == -4 and st["steps"] == 2 and st["t"] < 1.0
    bad = y.clone()
    bad[3] = float("nan")
    st = ctx.advance_to(0.01, bad, method="zon43", t0=0.0)
    assert st["rc"] == -7
    ctx.close()


@pytest.mark.parametrize("method", ["zon43", "mri"])
def test_device_loop_graph_equals_direct_launches(rt, method):
    """The device-side attempt loop (a CUDA graph with a WHILE node) runs the same kernels as
    direct launches with a host check after every attempt: identical states and counts."""
    m = ri.graphene_small(36)
    kw = dict(rtol=1e-5, atol_c=1e-9, atol_ph=1e-12)
    if method == "mri":
        kw["h_s"] = 0.01
    out = []
    for graphs in (True, False):
        ctx = rt.Context(m)
        ctx.upload_channels()
        ctx.set_graph_mode(graphs)
        y = torch.tensor(m.y0(), device="cuda")
        st = ctx.advance_to(0.03, y, method=method, t0=0.0, **kw)
        assert st["status"] == 0
        out.append((y.cpu().numpy(), st["steps"], st["attempts"]))
        ctx.close()
    assert np.array_equal(out[0][0], out[1][0])
    assert out[0][1:] == out[1][1:]


@pytest.mark.parametrize("prec,tol", [("fp32", 1e-5), ("fp64", 1e-12)])
def test_linearised_phph_rates_match_oracle(rt, oracle_lib, prec, tol):
    """rtbte_phph_rates against the oracle's sums over the same channel lists, at random
    populations and at the Bose-Einstein start; zero outside the ph-ph sub-lattice."""
    m = ri.graphene_small(36)
    o = oracle_lib.Oracle(m)
    o.build_lists()
    ctx = rt.Context(m, precision=prec)
    ctx.upload_channels()
    f, N = ri.random_populations(m, 9)
    for y_np in (np.concatenate([f, N]), m.y0()):
        got = ctx.phph_rates(torch.tensor(y_np, device="cuda")).cpu().numpy()
        ref = o.pp_rates(y_np)
        assert relL2(got, ref) < tol
        assert not got[ref == 0].any()
    ctx.close()


@pytest.mark.parametrize("method", ["zon43", "mri"])
def test_checkpoint_and_resume_continue_bit_for_bit(rt, method):
    """Two calls in one context with resume=1 on the second (the controller's step proposal and
    error history carry over) equal: first call, save (y, controller), destroy the context,
    new context, restore, second call -- bit for bit, with the same step counts."""
    m = ri.graphene_small(36)
    kw = dict(rtol=1e-5, atol_c=1e-9, atol_ph=1e-12)
    if method == "mri":
        kw["h_s"] = 0.01
    ctx = rt.Context(m)
    ctx.upload_channels()
    y = torch.tensor(m.y0(), device="cuda")
    s1 = ctx.advance_to(0.02, y, method=method, t0=0.0, **kw)
    y_mid = y.clone()
    saved = ctx.get_controller()
    s2 = ctx.advance_to(0.04, y, method=method, t0=0.02, resume=1, **kw)
    assert s1["status"] == 0 and s2["status"] == 0
    ctx.close()
    ctx2 = rt.Context(m)
    ctx2.upload_channels()
    ctx2.set_controller(saved)
    y2 = y_mid.clone()
    s3 = ctx2.advance_to(0.04, y2, method=method, t0=0.02, resume=1, **kw)
    ctx2.close()
    assert torch.equal(y, y2)
    assert (s2["steps"], s2["attempts"], s2["fails"]) == (s3["steps"], s3["attempts"], s3["fails"])
    assert saved.h > 0 and saved.first == 0


def test_population_range_violations_are_counted(rt):
    """Accepted step states with an occupation above 1 (beyond atol_c) are reported in
    rtbte_stats.range_violations; a physical start reports none."""
    m = ri.toy2d()
    ctx = rt.Context(m, precision="fp64")
    ctx.upload_channels()
    y = torch.tensor(m.y0(), device="cuda")
    st = ctx.advance_to(0.005, y, method="rk4", t0=0.0, h=0.001)
    assert st["status"] == 0 and st["range_violations"] == 0
    y0 = m.y0()
    y0[:3] = 1.5  # three electron states overfilled; two short steps keep them above 1
    y = torch.tensor(y0, device="cuda")
    st = ctx.advance_to(2e-5, y, method="rk4", t0=0.0, h=1e-5)
    assert st["status"] == 0 and st["steps"] == 2
    assert (y[:3] > 1.0).all() and st["range_violations"] == 6
    ctx.close()


def test_contexts_of_different_staging_sizes_coexist(rt):
    """The collision kernel's dynamic shared-memory limit is a property of the kernel function,
    shared by every context of the process: a context planned later with a smaller staging
    must not lower it below an earlier context's launches."""
    big, small = ri.graphene(n=90), ri.graphene_small(24)
    a = rt.Context(big)
    a.upload_channels()
    ya = torch.tensor(big.y0(), device="cuda")
    ra = a.rhs(ya).cpu().numpy()
    b = rt.Context(small)
    b.upload_channels()
    b.rhs(torch.tensor(small.y0(), device="cuda"))
    assert np.array_equal(a.rhs(ya).cpu().numpy(), ra)
    st = a.advance_to(0.01, ya, method="zon43", t0=0.0)
    assert st["status"] == 0
    a.close()
    b.close()
