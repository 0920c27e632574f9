"""GPU parity of the MRI with a tolerance-chosen slow step (RTBTE_MRI_ADAPT: step doubling on
the MIS Knoth-Wolke step) against the FP64 oracle's or_mri_adapt_solve, through the C ABI:
the same accepted / rejected slow steps and fast-step counts in FP64 mode, populations within
the parity tolerances of the fixed-step MRI (1e-11 FP64, 1e-6 FP32 collision sums), the
give-up path handing back the initial state, resuming the slow step proposal, and instances
in one context deciding together."""
import numpy as np
import pytest

import rtbte_inputs as ri

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KW = dict(atol_c=1e-9, atol_ph=1e-12)


@pytest.fixture(scope="module")
def rt():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_13402_gb300 import build

    build.build()
    import paper_2412_13402_gb300 as m

    return m


@pytest.fixture(scope="module")
def g36(oracle_lib):
    m = ri.graphene_small(36)
    o = oracle_lib.Oracle(m)
    o.build_lists()
    return m, o


def relL2(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


@pytest.mark.parametrize("prec,rtol,hs0,T,tol", [("fp64", 1e-8, 0.05, 0.1, 1e-11), ("fp32", 1e-6, 0.1, 0.2, 1e-6)])
def test_adaptive_slow_step_matches_oracle(rt, g36, prec, rtol, hs0, T, tol):
    m, o = g36
    ctx = rt.Context(m, precision=prec)
    ctx.upload_channels()
    y = torch.tensor(m.y0(), device="cuda")
    st = ctx.advance_to(T, y, method="mri_adapt", t0=0.0, h_s=hs0, rtol=rtol, **KW)
    yo, sto = o.mri_adapt(m.y0(), 0.0, T, hs0, rtol=rtol, **KW)
    assert st["status"] == 0 and sto["status"] == 0 and st["t"] == T
    assert sto["slow_fails"] >= 1 and sto["slow_steps"] >= 3  # the case exercises both branches
    assert relL2(y.cpu().numpy(), yo) < tol
    if prec == "fp64":
        assert st["slow_steps"] == sto["slow_steps"] and st["slow_fails"] == sto["slow_fails"]
        assert st["rhs_slow"] == sto["rhs_slow"]
        assert st["steps"] == sto["steps"] and st["rhs_fast"] == sto["rhs_evals"]
        # the estimate is a difference of states that agree to ~7 rtol = 7e-8 while the two sides'
        # states agree to ~1e-12 relative: eps to ~1.5e-5, the step factor eps^(-1/4) to ~4e-6
        assert st["h_slow_next"] == pytest.approx(sto["h_next"], rel=1e-4)
    ctx.close()


def test_give_up_hands_back_the_initial_state(rt, g36):
    """max_fail = 1 and a first slow step far too long: ERR_TEST_FAIL, y and t as they came in
    (the oracle agrees)."""
    m, o = g36
    ctx = rt.Context(m, precision="fp64")
    ctx.upload_channels()
    y0 = m.y0()
    y = torch.tensor(y0, device="cuda")
    st = ctx.advance_to(0.1, y, method="mri_adapt", t0=0.0, h_s=0.1, rtol=1e-9, slow_max_fail=1, **KW)
    yo, sto = o.mri_adapt(y0, 0.0, 0.1, 0.1, rtol=1e-9, slow=dict(max_fail=1), **KW)
    assert sto["status"] == -6 and st["rc"] == -6
    assert st["t"] == 0.0 and st["slow_fails"] == 1 and st["slow_steps"] == 0
    assert np.array_equal(y.cpu().numpy(), y0) and np.array_equal(yo, y0)
    ctx.close()


def test_resume_continues_with_the_slow_step_proposal(rt, g36):
    """Two calls over [0, 0.05] and [0.05, 0.1] with resume = 1 take the second call's first slow
    step from the first call's proposal (h_slow_next), not from h_s."""
    m, _ = g36
    ctx = rt.Context(m, precision="fp64")
    ctx.upload_channels()
    y = torch.tensor(m.y0(), device="cuda")
    a = ctx.advance_to(0.05, y, method="mri_adapt", t0=0.0, h_s=0.01, rtol=1e-7, **KW)
    assert a["status"] == 0 and a["h_slow_next"] > 0
    y_resumed, y_fresh = y.clone(), y.clone()
    b = ctx.advance_to(0.1, y_resumed, method="mri_adapt", t0=0.05, h_s=1e-4, rtol=1e-7, resume=1, **KW)
    c = ctx.advance_to(0.1, y_fresh, method="mri_adapt", t0=0.05, h_s=1e-4, rtol=1e-7, **KW)
    assert b["status"] == 0 and c["status"] == 0
    assert b["slow_steps"] + b["slow_fails"] < c["slow_steps"] + c["slow_fails"]  # no regrowth from 1e-4
    assert relL2(y_resumed.cpu().numpy(), y_fresh.cpu().numpy()) < 1e-6
    ctx.close()


def test_instances_share_the_slow_step(rt):
    """Two identical instances in one context decide every slow attempt on the same norm and
    end equal to a one-instance run."""
    m = ri.graphene_small(24)
    one = rt.Context(m, precision="fp64")
    one.upload_channels()
    two = rt.Context([m, m], precision="fp64")
    two.upload_channels(0)
    two.upload_channels(1)
    opts = dict(method="mri_adapt", t0=0.0, h_s=0.02, rtol=1e-7, **KW)
    y1 = torch.tensor(m.y0(), device="cuda")
    s1 = one.advance_to(0.06, y1, **opts)
    y2 = torch.tensor(np.concatenate([m.y0(), m.y0()]), device="cuda")
    s2 = two.advance_to(0.06, y2, **opts)
    assert s1["status"] == 0 and s2["status"] == 0
    assert s2["slow_steps"] == s1["slow_steps"] and s2["slow_fails"] == s1["slow_fails"]
    n = m.n_c + m.n_ph
    a, b = y2[:n].cpu().numpy(), y2[n:].cpu().numpy()
    assert np.array_equal(a, b)
    assert relL2(a, y1.cpu().numpy()) < 1e-13
    one.close()
    two.close()
