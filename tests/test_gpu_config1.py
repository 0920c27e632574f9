"""The toy 2D model's protocol (12x12 parabolic band, three phonon modes, e-ph only, FP64) run
to 1 ps on the GPU through the C ABI and compared with the FP64 oracle: fixed-step RK4 where it
is stable (0.1 fs, 10 000 steps) and where it is not (0.5 fs: both sides blow up, the library
stops with NONFINITE and hands back the last finite state), and adaptive Bogacki-Shampine 3(2)
at rtol 1e-8 (step counts within 1% of the oracle's, the end state within 1e-9 of the oracle's
and within the tolerance's reach of a tight Zonneveld reference)."""
import numpy as np
import pytest

import rtbte_inputs as ri

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def toy(oracle_lib):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_13402_gb300 import build

    build.build()
    import paper_2412_13402_gb300 as rt

    m = ri.toy2d()
    ctx = rt.Context(m, precision="fp64")
    ctx.upload_channels()
    o = oracle_lib.Oracle(m)
    o.build_lists()
    yield rt, m, ctx, o
    ctx.close()


def relL2(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def test_toy_rk4_to_1ps_matches_oracle(toy):
    rt, m, ctx, o = toy
    y = torch.tensor(m.y0(), device="cuda")
    st = ctx.advance_to(1.0, y, method="rk4", t0=0.0, h=1e-4)
    yo, sto = o.rk4(m.y0(), 0.0, 1.0, 1e-4)
    assert st["status"] == 0 and st["steps"] == sto["steps"] == 10000 and st["rhs_full"] == 40000
    assert relL2(y.cpu().numpy(), yo) < 1e-12


def test_toy_rk4_beyond_stability_is_nonfinite_on_both_sides(toy):
    rt, m, ctx, o = toy
    y = torch.tensor(m.y0(), device="cuda")
    st = ctx.advance_to(1.0, y, method="rk4", t0=0.0, h=5e-4)
    yo, _ = o.rk4(m.y0(), 0.0, 1.0, 5e-4)
    assert not np.all(np.isfinite(yo))
    assert st["rc"] == -7 and 0.0 < st["t"] < 1.0
    assert torch.isfinite(y).all()


def test_toy_bs3_to_1ps_matches_oracle(toy, oracle_lib):
    rt, m, ctx, o = toy
    kw = dict(rtol=1e-8, atol_c=1e-15, atol_ph=1e-15)
    y = torch.tensor(m.y0(), device="cuda")
    st = ctx.advance_to(1.0, y, method="bs32", t0=0.0, **kw)
    yo, sto = o.erk(m.y0(), 0.0, 1.0, method=oracle_lib.BS32, **kw)
    assert st["status"] == 0 and st["t"] == 1.0
    # over ~2100 adaptive steps a near-tie accept/reject decision can go either way with
    # last-bit differences (the oracle's exp and pow come from the host C library, whose
    # results differ in the last bit between CPU architectures: two steps here), so the step
    # sequence is compared, not required to be identical; the end states agree far below
    # the tolerance
    assert abs(st["steps"] - sto["steps"]) <= 0.01 * sto["steps"] and abs(st["fails"] - sto["fails"]) <= 3
    yg = y.cpu().numpy()
    assert relL2(yg, yo) < 1e-9
    ref, _ = o.erk(m.y0(), 0.0, 1.0, method=oracle_lib.ZON43, rtol=1e-12, atol_c=1e-16, atol_ph=1e-16)
    assert relL2(yg, ref) < 1e-8
