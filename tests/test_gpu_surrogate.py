"""GPU tests of the neural-operator surrogate of the ph-ph integral (librtbte's BF16
tensor-core training and inference kernels) against the FP64 oracle in
oracle/surrogate_oracle.py, and of its use in the MRI slow stage."""
import numpy as np
import pytest

import rtbte_inputs as ri
from oracle import surrogate_oracle as so

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ORDER = ["W1", "b1", "W2", "b2", "W3", "b3", "W4", "b4", "M1", "c1", "M2", "c2"]


@pytest.fixture(scope="module")
def rt():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_13402_gb300 import build

    build.build()
    import paper_2412_13402_gb300 as m

    return m


@pytest.fixture(scope="module")
def g36(rt):
    m = ri.graphene_small(36)
    ctx = rt.Context(m, precision="fp32")
    ctx.upload_channels()
    yield m, ctx
    ctx.close()


def flat(p):
    return np.concatenate([p[k].reshape(-1) for k in ORDER])


def unflat(v, like):
    out, o = {}, 0
    for k in ORDER:
        n = like[k].size
        out[k] = v[o:o + n].reshape(like[k].shape)
        o += n
    return out


def bf16_round(x):
    """Round FP32 values to the nearest BF16 (ties to even), returned as FP64."""
    b = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


def relL2(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


@pytest.mark.parametrize("width,B", [(64, 3), (24, 16)])
def test_loss_and_gradients_match_fp64_oracle(rt, g36, width, B):
    """Forward, loss and every parameter gradient of the GPU kernels (BF16 operands, FP32
    accumulation) against the FP64 oracle on the same weights and BF16-rounded inputs.  The
    sizes span several 64-row tiles with a ragged tail (3*144 points), ragged K (9*6 input
    columns) and N (width 24), and split-K weight gradients (16*144 points)."""
    m, ctx = g36
    s = rt.Surrogate(ctx, width=width, capacity=1, seed=5)
    rng = np.random.default_rng(width + B)
    p = so.init_params(c_in=m.nmodes, c_out=m.nmodes, width=width, seed=width)
    for k in p:
        p[k] = (p[k] + 0.05 * rng.standard_normal(p[k].shape)).astype(np.float32).astype(np.float64)
    s.set_params(flat(p))
    assert np.array_equal(s.get_params(), flat(p).astype(np.float32))
    ny, nx = s.nq_s[1], s.nq_s[0]
    x = rng.standard_normal((B, ny, nx, m.nmodes)).astype(np.float32)
    t = (0.3 * rng.standard_normal((B, ny, nx, m.nmodes))).astype(np.float32)
    loss, g, out = s.loss_grad(x, t)
    lo, go = so.loss_and_grads(p, bf16_round(x), t.astype(np.float64))
    oo, _ = so.forward(p, bf16_round(x))
    assert relL2(out, oo) < 1e-2
    assert abs(loss - lo) < 2e-2 * lo
    gg = unflat(g.astype(np.float64), p)
    for k in ORDER:
        assert relL2(gg[k], go[k]) < 2e-2, k
    s.close()


@pytest.mark.parametrize("width,B", [(64, 3), (24, 16), (64, 40)])
def test_tensor_core_engine_matches_mma_sync(rt, g36, width, B):
    """The default GEMM engine on this GPU is the tcgen05 one (forward layers and input gradients
    on the fifth-generation tensor cores, TMA-fed, accumulators in tensor memory).  On the same
    weights and inputs its output, loss and gradients agree with the mma.sync engine to FP32
    accumulation-order rounding; the sizes give ragged M tiles (3 x 144 and 40 x 144 points), N
    below 16 (the 6 output channels), N tiles of 256 + 256 + 64 (576-column input gradients)
    and N 24 / K 24 (width 24)."""
    m, ctx = g36
    s = rt.Surrogate(ctx, width=width, capacity=1, seed=9)
    rng = np.random.default_rng(7 * width + B)
    ny, nx = s.nq_s[1], s.nq_s[0]
    x = rng.standard_normal((B, ny, nx, m.nmodes)).astype(np.float32)
    t = (0.3 * rng.standard_normal((B, ny, nx, m.nmodes))).astype(np.float32)
    res = []
    for engine in (0, 1):
        s.set_gemm(engine)
        res.append(s.loss_grad(x, t))
    (l0, g0, o0), (l1, g1, o1) = res
    assert relL2(o0, o1) < 1e-5
    assert abs(l0 - l1) < 1e-5 * l1
    assert relL2(g0, g1) < 1e-4
    s.close()


def trajectory_states(rt, m, ctx, n_traj=4, per=6, t_end=0.06):
    """(device state, trajectory id) along the method's own trajectories from several initial
    conditions (excitation energy, amplitude, temperature) on the same channels."""
    states = []
    for j in range(n_traj):
        mj = ri.graphene(n=36, window=1.0, pp_stride=3, seed=ri.SEED_BASE + 11, sigma_eph=0.040, sigma_pp=0.008,
                         E_x=0.6 + 0.15 * j, amp=0.2 + 0.05 * j, T=250.0 + 40 * j)
        y = torch.tensor(mj.y0(), device="cuda")
        states.append((y.clone(), j))
        for i in range(1, per):
            st = ctx.advance_to(t_end * i / (per - 1), y, method="zon43", t0=t_end * (i - 1) / (per - 1), rtol=1e-5,
                                atol_c=1e-9, atol_ph=1e-12)
            assert st["status"] == 0
            states.append((y.clone(), j))
    return states


@pytest.fixture(scope="module")
def trained(rt, g36):
    """Width 64 (the fused inference kernels), trained on single pairs, then on differences."""
    m, ctx = g36
    states = trajectory_states(rt, m, ctx)
    s = rt.Surrogate(ctx, width=64, capacity=len(states), seed=7)
    for y, j in states[:-1]:
        s.collect(y, j)
    l_first = s.train(1, 4, 2e-3)
    l_last = s.train(400, 4, 2e-3)
    d_first = s.train(1, 4, 1e-3, horizon=3)
    d_last = s.train(300, 4, 1e-3, horizon=3)
    yield s, [y for y, _ in states], (l_first, l_last, d_first, d_last)
    s.close()


def test_collected_pairs_are_the_exact_slow_integral(rt, g36, trained):
    """Pairs hold N and the exact I^{ph-ph} of the sub-lattice: the normalisation the first
    training call fixed equals the FP64 statistics of those values read through rtbte_rhs."""
    m, ctx = g36
    s, states, _ = trained
    mu, sd, sc, n = s.stats()
    assert n == len(states) - 1
    full = m.pp_full_index().reshape(m.nmodes, -1) + m.n_c
    Ns, Is = [], []
    for y in states[:-1]:
        Ns.append(y.cpu().numpy()[full])
        Is.append(ctx.rhs(y, parts=rt.RTBTE_SLOW).cpu().numpy()[full])
    Ns, Is = np.array(Ns), np.array(Is)  # [n, C, P]
    assert np.allclose(mu, Ns.mean(axis=(0, 2)), rtol=1e-5)
    assert np.allclose(sc, np.sqrt((Is ** 2).mean(axis=(0, 2))), rtol=1e-4)


def test_training_lowers_the_loss(trained):
    _, _, (l_first, l_last, d_first, d_last) = trained
    assert l_last < 0.2 * l_first
    assert d_last < 0.5 * d_first


def oracle_prediction(s, m, y, width):
    mu, sd, sc, _ = s.stats()
    full = m.pp_full_index().reshape(m.nmodes, -1) + m.n_c
    ny, nx = s.nq_s[1], s.nq_s[0]
    N = y.cpu().numpy()[full].T.reshape(1, ny, nx, m.nmodes)
    like = so.init_params(m.nmodes, m.nmodes, width, 0)
    p = unflat(s.get_params().astype(np.float64), like)
    x = bf16_round(((N - mu) / sd).astype(np.float32))
    out, _ = so.forward(p, x)
    return full, (out * sc).reshape(-1, m.nmodes).T


def test_fused_prediction_matches_oracle_forward(rt, g36, trained):
    """rtbte_surrogate_predict (width 64: the fused inference kernels) scatters the scaled
    network output into the sub-lattice rows and zero elsewhere; it agrees with the FP64
    oracle forward on the trained weights."""
    m, ctx = g36
    s, states, _ = trained
    y = states[-1]
    pred = s.predict(y).cpu().numpy()
    full, ref = oracle_prediction(s, m, y, 64)
    assert relL2(pred[full], ref) < 2e-2
    mask = np.ones(m.n_y, dtype=bool)
    mask[full.ravel()] = False
    assert not pred[mask].any()


def test_fused_inference_equals_training_forward(rt, g36, trained):
    """The fused single-sample kernels and the training kernels compute the same network:
    same BF16 roundings and the same K order in every convolution, so they agree to FP32
    rounding of the last (64 -> C) product."""
    m, ctx = g36
    s, states, _ = trained
    y = states[-1]
    mu, sd, sc, _ = s.stats()
    full = m.pp_full_index().reshape(m.nmodes, -1) + m.n_c
    ny, nx = s.nq_s[1], s.nq_s[0]
    N = y.cpu().numpy()[full].T.reshape(1, ny, nx, m.nmodes)
    x = ((N - mu) / sd).astype(np.float32)
    _, _, out = s.loss_grad(x, np.zeros_like(x))
    pred = s.predict(y).cpu().numpy()[full]
    assert relL2(pred, (out[0] * sc).reshape(-1, m.nmodes).T) < 1e-4


def test_general_width_prediction_matches_oracle_forward(rt, g36):
    m, ctx = g36
    s = rt.Surrogate(ctx, width=32, capacity=1, seed=11)
    y = torch.tensor(m.y0(), device="cuda")
    pred = s.predict(y).cpu().numpy()
    full, ref = oracle_prediction(s, m, y, 32)
    assert relL2(pred[full], ref) < 2e-2
    s.close()


def test_trained_network_gains_over_holding_the_exact_value(rt, g36, trained):
    """What the trained network gains.  The surrogate slow stage (exact judge every 5 slow
    steps) evaluates the exact ph-ph integral 2 times instead of the 30 of plain MRI.  Without
    the network (output weights zero, so S(Y) - S(Y_ref) = 0) the slow value is the exact one
    held from the last judge; the trained network's control variate lowers both the judges'
    error of the slow value and the population error against a tight FP64 reference.  Plain
    MRI, exact at every stage, stays more accurate on this workload: the synthetic ph-ph
    integral changes by tens of percent between judges and a 9x9-point receptive field does
    not see its momentum-space couplings, so the population error is far above 1e-6 (the
    numbers are reported, not bounded above)."""
    m, ctx = g36
    s, _, _ = trained
    kw = dict(rtol=1e-5, atol_c=1e-9, atol_ph=1e-12)
    y0 = torch.tensor(m.y0(), device="cuda")
    ref_ctx = rt.Context(m, precision="fp64")
    ref_ctx.upload_channels()
    yr = y0.clone()
    assert ref_ctx.advance_to(0.1, yr, method="zon43", t0=0.0, rtol=1e-9, atol_c=1e-15, atol_ph=1e-15)["status"] == 0
    ref_ctx.close()
    yr = yr.cpu().numpy()
    yp = y0.clone()
    sp = ctx.advance_to(0.1, yp, method="mri", t0=0.0, h_s=0.01, **kw)
    assert sp["status"] == 0 and sp["slow_exact"] == 30 and sp["slow_surrogate"] == 0

    def run():
        s.attach(judge_period=5, judge_tol=10.0)
        ys = y0.clone()
        st = ctx.advance_to(0.1, ys, method="mri", t0=0.0, h_s=0.01, **kw)
        s.detach()
        assert st["status"] == 0 and st["surrogate_fallbacks"] == 0
        assert st["slow_exact"] == 2 and st["slow_surrogate"] == 28
        return relL2(ys.cpu().numpy(), yr), st["judge_err_max"]

    e_net, j_net = run()
    p = s.get_params()
    held = p.copy()
    held[-(64 * m.nmodes + m.nmodes):] = 0.0  # M2 and c2
    s.set_params(held)
    e_held, j_held = run()
    s.set_params(p)
    e_plain = relL2(yp.cpu().numpy(), yr)
    print(f"population error: plain MRI {e_plain:.3e}, held {e_held:.3e}, network {e_net:.3e}; "
          f"judge error: held {j_held:.3f}, network {j_net:.3f}")
    assert 0 < j_net < j_held
    assert e_net < 0.9 * e_held
    assert e_plain < e_net


def test_failed_judge_falls_back_to_the_exact_slow_part(rt, g36, trained):
    """A judge whose residual exceeds the tolerance detaches the surrogate for the rest of
    the call: every later slow value is exact and the call reports the fallback."""
    m, ctx = g36
    s, _, _ = trained
    s.attach(judge_period=2, judge_tol=1e-12)
    y = torch.tensor(m.y0(), device="cuda")
    st = ctx.advance_to(0.06, y, method="mri", t0=0.0, h_s=0.01, rtol=1e-5, atol_c=1e-9, atol_ph=1e-12)
    s.detach()
    assert st["status"] == 0 and st["surrogate_fallbacks"] == 1
    # steps 0-1 use the surrogate for 5 values (k=0 stages 2-3, k=1 all three); the judge at
    # k=2 fails, then 4 steps x 3 exact values
    assert st["slow_surrogate"] == 5 and st["slow_exact"] == 1 + 12
    assert np.isfinite(y.cpu().numpy()).all()


def test_surrogate_argument_checks(rt, g36):
    m, ctx = g36
    lib = rt.load()
    s = rt.Surrogate(ctx, width=16, capacity=1, seed=1)
    assert lib.rtbte_set_surrogate(ctx.ctx, s.h, 10, 1e-2) == -9  # not trained: no normalisation yet
    assert lib.rtbte_set_surrogate(ctx.ctx, s.h, 0, 1e-2) == -1
    assert lib.rtbte_surrogate_train(s.h, 1, 1, 0, 1e-3, None) == -9  # no pairs
    assert lib.rtbte_surrogate_train(s.h, 1, 1, -1, 1e-3, None) == -1
    y = torch.tensor(m.y0(), device="cuda")
    s.collect(y)
    assert lib.rtbte_surrogate_collect(s.h, y.data_ptr(), 0) == -1  # buffer full
    assert lib.rtbte_surrogate_train(s.h, 1, 1, 1, 1e-3, None) == -9  # one pair: no difference units
    s.close()
