"""Pins for the oracle's MRI with a tolerance-chosen slow step (step doubling on the MIS
Knoth-Wolke step; the extension the paper names as future work, Methods B): the error
estimate against exact matrix-exponential solutions, the accept / reject decision against
that estimate, the growth cap and end-point clipping on a problem with zero error, the
rejection path and its give-up status, and the step count's tolerance scaling.  CPU only."""
import numpy as np
import pytest
from scipy.linalg import expm

AF = np.array([[-20.0, 2.0], [1.0, -10.0]])  # fast part
AS = np.array([[-1.0, 0.5], [0.3, -0.8]])  # slow part (does not commute with AF)
Y0 = np.array([1.0, 2.0])
TIGHT = 1e-13  # fast-solve tolerance that makes the fast error negligible


def fast(t, y):
    return AF @ y


def slow(t, y):
    return AS @ y


def one_and_two_steps(oracle_lib, H):
    """One MIS step of H and two of H/2 from Y0 (fixed-step oracle MRI, fast solves at TIGHT)."""
    y1, _ = oracle_lib.ode_mri(fast, slow, Y0, 0.0, H, H, TIGHT, 1e-16)
    y2, _ = oracle_lib.ode_mri(fast, slow, Y0, 0.0, H, H / 2, TIGHT, 1e-16)
    return y1, y2


def test_step_doubling_estimate_converges_to_the_true_local_error(oracle_lib):
    """(y_1 - y_2) / (2^3 - 1) estimates the local error of y_2 for an order-3 slow method: its
    deviation from the exact error y_2 - y(H) (matrix exponential) is of relative size O(H).
    A wrong order in the denominator (2^p - 1 with p != 3) would leave an O(1) deviation."""
    devs = []
    for H in (0.02, 0.01, 0.005):
        y1, y2 = one_and_two_steps(oracle_lib, H)
        true = y2 - expm((AF + AS) * H) @ Y0
        est = (y1 - y2) / 7.0
        devs.append(np.linalg.norm(est - true) / np.linalg.norm(true))
    assert devs[1] < 0.1
    assert 0.35 < devs[1] / devs[0] < 0.65 and 0.35 < devs[2] / devs[1] < 0.65


@pytest.mark.parametrize("eps_target,accepted", [(0.8, True), (1.25, False)])
def test_a_slow_step_is_accepted_exactly_when_the_estimate_is_within_tolerance(oracle_lib, eps_target, accepted):
    """A single attempt over [0, H]: with rtol set so that the WRMS norm of the estimate
    (weights 1/(rtol |y_0| + atol), atol negligible) is 0.8, the step is accepted and the result
    is the two half steps bit for bit; at 1.25 it is rejected first and retried shorter."""
    H = 0.01
    y1, y2 = one_and_two_steps(oracle_lib, H)
    est = (y1 - y2) / 7.0
    atol = 1e-30
    eps_at_rtol1 = np.sqrt(np.mean((est / (np.abs(Y0) + atol)) ** 2))
    rtol = eps_at_rtol1 / eps_target
    y, st = oracle_lib.ode_mri_adapt(fast, slow, Y0, 0.0, H, H, rtol, atol, slow=dict(fast_scale=TIGHT / rtol))
    assert st["status"] == 0 and st["t"] == H
    if accepted:
        assert st["slow_fails"] == 0 and st["slow_steps"] == 1
        ref, _ = oracle_lib.ode_mri(fast, slow, Y0, 0.0, H, H / 2, rtol * (TIGHT / rtol), atol * (TIGHT / rtol))
        assert np.array_equal(y, ref)
        assert st["h_next"] == pytest.approx(H * 0.9 * 0.8 ** -0.25, rel=1e-4)
    else:
        assert st["slow_fails"] >= 1 and st["slow_steps"] >= 2


def test_zero_error_grows_the_slow_step_by_the_cap_and_clips_at_the_end(oracle_lib):
    """y' = 0: every estimate is 0, so each accepted step grows H by the cap (5): 0.01, 0.05,
    0.25, then 1.25 is clipped to the 0.69 left before t1 = 1."""
    z = lambda t, y: 0.0 * y
    y, st = oracle_lib.ode_mri_adapt(z, z, Y0, 0.0, 1.0, 0.01, 1e-6, 1e-12)
    assert st["status"] == 0 and st["t"] == 1.0
    assert np.array_equal(y, Y0)
    assert st["slow_steps"] == 4 and st["slow_fails"] == 0
    assert st["h_last"] == pytest.approx(0.69, rel=1e-12)
    assert st["h_next"] == pytest.approx(0.69 * 5.0, rel=1e-12)
    assert st["rhs_slow"] == 3 * 3 * 4  # three stages, one + two steps per attempt


def test_rejections_restore_the_state_and_give_up_after_max_fail(oracle_lib):
    """A first slow step far too long for the tolerance is rejected; with max_fail = 1 the call
    stops with 'repeated error-test failures' and hands back the initial state at t0."""
    y, st = oracle_lib.ode_mri_adapt(fast, slow, Y0, 0.0, 1.0, 0.5, 1e-8, 1e-12, slow=dict(max_fail=1))
    assert st["status"] == -6
    assert st["t"] == 0.0 and np.array_equal(y, Y0)
    assert st["slow_fails"] == 1 and st["slow_steps"] == 0
    # with the default limit the same call recovers and meets the tolerance's scale
    y, st = oracle_lib.ode_mri_adapt(fast, slow, Y0, 0.0, 1.0, 0.5, 1e-6, 1e-12)
    assert st["status"] == 0 and st["slow_fails"] >= 1
    exact = expm((AF + AS) * 1.0) @ Y0
    assert np.linalg.norm(y - exact) / np.linalg.norm(exact) < 1e-3


def test_slow_step_count_scales_as_the_fourth_root_of_the_tolerance(oracle_lib):
    """Local error ~ C H^4 at order 3, so H ~ rtol^(1/4): the number of slow steps grows by
    about 10^(1/4) = 1.78 per decade of rtol, and the global error falls with rtol."""
    T = 2.0
    exact = expm((AF + AS) * T) @ Y0
    steps, errs = [], []
    for rtol in (1e-3, 1e-4, 1e-5, 1e-6):
        y, st = oracle_lib.ode_mri_adapt(fast, slow, Y0, 0.0, T, 0.01, rtol, 1e-14)
        assert st["status"] == 0 and st["t"] == T
        steps.append(st["slow_steps"])
        errs.append(np.linalg.norm(y - exact) / np.linalg.norm(exact))
    ratios = [b / a for a, b in zip(steps, steps[1:])]
    assert all(1.4 < r < 2.2 for r in ratios), steps
    assert all(b < a for a, b in zip(errs, errs[1:])), errs
