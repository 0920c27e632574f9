"""Pins for the oracle's time integrators (Methods B): tableaux against exact rationals and
their order conditions, observed convergence orders against closed-form ODE solutions,
the MIS coupling (Eq. mis_coef) through its reduction to the base method, and the
adaptive controller's tolerance proportionality.  CPU only."""
import json
import os
from fractions import Fraction as Fr

import numpy as np
import pytest
from scipy.linalg import expm

HERE = os.path.dirname(os.path.abspath(__file__))
GOLD = json.load(open(os.path.join(HERE, "golden", "tableaux.json")))


def rat(M):
    if isinstance(M, list):
        return [rat(x) for x in M]
    return Fr(M)


def order_conditions(A, b, c, p):
    """Butcher order conditions up to order p (p <= 4) as exact residuals."""
    S = len(b)
    Ac = [sum(A[i][j] * c[j] for j in range(S)) for i in range(S)]
    AAc = [sum(A[i][j] * Ac[j] for j in range(S)) for i in range(S)]
    Acc = [sum(A[i][j] * c[j] ** 2 for j in range(S)) for i in range(S)]
    conds = {1: [sum(b) - 1]}
    conds[2] = [sum(b[i] * c[i] for i in range(S)) - Fr(1, 2)]
    conds[3] = [sum(b[i] * c[i] ** 2 for i in range(S)) - Fr(1, 3),
                sum(b[i] * Ac[i] for i in range(S)) - Fr(1, 6)]
    conds[4] = [sum(b[i] * c[i] ** 3 for i in range(S)) - Fr(1, 4),
                sum(b[i] * c[i] * Ac[i] for i in range(S)) - Fr(1, 8),
                sum(b[i] * Acc[i] for i in range(S)) - Fr(1, 12),
                sum(b[i] * AAc[i] for i in range(S)) - Fr(1, 24)]
    return [r for k in range(1, p + 1) for r in conds[k]]


@pytest.mark.parametrize("name", ["RK4", "BS32", "ZON43", "KW3"])
def test_golden_tableaux_order_conditions(name):
    g = GOLD[name]
    A, b, c = rat(g["A"]), rat(g["b"]), rat(g["c"])
    S = len(b)
    for i in range(S):
        assert sum(A[i]) == c[i]                       # row sums give the abscissae
        assert all(A[i][j] == 0 for j in range(i, S))  # explicit
    assert all(r == 0 for r in order_conditions(A, b, c, g["p"]))
    if g["p"] < 4:  # not of one order higher
        assert any(r != 0 for r in order_conditions(A, b, c, g["p"] + 1))
    if "bt" in g:
        bt = rat(g["bt"])
        assert all(r == 0 for r in order_conditions(A, bt, c, g["q"]))
        assert any(r != 0 for r in order_conditions(A, bt, c, g["q"] + 1))


@pytest.mark.parametrize("name,mid", [("RK4", 0), ("BS32", 1), ("ZON43", 2), ("KW3", 3)])
def test_oracle_tableaux_equal_golden(oracle_lib, name, mid):
    g = GOLD[name]
    t = oracle_lib.tableau(mid)
    S = len(g["b"])
    assert t["S"] == S and t["p"] == g["p"]
    assert np.array_equal(t["A"], np.array([[float(Fr(x)) for x in row] for row in g["A"]]))
    assert np.array_equal(t["b"], np.array([float(Fr(x)) for x in g["b"]]))
    assert np.array_equal(t["c"], np.array([float(Fr(x)) for x in g["c"]]))
    if "bt" in g:
        assert np.array_equal(t["bt"], np.array([float(Fr(x)) for x in g["bt"]]))


def test_mis_coefficients_telescope(oracle_lib):
    """The MIS couplings of each slow stage sum to the base method's weights, and the partial
    sums up to stage i give row i of A (so with a vanishing fast part the MRI stages are the
    base method's stages)."""
    Om, ch = oracle_lib.mis_coef()
    g = GOLD["KW3"]
    A = np.array([[float(Fr(x)) for x in row] for row in g["A"]])
    b = np.array([float(Fr(x)) for x in g["b"]])
    assert np.allclose(ch, [0, 1 / 3, 3 / 4, 1], atol=0, rtol=1e-15)
    assert np.allclose(Om[0], 0)
    for i in range(1, 3):
        assert np.allclose(Om[1:i + 1].sum(axis=0), A[i], atol=1e-15)
    assert np.allclose(Om[1:].sum(axis=0), b, atol=1e-15)


# ---------------------------------------------------------------------------
# Observed orders on problems with closed-form solutions
# ---------------------------------------------------------------------------
Y0 = np.array([0.1, 0.2, 0.5, 0.8])


def logistic(t, y):
    return y * (1.0 - y)


def logistic_exact(t):
    return 1.0 / (1.0 + (1.0 / Y0 - 1.0) * np.exp(-t))


def relax(t, y, tau=0.7, yeq=0.3):
    return -(y - yeq) / tau


def relax_exact(t, tau=0.7, yeq=0.3):
    return yeq + (Y0 - yeq) * np.exp(-t / tau)


def observed_order(errs, hs):
    return np.polyfit(np.log(hs), np.log(errs), 1)[0]


@pytest.mark.parametrize("f,exact", [(logistic, logistic_exact), (relax, relax_exact)])
def test_rk4_order(oracle_lib, f, exact):
    hs = [0.2, 0.1, 0.05, 0.025]
    errs = [np.abs(oracle_lib.ode_rk4(f, Y0, 0.0, 2.0, h)[0] - exact(2.0)).max() for h in hs]
    assert 3.8 < observed_order(errs, hs) < 4.3


@pytest.mark.parametrize("mid,p", [(2, 4), (1, 3)])
@pytest.mark.parametrize("f,exact", [(logistic, logistic_exact), (relax, relax_exact)])
def test_erk_main_method_order_fixed_steps(oracle_lib, mid, p, f, exact):
    """With the error test disabled (huge tolerances) and h0 = hmax = h the adaptive ERK takes
    fixed steps of its main method."""
    hs = [0.2, 0.1, 0.05, 0.025]
    errs = []
    for h in hs:
        y, st = oracle_lib.ode_erk(f, Y0, 0.0, 2.0, mid, 1e30, 1e30, h0=h, hmax=h)
        assert st["fails"] == 0
        errs.append(np.abs(y - exact(2.0)).max())
    assert p - 0.25 < observed_order(errs, hs) < p + 0.35


def test_erk_tolerance_proportionality_and_counts(oracle_lib):
    errs, evals = [], []
    for rtol in (1e-4, 1e-6, 1e-8, 1e-10):
        y, st = oracle_lib.ode_erk(logistic, Y0, 0.0, 5.0, 2, rtol, 1e-14)
        assert st["status"] == 0 and st["t"] == 5.0
        errs.append(np.abs(y - logistic_exact(5.0)).max())
        evals.append(st["rhs_evals"])
        # 5 stages per attempt plus two evaluations of the starting-step estimate
        assert st["rhs_evals"] == 5 * st["attempts"] + 2
    for a, b in zip(errs, errs[1:]):
        assert b < a / 10
    assert errs[-1] < 1e-8
    assert evals == sorted(evals)


def test_erk_rejects_and_recovers(oracle_lib):
    """A stiff start (fast transient) forces error-test failures; the controller recovers and
    still meets the tolerance."""
    lam = 200.0
    f = lambda t, y: -lam * (y - np.cos(t))
    exact = lambda t: (lam ** 2 * np.cos(t) + lam * np.sin(t)) / (lam ** 2 + 1) + (
        Y0 - lam ** 2 / (lam ** 2 + 1)) * np.exp(-lam * t)
    y, st = oracle_lib.ode_erk(f, Y0, 0.0, 1.0, 2, 1e-7, 1e-10, h0=0.05)
    assert st["fails"] > 0 and st["status"] == 0
    assert np.abs(y - exact(1.0)).max() < 1e-5


# split linear test problem with non-commuting fast and slow parts
AF = np.array([[-2.0, 1.0, 0.0], [0.0, -3.0, 0.5], [0.3, 0.0, -1.5]])
AS = np.array([[-0.5, 0.0, 0.2], [0.4, -0.2, 0.0], [0.0, 0.1, -0.3]])
Z0 = np.array([1.0, -0.5, 0.25])


def test_mri_mis_order_three(oracle_lib):
    T = 1.0
    exact = expm((AF + AS) * T) @ Z0
    hs = [0.2, 0.1, 0.05, 0.025]
    errs = []
    for h in hs:
        y, st = oracle_lib.ode_mri(lambda t, y: AF @ y, lambda t, y: AS @ y, Z0, 0.0, T, h, 1e-13, 1e-15)
        assert st["status"] == 0
        assert st["rhs_slow"] == 3 * round(T / h)
        errs.append(np.abs(y - exact).max())
    assert 2.7 < observed_order(errs, hs) < 3.4


def test_mri_with_vanishing_fast_part_is_the_base_method(oracle_lib):
    """f_fast = 0: the fast solves integrate constant forcings exactly, so the MRI step is the
    Knoth-Wolke step; its order on the logistic equation is 3."""
    hs = [0.2, 0.1, 0.05, 0.025]
    errs = []
    for h in hs:
        y, _ = oracle_lib.ode_mri(lambda t, y: 0.0 * y, logistic, Y0, 0.0, 2.0, h, 1e-10, 1e-14)
        errs.append(np.abs(y - logistic_exact(2.0)).max())
    assert 2.8 < observed_order(errs, hs) < 3.3


def test_split_rk4_is_first_order(oracle_lib):
    T = 1.0
    exact = expm((AF + AS) * T) @ Z0
    hs = [0.1, 0.05, 0.025, 0.0125]
    errs = [np.abs(oracle_lib.ode_split_rk4(lambda t, y: AF @ y, lambda t, y: AS @ y, Z0, 0.0, T, h, h / 4)[0]
                   - exact).max() for h in hs]
    assert 0.85 < observed_order(errs, hs) < 1.2


def test_wrms_norm_definition(oracle_lib):
    import ctypes as C

    v = np.array([1e-6, -2e-6, 3e-9])
    yr = np.array([0.5, 1.0, 0.0])
    atol = np.array([1e-9, 1e-9, 1e-12])
    got = oracle_lib.lib().or_wrms(3, v.ctypes.data, yr.ctypes.data, 1e-5, atol.ctypes.data)
    # component weights 1/(rtol|y|+atol): 1/(5.001e-6), 1/(1.0001e-5), 1/1e-12
    ref = np.sqrt(((1e-6 / 5.001e-6) ** 2 + (2e-6 / 1.0001e-5) ** 2 + (3e-9 / 1e-12) ** 2) / 3)
    assert abs(got - ref) < 1e-13 * ref
