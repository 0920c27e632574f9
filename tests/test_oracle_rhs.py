"""Pins for the oracle's collision integrals (Eq. e-ph, Eq. ph-ph and their F/G factors).

Each check compares the oracle with something other than itself: closed-form
equilibrium identities, exact detailed balance on an exactly resonant model,
conservation laws, brute force without stored lists, and index conventions probed
with single-phonon populations.  CPU only.
"""
import math

import numpy as np
import pytest

import rtbte_inputs as ri

KB = ri.KB_EV_K


def inv_phonon_index(model):
    """p -> index of (nu, -q)."""
    nx, ny, nz = model.nq
    q = np.arange(model.N_q)
    x, y, z = q % nx, (q // nx) % ny, q // (nx * ny)
    qi = ((-z % nz) * ny + (-y % ny)) * nx + (-x % nx)
    return (np.arange(model.nmodes)[:, None] * model.N_q + qi[None, :]).ravel()


def symmetric_state(model, seed):
    """Random populations with N(nu, q) == N(nu, -q) bit for bit (the inversion symmetry the
    paper's literal emission term relies on)."""
    f, N = ri.random_populations(model, seed)
    inv = inv_phonon_index(model)
    N = 0.5 * (N + N[inv])
    return np.concatenate([f, N])


# ---------------------------------------------------------------------------
# Gaussian delta (Methods A, normalised reading)
# ---------------------------------------------------------------------------
def test_gaussian_delta_normalisation_and_width(oracle_lib):
    sig = 0.02
    E = np.linspace(-3 * sig, 3 * sig, 200001)
    d = np.array([oracle_lib.gauss_delta(e, sig) for e in E[::100]])
    Ec = E[::100]
    # truncated integral equals erf(3); second moment of the full Gaussian is sigma^2/2
    from scipy.integrate import simpson

    assert abs(simpson(d, x=Ec) - math.erf(3.0)) < 1e-9
    E2 = np.linspace(-12 * sig, 12 * sig, 40001)
    d2 = np.array([oracle_lib.gauss_delta(e, sig) for e in E2])
    assert abs(simpson(d2 * E2 ** 2, x=E2) - sig ** 2 / 2) < 1e-12


# ---------------------------------------------------------------------------
# F and G factors: equilibrium closed forms
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("seed", range(5))
def test_population_factors_equilibrium_closed_form(oracle_lib, seed):
    """At Fermi-Dirac / Bose-Einstein populations of one temperature,
    F_em  = f(1-f')(1+N)(1 - exp(beta*(eps - hw - eps'))),
    F_abs = f(1-f') N   (1 - exp(beta*(eps + hw - eps'))),
    G_em  = N(N'+1)(N''+1)(1 - exp(beta*(hw - hw' - hw''))),
    G_abs = N(N'+1) N''   (1 - exp(beta*(hw - hw' + hw''))).
    These follow from the ratios of the occupation factors alone, so a swapped
    population, a sign slip or a dropped +1 breaks them."""
    rng = np.random.default_rng(seed)
    T = 150 + 500 * rng.random()
    b = 1.0 / (KB * T)
    mu = 0.2 * rng.standard_normal()
    for _ in range(50):
        # keep every occupation and its complement >= ~1e-2 so that 1-f is well conditioned
        e, ep = mu + rng.uniform(-4, 4, 2) * KB * T
        w, w1, w2 = rng.uniform(0.05, 4, 3) * KB * T
        f, fp = [float(ri.fermi_dirac(x, mu, T)) for x in (e, ep)]
        N, N1, N2 = [float(ri.bose_einstein(np.array([x]), T)[0]) for x in (w, w1, w2)]
        fem = f * (1 - fp) * (1 + N) * (-math.expm1(b * (e - w - ep)))
        fab = f * (1 - fp) * N * (-math.expm1(b * (e + w - ep)))
        gem = N * (N1 + 1) * (N2 + 1) * (-math.expm1(b * (w - w1 - w2)))
        gab = N * (N1 + 1) * N2 * (-math.expm1(b * (w - w1 + w2)))
        # tolerance scale: the gross forward + reverse magnitude of each factor
        sf = f * (1 - fp) * (1 + N) + (1 - f) * fp * (1 + N)
        sg = (N + 1) * (N1 + 1) * (N2 + 1) + N * N1 * N2
        for got, ref, scale in ((oracle_lib.F_em(f, fp, N), fem, sf), (oracle_lib.F_abs(f, fp, N), fab, sf),
                                (oracle_lib.G_em(N, N1, N2), gem, sg), (oracle_lib.G_abs(N, N1, N2), gab, sg)):
            assert abs(got - ref) <= 1e-13 * scale


def test_population_factor_limits(oracle_lib):
    """Pauli blocking and spontaneous emission limits: a full final state blocks, an empty
    initial state gives only the reverse process, spontaneous emission survives at N=0."""
    assert oracle_lib.F_em(1.0, 0.0, 0.0) == 1.0          # spontaneous emission
    assert oracle_lib.F_abs(1.0, 0.0, 0.0) == 0.0         # nothing to absorb
    assert abs(oracle_lib.F_em(0.75, 1.0, 2.0) + 0.5) < 1e-15  # full final state: reverse only, -(1-f) f' N
    assert oracle_lib.G_em(1.0, 0.0, 0.0) == 1.0          # spontaneous decay a -> b + c
    assert oracle_lib.G_abs(0.0, 1.0, 0.0) == -1.0        # b decays into a + c's absence: reverse only


# ---------------------------------------------------------------------------
# Detailed balance on the exact-resonance ("ladder") model
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("T,mu", [(300.0, 0.0), (120.0, 0.05), (900.0, -0.03)])
def test_detailed_balance_exact_resonance(oracle_lib, T, mu):
    m = ri.ladder(n=6, T=T, mu=mu)
    o = oracle_lib.Oracle(m)
    o.build_lists()
    y = m.y0()
    for rhs in (o.rhs(y), o.rhs_literal(y)):
        # scale: the rates of the same model away from equilibrium
        ref = np.abs(o.rhs(symmetric_state(m, 3))).max()
        assert ref > 1e-3
        assert np.abs(rhs).max() < 1e-12 * ref
    # away from equilibrium the rates do not vanish
    ne = o.rhs(symmetric_state(m, 4))
    assert np.abs(ne[: m.n_c]).max() > 1e-3 and np.abs(ne[m.n_c:]).max() > 1e-6


# ---------------------------------------------------------------------------
# Conservation laws
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("mk", [lambda: ri.toy2d(), lambda: ri.graphene_small(24),
                                lambda: ri.tiny((4, 4, 4), fold=2, nbands=2, nmodes=2), lambda: ri.silicon(16)])
def test_carrier_number_conservation(oracle_lib, mk):
    m = mk()
    o = oracle_lib.Oracle(m)
    o.build_lists(oracle_lib.FAST)
    y = symmetric_state(m, 11)
    r = o.rhs(y, oracle_lib.EPH)[: m.n_c]
    assert abs(r.sum()) <= 1e-12 * np.abs(r).sum()
    assert np.abs(r).max() > 0


def test_energy_conservation_exact_resonance(oracle_lib):
    """With every kept channel exactly resonant, d/dt [(2/N_k) sum eps f + (1/N_q) sum hw N]
    vanishes for the e-ph + ph-e pair (this fixes the ph-e prefactor 4 pi/(hbar N_k) relative to
    the e-ph one and the phonon each absorption feeds), and sum hw dN/dt vanishes for ph-ph (this
    fixes the factor 2 on absorption and the pair counting of emission)."""
    m = ri.ladder(n=6)
    o = oracle_lib.Oracle(m)
    o.build_lists()
    y = symmetric_state(m, 5)
    r = o.rhs(y, oracle_lib.FAST)
    eps, w = m.e_eps, m.ph_omega
    e_el = (2.0 / m.N_k) * np.dot(eps, r[: m.n_c])
    e_ph = (1.0 / m.N_q) * np.dot(w, r[m.n_c:])
    assert abs(e_el) > 1e-6
    assert abs(e_el + e_ph) < 1e-12 * abs(e_el)
    rl = o.rhs_literal(y, oracle_lib.FAST)
    assert abs((2.0 / m.N_k) * np.dot(eps, rl[: m.n_c]) + (1.0 / m.N_q) * np.dot(w, rl[m.n_c:])) < 1e-12 * abs(e_el)
    rp = o.rhs(y, oracle_lib.SLOW)[m.n_c:]
    assert np.abs(rp).max() > 1e-8
    assert abs(np.dot(w, rp)) < 1e-12 * np.dot(w, np.abs(rp))


@pytest.mark.parametrize("T,mu", [(300.0, 0.0), (150.0, 0.04)])
def test_detailed_balance_exact_resonance_folded_3d(oracle_lib, T, mu):
    """Detailed balance on the folded 3D exact-resonance model (fold 2, N_k = 8 N_q): at
    Fermi-Dirac / Bose-Einstein populations of one temperature every rate vanishes, from the
    stored lists and from the literal sums."""
    m = ri.ladder3d(n=8, T=T, mu=mu)
    assert m.N_k == 8 * m.N_q
    o = oracle_lib.Oracle(m)
    o.build_lists()
    ref = np.abs(o.rhs(symmetric_state(m, 3))).max()
    assert ref > 1e-3
    for rhs in (o.rhs(m.y0()), o.rhs_literal(m.y0())):
        assert np.abs(rhs).max() < 1e-12 * ref


def test_energy_conservation_exact_resonance_folded_3d(oracle_lib):
    """Energy conservation of the e-ph + ph-e pair on a grid where N_k != N_q (fold 2 in 3D,
    N_k = 8 N_q): d/dt [(2/N_k) sum eps f + (1/N_q) sum hw N] = 0 for arbitrary (inversion
    symmetric) populations.  Each process moves hw from the electrons to one phonon, so this
    holds only with the e-ph weight (2 pi/hbar)(1/N_q) and the ph-e weight (4 pi/hbar)(1/N_k)
    of Eq. e-ph: exchanging N_k and N_q in either prefactor scales that side's rates by 8 and
    breaks the balance (checked below on the oracle's own rows, rescaled as such a swap would)."""
    m = ri.ladder3d(n=8)
    o = oracle_lib.Oracle(m)
    o.build_lists(oracle_lib.FAST)
    y = symmetric_state(m, 5)
    eps, w = m.e_eps, m.ph_omega
    for r in (o.rhs(y, oracle_lib.FAST), o.rhs_literal(y, oracle_lib.FAST)):
        e_el = (2.0 / m.N_k) * np.dot(eps, r[: m.n_c])
        e_ph = (1.0 / m.N_q) * np.dot(w, r[m.n_c:])
        assert abs(e_el) > 1e-6
        assert abs(e_el + e_ph) < 1e-12 * abs(e_el)
        # a swapped N_k <-> N_q in the ph-e weight (x N_k/N_q) or in the e-ph weight (x N_q/N_k)
        ratio = m.N_k / m.N_q
        assert abs(e_el + ratio * e_ph) > 1.0 * abs(e_el)
        assert abs(e_el / ratio + e_ph) > 0.5 * abs(e_el)


def test_energy_balance_equals_detuning_sum(oracle_lib):
    """Off resonance the e-ph energy change is the detuning-weighted rate sum:
    d/dt E = -(2/N_k) sum_{emission entries} W F_em (eps_d - hw - eps_s), exactly (to rounding)."""
    m = ri.graphene_small(24)
    o = oracle_lib.Oracle(m)
    o.build_lists(oracle_lib.FAST)
    y = symmetric_state(m, 6)
    r = o.rhs(y, oracle_lib.FAST)
    dE = (2.0 / m.N_k) * np.dot(m.e_eps, r[: m.n_c]) + (1.0 / m.N_q) * np.dot(m.ph_omega, r[m.n_c:])
    L = o.lists["eph"]
    f, N = y[: m.n_c], y[m.n_c:]
    acc = 0.0
    for d in range(m.n_c):
        sl = slice(L["off"][2 * d], L["off"][2 * d + 1])
        s, p, W = L["src"][sl], L["ph"][sl], L["W"][sl]
        fe = f[d] * (1 - f[s]) * (1 + N[p]) - (1 - f[d]) * f[s] * N[p]
        acc += np.sum(W * fe * (m.e_eps[d] - m.ph_omega[p] - m.e_eps[s]))
    ref = (2.0 / m.N_k) * np.sum(np.abs(m.e_eps * r[: m.n_c]))
    assert abs(dE - (-(2.0 / m.N_k) * acc)) < 1e-11 * ref


# ---------------------------------------------------------------------------
# Stored lists reproduce the plain sums (brute force)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("mk", [lambda: ri.tiny((4, 4, 1)), lambda: ri.tiny((6, 6, 1), nbands=1, nmodes=4),
                                lambda: ri.tiny((4, 4, 4), fold=2, nbands=2, nmodes=2, pp_stride=1),
                                lambda: ri.tiny((6, 6, 1), pp_stride=2, sigma_pp=0.03),
                                lambda: ri.toy2d(), lambda: ri.graphene_small(24)])
def test_lists_equal_plain_sums(oracle_lib, mk):
    m = mk()
    o = oracle_lib.Oracle(m)
    o.build_lists()
    f, N = ri.random_populations(m, 21)
    y = np.concatenate([f, N])
    a = o.rhs(y)
    b = o.rhs_literal(y)
    assert np.abs(a - b).max() <= 1e-12 * max(np.abs(b).max(), 1e-300)
    assert np.abs(b).max() > 0


def test_phe_list_is_the_absorption_half_of_eph(oracle_lib):
    """Every ph-e entry is an e-ph absorption entry regrouped by phonon, with the weight
    rescaled by (4pi/(hbar N_k)) / (2pi/(hbar N_q)) = 2 N_q / N_k."""
    m = ri.tiny((4, 4, 4), fold=2, nbands=2, nmodes=2)
    o = oracle_lib.Oracle(m)
    L = o.build_lists()
    e, h = L["eph"], L["phe"]
    abs_set = {}
    for d in range(m.n_c):
        for k in range(e["off"][2 * d + 1], e["off"][2 * d + 2]):
            abs_set[(int(e["ph"][k]), d, int(e["src"][k]))] = e["W"][k]
    phe_set = {}
    for p in range(m.n_ph):
        for k in range(h["off"][p], h["off"][p + 1]):
            phe_set[(p, int(h["dst"][k]), int(h["src"][k]))] = h["W"][k]
    assert set(abs_set) == set(phe_set) and len(phe_set) > 0
    ratio = 2.0 * m.N_q / m.N_k
    for k, w in abs_set.items():
        assert abs(phe_set[k] - ratio * w) <= 1e-14 * phe_set[k]


# ---------------------------------------------------------------------------
# Index conventions: final state k + q, phonon momentum bookkeeping
# ---------------------------------------------------------------------------
def test_emission_reads_phonon_at_final_minus_initial_momentum(oracle_lib):
    """Put a single phonon population at (nu*, q*); the e-ph rate of destination k changes only
    through sources at k' with q* = k' - k (final state k+q, Eq. e-ph)."""
    m = ri.tiny((6, 6, 1), nbands=1, nmodes=2, sigma_eph=0.2)
    o = oracle_lib.Oracle(m)
    f = np.linspace(0.1, 0.9, m.n_c)
    nu, qx, qy = 1, 2, 1
    p = nu * m.N_q + qy * m.nq[0] + qx
    y0 = np.concatenate([f, np.zeros(m.n_ph)])
    y1 = y0.copy()
    y1[m.n_c + p] = 1.0
    d = o.rhs_literal(y1, oracle_lib.EPH)[: m.n_c] - o.rhs_literal(y0, oracle_lib.EPH)[: m.n_c]
    # the changed term for destination k involves source k + q* only
    for s in range(m.n_c):
        if abs(d[s]) < 1e-14:
            continue
        kx, ky = m.e_k[s, 0], m.e_k[s, 1]
        t = [j for j in range(m.n_c) if m.e_k[j, 0] == (kx + qx) % 6 and m.e_k[j, 1] == (ky + qy) % 6][0]
        fe = f[s] * (1 - f[t]) - (1 - f[s]) * f[t]  # dF/dN, same for emission and absorption
        assert np.sign(d[s]) == -np.sign(fe) or abs(fe) < 1e-12
    assert np.count_nonzero(np.abs(d) > 1e-14) > 0


def test_phph_momentum_rule(oracle_lib):
    """Every ph-ph entry satisfies q_a = q_b + q_c (emission) or q_b = q_a + q_c (absorption)
    on the sub-lattice."""
    m = ri.tiny((6, 6, 1), pp_stride=2, sigma_pp=0.03)
    o = oracle_lib.Oracle(m)
    L = o.pp_lists()
    nqs = m.nq_pp
    Nqs = m.N_q_pp
    M = L["full"].shape[0]
    q = lambda a: ((a % Nqs) % nqs[0], (a % Nqs) // nqs[0])
    n_checked = 0
    for a in range(M):
        for proc in (0, 1):
            for k in range(L["off"][2 * a + proc], L["off"][2 * a + proc + 1]):
                qa, qb, qc = q(a), q(int(L["b"][k])), q(int(L["c"][k]))
                if proc == 0:
                    assert ((qb[0] + qc[0]) % nqs[0], (qb[1] + qc[1]) % nqs[1]) == qa
                    assert L["b"][k] <= L["c"][k]
                else:
                    assert ((qa[0] + qc[0]) % nqs[0], (qa[1] + qc[1]) % nqs[1]) == qb
                n_checked += 1
    assert n_checked > 100


def test_frozen_modes_do_not_scatter(oracle_lib):
    m = ri.graphene_small(24)
    o = oracle_lib.Oracle(m)
    L = o.build_lists()
    fr = m.frozen()
    assert fr.any()
    assert not fr[L["eph"]["ph"]].any()
    cnt = np.diff(L["phe"]["off"])
    assert (cnt[fr] == 0).all()
    r = o.rhs(symmetric_state(m, 1))
    assert (r[m.n_c:][fr] == 0).all()


def test_linearised_phph_rates_are_the_derivative_of_the_integral(oracle_lib):
    """The linearised ph-ph rate of a sub-lattice phonon (partners held fixed) equals minus
    the derivative of its literal Eq. ph-ph integral with respect to its own population,
    checked by central differences of the plain sums on phonons that are not their own
    partner in any channel (there the integral is affine in the population; a phonon can
    absorb one of its own kind, a + a -> b, which makes the full derivative differ)."""
    m = ri.graphene_small(24)
    o = oracle_lib.Oracle(m)
    L = o.build_lists()["pp"]
    f, N = ri.random_populations(m, 8)
    y = np.concatenate([f, N])
    rates = o.pp_rates(y)
    full = o.pp_full_index()
    off = L["off"]
    own = [a for a in range(full.shape[0])
           if not np.any(L["b"][off[2 * a]:off[2 * a + 2]] == a) and not np.any(L["c"][off[2 * a]:off[2 * a + 2]] == a)]
    assert len(own) > full.shape[0] // 4
    rng = np.random.default_rng(2)
    for a in rng.choice(own, 8, replace=False):
        r = m.n_c + full[a]
        pmask = np.zeros(m.n_ph, np.uint8)
        pmask[full[a]] = 1
        d = 1e-3 * max(1.0, y[r])
        yp, ym = y.copy(), y.copy()
        yp[r] += d
        ym[r] -= d
        ip = o.rhs_literal(yp, parts=oracle_lib.PHPH, pmask=pmask)[r]
        im = o.rhs_literal(ym, parts=oracle_lib.PHPH, pmask=pmask)[r]
        assert -(ip - im) / (2 * d) == pytest.approx(rates[r], rel=1e-9, abs=1e-12 * abs(rates).max())
    mask = np.ones(m.n_y, bool)
    mask[m.n_c + full] = False
    assert not rates[mask].any()
    # at Bose-Einstein populations (one temperature) the optical branches relax (positive rates)
    rb = o.pp_rates(m.y0())[m.n_c + full].reshape(m.nmodes, -1)
    assert (rb[3:] > 0).all()
