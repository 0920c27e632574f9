"""Checks of the synthetic workloads themselves (sizes and physical scales), computed with
the oracle.  These pin the input recipe to the shapes of the paper's graphene workload
(Methods A: 1 meV frequency cutoff, 20 meV e-ph and 2 meV ph-ph broadening) and to the
scale of the ph-ph coupling (optical phonons decay in 1-10 ps, Results)."""
import numpy as np

import rtbte_inputs as ri


def test_graphene_sizes(oracle_lib):
    m = ri.graphene()
    assert m.n_c == 12722 and m.n_ph == 6 * 180 * 180 and m.n_pp == 6 * 60 * 60
    assert m.sigma_eph == 0.020 and m.sigma_pp == 0.002 and m.omega_cut == 0.001
    o = oracle_lib.Oracle(m)
    rng = np.random.default_rng(1)
    L = o.eph_lists(dests=rng.choice(m.n_c, 24, replace=False))
    est = np.diff(L["off"]).mean() * 2 * m.n_c
    assert 0.8e8 < est < 2.0e8  # "~1e8 e-ph channels"


def test_graphene_optical_phonon_decay_rate(oracle_lib):
    """Linearised 300 K out-scattering rate of the top optical branch, by a finite difference
    of the literal ph-ph integral at Bose-Einstein populations: within [0.1, 1] 1/ps."""
    m = ri.graphene()
    o = oracle_lib.Oracle(m)
    full = o.pp_full_index()
    y = m.y0()
    rng = np.random.default_rng(0)
    rates = []
    for a in rng.choice(m.N_q_pp, 6, replace=False):
        p = int(full[5 * m.N_q_pp + a])
        mask = np.zeros(m.n_ph, np.uint8)
        mask[p] = 1
        em = np.zeros(m.n_c, np.uint8)
        r0 = o.rhs_literal(y, oracle_lib.SLOW, em, mask)[m.n_c + p]
        y1 = y.copy()
        y1[m.n_c + p] += 1e-3
        r1 = o.rhs_literal(y1, oracle_lib.SLOW, em, mask)[m.n_c + p]
        rates.append(-(r1 - r0) / 1e-3)
    assert 0.1 < np.mean(rates) < 1.0


def test_initial_states_are_inversion_symmetric():
    for m in (ri.toy2d(), ri.graphene(n=60)):
        nx, ny, _ = m.nq
        q = np.arange(m.N_q)
        x, y = q % nx, q // nx
        qi = ((-y) % ny) * nx + (-x) % nx
        for nu in range(m.nmodes):
            assert np.array_equal(m.N0[nu * m.N_q + q], m.N0[nu * m.N_q + qi])
            assert np.array_equal(m.ph_omega[nu * m.N_q + q], m.ph_omega[nu * m.N_q + qi])


def test_silicon_like_model_shape(oracle_lib):
    """The silicon-like 3D model (fold 2): states within the 0.4 eV window of three ellipsoidal
    valley pairs, each band holding both valleys of its axis in equal numbers; ph-ph channels
    exist on the full q-grid (carrier conservation is checked with the other models)."""
    m = ri.silicon(16)
    assert m.dim == 3 and m.fold == 2 and m.nq == (8, 8, 8)
    assert (m.e_eps <= 0.4).all() and (m.e_eps >= 0).all()
    assert sorted(set(m.e_band.tolist())) == [0, 1, 2]
    for b in range(3):
        kb = m.e_k[m.e_band == b][:, b]
        lo = (kb < m.nk[b] // 2).sum()
        assert lo > 0 and abs(2 * lo - kb.shape[0]) <= kb.shape[0] // 4
    o = oracle_lib.Oracle(m)
    assert o.pp_lists()["off"][-1] > 0
