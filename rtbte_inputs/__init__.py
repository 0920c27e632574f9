"""Seeded synthetic inputs for the coupled electron/phonon real-time Boltzmann equation.

This module is shared by the CUDA path and by the CPU oracle.  It holds the *model
definition only*: momentum grids, band energies, phonon frequencies, coupling
look-up tables, seeds and initial populations.  It contains none of the method's
arithmetic (no channel enumeration, no delta functions, no collision integrals,
no time stepping); those live separately in ``oracle/`` and in the CUDA library.

Units: energies in eV (phonon tables hold hbar*omega in eV), time in ps, momenta
in 1/Angstrom.  The paper's first-principles inputs (DFT bands, DFPT e-ph matrix
elements, TDEP force constants; Methods A) are replaced by smooth model
dispersions and lognormal coupling strengths drawn from a counter-based hash.

Layouts (all arrays C-contiguous):
  electron state s (windowed):   e_band[s], e_k[s, 3] (grid indices), e_eps[s]
      states are ordered by (band, k_lin), k_lin = (kz*nky + ky)*nkx + kx
  phonon state p = nu*N_q + q_lin, q_lin = (qz*nqy + qy)*nqx + qx
      ph_omega[p] = hbar*omega (eV)
  state vector y = [f_s (N_c values); N_p (N_ph values)]   (Eq. state_vec)
"""
from __future__ import annotations

import dataclasses
import math
from dataclasses import dataclass, field

import numpy as np

HBAR_EV_PS = 6.582119569e-4      # eV*ps (CODATA)
KB_EV_K = 8.617333262e-5         # eV/K (CODATA)
HB2_2ME = 3.80998                # hbar^2/(2 m_e) in eV*Angstrom^2
HBAR_V_GRAPHENE = 6.582119569    # hbar * 1e6 m/s in eV*Angstrom

SEED_BASE = 13402 * 10


def fermi_dirac(e, mu, T):
    x = (np.asarray(e, dtype=np.float64) - mu) / (KB_EV_K * T)
    return 0.5 * (1.0 - np.tanh(0.5 * x))


def bose_einstein(w, T):
    w = np.asarray(w, dtype=np.float64)
    out = np.zeros_like(w)
    pos = w > 0
    out[pos] = 1.0 / np.expm1(w[pos] / (KB_EV_K * T))
    return out


def lognormal_lut(bits: int, log_sd: float) -> np.ndarray:
    """Shape factors exp(s*z_i) at the 2^bits equiprobable midpoints of N(0,1).

    A coupling strength is median * lut[i] with i taken from the top bits of a
    64-bit hash of the process key, i.e. a discretised lognormal draw that every
    implementation reproduces bit for bit from integer arithmetic alone.
    """
    from scipy.special import ndtri

    L = 1 << bits
    z = ndtri((np.arange(L, dtype=np.float64) + 0.5) / L)
    return np.exp(log_sd * z)


def _min_image(i, n):
    i = np.asarray(i, dtype=np.int64)
    d = np.where(i > n // 2, i - n, i)
    return d


def _grid_coords(n3):
    nx, ny, nz = n3
    iz, iy, ix = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return np.stack([ix.ravel(), iy.ravel(), iz.ravel()], axis=1).astype(np.int64)


def _shape_s(n3, dim):
    """s(q) = sqrt((1/D) sum_c sin^2(pi |d_c| / n_c)) in [0, 1], from min-image |d_c| so that
    s(-q) equals s(q) bit for bit."""
    c = _grid_coords(n3)
    acc = np.zeros(c.shape[0], dtype=np.float64)
    for ax in range(dim):
        n = n3[ax]
        d = np.abs(_min_image(c[:, ax], n)).astype(np.float64)
        acc += np.sin(np.pi * d / n) ** 2
    return np.sqrt(acc / dim)


@dataclass
class Model:
    name: str
    dim: int
    nk: tuple
    nq: tuple
    fold: int
    nbands: int
    e_band: np.ndarray
    e_k: np.ndarray
    e_eps: np.ndarray
    nmodes: int
    ph_omega: np.ndarray
    pp_stride: int
    sigma_eph: float
    sigma_pp: float
    omega_cut: float
    g2_seed: int
    v3_seed: int
    g2_coef: np.ndarray
    v3_coef: float
    lut_bits: int
    lut: np.ndarray
    f0: np.ndarray
    N0: np.ndarray
    integ: dict = field(default_factory=dict)
    note: str = ""

    # ---- derived sizes -------------------------------------------------
    @property
    def n_c(self) -> int:
        return int(self.e_eps.shape[0])

    @property
    def N_k(self) -> int:
        return int(np.prod(self.nk))

    @property
    def N_q(self) -> int:
        return int(np.prod(self.nq))

    @property
    def n_ph(self) -> int:
        return int(self.nmodes * self.N_q)

    @property
    def n_y(self) -> int:
        return self.n_c + self.n_ph

    @property
    def nq_pp(self) -> tuple:
        if self.pp_stride <= 0:
            return (0, 0, 0)
        return tuple(int(n // self.pp_stride) if n > 1 else 1 for n in self.nq)

    @property
    def N_q_pp(self) -> int:
        return int(np.prod(self.nq_pp)) if self.pp_stride > 0 else 0

    @property
    def n_pp(self) -> int:
        return self.nmodes * self.N_q_pp

    def y0(self) -> np.ndarray:
        return np.concatenate([self.f0, self.N0]).astype(np.float64)

    def frozen(self) -> np.ndarray:
        return self.ph_omega < self.omega_cut

    def pp_full_index(self) -> np.ndarray:
        """Full phonon index p of every ph-ph sub-lattice state a = nu*N_q_pp + qs_lin."""
        if self.pp_stride <= 0:
            return np.zeros(0, dtype=np.int64)
        s = self.pp_stride
        c = _grid_coords(self.nq_pp) * np.array([s if n > 1 else 1 for n in self.nq])
        nx, ny, _ = self.nq
        qlin = (c[:, 2] * ny + c[:, 1]) * nx + c[:, 0]
        return (np.arange(self.nmodes)[:, None] * self.N_q + qlin[None, :]).ravel()

    def with_populations(self, f0=None, N0=None) -> "Model":
        return dataclasses.replace(
            self,
            f0=self.f0 if f0 is None else np.ascontiguousarray(f0, dtype=np.float64),
            N0=self.N0 if N0 is None else np.ascontiguousarray(N0, dtype=np.float64),
        )


def _electron_states(nk, nbands, eps_fn, keep_fn):
    """Windowed electron states ordered by (band, k_lin)."""
    c = _grid_coords(nk)
    bands, ks, eps = [], [], []
    for b in range(nbands):
        e = eps_fn(b, c)
        keep = keep_fn(b, e)
        bands.append(np.full(int(keep.sum()), b, dtype=np.int32))
        ks.append(c[keep].astype(np.int32))
        eps.append(e[keep])
    return (np.concatenate(bands), np.ascontiguousarray(np.concatenate(ks), dtype=np.int32),
            np.ascontiguousarray(np.concatenate(eps), dtype=np.float64))


def _kvec(c, nk, dk):
    out = np.zeros(c.shape, dtype=np.float64)
    for ax in range(3):
        if nk[ax] > 1:
            out[:, ax] = _min_image(c[:, ax], nk[ax]).astype(np.float64) * dk[ax]
    # |d| is used through squares, so k(-d) and k(d) agree bit for bit.
    return out


# ---------------------------------------------------------------------------
# Workloads (synthetic stand-ins for the paper's graphene and silicon runs)
# ---------------------------------------------------------------------------

def toy2d(n: int = 12, seed: int = SEED_BASE + 0) -> Model:
    """Toy 2D model, e-ph only: one parabolic band (m* = 0.2 m_e) on an n x n periodic
    k-grid with lattice constant 20 Angstrom, three phonon modes on the same grid
    (acoustic 10 meV zone-corner scale, flat 40 and 80 meV), sigma = 10 meV,
    hot-carrier Gaussian at 0.3 eV over a 300 K Fermi-Dirac, Bose-Einstein phonons."""
    nk = (n, n, 1)
    a = 20.0
    dk = (2 * np.pi / (n * a),) * 2 + (0.0,)

    def eps_fn(b, c):
        k = _kvec(c, nk, dk)
        return (HB2_2ME / 0.2) * (k[:, 0] ** 2 + k[:, 1] ** 2 + k[:, 2] ** 2)

    e_band, e_k, e_eps = _electron_states(nk, 1, eps_fn, lambda b, e: np.ones(e.shape, bool))
    s = _shape_s(nk, 2)
    omega = np.concatenate([0.010 * s, np.full_like(s, 0.040), np.full_like(s, 0.080)])
    T = 300.0
    f0 = fermi_dirac(e_eps, -0.1, T) + 0.1 * np.exp(-((e_eps - 0.3) ** 2) / (2 * 0.05 ** 2))
    N0 = bose_einstein(omega, T)
    N0[omega < 0.001] = 0.0
    return Model(
        name=f"toy2d_{n}", dim=2, nk=nk, nq=nk, fold=1, nbands=1,
        e_band=e_band, e_k=e_k, e_eps=e_eps, nmodes=3, ph_omega=omega, pp_stride=0,
        sigma_eph=0.010, sigma_pp=0.002, omega_cut=0.001,
        g2_seed=seed, v3_seed=seed + 1000003, g2_coef=np.full(3, 1e-3), v3_coef=0.0,
        lut_bits=12, lut=lognormal_lut(12, 1.0), f0=f0, N0=N0,
        integ=dict(t_end=1.0, rk4_h=[5e-3, 2e-3, 1e-3, 5e-4, 1e-4, 1e-5],
                   bs3_rtol=1e-8, atol_c=1e-15, atol_ph=1e-15),
        note="config 1: toy 2D e-ph only, FP64",
    )


GRAPHENE_MODES = (("LA", "ac", 0.120), ("TA", "ac", 0.090), ("ZA", "ac", 0.060),
                  ("ZO", "op", 0.110), ("TO", "op", 0.190), ("LO", "op", 0.196))

# |V3|^2 median (eV^3 scale absorbed) chosen so that the 300 K out-scattering rate of the
# top optical branch on the 60 x 60 ph-ph sub-lattice is ~0.3 1/ps (optical phonons decay
# in 1-10 ps); tests/test_oracle_model.py checks the rate lies in [0.1, 1] 1/ps.
GRAPHENE_V3_COEF = 8.0e-9


def graphene(n: int = 180, window: float = 1.0, k_max_eV: float = 1.0, pp_stride: int = 3,
             seed: int = SEED_BASE + 1, T: float = 300.0, E_x: float = 1.0, amp: float = 0.3,
             width: float = 0.05, sigma_eph: float = 0.020, sigma_pp: float = 0.002,
             v3_coef: float | None = None) -> Model:
    """Graphene-like 2D model: two Dirac bands eps = +-hbar v |k| (v = 1e6 m/s) on an n x n
    torus of side 4 k_max (k_max = k_max_eV / hbar v), states with |eps| <= window kept,
    six phonon branches (LA/TA/ZA acoustic, ZO/TO/LO optical) on the same q-grid, ph-ph on
    the stride-`pp_stride` sub-lattice, hot carriers at +-E_x/2 over 300 K Fermi-Dirac."""
    nk = (n, n, 1)
    L = 4.0 * k_max_eV / HBAR_V_GRAPHENE
    dk = (L / n, L / n, 0.0)

    def eps_fn(b, c):
        k = _kvec(c, nk, dk)
        kk = np.sqrt(k[:, 0] ** 2 + k[:, 1] ** 2)
        return (1.0 if b == 1 else -1.0) * HBAR_V_GRAPHENE * kk

    e_band, e_k, e_eps = _electron_states(nk, 2, eps_fn, lambda b, e: np.abs(e) <= window)
    s = _shape_s(nk, 2)
    om = []
    for _, kind, w in GRAPHENE_MODES:
        om.append(w * s if kind == "ac" else w - 0.004 * s * s)
    omega = np.concatenate(om)
    G = lambda x: np.exp(-(x ** 2) / (2 * width ** 2))
    f0 = np.where(e_band == 1,
                  fermi_dirac(e_eps, 0.0, T) + amp * G(e_eps - E_x / 2),
                  fermi_dirac(e_eps, 0.0, T) - amp * G(e_eps + E_x / 2))
    N0 = bose_einstein(omega, T)
    N0[omega < 0.001] = 0.0
    return Model(
        name=f"graphene_{n}", dim=2, nk=nk, nq=nk, fold=1, nbands=2,
        e_band=e_band, e_k=e_k, e_eps=e_eps, nmodes=6, ph_omega=omega, pp_stride=pp_stride,
        sigma_eph=sigma_eph, sigma_pp=sigma_pp, omega_cut=0.001,
        g2_seed=seed, v3_seed=seed + 1000003, g2_coef=np.full(6, 1e-3),
        v3_coef=GRAPHENE_V3_COEF if v3_coef is None else v3_coef,
        lut_bits=12, lut=lognormal_lut(12, 1.0), f0=np.ascontiguousarray(f0), N0=N0,
        integ=dict(t_end=100.0, h_s=0.020, rtol=1e-5, atol_c=1e-9, atol_ph=1e-12),
        note="config 2: graphene-like 2D, plain GPU form",
    )


def graphene_small(n: int = 36, seed: int = SEED_BASE + 11) -> Model:
    """Parity-sized graphene-like model: the same physics on a coarse grid (the window is
    scaled with the grid so the state count stays small), wider broadening so that the
    coarse energy grid still yields resonant channels."""
    return graphene(n=n, window=1.0, k_max_eV=1.0, pp_stride=3, seed=seed,
                    sigma_eph=0.040, sigma_pp=0.008)


def ladder(n: int = 6, quantum: float = 2.0 ** -5, T: float = 300.0, mu: float = 0.0,
           seed: int = 7, pp_stride: int = 1, with_pp: bool = True) -> Model:
    """Exact-resonance test model.  Electron energies are integer multiples of `quantum`
    (a power of two, so every energy difference is exact in binary floating point),
    phonon branches are dispersionless at 1, 2 and 3 quanta, and sigma = quantum/4 so a
    channel is either exactly resonant or outside the 3-sigma window.  With Fermi-Dirac
    electrons and Bose-Einstein phonons at one temperature every collision term vanishes."""
    nk = (n, n, 1)
    c = _grid_coords(nk)

    def eps_fn(b, cc):
        dx = np.abs(_min_image(cc[:, 0], n))
        dy = np.abs(_min_image(cc[:, 1], n))
        return (dx + dy + 3 * b).astype(np.float64) * quantum

    e_band, e_k, e_eps = _electron_states(nk, 2, eps_fn, lambda b, e: np.ones(e.shape, bool))
    Nq = n * n
    omega = np.concatenate([np.full(Nq, 1 * quantum), np.full(Nq, 2 * quantum),
                            np.full(Nq, 3 * quantum)])
    f0 = fermi_dirac(e_eps, mu, T)
    N0 = bose_einstein(omega, T)
    return Model(
        name=f"ladder_{n}", dim=2, nk=nk, nq=nk, fold=1, nbands=2,
        e_band=e_band, e_k=e_k, e_eps=e_eps, nmodes=3, ph_omega=omega,
        pp_stride=pp_stride if with_pp else 0,
        sigma_eph=quantum / 4, sigma_pp=quantum / 4, omega_cut=0.001,
        g2_seed=seed, v3_seed=seed + 1000003, g2_coef=np.array([1e-3, 2e-3, 0.5e-3]),
        v3_coef=1e-5, lut_bits=8, lut=lognormal_lut(8, 1.0), f0=f0, N0=N0,
        note="exact-resonance detailed-balance model",
    )


def ladder3d(n: int = 8, quantum: float = 2.0 ** -5, T: float = 300.0, mu: float = 0.0,
             seed: int = 17, pp_stride: int = 1, with_pp: bool = True) -> Model:
    """Exact-resonance test model on a folded 3D grid: electrons on an n^3 k-grid, phonons on
    the (n/2)^3 q-grid (fold 2, so N_k = 8 N_q), electron energies (|dx| + |dy| + |dz| + 3 b)
    quanta from the min-image grid displacement, dispersionless phonon branches at 1, 2 and
    3 quanta, sigma = quantum/4.  Every kept channel is exactly resonant (a power-of-two
    quantum makes every energy difference exact in binary floating point), so populations of
    one temperature give a vanishing RHS and the total energy is conserved exactly for any
    populations -- on a grid where the e-ph (1/N_q) and ph-e (1/N_k) normalisations differ."""
    assert n % 2 == 0
    nk = (n, n, n)
    nq = (n // 2,) * 3

    def eps_fn(b, cc):
        d = sum(np.abs(_min_image(cc[:, ax], n)) for ax in range(3))
        return (d + 3 * b).astype(np.float64) * quantum

    e_band, e_k, e_eps = _electron_states(nk, 2, eps_fn, lambda b, e: np.ones(e.shape, bool))
    Nq = int(np.prod(nq))
    omega = np.concatenate([np.full(Nq, 1 * quantum), np.full(Nq, 2 * quantum), np.full(Nq, 3 * quantum)])
    f0 = fermi_dirac(e_eps, mu, T)
    N0 = bose_einstein(omega, T)
    return Model(
        name=f"ladder3d_{n}_f2", dim=3, nk=nk, nq=nq, fold=2, nbands=2,
        e_band=e_band, e_k=e_k, e_eps=e_eps, nmodes=3, ph_omega=omega,
        pp_stride=pp_stride if with_pp else 0,
        sigma_eph=quantum / 4, sigma_pp=quantum / 4, omega_cut=0.001,
        g2_seed=seed, v3_seed=seed + 1000003, g2_coef=np.array([1e-3, 2e-3, 0.5e-3]),
        v3_coef=1e-5, lut_bits=8, lut=lognormal_lut(8, 1.0), f0=f0, N0=N0,
        note="exact-resonance detailed-balance model, folded 3D grid (N_k != N_q)",
    )


def tiny(n=(4, 4, 1), nbands: int = 2, nmodes: int = 3, fold: int = 1, pp_stride: int = 1,
         seed: int = 99, sigma_eph: float = 0.05, sigma_pp: float = 0.02,
         rng_seed: int = 5) -> Model:
    """Small random model for brute-force checks: random (inversion-symmetric) band energies
    and phonon frequencies on tiny 2D or 3D grids, random populations."""
    nk = tuple(n)
    dim = 3 if nk[2] > 1 else 2
    nq = tuple(max(1, x // fold) if x > 1 else 1 for x in nk)
    rng = np.random.default_rng(rng_seed)
    c = _grid_coords(nk)
    Nk = c.shape[0]

    # inversion-symmetric random energies: value depends on the min-image |d| pattern
    def sym_table(shape_n, scale, offset):
        cc = _grid_coords(shape_n)
        key = np.zeros(cc.shape[0], dtype=np.int64)
        for ax in range(3):
            d = np.abs(_min_image(cc[:, ax], shape_n[ax]))
            key = key * 1009 + d
        uniq, inv = np.unique(key, return_inverse=True)
        vals = offset + scale * rng.random(uniq.shape[0])
        return vals[inv]

    eps_list = [sym_table(nk, 0.4, -0.2 + 0.15 * b) for b in range(nbands)]

    def eps_fn(b, cc):
        return eps_list[b]

    e_band, e_k, e_eps = _electron_states(nk, nbands, eps_fn, lambda b, e: np.ones(e.shape, bool))
    om = [sym_table(nq, 0.08, 0.0005 + 0.02 * v) for v in range(nmodes)]
    omega = np.concatenate(om)
    f0 = rng.random(e_eps.shape[0]) * 0.9 + 0.05
    N0 = rng.random(omega.shape[0]) * 2.0
    return Model(
        name=f"tiny_{'x'.join(map(str, nk))}_f{fold}", dim=dim, nk=nk, nq=nq, fold=fold,
        nbands=nbands, e_band=e_band, e_k=e_k, e_eps=e_eps, nmodes=nmodes, ph_omega=omega,
        pp_stride=pp_stride, sigma_eph=sigma_eph, sigma_pp=sigma_pp, omega_cut=0.001,
        g2_seed=seed, v3_seed=seed + 1000003, g2_coef=np.linspace(1e-3, 2e-3, nmodes),
        v3_coef=1e-5, lut_bits=8, lut=lognormal_lut(8, 1.0), f0=f0, N0=N0,
        note="random brute-force model",
    )


SILICON_MODES = (("TA1", "ac", 0.020), ("TA2", "ac", 0.022), ("LA", "ac", 0.050),
                  ("TO1", "op", 0.060), ("TO2", "op", 0.061), ("LO", "op", 0.063))


def silicon(n: int = 32, fold: int = 2, window: float = 0.4, seed: int = SEED_BASE + 2, T: float = 300.0,
            E_x: float = 0.2, amp: float = 0.2, width: float = 0.03, sigma_eph: float | None = None,
            sigma_pp: float | None = None, v3_coef: float = 2.0e-8, pp_stride: int = 1) -> Model:
    """Bulk-silicon-like 3D model (the precision-study workload): three conduction bands, band b
    being the pair of ellipsoidal valleys on axis b at +-0.85 of the zone half-width (m_l = 0.92,
    m_t = 0.19, lattice 5.43 Angstrom, simple cubic zone), states within `window` of the band
    minimum on an n^3 k-grid; six phonon branches (two TA and one LA Debye-like acoustic, three
    flat ~60 meV optical) on the (n/fold)^3 q-grid, ph-ph on its stride-`pp_stride` sub-lattice
    (the full q-grid by default); hot electrons
    at E_x over a 300 K Fermi-Dirac tail.  Broadenings default to the paper's 5 meV and 1.1 meV
    scaled by 80/n and 40/(n/fold) so that coarse grids keep resonant channels."""
    nk = (n, n, n)
    nq = tuple(x // fold for x in nk)
    a = 5.43
    dk = (2 * np.pi / (n * a),) * 3
    k0 = 0.85 * np.pi / a  # valley centre on its axis

    def eps_fn(b, c):
        k = _kvec(c, nk, dk)
        kl = np.abs(k[:, b]) - k0
        kt2 = sum(k[:, ax] ** 2 for ax in range(3) if ax != b)
        return HB2_2ME * (kl ** 2 / 0.92 + kt2 / 0.19)

    e_band, e_k, e_eps = _electron_states(nk, 3, eps_fn, lambda b, e: e <= window)
    s = _shape_s(nq, 3)
    om = [w * s if kind == "ac" else w - 0.004 * s * s for _, kind, w in SILICON_MODES]
    omega = np.concatenate(om)
    f0 = fermi_dirac(e_eps, -0.15, T) + amp * np.exp(-((e_eps - E_x) ** 2) / (2 * width ** 2))
    N0 = bose_einstein(omega, T)
    N0[omega < 0.0002] = 0.0
    return Model(
        name=f"silicon_{n}_f{fold}", dim=3, nk=nk, nq=nq, fold=fold, nbands=3,
        e_band=e_band, e_k=e_k, e_eps=e_eps, nmodes=6, ph_omega=omega, pp_stride=pp_stride,
        sigma_eph=0.005 * 80.0 / n if sigma_eph is None else sigma_eph,
        sigma_pp=0.0011 * 40.0 / nq[0] if sigma_pp is None else sigma_pp, omega_cut=0.0002,
        g2_seed=seed, v3_seed=seed + 1000003, g2_coef=np.full(6, 1e-3), v3_coef=v3_coef,
        lut_bits=12, lut=lognormal_lut(12, 1.0), f0=np.ascontiguousarray(f0), N0=N0,
        integ=dict(t_end=20.0, h_s=0.050, rtol=1e-5, atol_c=1e-9, atol_ph=1e-11),
        note="config 3: silicon-like 3D, precision study (reduced grids)",
    )


def silicon_printed() -> Model:
    """The silicon-like workload at the printed grids: 80^3 k-grid, 0.4 eV window (36 321
    states), six branches on the 40^3 q-grid (384 000 phonons), fold 2, ph-ph on the stride-2
    sub-lattice (20^3 points, 48 000 phonons), the paper's 5 meV and 1.1 meV broadenings.
    About 1.2e9 e-ph, 0.6e9 ph-e and 0.37e9 ph-ph stored entries (17.6 GB in FP32)."""
    m = silicon(80, fold=2, pp_stride=2)
    m.name = "silicon_80_f2_pp2"
    m.note = "config 3: silicon-like 3D at the printed 80^3 / 40^3 grids, ph-ph on the stride-2 sub-lattice"
    return m


def ensemble(n_inst: int = 64, seed: int = SEED_BASE + 3, sides=tuple(range(24, 97, 3))) -> list:
    """Batched ensemble: independent graphene-like instances with uneven grids (side drawn
    uniformly from `sides`), excitation energies E_x ~ U[0.1, 1.0] eV and temperatures
    T ~ U[100, 500] K drawn from the seed.  Broadenings scale as sqrt(180/side) so that coarse
    grids keep resonant channels (sigma_eph = 20 meV and sigma_pp = 2 meV at side 180)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_inst):
        n = int(rng.choice(sides))
        E_x = float(rng.uniform(0.1, 1.0))
        T = float(rng.uniform(100.0, 500.0))
        f = math.sqrt(180.0 / n)
        m = graphene(n=n, window=1.0, seed=seed * 1000 + i, T=T, E_x=E_x, sigma_eph=0.020 * f, sigma_pp=0.002 * f)
        m.name = f"ensemble{i}_n{n}"
        m.note = f"config 4 instance {i}: side {n}, E_x {E_x:.3f} eV, T {T:.1f} K"
        out.append(m)
    return out


def random_populations(model: Model, seed: int, spread: float = 1.0):
    """Seeded random populations of the model's shape: f in (0.02, 0.98), N in (0, 3*spread),
    zero on frozen phonon states."""
    rng = np.random.default_rng(seed)
    f = 0.02 + 0.96 * rng.random(model.n_c)
    N = 3.0 * spread * rng.random(model.n_ph)
    N[model.frozen()] = 0.0
    return f, N


def by_name(name: str, **kw) -> Model:
    table = {"toy2d": toy2d, "graphene": graphene, "graphene_small": graphene_small,
             "ladder": ladder, "ladder3d": ladder3d, "tiny": tiny, "silicon": silicon, "silicon_printed": silicon_printed}
    return table[name](**kw)
