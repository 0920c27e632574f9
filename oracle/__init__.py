"""FP64 CPU oracle for the rt-BTE collision integrals and time integrators.

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and the
cpu_baseline / reference legs of bench.py.  The product path (the CUDA library and
its Python binding) never imports this package, and this package never imports the
product.  Both consume the seeded model tables from ``rtbte_inputs``.

Parity pins for every function live in tests/test_oracle_*.py; the one function
without an independent pin (the adaptive controller's constants, which the paper
leaves to ARKODE's defaults) is marked "parity unpinned" below.

Python wrapper over oracle/rtbte_oracle.c (plain C, FP64, OpenMP over destinations
only, so results do not depend on the thread count).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import sys
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rtbte_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "librtbte_oracle.so")
_lock = threading.Lock()
_lib = None

EPH, PHE, PHPH = 1, 2, 4
FAST, SLOW, ALL = EPH | PHE, PHPH, EPH | PHE | PHPH
RK4, BS32, ZON43, KW3 = 0, 1, 2, 3
HBAR = 6.582119569e-4  # eV*ps, CODATA (restated here; the oracle takes it as an input)


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc, -O2, IEEE semantics, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


class OrModel(C.Structure):
    _fields_ = [("dim", C.c_int32), ("fold", C.c_int32), ("nbands", C.c_int32), ("nmodes", C.c_int32),
                ("nk", C.c_int32 * 3), ("nq", C.c_int32 * 3),
                ("n_c", C.c_int32), ("pp_stride", C.c_int32), ("lut_bits", C.c_int32), ("pad0", C.c_int32),
                ("e_band", C.c_void_p), ("e_k", C.c_void_p), ("e_eps", C.c_void_p), ("ph_omega", C.c_void_p),
                ("g2_coef", C.c_void_p), ("lut", C.c_void_p),
                ("v3_coef", C.c_double), ("sigma_eph", C.c_double), ("sigma_pp", C.c_double),
                ("omega_cut", C.c_double), ("hbar", C.c_double),
                ("g2_seed", C.c_uint64), ("v3_seed", C.c_uint64)]


class OrProblem(C.Structure):
    _fields_ = [("m", C.c_void_p),
                ("eph_off", C.c_void_p), ("eph_src", C.c_void_p), ("eph_ph", C.c_void_p), ("eph_W", C.c_void_p),
                ("phe_off", C.c_void_p), ("phe_dst", C.c_void_p), ("phe_src", C.c_void_p), ("phe_W", C.c_void_p),
                ("n_pp", C.c_int64), ("pp_full", C.c_void_p), ("pp_off", C.c_void_p), ("pp_b", C.c_void_p),
                ("pp_c", C.c_void_p), ("pp_W", C.c_void_p),
                ("parts", C.c_uint), ("forcing", C.c_void_p), ("nrhs", C.c_int64)]


class OrErkOpts(C.Structure):
    _fields_ = [("method", C.c_int), ("pid_sign_mode", C.c_int), ("rtol", C.c_double), ("atol", C.c_void_p),
                ("h0", C.c_double), ("hmin", C.c_double), ("hmax", C.c_double), ("max_steps", C.c_int64),
                ("a1", C.c_double), ("a2", C.c_double), ("a3", C.c_double),
                ("safety", C.c_double), ("growth", C.c_double), ("growth_first", C.c_double),
                ("etamxf", C.c_double), ("etamin", C.c_double), ("small_nef", C.c_int), ("max_nef", C.c_int)]


class OrStats(C.Structure):
    _fields_ = [("steps", C.c_int64), ("attempts", C.c_int64), ("fails", C.c_int64), ("rhs_evals", C.c_int64),
                ("rhs_slow", C.c_int64), ("slow_steps", C.c_int64), ("t", C.c_double), ("h_last", C.c_double),
                ("h_next", C.c_double), ("status", C.c_int), ("slow_fails", C.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class OrSlowOpts(C.Structure):
    _fields_ = [("hs0", C.c_double), ("safety", C.c_double), ("fac_min", C.c_double), ("fac_max", C.c_double),
                ("fast_scale", C.c_double), ("max_fail", C.c_int)]


def slow_opts(hs0, safety=0.9, fac_min=0.2, fac_max=5.0, fast_scale=0.1, max_fail=7):
    """Slow-step control of the tolerance-chosen MRI (library constants; not in the paper)."""
    o = OrSlowOpts()
    o.hs0, o.safety, o.fac_min, o.fac_max, o.fast_scale, o.max_fail = hs0, safety, fac_min, fac_max, fast_scale, max_fail
    return o


RHS_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_double, C.POINTER(C.c_double), C.POINTER(C.c_double))


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = C.CDLL(build())
            L = _lib
            vp, i64, i32, dbl = C.c_void_p, C.c_int64, C.c_int, C.c_double
            L.or_eph_count.argtypes = [vp, i32, vp, vp]
            L.or_eph_fill.argtypes = [vp, i32, vp, vp, vp, vp, vp]
            L.or_phe_count.argtypes = [vp, i32, vp, vp]
            L.or_phe_fill.argtypes = [vp, i32, vp, vp, vp, vp, vp]
            L.or_pp_size.argtypes = [vp]
            L.or_pp_size.restype = C.c_long
            L.or_pp_full_index.argtypes = [vp, vp]
            L.or_pp_count.argtypes = [vp, i32, vp, vp]
            L.or_pp_fill.argtypes = [vp, i32, vp, vp, vp, vp, vp]
            L.or_rhs_literal.argtypes = [vp, vp, vp, C.c_uint, vp, vp]
            L.or_rhs_lists.argtypes = [vp, vp, vp, C.c_uint]
            for fn in ("or_F_em", "or_F_abs", "or_G_em", "or_G_abs"):
                getattr(L, fn).argtypes = [dbl, dbl, dbl]
                getattr(L, fn).restype = dbl
            L.or_gauss_delta.argtypes = [dbl, dbl]
            L.or_gauss_delta.restype = dbl
            L.or_tableau_get.argtypes = [i32, vp, vp, vp, vp, vp, vp]
            L.or_wrms.argtypes = [C.c_long, vp, vp, dbl, vp]
            L.or_wrms.restype = dbl
            L.or_erk_solve.argtypes = [vp, vp, C.c_long, dbl, dbl, vp, vp, vp, vp]
            L.or_rk4_solve.argtypes = [vp, vp, C.c_long, dbl, dbl, dbl, vp, vp]
            L.or_mri_solve.argtypes = [vp, vp, vp, vp, C.c_long, dbl, dbl, dbl, vp, vp, vp]
            L.or_mri_adapt_solve.argtypes = [vp, vp, vp, vp, C.c_long, dbl, dbl, vp, vp, vp, vp]
            L.or_split_rk4_solve.argtypes = [vp, vp, vp, vp, C.c_long, dbl, dbl, dbl, dbl, vp, vp]
            L.or_mis_coef.argtypes = [i32, vp, vp]
            L.or_num_threads.restype = i32
            L.or_set_threads.argtypes = [i32]
        return _lib


def _p(a):
    return None if a is None else a.ctypes.data


class Oracle:
    """Oracle bound to one model (keeps the numpy arrays alive for the C side)."""

    def __init__(self, model):
        self.model = model
        m = model
        self._keep = [np.ascontiguousarray(m.e_band, np.int32), np.ascontiguousarray(m.e_k, np.int32),
                      np.ascontiguousarray(m.e_eps, np.float64), np.ascontiguousarray(m.ph_omega, np.float64),
                      np.ascontiguousarray(m.g2_coef, np.float64), np.ascontiguousarray(m.lut, np.float64)]
        eb, ek, ee, om, g2, lut = self._keep
        s = OrModel()
        s.dim, s.fold, s.nbands, s.nmodes = m.dim, m.fold, m.nbands, m.nmodes
        for i in range(3):
            s.nk[i] = m.nk[i]
            s.nq[i] = m.nq[i]
        s.n_c, s.pp_stride, s.lut_bits = m.n_c, m.pp_stride, m.lut_bits
        s.e_band, s.e_k, s.e_eps, s.ph_omega = _p(eb), _p(ek), _p(ee), _p(om)
        s.g2_coef, s.lut = _p(g2), _p(lut)
        s.v3_coef, s.sigma_eph, s.sigma_pp, s.omega_cut, s.hbar = (m.v3_coef, m.sigma_eph, m.sigma_pp,
                                                                    m.omega_cut, HBAR)
        s.g2_seed, s.v3_seed = m.g2_seed, m.v3_seed
        self.s = s
        self.ptr = C.addressof(s)
        self.lists = None

    # ---- channel lists -------------------------------------------------
    def eph_lists(self, dests=None):
        """e-ph CSR lists for `dests` (all electron states if None): off[2n+1] (emission,
        absorption per destination), src, ph, W (FP64)."""
        L = lib()
        d = None if dests is None else np.ascontiguousarray(dests, np.int32)
        n = self.model.n_c if d is None else d.shape[0]
        cnt = np.zeros(2 * n, np.int64)
        L.or_eph_count(self.ptr, n, _p(d), _p(cnt))
        off = np.zeros(2 * n + 1, np.int64)
        np.cumsum(cnt, out=off[1:])
        E = int(off[-1])
        src, ph, W = np.zeros(E, np.int32), np.zeros(E, np.int32), np.zeros(E, np.float64)
        L.or_eph_fill(self.ptr, n, _p(d), _p(off), _p(src), _p(ph), _p(W))
        return dict(off=off, src=src, ph=ph, W=W)

    def phe_lists(self, phonons=None):
        """ph-e CSR lists (one segment per phonon): off[n+1], dst, src, W (FP64, with the
        (4 pi/hbar)(1/N_k) prefactor of the ph-e integral)."""
        L = lib()
        q = None if phonons is None else np.ascontiguousarray(phonons, np.int64)
        n = self.model.n_ph if q is None else q.shape[0]
        cnt = np.zeros(n, np.int64)
        L.or_phe_count(self.ptr, n, _p(q), _p(cnt))
        off = np.zeros(n + 1, np.int64)
        np.cumsum(cnt, out=off[1:])
        E = int(off[-1])
        dst, src, W = np.zeros(E, np.int32), np.zeros(E, np.int32), np.zeros(E, np.float64)
        L.or_phe_fill(self.ptr, n, _p(q), _p(off), _p(dst), _p(src), _p(W))
        return dict(off=off, dst=dst, src=src, W=W)

    def pp_full_index(self):
        L = lib()
        M = int(L.or_pp_size(self.ptr))
        out = np.zeros(M, np.int64)
        L.or_pp_full_index(self.ptr, _p(out))
        return out

    def pp_lists(self, dests=None):
        """ph-ph CSR lists on the sub-lattice: off[2n+1] (emission pairs b<=c, absorption),
        b, c (sub-lattice indices), W (FP64, including the pair/absorption factors)."""
        L = lib()
        full = self.pp_full_index()
        d = None if dests is None else np.ascontiguousarray(dests, np.int64)
        n = full.shape[0] if d is None else d.shape[0]
        cnt = np.zeros(2 * n, np.int64)
        L.or_pp_count(self.ptr, n, _p(d), _p(cnt))
        off = np.zeros(2 * n + 1, np.int64)
        np.cumsum(cnt, out=off[1:])
        E = int(off[-1])
        b, c, W = np.zeros(E, np.int32), np.zeros(E, np.int32), np.zeros(E, np.float64)
        L.or_pp_fill(self.ptr, n, _p(d), _p(off), _p(b), _p(c), _p(W))
        return dict(off=off, b=b, c=c, W=W, full=full)

    def pp_rates(self, y):
        """Linearised ph-ph rates (Eq. ph-ph differentiated in the destination population):
        for every sub-lattice phonon a, -dI_a/dN_a = sum_em W (N_b + N_c + 1) + sum_abs W (N_c - N_b)
        over its stored channels (W with the pair and absorption factors).  Returns a
        state-size vector, 0 outside the sub-lattice rows."""
        y = np.ascontiguousarray(y, np.float64)
        m = self.model
        L = self.lists["pp"] if self.lists is not None and self.lists.get("pp") is not None else self.pp_lists()
        N = y[m.n_c:][L["full"]]  # populations of the sub-lattice, compact order
        out = np.zeros_like(y)
        off, b, c, W = L["off"], L["b"], L["c"], L["W"]
        for a in range(L["full"].shape[0]):
            e0, e1, e2 = off[2 * a], off[2 * a + 1], off[2 * a + 2]
            em = np.sum(W[e0:e1] * (N[b[e0:e1]] + N[c[e0:e1]] + 1.0))
            ab = np.sum(W[e1:e2] * (N[c[e1:e2]] - N[b[e1:e2]]))
            out[m.n_c + L["full"][a]] = em + ab
        return out

    def build_lists(self, parts=ALL):
        self.lists = dict(eph=self.eph_lists() if parts & (EPH | PHE) else None,
                          phe=self.phe_lists() if parts & PHE else None,
                          pp=self.pp_lists() if (parts & PHPH) and self.model.pp_stride > 0 else None)
        self._problem = None
        return self.lists

    # ---- right-hand side -------------------------------------------------
    def rhs_literal(self, y, parts=ALL, emask=None, pmask=None):
        """RHS straight from Eq. e-ph / Eq. ph-ph (no stored list)."""
        y = np.ascontiguousarray(y, np.float64)
        out = np.zeros_like(y)
        em = None if emask is None else np.ascontiguousarray(emask, np.uint8)
        pm = None if pmask is None else np.ascontiguousarray(pmask, np.uint8)
        lib().or_rhs_literal(self.ptr, _p(y), _p(out), parts, _p(em), _p(pm))
        return out

    def problem(self, parts=ALL, forcing=None):
        if self.lists is None:
            self.build_lists()
        P = OrProblem()
        P.m = self.ptr
        e, h, q = self.lists["eph"], self.lists["phe"], self.lists["pp"]
        if e is not None:
            P.eph_off, P.eph_src, P.eph_ph, P.eph_W = _p(e["off"]), _p(e["src"]), _p(e["ph"]), _p(e["W"])
        else:
            # an empty e-ph list: every destination has two empty segments
            self._empty_off = np.zeros(2 * self.model.n_c + 1, np.int64)
            P.eph_off = _p(self._empty_off)
        if h is not None:
            P.phe_off, P.phe_dst, P.phe_src, P.phe_W = _p(h["off"]), _p(h["dst"]), _p(h["src"]), _p(h["W"])
        if q is not None:
            P.n_pp = q["full"].shape[0]
            P.pp_full, P.pp_off, P.pp_b, P.pp_c, P.pp_W = (_p(q["full"]), _p(q["off"]), _p(q["b"]),
                                                           _p(q["c"]), _p(q["W"]))
        P.parts = parts
        P.forcing = _p(forcing)
        return P

    def rhs(self, y, parts=ALL):
        """RHS from the oracle's stored lists (FP64, literal F/G forms)."""
        P = self.problem(parts)
        y = np.ascontiguousarray(y, np.float64)
        out = np.zeros_like(y)
        lib().or_rhs_lists(C.addressof(P), _p(y), _p(out), parts)
        return out

    # ---- integrators -----------------------------------------------------
    def _fn(self):
        return C.cast(lib().or_problem_rhs, C.c_void_p).value

    def atol_vec(self, atol_c, atol_ph):
        m = self.model
        return np.concatenate([np.full(m.n_c, atol_c), np.full(m.n_ph, atol_ph)]).astype(np.float64)

    def rk4(self, y0, t0, t1, h, parts=ALL):
        P = self.problem(parts)
        y = np.array(y0, np.float64, copy=True)
        st = OrStats()
        lib().or_rk4_solve(self._fn(), C.addressof(P), y.shape[0], t0, t1, h, _p(y), C.addressof(st))
        return y, st.as_dict()

    def erk(self, y0, t0, t1, method=ZON43, rtol=1e-5, atol_c=1e-9, atol_ph=1e-12, parts=ALL, **kw):
        P = self.problem(parts)
        y = np.array(y0, np.float64, copy=True)
        atol = self.atol_vec(atol_c, atol_ph)
        o = erk_opts(method, rtol, atol, **kw)
        st = OrStats()
        h = C.c_double(kw.get("h0", 0.0))
        lib().or_erk_solve(self._fn(), C.addressof(P), y.shape[0], t0, t1, _p(y), C.addressof(o),
                           C.addressof(h), C.addressof(st))
        return y, st.as_dict()

    def mri(self, y0, t0, t1, hs, rtol=1e-5, atol_c=1e-9, atol_ph=1e-12, **kw):
        Pf = self.problem(FAST)
        Ps = self.problem(SLOW)
        y = np.array(y0, np.float64, copy=True)
        atol = self.atol_vec(atol_c, atol_ph)
        o = erk_opts(kw.pop("method", ZON43), rtol, atol, **kw)
        st = OrStats()
        fn = self._fn()
        lib().or_mri_solve(fn, C.addressof(Pf), fn, C.addressof(Ps), y.shape[0], t0, t1, hs, _p(y),
                           C.addressof(o), C.addressof(st))
        return y, st.as_dict()

    def mri_adapt(self, y0, t0, t1, hs0, rtol=1e-5, atol_c=1e-9, atol_ph=1e-12, slow=None, **kw):
        """MRI with the slow step chosen from (rtol, atol) by step doubling; `slow`: dict of
        slow_opts keywords other than hs0."""
        Pf = self.problem(FAST)
        Ps = self.problem(SLOW)
        y = np.array(y0, np.float64, copy=True)
        atol = self.atol_vec(atol_c, atol_ph)
        o = erk_opts(kw.pop("method", ZON43), rtol, atol, **kw)
        so = slow_opts(hs0, **(slow or {}))
        st = OrStats()
        fn = self._fn()
        lib().or_mri_adapt_solve(fn, C.addressof(Pf), fn, C.addressof(Ps), y.shape[0], t0, t1, C.addressof(so),
                                 _p(y), C.addressof(o), C.addressof(st))
        return y, st.as_dict()

    def split_rk4(self, y0, t0, t1, hs, hf):
        Pf = self.problem(FAST)
        Ps = self.problem(SLOW)
        y = np.array(y0, np.float64, copy=True)
        st = OrStats()
        fn = self._fn()
        lib().or_split_rk4_solve(fn, C.addressof(Pf), fn, C.addressof(Ps), y.shape[0], t0, t1, hs, hf,
                                 _p(y), C.addressof(st))
        return y, st.as_dict()


def erk_opts(method, rtol, atol, h0=0.0, hmin=0.0, hmax=0.0, max_steps=10 ** 7, a1=0.58, a2=0.21, a3=0.1,
             pid_sign_mode=0, safety=0.96, growth=20.0, growth_first=1e4, etamxf=0.3, etamin=0.1,
             small_nef=2, max_nef=7):
    """Adaptive-ERK options.  The PID gains are the paper's (a1=.58, a2=.21, a3=.1, p*=p).
    The remaining constants (safety, growth limits, failure reductions) are not in the
    paper; they follow ARKODE's documented defaults.  Parity unpinned: no ARKODE run is
    available to compare step sequences against."""
    o = OrErkOpts()
    o.method, o.pid_sign_mode, o.rtol = method, pid_sign_mode, rtol
    o._atol = np.ascontiguousarray(atol, np.float64)
    o.atol = _p(o._atol)
    o.h0, o.hmin, o.hmax, o.max_steps = h0, hmin, hmax, max_steps
    o.a1, o.a2, o.a3 = a1, a2, a3
    o.safety, o.growth, o.growth_first, o.etamxf, o.etamin = safety, growth, growth_first, etamxf, etamin
    o.small_nef, o.max_nef = small_nef, max_nef
    return o


# ---- generic-ODE entry points (Python callbacks), used by the order tests ----
def _wrap_py(f, n):
    def cb(user, t, y, ydot):
        yy = np.ctypeslib.as_array(y, shape=(n,))
        out = np.ctypeslib.as_array(ydot, shape=(n,))
        out[:] = f(t, yy)
    return RHS_FN(cb)


def ode_rk4(f, y0, t0, t1, h):
    y = np.array(y0, np.float64, copy=True)
    cb = _wrap_py(f, y.shape[0])
    st = OrStats()
    lib().or_rk4_solve(C.cast(cb, C.c_void_p), None, y.shape[0], t0, t1, h, _p(y), C.addressof(st))
    return y, st.as_dict()


def ode_erk(f, y0, t0, t1, method, rtol, atol, **kw):
    y = np.array(y0, np.float64, copy=True)
    n = y.shape[0]
    cb = _wrap_py(f, n)
    o = erk_opts(method, rtol, np.broadcast_to(np.asarray(atol, np.float64), (n,)).copy(), **kw)
    st = OrStats()
    h = C.c_double(kw.get("h0", 0.0))
    lib().or_erk_solve(C.cast(cb, C.c_void_p), None, n, t0, t1, _p(y), C.addressof(o), C.addressof(h),
                       C.addressof(st))
    return y, st.as_dict()


def ode_mri(ff, fs, y0, t0, t1, hs, rtol, atol, **kw):
    y = np.array(y0, np.float64, copy=True)
    n = y.shape[0]
    cf, cs = _wrap_py(ff, n), _wrap_py(fs, n)
    o = erk_opts(kw.pop("method", ZON43), rtol, np.broadcast_to(np.asarray(atol, np.float64), (n,)).copy(), **kw)
    st = OrStats()
    lib().or_mri_solve(C.cast(cf, C.c_void_p), None, C.cast(cs, C.c_void_p), None, n, t0, t1, hs, _p(y),
                       C.addressof(o), C.addressof(st))
    return y, st.as_dict()


def ode_mri_adapt(ff, fs, y0, t0, t1, hs0, rtol, atol, slow=None, **kw):
    y = np.array(y0, np.float64, copy=True)
    n = y.shape[0]
    cf, cs = _wrap_py(ff, n), _wrap_py(fs, n)
    o = erk_opts(kw.pop("method", ZON43), rtol, np.broadcast_to(np.asarray(atol, np.float64), (n,)).copy(), **kw)
    so = slow_opts(hs0, **(slow or {}))
    st = OrStats()
    lib().or_mri_adapt_solve(C.cast(cf, C.c_void_p), None, C.cast(cs, C.c_void_p), None, n, t0, t1,
                             C.addressof(so), _p(y), C.addressof(o), C.addressof(st))
    return y, st.as_dict()


def ode_split_rk4(ff, fs, y0, t0, t1, hs, hf):
    y = np.array(y0, np.float64, copy=True)
    n = y.shape[0]
    cf, cs = _wrap_py(ff, n), _wrap_py(fs, n)
    st = OrStats()
    lib().or_split_rk4_solve(C.cast(cf, C.c_void_p), None, C.cast(cs, C.c_void_p), None, n, t0, t1, hs, hf,
                             _p(y), C.addressof(st))
    return y, st.as_dict()


def tableau(method):
    S, p = C.c_int(), C.c_int()
    A, b, bt, c = np.zeros(36), np.zeros(6), np.zeros(6), np.zeros(6)
    lib().or_tableau_get(method, C.byref(S), C.byref(p), _p(A), _p(b), _p(bt), _p(c))
    s = S.value
    return dict(S=s, p=p.value, A=A.reshape(6, 6)[:s, :s].copy(), b=b[:s].copy(), bt=bt[:s].copy(),
                c=c[:s].copy())


def mis_coef():
    Om, ch = np.zeros(36), np.zeros(6)
    lib().or_mis_coef(KW3, _p(Om), _p(ch))
    return Om.reshape(6, 6)[:4, :3].copy(), ch[:4].copy()


def F_em(f, fp, N):
    return lib().or_F_em(f, fp, N)


def F_abs(f, fp, N):
    return lib().or_F_abs(f, fp, N)


def G_em(N, N1, N2):
    return lib().or_G_em(N, N1, N2)


def G_abs(N, N1, N2):
    return lib().or_G_abs(N, N1, N2)


def gauss_delta(E, sigma):
    return lib().or_gauss_delta(E, sigma)


def threads():
    return int(lib().or_num_threads())


def set_threads(n):
    lib().or_set_threads(int(n))
