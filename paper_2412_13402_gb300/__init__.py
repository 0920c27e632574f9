"""Python binding of librtbte, the GB300 (sm_103a) library for the coupled electron/phonon
real-time Boltzmann equation of arXiv 2412.13402.

Argument marshalling only: every step of the right-hand side and of the integrators runs
in the library's CUDA kernels.  The functions ``rtbte_create``, ``rtbte_upload_channels``,
``rtbte_rhs``, ``rtbte_advance_to`` and ``rtbte_destroy`` mirror the C ABI of
include/rtbte.h one to one; ``Context`` is a convenience wrapper that builds the
descriptors from model tables and takes PyTorch tensors for device memory and streams.

There is no CPU fallback: importing works without a GPU, but any call raises if the
compiled library is missing or no CUDA device is present.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librtbte.so")

RTBTE_OK = 0
STATUS = {0: "ok", -1: "invalid argument", -2: "out of memory", -3: "CUDA error", -4: "too many steps",
          -5: "step size underflow", -6: "repeated error-test failures", -7: "non-finite value",
          -8: "device wait timed out", -9: "call out of order", -10: "unsupported size"}
RTBTE_EPH, RTBTE_PHE, RTBTE_PHPH = 1, 2, 4
RTBTE_FAST, RTBTE_SLOW, RTBTE_ALL = 3, 4, 7
RTBTE_PREC_FP32_COMP, RTBTE_PREC_FP64 = 0, 1
RTBTE_CH_BUILD, RTBTE_CH_PREBUILT, RTBTE_CH_COUNT = 0, 1, 2
RTBTE_RK4, RTBTE_BS32, RTBTE_ZON43, RTBTE_MRI_KW3, RTBTE_SPLIT_RK4, RTBTE_MRI_ADAPT = 0, 1, 2, 3, 4, 5
HBAR_EV_PS = 6.582119569e-4

EXPORTS = ["rtbte_desc_defaults", "rtbte_integ_defaults", "rtbte_create", "rtbte_upload_channels", "rtbte_rhs",
           "rtbte_advance_to", "rtbte_get_controller", "rtbte_set_controller", "rtbte_phph_rates", "rtbte_get_sizes", "rtbte_row_entries", "rtbte_download_channels", "rtbte_download_segments", "rtbte_set_stream",
           "rtbte_autotune", "rtbte_get_tuning", "rtbte_set_graph_mode", "rtbte_set_kernel_timing", "rtbte_kernel_time", "rtbte_launch_count", "rtbte_last_error",
           "rtbte_status_string", "rtbte_eph_rhs_noalloc", "rtbte_surrogate_create", "rtbte_surrogate_collect",
           "rtbte_surrogate_train", "rtbte_surrogate_predict", "rtbte_surrogate_loss_grad",
           "rtbte_surrogate_num_params", "rtbte_surrogate_get_params", "rtbte_surrogate_set_params",
           "rtbte_surrogate_stats", "rtbte_set_surrogate", "rtbte_surrogate_set_gemm", "rtbte_surrogate_destroy",
           "rtbte_destroy"]


class InstanceDesc(C.Structure):
    _fields_ = [("dim", C.c_int32), ("fold", C.c_int32), ("nbands", C.c_int32), ("nmodes", C.c_int32),
                ("nk", C.c_int32 * 3), ("nq", C.c_int32 * 3), ("n_c", C.c_int32), ("pp_stride", C.c_int32),
                ("lut_bits", C.c_int32), ("reserved0", C.c_int32),
                ("e_band", C.c_void_p), ("e_k", C.c_void_p), ("e_eps", C.c_void_p), ("ph_omega", C.c_void_p),
                ("lut", C.c_void_p), ("g2_coef", C.c_void_p),
                ("v3_coef", C.c_double), ("sigma_eph", C.c_double), ("sigma_pp", C.c_double),
                ("omega_cut", C.c_double), ("g2_seed", C.c_uint64), ("v3_seed", C.c_uint64)]


class Desc(C.Structure):
    _fields_ = [("n_instances", C.c_int32), ("precision", C.c_int32), ("inst", C.c_void_p), ("hbar", C.c_double),
                ("stream", C.c_void_p), ("device", C.c_int32), ("eph_q_blocks", C.c_int32),
                ("row_begin", C.c_int64), ("row_end", C.c_int64)]


class Channels(C.Structure):
    _fields_ = [("mode", C.c_int32), ("reserved", C.c_int32)] + [
        (n, C.c_void_p) for n in ("eph_off", "eph_src", "eph_ph", "eph_W", "phe_off", "phe_dst", "phe_src", "phe_W",
                                  "pp_off", "pp_b", "pp_c", "pp_W")]


class Sizes(C.Structure):
    _fields_ = [(n, C.c_int64) for n in ("n_c", "n_ph", "n_pp", "y_offset", "n_y_total", "eph_entries",
                                         "phe_entries", "pp_entries", "eph_stored", "phe_stored", "pp_stored",
                                         "work_items", "channel_bytes", "eph_q_blocks")]


class Integ(C.Structure):
    _fields_ = [("method", C.c_int32), ("fast_method", C.c_int32), ("t0", C.c_double), ("h", C.c_double),
                ("h_s", C.c_double), ("rtol", C.c_double), ("atol_c", C.c_double), ("atol_ph", C.c_double),
                ("h0", C.c_double), ("hmin", C.c_double), ("hmax", C.c_double), ("max_steps", C.c_int64),
                ("a1", C.c_double), ("a2", C.c_double), ("a3", C.c_double), ("pid_sign_mode", C.c_int32),
                ("max_nef", C.c_int32), ("safety", C.c_double), ("growth", C.c_double),
                ("growth_first", C.c_double), ("etamxf", C.c_double), ("etamin", C.c_double),
                ("small_nef", C.c_int32), ("chunk", C.c_int32), ("resume", C.c_int32), ("reserved2", C.c_int32),
                ("fast_tol_scale", C.c_double), ("slow_safety", C.c_double), ("slow_fac_min", C.c_double),
                ("slow_fac_max", C.c_double), ("slow_max_fail", C.c_int32), ("reserved3", C.c_int32)]


class Controller(C.Structure):
    _fields_ = [("t", C.c_double), ("h", C.c_double), ("eps1", C.c_double), ("eps2", C.c_double),
                ("first", C.c_int32), ("nef", C.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Stats(C.Structure):
    _fields_ = [("steps", C.c_int64), ("attempts", C.c_int64), ("fails", C.c_int64), ("rhs_full", C.c_int64),
                ("rhs_fast", C.c_int64), ("rhs_slow", C.c_int64), ("slow_steps", C.c_int64), ("t", C.c_double),
                ("h_last", C.c_double), ("h_next", C.c_double), ("status", C.c_int32),
                ("surrogate_fallbacks", C.c_int32), ("slow_exact", C.c_int64), ("slow_surrogate", C.c_int64),
                ("judge_err_max", C.c_double), ("range_violations", C.c_int64), ("slow_fails", C.c_int64),
                ("h_slow_next", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lock = threading.Lock()
_lib = None


class RtbteError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)} ({code}): {msg}")
        self.code = code


def load():
    """Load librtbte.so (built in-tree by paper_2412_13402_gb300.build).  Raises if missing."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is not built: run `python -c 'import __graft_entry__ as g; g.build()'`")
        L = C.CDLL(LIB_PATH)
        vp, i32, i64, dbl = C.c_void_p, C.c_int, C.c_int64, C.c_double
        L.rtbte_desc_defaults.argtypes = [vp]
        L.rtbte_integ_defaults.argtypes = [vp]
        L.rtbte_create.argtypes = [vp, C.POINTER(vp)]
        L.rtbte_upload_channels.argtypes = [vp, i32, vp]
        L.rtbte_rhs.argtypes = [vp, dbl, vp, vp, C.c_uint]
        L.rtbte_advance_to.argtypes = [vp, dbl, vp, vp, vp]
        L.rtbte_phph_rates.argtypes = [vp, vp, vp]
        L.rtbte_get_controller.argtypes = [vp, i32, vp]
        L.rtbte_set_controller.argtypes = [vp, i32, vp]
        L.rtbte_get_sizes.argtypes = [vp, i32, vp]
        L.rtbte_row_entries.argtypes = [vp, i32, vp]
        L.rtbte_download_channels.argtypes = [vp, i32, C.c_uint, vp, vp, vp, vp]
        L.rtbte_download_segments.argtypes = [vp, i32, C.c_uint, i64, i64, vp, vp, vp, vp, i64]
        L.rtbte_set_stream.argtypes = [vp, vp]
        L.rtbte_autotune.argtypes = [vp, C.c_uint, vp]
        L.rtbte_get_tuning.argtypes = [vp, vp, vp, vp]
        L.rtbte_set_graph_mode.argtypes = [vp, i32]
        L.rtbte_set_kernel_timing.argtypes = [vp, i32]
        L.rtbte_kernel_time.argtypes = [vp, vp, vp]
        L.rtbte_launch_count.argtypes = [vp]
        L.rtbte_launch_count.restype = i64
        L.rtbte_last_error.argtypes = [vp]
        L.rtbte_last_error.restype = C.c_char_p
        L.rtbte_status_string.argtypes = [i32]
        L.rtbte_status_string.restype = C.c_char_p
        L.rtbte_eph_rhs_noalloc.argtypes = [C.c_int32, i64, C.c_int32, vp, vp, vp, vp, vp, vp, vp]
        fp = C.c_float
        L.rtbte_surrogate_create.argtypes = [vp, i32, i32, i32, C.c_uint64, C.POINTER(vp)]
        L.rtbte_surrogate_collect.argtypes = [vp, vp, i32]
        L.rtbte_surrogate_train.argtypes = [vp, i32, i32, i32, fp, vp]
        L.rtbte_surrogate_predict.argtypes = [vp, vp, vp]
        L.rtbte_surrogate_loss_grad.argtypes = [vp, vp, vp, i32, vp, vp, vp]
        L.rtbte_surrogate_num_params.argtypes = [vp]
        L.rtbte_surrogate_num_params.restype = i64
        L.rtbte_surrogate_get_params.argtypes = [vp, vp]
        L.rtbte_surrogate_set_params.argtypes = [vp, vp]
        L.rtbte_surrogate_stats.argtypes = [vp, vp, vp, vp, vp]
        L.rtbte_surrogate_stats.restype = None
        L.rtbte_set_surrogate.argtypes = [vp, vp, i32, dbl]
        L.rtbte_surrogate_set_gemm.argtypes = [vp, i32]
        L.rtbte_surrogate_destroy.argtypes = [vp]
        L.rtbte_surrogate_destroy.restype = None
        L.rtbte_destroy.argtypes = [vp]
        L.rtbte_destroy.restype = None
        _lib = L
        return L


def _check(ctx, rc):
    if rc != RTBTE_OK:
        msg = load().rtbte_last_error(ctx).decode() if ctx else ""
        raise RtbteError(rc, msg)


# ---- one-to-one wrappers of the C ABI -------------------------------------------------
def rtbte_create(desc: Desc) -> int:
    h = C.c_void_p()
    rc = load().rtbte_create(C.addressof(desc), C.byref(h))
    _check(None, rc)
    return h.value


def rtbte_upload_channels(ctx: int, inst: int, ch: Channels) -> None:
    _check(ctx, load().rtbte_upload_channels(ctx, inst, C.addressof(ch)))


def rtbte_rhs(ctx: int, t: float, y_ptr: int, ydot_ptr: int, parts: int) -> None:
    _check(ctx, load().rtbte_rhs(ctx, t, y_ptr, ydot_ptr, parts))


def rtbte_advance_to(ctx: int, t_out: float, y_ptr: int, opt: Integ, st: Stats) -> int:
    rc = load().rtbte_advance_to(ctx, t_out, y_ptr, C.addressof(opt), C.addressof(st))
    if rc < 0 and rc not in (-4, -5, -6, -7):
        _check(ctx, rc)
    return rc


def rtbte_destroy(ctx: int) -> None:
    load().rtbte_destroy(ctx)


def _p(a):
    return a.ctypes.data if a is not None else None


def instance_desc(model, keep: list) -> InstanceDesc:
    """Descriptor of one model (rtbte_inputs.Model or any object with the same fields);
    the numpy arrays referenced are appended to `keep` so they outlive the call."""
    arrs = [np.ascontiguousarray(model.e_band, np.int32), np.ascontiguousarray(model.e_k, np.int32),
            np.ascontiguousarray(model.e_eps, np.float64), np.ascontiguousarray(model.ph_omega, np.float64),
            np.ascontiguousarray(model.lut, np.float64), np.ascontiguousarray(model.g2_coef, np.float64)]
    keep.extend(arrs)
    d = InstanceDesc()
    d.dim, d.fold, d.nbands, d.nmodes = model.dim, model.fold, model.nbands, model.nmodes
    for i in range(3):
        d.nk[i], d.nq[i] = model.nk[i], model.nq[i]
    d.n_c, d.pp_stride, d.lut_bits = model.n_c, model.pp_stride, model.lut_bits
    d.e_band, d.e_k, d.e_eps, d.ph_omega, d.lut, d.g2_coef = [_p(a) for a in arrs]
    d.v3_coef, d.sigma_eph, d.sigma_pp, d.omega_cut = model.v3_coef, model.sigma_eph, model.sigma_pp, model.omega_cut
    d.g2_seed, d.v3_seed = model.g2_seed, model.v3_seed
    return d


def integ_options(**kw) -> Integ:
    o = Integ()
    load().rtbte_integ_defaults(C.addressof(o))
    names = {"method": {"rk4": 0, "bs32": 1, "zon43": 2, "mri": 3, "split_rk4": 4, "mri_adapt": 5}}
    for k, v in kw.items():
        if k in names and isinstance(v, str):
            v = names[k][v]
        if k == "fast_method" and isinstance(v, str):
            v = names["method"][v]
        setattr(o, k, v)
    return o


class Context:
    """One library context over one or more independent instances sharing a state vector."""

    def __init__(self, models, precision: str = "fp32", stream=None, device: int = 0, hbar: float = HBAR_EV_PS,
                 eph_q_blocks: int = 0, row_range: tuple | None = None):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("librtbte needs a CUDA device")
        load()
        self.models = list(models) if isinstance(models, (list, tuple)) else [models]
        self._keep = []
        descs = (InstanceDesc * len(self.models))()
        for i, m in enumerate(self.models):
            descs[i] = instance_desc(m, self._keep)
        self._descs = descs
        d = Desc()
        load().rtbte_desc_defaults(C.addressof(d))
        d.n_instances = len(self.models)
        d.precision = RTBTE_PREC_FP64 if precision == "fp64" else RTBTE_PREC_FP32_COMP
        d.inst = C.addressof(descs)
        d.hbar = hbar
        torch.cuda.set_device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(device)
        d.stream = self.stream.cuda_stream
        d.device = device
        d.eph_q_blocks = eph_q_blocks
        if row_range is not None:  # evaluate only the state rows [begin, end) (see rtbte_desc)
            d.row_begin, d.row_end = int(row_range[0]), int(row_range[1])
        self.row_range = row_range
        self.device = device
        self.ctx = rtbte_create(d)

    # ---- setup --------------------------------------------------------------------
    def upload_channels(self, inst: int = 0, prebuilt: dict | None = None, count_only: bool = False):
        """Build the channel lists on the device, or copy `prebuilt` host lists (dict with
        keys eph/phe/pp as produced by the oracle's list builders, FP64 weights), or with
        count_only only count every row's channels (for row_entries)."""
        ch = Channels()
        if count_only:
            ch.mode = RTBTE_CH_COUNT
        elif prebuilt is None:
            ch.mode = RTBTE_CH_BUILD
        else:
            ch.mode = RTBTE_CH_PREBUILT
            keep = []
            m = self.models[inst]
            e = prebuilt["eph"]
            # the library's e-ph segments are (mode, destination, process); regroup the
            # destination-major lists mode-blocked
            off, src, ph, W = _mode_blocked_eph(m, e)
            h = prebuilt["phe"]
            arrs = [off, src, ph, W, np.ascontiguousarray(h["off"], np.int64), np.ascontiguousarray(h["dst"], np.int32),
                    np.ascontiguousarray(h["src"], np.int32), np.ascontiguousarray(h["W"], np.float64)]
            q = prebuilt.get("pp")
            if q is not None:
                arrs += [np.ascontiguousarray(q["off"], np.int64), np.ascontiguousarray(q["b"], np.int32),
                         np.ascontiguousarray(q["c"], np.int32), np.ascontiguousarray(q["W"], np.float64)]
            else:
                arrs += [None] * 4
            keep.extend(arrs)
            (ch.eph_off, ch.eph_src, ch.eph_ph, ch.eph_W, ch.phe_off, ch.phe_dst, ch.phe_src, ch.phe_W,
             ch.pp_off, ch.pp_b, ch.pp_c, ch.pp_W) = [_p(a) for a in arrs]
        rtbte_upload_channels(self.ctx, inst, ch)

    def sizes(self, inst: int = 0) -> dict:
        s = Sizes()
        _check(self.ctx, load().rtbte_get_sizes(self.ctx, inst, C.addressof(s)))
        return {k: getattr(s, k) for k, _ in s._fields_}

    def row_entries(self, inst: int = 0) -> np.ndarray:
        """Logical channel entries per state row (the cost weights of row slices)."""
        m = self.models[inst]
        out = np.zeros(m.n_c + m.n_ph, np.int64)
        _check(self.ctx, load().rtbte_row_entries(self.ctx, inst, _p(out)))
        return out

    def download_channels(self, inst: int, which: int) -> dict:
        s = self.sizes(inst)
        m = self.models[inst]
        if which == RTBTE_EPH:
            nseg, E = 2 * m.nmodes * m.n_c, s["eph_entries"]
        elif which == RTBTE_PHE:
            nseg, E = m.n_ph, s["phe_entries"]
        else:
            nseg, E = 2 * m.n_pp, s["pp_entries"]
        off = np.zeros(nseg + 1, np.int64)
        a, b, W = np.zeros(max(E, 1), np.int32), np.zeros(max(E, 1), np.int32), np.zeros(max(E, 1), np.float64)
        _check(self.ctx, load().rtbte_download_channels(self.ctx, inst, which, _p(off), _p(a), _p(b), _p(W)))
        return dict(off=off, a=a[:E], b=b[:E], W=W[:E])

    def download_segments(self, inst: int, which: int, seg_begin: int, seg_end: int) -> dict:
        """Segments [seg_begin, seg_end) of download_channels' order only (large lists)."""
        L = load()
        off = np.zeros(seg_end - seg_begin + 1, np.int64)
        _check(self.ctx, L.rtbte_download_segments(self.ctx, inst, which, seg_begin, seg_end, _p(off), None, None,
                                                   None, 0))
        E = int(off[-1])
        a, b, W = np.zeros(max(E, 1), np.int32), np.zeros(max(E, 1), np.int32), np.zeros(max(E, 1), np.float64)
        _check(self.ctx, L.rtbte_download_segments(self.ctx, inst, which, seg_begin, seg_end, _p(off), _p(a), _p(b),
                                                   _p(W), E))
        return dict(off=off, a=a[:E], b=b[:E], W=W[:E])

    # ---- compute ------------------------------------------------------------------
    @property
    def n_y(self) -> int:
        return self.sizes(0)["n_y_total"]

    def rhs(self, y, ydot=None, parts: int = RTBTE_ALL, t: float = 0.0):
        """ydot = RHS(y) for FP64 torch tensors (both on the device, or both on the host)."""
        import torch

        if ydot is None:
            ydot = torch.empty_like(y)
        assert y.dtype == torch.float64 and ydot.dtype == torch.float64 and y.is_contiguous() and ydot.is_contiguous()
        rtbte_rhs(self.ctx, t, y.data_ptr(), ydot.data_ptr(), parts)
        return ydot

    def advance_to(self, t_out: float, y, options: "Integ | None" = None, stats: "Stats | None" = None, **opts):
        """Integrate the state y (FP64 torch tensor on the device, or in host memory -- pinned
        copies fastest -- which the library stages in and out) to t_out.  With keyword options:
        returns a dict of the statistics.  With a prebuilt `options` (integ_options(...)) and a
        reusable `stats` object: fills and returns `stats` (no per-call allocation, for tight
        driver loops)."""
        import torch

        assert y.dtype == torch.float64 and y.is_contiguous()
        if options is not None:
            st = stats if stats is not None else Stats()
            rtbte_advance_to(self.ctx, t_out, y.data_ptr(), options, st)
            return st
        o = integ_options(**opts)
        st = Stats()
        rc = rtbte_advance_to(self.ctx, t_out, y.data_ptr(), o, st)
        d = st.as_dict()
        d["rc"] = rc
        return d

    def get_controller(self, inst: int = 0) -> Controller:
        """Step-size controller state of an instance (checkpointing)."""
        c = Controller()
        _check(self.ctx, load().rtbte_get_controller(self.ctx, inst, C.byref(c)))
        return c

    def set_controller(self, c: Controller, inst: int = 0):
        """Restore a saved controller state; the next advance_to with resume=1 continues it."""
        _check(self.ctx, load().rtbte_set_controller(self.ctx, inst, C.byref(c)))

    def phph_rates(self, y):
        """Linearised ph-ph rates -dI^{ph-ph}_a/dN_a on the sub-lattice rows (0 elsewhere)."""
        import torch

        assert y.is_cuda and y.dtype == torch.float64 and y.is_contiguous()
        out = torch.empty_like(y)
        _check(self.ctx, load().rtbte_phph_rates(self.ctx, y.data_ptr(), out.data_ptr()))
        return out

    def autotune(self, parts: int = RTBTE_ALL) -> int:
        """Pick the collision kernel's work-split weight by timing; returns the chosen weight."""
        w = C.c_int()
        _check(self.ctx, load().rtbte_autotune(self.ctx, parts, C.byref(w)))
        return w.value

    def tuning(self) -> dict:
        """Launch parameters of the collision kernel in use (see rtbte_autotune)."""
        w, d, sh = C.c_int32(), C.c_int32(), C.c_double()
        _check(self.ctx, load().rtbte_get_tuning(self.ctx, C.byref(w), C.byref(d), C.byref(sh)))
        return {"item_weight": w.value, "prefetch_items": d.value, "static_share": sh.value}

    def set_graph_mode(self, use_graphs: bool):
        """Attempts through the device-loop graph (default) or by direct launches."""
        _check(self.ctx, load().rtbte_set_graph_mode(self.ctx, int(bool(use_graphs))))

    def set_kernel_timing(self, enable: bool):
        _check(self.ctx, load().rtbte_set_kernel_timing(self.ctx, int(bool(enable))))

    def kernel_time(self):
        """(summed milliseconds, launches) of collision-kernel launches timed since the last query."""
        ms, n = C.c_double(), C.c_int64()
        _check(self.ctx, load().rtbte_kernel_time(self.ctx, C.byref(ms), C.byref(n)))
        return ms.value, n.value

    def launch_count(self) -> int:
        return int(load().rtbte_launch_count(self.ctx))

    def set_stream(self, stream):
        self.stream = stream
        _check(self.ctx, load().rtbte_set_stream(self.ctx, stream.cuda_stream))

    def close(self):
        if getattr(self, "ctx", None):
            rtbte_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _mode_blocked_eph(model, e):
    """Destination-major e-ph lists (segments (d, proc), entries sorted by (mode, src)) ->
    the library's mode-blocked logical order (segments (mode, d, proc), entries by src)."""
    nc, nm, Nq = model.n_c, model.nmodes, model.N_q
    off_in = np.asarray(e["off"], np.int64)
    src, ph, W = np.asarray(e["src"]), np.asarray(e["ph"]), np.asarray(e["W"])
    nu = ph // Nq
    seg_in = np.repeat(np.arange(2 * nc), np.diff(off_in))
    d, proc = seg_in // 2, seg_in % 2
    seg_out = (nu * nc + d) * 2 + proc
    order = np.argsort(seg_out, kind="stable")
    cnt = np.bincount(seg_out, minlength=2 * nm * nc)
    off = np.zeros(2 * nm * nc + 1, np.int64)
    np.cumsum(cnt, out=off[1:])
    return (off, np.ascontiguousarray(src[order], np.int32), np.ascontiguousarray(ph[order], np.int32),
            np.ascontiguousarray(W[order], np.float64))


class Surrogate:
    """Neural-operator surrogate of the ph-ph integral of instance `inst` of a Context
    (2-D sub-lattice, one channel per branch).  Training and inference run in librtbte's
    BF16 tensor-core kernels; this class only marshals arguments."""

    def __init__(self, ctx: "Context", inst: int = 0, width: int = 64, capacity: int = 1024, seed: int = 0):
        self.context = ctx
        m = ctx.models[inst]
        self.nmodes = m.nmodes
        self.nq_s = tuple(n // m.pp_stride if n > 1 else 1 for n in m.nq)
        h = C.c_void_p()
        _check(ctx.ctx, load().rtbte_surrogate_create(ctx.ctx, inst, width, capacity, seed, C.byref(h)))
        self.h = h

    def _chk(self, rc):
        if rc != RTBTE_OK:
            raise RtbteError(rc, load().rtbte_last_error(self.context.ctx).decode())

    def collect(self, y, trajectory: int = 0):
        """Store the pair (N, exact I^{ph-ph}) at the device state y (FP64 [n_y])."""
        self._chk(load().rtbte_surrogate_collect(self.h, y.data_ptr(), trajectory))

    def train(self, steps: int, batch: int, lr: float, horizon: int = 0) -> float:
        """Adam steps on single pairs (horizon 0) or on differences of pairs of one trajectory
        at most `horizon` collections apart; returns the last minibatch loss."""
        loss = C.c_float()
        self._chk(load().rtbte_surrogate_train(self.h, steps, batch, horizon, lr, C.byref(loss)))
        return loss.value

    def predict(self, y):
        import torch

        out = torch.empty_like(y)
        self._chk(load().rtbte_surrogate_predict(self.h, y.data_ptr(), out.data_ptr()))
        return out

    @property
    def num_params(self) -> int:
        return int(load().rtbte_surrogate_num_params(self.h))

    def get_params(self) -> np.ndarray:
        out = np.empty(self.num_params, dtype=np.float32)
        self._chk(load().rtbte_surrogate_get_params(self.h, out.ctypes.data))
        return out

    def set_params(self, flat: np.ndarray):
        flat = np.ascontiguousarray(flat, dtype=np.float32)
        assert flat.size == self.num_params
        self._chk(load().rtbte_surrogate_set_params(self.h, flat.ctypes.data))

    def loss_grad(self, x: np.ndarray, t: np.ndarray):
        """(loss, flat gradients, output) for normalised host batches x, t [B, ny, nx, C]."""
        x = np.ascontiguousarray(x, dtype=np.float32)
        t = np.ascontiguousarray(t, dtype=np.float32)
        assert x.shape == t.shape and x.shape[1:] == (self.nq_s[1], self.nq_s[0], self.nmodes)
        loss = C.c_float()
        g = np.empty(self.num_params, dtype=np.float32)
        out = np.empty_like(x)
        self._chk(load().rtbte_surrogate_loss_grad(self.h, x.ctypes.data, t.ctypes.data, x.shape[0], C.byref(loss),
                                                   g.ctypes.data, out.ctypes.data))
        return loss.value, g, out

    def stats(self):
        mu, sd, so = (np.zeros(self.nmodes, dtype=np.float32) for _ in range(3))
        n = C.c_int()
        load().rtbte_surrogate_stats(self.h, mu.ctypes.data, sd.ctypes.data, so.ctypes.data, C.byref(n))
        return mu, sd, so, n.value

    def set_gemm(self, engine: int):
        """0: tcgen05 tensor cores where both operands are K-major (default); 1: mma.sync for all."""
        self._chk(load().rtbte_surrogate_set_gemm(self.h, engine))

    def attach(self, judge_period: int = 10, judge_tol: float = 1e-2):
        """Use this surrogate for the slow part of the context's MRI integrations."""
        self._chk(load().rtbte_set_surrogate(self.context.ctx, self.h, judge_period, judge_tol))

    def detach(self):
        self._chk(load().rtbte_set_surrogate(self.context.ctx, None, 1, 1.0))

    def close(self):
        if getattr(self, "h", None):
            load().rtbte_surrogate_destroy(self.h)
            self.h = None
