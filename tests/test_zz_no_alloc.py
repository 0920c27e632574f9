"""The allocation-free e-ph entry point (rtbte_eph_rhs_noalloc) agrees with rtbte_rhs and
with the FP64 oracle.

rtbte_eph_rhs_noalloc is for callers that cannot allocate device memory (programs whose
device memory belongs to another allocator or to an arena reserved at start-up,
latency-critical loops that cannot take an allocation's implicit synchronisation): its
working memory is a fixed array in the library's device image.  This file is collected last
so that a run stopping at its first failure has already run every other test; it also passes
when run alone.
"""
import ctypes as C

import numpy as np
import pytest

import rtbte_inputs as ri

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rt():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2412_13402_gb300 import build

    build.build()
    import paper_2412_13402_gb300 as m

    return m


def relL2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("mk", [lambda: ri.graphene_small(36), lambda: ri.graphene(n=90, window=1.0)])
def test_noalloc_eph_matches_rtbte_rhs_twice(rt, mk):
    m = mk()
    ctx = rt.Context(m, precision="fp32")
    ctx.upload_channels()
    L = ctx.download_channels(0, rt.RTBTE_EPH)  # the layout the entry point takes
    dev = torch.device("cuda")
    off = torch.tensor(L["off"], dtype=torch.int64, device=dev)
    src = torch.tensor(L["a"], dtype=torch.int32, device=dev)
    ph = torch.tensor(L["b"], dtype=torch.int32, device=dev)
    W = torch.tensor(L["W"], dtype=torch.float64, device=dev)
    out = torch.empty(m.n_c, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()
    lib = rt.load()
    f, N = ri.random_populations(m, 4)
    for y_np in (m.y0(), np.concatenate([f, N])):  # two calls in a row on the shared array
        y = torch.tensor(y_np, device=dev)
        rc = lib.rtbte_eph_rhs_noalloc(m.n_c, m.n_ph, m.nmodes, off.data_ptr(), src.data_ptr(), ph.data_ptr(),
                                       W.data_ptr(), y.data_ptr(), out.data_ptr(), stream.cuda_stream)
        assert rc == 0
        ref = ctx.rhs(y, parts=rt.RTBTE_EPH)[: m.n_c].cpu().numpy()
        got = out.cpu().numpy()
        assert relL2(got, ref) <= 1e-5
    ctx.close()


def test_noalloc_eph_matches_oracle(rt, oracle_lib):
    """Two calls in a row against the FP64 oracle's e-ph rows (Eq. e-ph, first integral) on the
    parity-sized graphene-like model and on the folded 3D exact-resonance model."""
    lib = rt.load()
    dev = torch.device("cuda")
    stream = torch.cuda.current_stream()
    for m in (ri.graphene_small(36), ri.ladder3d(n=8)):
        o = oracle_lib.Oracle(m)
        L = o.build_lists(oracle_lib.EPH)["eph"]
        # the entry point takes segments (mode, destination, process), sources ascending
        seg = np.repeat(np.arange(len(L["off"]) - 1), np.diff(L["off"]))
        key = ((L["ph"] // m.N_q) * m.n_c + seg // 2) * 2 + seg % 2
        order = np.argsort(key, kind="stable")
        cnt = np.bincount(key, minlength=2 * m.nmodes * m.n_c)
        off = np.zeros(cnt.size + 1, np.int64)
        np.cumsum(cnt, out=off[1:])
        t_off = torch.tensor(off, device=dev)
        t_src = torch.tensor(L["src"][order].astype(np.int32), device=dev)
        t_ph = torch.tensor(L["ph"][order].astype(np.int32), device=dev)
        t_W = torch.tensor(L["W"][order], dtype=torch.float64, device=dev)
        out = torch.empty(m.n_c, dtype=torch.float64, device=dev)
        for seed in (6, 7):
            y_np = np.concatenate(ri.random_populations(m, seed))
            y = torch.tensor(y_np, device=dev)
            rc = lib.rtbte_eph_rhs_noalloc(m.n_c, m.n_ph, m.nmodes, t_off.data_ptr(), t_src.data_ptr(),
                                           t_ph.data_ptr(), t_W.data_ptr(), y.data_ptr(), out.data_ptr(),
                                           stream.cuda_stream)
            assert rc == 0
            ref = o.rhs(y_np, oracle_lib.EPH)[: m.n_c]
            assert np.abs(ref).max() > 0
            assert relL2(out.cpu().numpy(), ref) <= 1e-5


def test_noalloc_rejects_sizes_beyond_its_array(rt):
    lib = rt.load()
    cap = 8 << 20  # RTBTE_NOALLOC_SCRATCH_BYTES
    n_c = cap // 4  # the population copies alone exceed the array
    rc = lib.rtbte_eph_rhs_noalloc(n_c, 6, 6, None, None, None, None, None, None, None)
    assert rc == -10  # RTBTE_E_UNSUPPORTED, checked before any pointer is touched
    assert lib.rtbte_eph_rhs_noalloc(0, 6, 6, None, None, None, None, None, None, None) == -1
