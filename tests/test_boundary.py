"""The C-ABI library builds for sm_103a, loads without a GPU, and exports every entry point
include/rtbte.h declares; descriptor layouts agree between the header and the binding.
No compute calls (CPU only)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="session")
def rtlib():
    from paper_2412_13402_gb300 import build

    build.build()
    import paper_2412_13402_gb300 as rt

    return rt


def declared_functions():
    txt = open(os.path.join(ROOT, "include", "rtbte.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(rtbte_[a-z_]+)\s*\(", txt)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("rtbte_create", "rtbte_upload_channels", "rtbte_rhs", "rtbte_advance_to", "rtbte_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol(rtlib):
    L = C.CDLL(rtlib.LIB_PATH)
    for n in declared_functions():
        assert hasattr(L, n), n
    assert sorted(rtlib.EXPORTS) == declared_functions()


def test_binding_layouts_match_the_header(rtlib):
    L = rtlib.load()
    o = rtlib.Integ()
    L.rtbte_integ_defaults(C.addressof(o))
    # the paper's PID gains (Methods B) and the documented defaults land in their fields
    assert (o.method, o.fast_method) == (rtlib.RTBTE_ZON43, rtlib.RTBTE_ZON43)
    assert (o.a1, o.a2, o.a3) == (0.58, 0.21, 0.1)
    assert (o.rtol, o.atol_c, o.atol_ph) == (1e-5, 1e-9, 1e-12)
    assert (o.safety, o.growth, o.growth_first, o.etamxf, o.etamin) == (0.96, 20.0, 1e4, 0.3, 0.1)
    assert (o.small_nef, o.max_nef, o.chunk, o.pid_sign_mode) == (2, 7, 0, 0)
    d = rtlib.Desc()
    L.rtbte_desc_defaults(C.addressof(d))
    assert (d.n_instances, d.precision, d.device) == (1, 0, 0)
    assert d.hbar == 6.582119569e-4


def test_struct_sizes_match_a_c_compiler(rtlib, tmp_path):
    import subprocess

    src = tmp_path / "sz.c"
    src.write_text('#include <stdio.h>\n#include "rtbte.h"\nint main(void){printf("%zu %zu %zu %zu %zu %zu\\n",'
                   'sizeof(rtbte_instance_desc), sizeof(rtbte_desc), sizeof(rtbte_channels), sizeof(rtbte_sizes),'
                   'sizeof(rtbte_integ), sizeof(rtbte_stats)); return 0;}\n')
    exe = tmp_path / "sz"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    want = [C.sizeof(t) for t in (rtlib.InstanceDesc, rtlib.Desc, rtlib.Channels, rtlib.Sizes, rtlib.Integ,
                                  rtlib.Stats)]
    assert got == want


def test_status_strings(rtlib):
    L = rtlib.load()
    for code, text in rtlib.STATUS.items():
        assert L.rtbte_status_string(code).decode() == text


def test_create_without_device_fails_cleanly(rtlib):
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import rtbte_inputs as ri

    m = ri.toy2d()
    keep = []
    descs = (rtlib.InstanceDesc * 1)()
    descs[0] = rtlib.instance_desc(m, keep)
    d = rtlib.Desc()
    rtlib.load().rtbte_desc_defaults(C.addressof(d))
    d.inst = C.addressof(descs)
    h = C.c_void_p()
    rc = rtlib.load().rtbte_create(C.addressof(d), C.byref(h))
    assert rc == -3 and not h.value
    assert rtlib.load().rtbte_create(None, C.byref(h)) == -1
