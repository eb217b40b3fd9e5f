"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
entry point that include/rid.h declares; host-side argument checks answer
before any device work.  CPU only."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_2408_14070_gb300 import build, rid
    build.build()
    return rid.lib()


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "rid.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(rid_[a-z0-9_]+)\s*\(", txt)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for n in ("rid_create_system", "rid_set_ensemble", "rid_explore", "rid_label", "rid_destroy_system"):
        assert n in names


def test_library_exports_every_declared_symbol(L):
    from paper_2408_14070_gb300 import rid
    for n in declared_symbols():
        assert hasattr(L, n), n
    assert set(declared_symbols()) <= set(rid.EXPORTS) | {"rid_server_create", "rid_server_destroy",
                                                          "rid_submit", "rid_poll", "rid_cancel",
                                                          "rid_server_stats"}


def test_version_and_status_strings(L):
    assert L.rid_version() >= 100
    assert L.rid_status_string(0) == b"ok"
    assert b"argument" in L.rid_status_string(1)


def test_null_arguments_rejected_before_device_work(L):
    from paper_2408_14070_gb300 import rid
    h = C.c_void_p()
    assert L.rid_create_system(None, C.byref(h)) == rid.RID_ERR_ARG
    assert b"NULL" in L.rid_last_error()
    d = rid.SystemDesc()
    d.n_beads = 3
    assert L.rid_create_system(C.byref(d), C.byref(h)) == rid.RID_ERR_ARG
    assert b"n_beads" in L.rid_last_error()
    assert L.rid_explore(None, 1, None, None, 0, 1, None, None, None, None, None, 0, None) == rid.RID_ERR_ARG
    assert L.rid_philox(-1, None, 0, None, None, 0, None) == rid.RID_ERR_ARG
    assert L.rid_destroy_system(None) == rid.RID_OK
