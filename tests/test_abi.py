"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
entry point that include/rid.h declares; host-side argument checks answer
before any device work.  CPU only."""
import ctypes as C
import os
import re
import shutil
import subprocess

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


def test_ctypes_structures_match_the_header(tmp_path):
    # sizes and field offsets of every descriptor the binding passes, as gcc
    # lays out include/rid.h, against the binding's ctypes structures
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    from paper_2408_14070_gb300 import rid
    structs = {"rid_system_desc": rid.SystemDesc, "rid_ensemble_desc": rid.EnsembleDesc,
               "rid_train_desc": rid.TrainDesc, "rid_mcmc_desc": rid.McmcDesc, "rid_mcmc_path": rid.McmcPath,
               "rid_select_desc": rid.SelectDesc, "rid_label_job": rid.LabelJob, "rid_request": rid.Request,
               "rid_job_info": rid.JobInfo}
    hdr = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "rid.h")).read(), flags=re.S)
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "rid.h"', "int main(void) {"]
    want = []
    for cname, py in structs.items():
        assert re.search(r"\}\s*" + cname + r"\s*;", hdr), cname
        lines.append(f'printf("%zu\\n", sizeof({cname}));')
        want.append(C.sizeof(py))
        # C field names in declaration order: the ctypes fields follow the same order
        body = re.search(r"typedef struct\s*\{([^{}]*)\}\s*" + cname + r"\s*;", hdr).group(1)
        names = []
        for decl in body.split(";"):
            decl = decl.strip()
            if not decl:
                continue
            for part in decl.split(","):
                names.append(re.findall(r"[A-Za-z_][A-Za-z0-9_]*", part)[-1])
        assert len(names) == len(py._fields_), (cname, names, [f[0] for f in py._fields_])
        for n, (pn, _) in zip(names, py._fields_):
            lines.append(f'printf("%zu\\n", offsetof({cname}, {n}));')
            want.append(getattr(py, pn).offset)
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()]
    assert got == want
