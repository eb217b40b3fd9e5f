"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
entry point that include/rid.h declares; host-side argument checks answer
before any device work.  CPU only."""
import ctypes as C
import os
import re
import shutil
import subprocess

import numpy as np
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
    assert set(declared_symbols()) == set(rid.EXPORTS)


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
    # the per-system switches and the request loop answer a NULL handle
    i32 = C.c_int32()
    for call in (lambda: L.rid_set_fused_steps(None, 1), lambda: L.rid_set_mlp_cluster(None, 0),
                 lambda: L.rid_set_ff_threads(None, 0), lambda: L.rid_get_ff_threads(None, C.byref(i32)),
                 lambda: L.rid_get_mlp_cluster(None, C.byref(i32)), lambda: L.rid_profile_enable(None, 1),
                 lambda: L.rid_submit(None, None, None), lambda: L.rid_poll(None, 1, None),
                 lambda: L.rid_cancel(None, 1),
                 lambda: L.rid_server_load(None, None, None, None)):
        assert call() == rid.RID_ERR_ARG
        assert b"NULL" in L.rid_last_error()
    assert L.rid_launch_count(None) == -1


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


def test_descriptor_checks_answer_before_device_work(L):
    # the argument checks of the training, MCMC, selection and constrained
    # entry points run before any device call, so they answer on a machine
    # without a GPU
    from paper_2408_14070_gb300 import rid
    w = np.zeros(1024, np.float32)
    P = C.POINTER(C.c_float)
    h = C.c_void_p()
    good = dict(n_models=1, n_cv=1, n_layers=1, width=8, resnet=0, batch_size=4, init_lr=1e-3, decay_rate=0.9,
                decay_steps=10, beta1=0.9, beta2=0.999, adam_eps=1e-8, dropout_rate=0.0, dropout_seed=0)
    for bad in ({"n_models": 0}, {"width": 0}, {"batch_size": 0}, {"init_lr": 0.0}, {"beta1": 1.0},
                {"dropout_rate": 1.0}, {"dropout_rate": -0.5}):
        d = rid.TrainDesc(**{**good, **bad})
        assert L.rid_trainer_create(C.byref(d), w.ctypes.data_as(P), C.byref(h)) == rid.RID_ERR_ARG, bad
    s0 = np.zeros((4, 2), np.float32)
    cv = np.array([0, 1], np.int32)
    nodes = np.zeros((3, 2), np.float32)
    mgood = dict(n_models=1, n_cv=2, n_layers=1, width=8, resnet=0, weights=w.ctypes.data, n_walkers=4, n_steps=5,
                 n_burn=0, kT=1.0, step_size=0.3, seed=1, bins=10, proj_i=0, proj_j=1, path_n_nodes=0, path_n_cv=0,
                 path_cv=None, path_nodes=None, path_lambda=1.0, path_z_lo=0.0, path_z_hi=1.0)
    path = dict(path_n_nodes=3, path_n_cv=2, path_cv=cv.ctypes.data, path_nodes=nodes.ctypes.data)
    for bad in ({"bins": 0}, {"kT": 0.0}, {"proj_j": 2}, {"n_walkers": 0}, {**path, "path_n_nodes": 1},
                {**path, "path_lambda": 0.0}, {**path, "path_z_hi": 0.0}, {**path, "path_n_cv": 3}):
        d = rid.McmcDesc(**{**mgood, **bad})
        assert L.rid_mcmc(C.byref(d), s0.ctypes.data, *([None] * 8), 0, None) == rid.RID_ERR_ARG, bad
    bad_cv = np.array([0, 5], np.int32)
    d = rid.McmcDesc(**{**mgood, **path, "path_cv": bad_cv.ctypes.data})
    assert L.rid_mcmc(C.byref(d), s0.ctypes.data, *([None] * 8), 0, None) == rid.RID_ERR_ARG
    assert b"path CV index" in L.rid_last_error()
    eps = np.zeros(4, np.float32)
    sel = np.zeros(4, np.int32)
    sgood = dict(n_cv=2, weights=None, periodic=None, trust_lo=0.0, trust_hi=1.0, cluster_threshold=1.0,
                 numb_cluster_lower=1, numb_cluster_upper=5, adapt=0, max_selection=4)
    for bad in ({"n_cv": 0}, {"cluster_threshold": 0.0}, {"adapt": 1, "numb_cluster_upper": 0}):
        d = rid.SelectDesc(**{**sgood, **bad})
        n1, n2, t = C.c_int32(), C.c_int32(), C.c_double()
        assert L.rid_select(C.byref(d), 4, s0.ctypes.data, eps.ctypes.data, sel.ctypes.data, C.byref(n1),
                            C.byref(n2), C.byref(t), 0, None) == rid.RID_ERR_ARG, bad
    assert L.rid_mcmc_system(None, 4, s0.ctypes.data, 5, 0, 1.0, 0.3, 1, 10, 0, 1, None, None, None, *([None] * 7),
                             None, 0, None) == rid.RID_ERR_ARG
    assert L.rid_label_constrained(None, 1, None, None, 1, None, None, 0, 10, 0, 2, None, None, None, None, None, 0,
                                   None) == rid.RID_ERR_ARG
