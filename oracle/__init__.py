"""FP64 CPU oracle for the RiD biased / restrained Langevin step (ctypes wrapper).

TEST INFRASTRUCTURE ONLY: imported by the tests, by the package's smoke check
and by the benchmark's CPU-baseline leg -- never by the product path.  It
shares no code with the CUDA library; both read the arrays made by
``paper_2408_14070_gb300.inputs``.

The arithmetic lives in ``rid_oracle.c`` (plain C, double precision); this file
only marshals numpy arrays.  ``build()`` compiles it with gcc.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rid_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "librid_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc, -ffp-contract=off)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-pthread",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _P(a, t):
    return a.ctypes.data_as(C.POINTER(t)) if a is not None else None


_d = C.POINTER(C.c_double)
_f = C.POINTER(C.c_float)
_i32 = C.POINTER(C.c_int32)
_u32 = C.POINTER(C.c_uint32)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = C.CDLL(build())
            L = _lib
            sys_args = [_d, _i32, C.c_uint64, _d, _d, _i32]
            L.orc_philox_batch.argtypes = [C.c_int64, _u32, C.c_uint64, _u32]
            L.orc_normals_batch.argtypes = [C.c_int64, _u32, C.c_uint64, _d]
            L.orc_dihedral.argtypes = [_d, _d]
            L.orc_dihedral.restype = C.c_double
            L.orc_wrap_pi.argtypes = [C.c_double]
            L.orc_wrap_pi.restype = C.c_double
            L.orc_switch.argtypes = [C.c_double, C.c_double, C.c_double]
            L.orc_switch.restype = C.c_double
            L.orc_model_param_count.argtypes = [C.c_int, C.c_int, C.c_int]
            L.orc_model_param_count.restype = C.c_int64
            L.orc_lj_pairs.argtypes = [C.c_int, _f, C.c_double, C.c_int64, _i32]
            L.orc_lj_pairs.restype = C.c_int64
            L.orc_eval_ff.argtypes = sys_args + [_d, _d, _d]
            L.orc_eval_ff.restype = C.c_double
            L.orc_eval_cvs.argtypes = sys_args + [_d, _d, _d]
            L.orc_mlp.argtypes = [C.c_int] * 5 + [_d, C.c_int, _d, _d, _d]
            L.orc_eval_ensemble.argtypes = [_i32, _d, _d, C.c_int, _i32, _d, _d, _d, _d]
            L.orc_eval_total.argtypes = sys_args + [_i32, _d, _d, C.c_int, _d, _d, _d, _d, _d, _d]
            L.orc_explore.argtypes = sys_args + [_i32, _d, _d, C.c_int, _f, _f, C.c_uint64, C.c_int64,
                                                 _f, _f, _d, _d, _d, C.c_int]
            L.orc_explore.restype = C.c_int
            L.orc_label.argtypes = sys_args + [C.c_int, _f, _f, _d, _d, C.c_uint64, C.c_int64, C.c_int64,
                                               C.c_int, _d, _d, _d, _d, _d, C.c_int]
            L.orc_label.restype = C.c_int
            L.orc_harmonic1d.argtypes = [C.c_double] * 8 + [C.c_uint64, C.c_int64, C.c_int64, C.c_int,
                                                            _d, _d, _d, _d]
            L.orc_label_stats.argtypes = [C.c_int64, C.c_int, C.c_int, _d, _d, _d, _d, _d]
            L.orc_label_constrained.argtypes = sys_args + [C.c_int, _f, _f, C.c_int, _i32, _d, C.c_uint64,
                                                           C.c_int64, C.c_int64, C.c_int, _d, _d, _d, _d, _d]
            L.orc_label_constrained.restype = C.c_int
        return _lib


# --------------------------------------------------------------------------
def _sys(sp):
    sd = np.array([sp.mass, sp.kT, sp.dt, sp.gamma, sp.bond_k, sp.bond_r0, sp.angle_k,
                   sp.angle_theta0, sp.lj_eps, sp.lj_sigma, sp.lj_rc], dtype=np.float64)
    si = np.array([sp.n_beads, sp.n_cv, sp.output_freq], dtype=np.int32)
    dk = np.ascontiguousarray(sp.dihedral_k, dtype=np.float64)
    dd = np.ascontiguousarray(sp.dihedral_delta, dtype=np.float64)
    cv = np.ascontiguousarray(sp.cv_atoms, dtype=np.int32)
    keep = (sd, si, dk, dd, cv)
    return keep, [_P(sd, C.c_double), _P(si, C.c_int32), C.c_uint64(int(sp.seed)),
                  _P(dk, C.c_double), _P(dd, C.c_double), _P(cv, C.c_int32)]


def _ens(ens):
    if ens is None:
        return (), [None, None, None]
    ei = np.array([ens.n_models, ens.n_in, ens.n_layers, ens.width, int(ens.resnet)], dtype=np.int32)
    ed = np.array([ens.trust_lo, ens.trust_hi], dtype=np.float64)
    w = np.ascontiguousarray(ens.weights, dtype=np.float64)
    return (ei, ed, w), [_P(ei, C.c_int32), _P(ed, C.c_double), _P(w, C.c_double)]


def philox(ctr, seed):
    ctr = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    out = np.empty_like(ctr)
    lib().orc_philox_batch(ctr.shape[0], _P(ctr, C.c_uint32), C.c_uint64(int(seed)), _P(out, C.c_uint32))
    return out


def normals(bwss, seed):
    """bwss: [n][4] = (bead, walker, step, stream) -> [n][3] standard normals."""
    bwss = np.ascontiguousarray(bwss, dtype=np.uint32).reshape(-1, 4)
    out = np.empty((bwss.shape[0], 3), dtype=np.float64)
    lib().orc_normals_batch(bwss.shape[0], _P(bwss, C.c_uint32), C.c_uint64(int(seed)), _P(out, C.c_double))
    return out


def dihedral(p, grad=True):
    p = np.ascontiguousarray(p, dtype=np.float64).reshape(4, 3)
    g = np.zeros((4, 3))
    phi = lib().orc_dihedral(_P(p, C.c_double), _P(g, C.c_double) if grad else None)
    return (phi, g) if grad else phi


def wrap_pi(d):
    return lib().orc_wrap_pi(float(d))


def switch(eps, e0, e1):
    return lib().orc_switch(float(eps), float(e0), float(e1))


def lj_pairs(xf, rc):
    xf = np.ascontiguousarray(xf, dtype=np.float32).reshape(-1, 3)
    n = xf.shape[0]
    cap = n * n // 2 + 1
    out = np.empty((cap, 2), dtype=np.int32)
    c = lib().orc_lj_pairs(n, _P(xf, C.c_float), float(rc), cap, _P(out, C.c_int32))
    return out[:c].copy()


def ff(sp, x, forces=True):
    keep, sa = _sys(sp)
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 3)
    f = np.zeros_like(x) if forces else None
    terms = np.zeros(4)
    U = lib().orc_eval_ff(*sa, _P(x, C.c_double), _P(f, C.c_double), _P(terms, C.c_double))
    return U, f, terms


def cvs(sp, x):
    keep, sa = _sys(sp)
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 3)
    s = np.zeros(sp.n_cv)
    J = np.zeros((sp.n_cv, 4, 3))
    lib().orc_eval_cvs(*sa, _P(x, C.c_double), _P(s, C.c_double), _P(J, C.c_double))
    return s, J


def mlp(ens, m, u):
    w = np.ascontiguousarray(ens.weights, dtype=np.float64)
    u = np.ascontiguousarray(u, dtype=np.float64)
    A = np.zeros(1)
    du = np.zeros(ens.n_in)
    lib().orc_mlp(ens.n_models, ens.n_in, ens.n_layers, ens.width, int(ens.resnet), _P(w, C.c_double),
                  int(m), _P(u, C.c_double), _P(A, C.c_double), _P(du, C.c_double))
    return A[0], du


def ensemble(ens, s, cv_atoms=None):
    """Ensemble at CV point s; cv_atoms [C][4] gives the CV kinds (a row
    ending in -1, -1 is a distance), None for torsions only."""
    keep, ea = _ens(ens)
    s = np.ascontiguousarray(s, dtype=np.float64)
    Cn = s.shape[0]
    cva = None if cv_atoms is None else np.ascontiguousarray(cv_atoms, dtype=np.int32)
    Fs = np.zeros(Cn)
    o3 = np.zeros(3)
    gA = np.zeros((ens.n_models, Cn))
    lib().orc_eval_ensemble(ea[0], ea[1], ea[2], Cn, _P(cva, C.c_int32), _P(s, C.c_double), _P(Fs, C.c_double),
                            _P(o3, C.c_double), _P(gA, C.c_double))
    return dict(Fs=Fs, eps=o3[0], Abar=o3[1], sigma=o3[2], gradA=gA)


def total(sp, x, ens=None, mode=None, s0=None, kappa=None):
    """Total force at one configuration.  mode: 0 none, 1 bias, 2 restraint."""
    if mode is None:
        mode = 1 if ens is not None else 0
    keep, sa = _sys(sp)
    keepe, ea = _ens(ens)
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 3)
    f = np.zeros_like(x)
    s = np.zeros(sp.n_cv)
    o4 = np.zeros(4)
    s0a = None if s0 is None else np.ascontiguousarray(s0, dtype=np.float64)
    ka = None if kappa is None else np.ascontiguousarray(np.broadcast_to(kappa, (sp.n_cv,)), dtype=np.float64)
    lib().orc_eval_total(*sa, *ea, int(mode), _P(s0a, C.c_double), _P(ka, C.c_double), _P(x, C.c_double),
                         _P(f, C.c_double), _P(s, C.c_double), _P(o4, C.c_double))
    return dict(f=f, s=s, U_ff=o4[0], eps=o4[1], Abar=o4[2], U_restraint=o4[3])


def explore(sp, x0, n_steps, ens=None, v0=None, step0=0, energy=False, n_threads=0):
    keep, sa = _sys(sp)
    keepe, ea = _ens(ens)
    x0 = np.ascontiguousarray(x0, dtype=np.float32)
    W, N = x0.shape[0], sp.n_beads
    v0a = None if v0 is None else np.ascontiguousarray(v0, dtype=np.float32)
    T = n_steps // sp.output_freq if sp.output_freq > 0 else 0
    cv = np.zeros((W, T, sp.n_cv), dtype=np.float32)
    eps = np.zeros((W, T), dtype=np.float32)
    en = np.zeros((W, T, 3)) if energy else None
    xo = np.zeros((W, N, 3))
    vo = np.zeros((W, N, 3))
    nt = lib().orc_explore(*sa, *ea, W, _P(x0, C.c_float), _P(v0a, C.c_float), C.c_uint64(step0),
                           C.c_int64(n_steps), _P(cv, C.c_float), _P(eps, C.c_float), _P(en, C.c_double),
                           _P(xo, C.c_double), _P(vo, C.c_double), int(n_threads))
    return dict(cv=cv, eps=eps, energy=en, x=xo, v=vo, threads=nt)


def label(sp, x0, s0, kappa, n_steps, n_equil, n_blocks=20, v0=None, step0=0, n_threads=0):
    keep, sa = _sys(sp)
    x0 = np.ascontiguousarray(x0, dtype=np.float32)
    R, N, Cn = x0.shape[0], sp.n_beads, sp.n_cv
    v0a = None if v0 is None else np.ascontiguousarray(v0, dtype=np.float32)
    s0 = np.ascontiguousarray(np.broadcast_to(s0, (R, Cn)), dtype=np.float64)
    kappa = np.ascontiguousarray(np.broadcast_to(kappa, (R, Cn)), dtype=np.float64)
    mf, se, sd = (np.zeros((R, Cn)) for _ in range(3))
    xo = np.zeros((R, N, 3))
    vo = np.zeros((R, N, 3))
    nt = lib().orc_label(*sa, R, _P(x0, C.c_float), _P(v0a, C.c_float), _P(s0, C.c_double),
                         _P(kappa, C.c_double), C.c_uint64(step0), C.c_int64(n_steps), C.c_int64(n_equil),
                         int(n_blocks), _P(mf, C.c_double), _P(se, C.c_double), _P(sd, C.c_double),
                         _P(xo, C.c_double), _P(vo, C.c_double), int(n_threads))
    if nt < 0:
        raise ValueError("invalid label arguments")
    return dict(mf=mf, se=se, std=sd, x=xo, v=vo, threads=nt)


def label_constrained(sp, x0, pairs, d0, n_steps, n_equil, n_blocks=20, v0=None, step0=0):
    """Constrained-MD mean forces on distance CVs (orc_label_constrained):
    pairs [C][2] bead indices, d0 [R][C] targets; returns dict(mf, se, std, x, v)."""
    keep, sa = _sys(sp)
    x0 = np.ascontiguousarray(x0, dtype=np.float32)
    R, N = x0.shape[0], x0.shape[1]
    v0 = None if v0 is None else np.ascontiguousarray(v0, dtype=np.float32)
    pr = np.ascontiguousarray(pairs, dtype=np.int32)
    Cn = pr.shape[0]
    d0 = np.ascontiguousarray(d0, dtype=np.float64).reshape(R, Cn)
    mf, se, sd = (np.zeros((R, Cn)) for _ in range(3))
    xo, vo = np.zeros((R, N, 3)), np.zeros((R, N, 3))
    rc = lib().orc_label_constrained(*sa, R, _P(x0, C.c_float), _P(v0, C.c_float), Cn, _P(pr, C.c_int32),
                                     _P(d0, C.c_double), C.c_uint64(int(step0)), int(n_steps), int(n_equil),
                                     int(n_blocks), _P(mf, C.c_double), _P(se, C.c_double), _P(sd, C.c_double),
                                     _P(xo, C.c_double), _P(vo, C.c_double))
    if rc != 0:
        raise ValueError("orc_label_constrained: bad arguments")
    return dict(mf=mf, se=se, std=sd, x=xo, v=vo)


def harmonic1d(a, c, kappa, s0, n_steps, n_equil, n_blocks=20, m=1.0, kT=1.0, dt=0.01, gamma=1.0, seed=1):
    mf, se, sd, mom = np.zeros(1), np.zeros(1), np.zeros(1), np.zeros(2)
    lib().orc_harmonic1d(float(a), float(c), float(kappa), float(s0), float(m), float(kT), float(dt),
                         float(gamma), C.c_uint64(seed), C.c_int64(n_steps), C.c_int64(n_equil),
                         int(n_blocks), _P(mf, C.c_double), _P(se, C.c_double), _P(sd, C.c_double),
                         _P(mom, C.c_double))
    return dict(mf=mf[0], se=se[0], std=sd[0], mean=mom[0], mean2=mom[1])


def label_stats(d, kappa, n_blocks):
    d = np.ascontiguousarray(d, dtype=np.float64)
    K, Cn = d.shape
    kappa = np.ascontiguousarray(np.broadcast_to(kappa, (Cn,)), dtype=np.float64)
    mf, se, sd = np.zeros(Cn), np.zeros(Cn), np.zeros(Cn)
    lib().orc_label_stats(K, Cn, int(n_blocks), _P(d, C.c_double), _P(kappa, C.c_double),
                          _P(mf, C.c_double), _P(se, C.c_double), _P(sd, C.c_double))
    return dict(mf=mf, se=se, std=sd)
