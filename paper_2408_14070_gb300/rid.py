"""Python binding of librid (ctypes).  Argument marshalling only: every step
of the computation runs in the library's CUDA kernels.

Arrays may be numpy arrays (host memory) or CUDA torch tensors (device
memory); all arrays of one call must live on the same side.  The binding
raises ``RidError`` carrying the library's status code and message.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

# The request loop runs exploration jobs on up to 16 streams.  The CUDA runtime
# maps streams onto CUDA_DEVICE_MAX_CONNECTIONS hardware work queues (8 unless
# set), and streams that share a queue wait on one another's launches: with 32
# queues the served mix overlaps fully (measured: 1.06 -> 1.58 M walker-steps/s
# on the serving stream at 200 requests/s).  The runtime reads the variable
# when the process creates its CUDA context, so it is set here, before any
# CUDA call the binding makes, unless the caller chose a value.
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "librid.so")

RID_OK, RID_ERR_ARG, RID_ERR_OOM, RID_ERR_CUDA, RID_ERR_NONFINITE = 0, 1, 2, 3, 4
RID_ERR_TIMEOUT, RID_NOT_READY, RID_ERR_STATE, RID_ERR_CANCELLED = 5, 6, 7, 8
RID_MEM_HOST, RID_MEM_DEVICE = 0, 1
RID_PREC_FP32, RID_PREC_BF16, RID_PREC_FP8 = 0, 1, 2
RID_BIAS_NONE, RID_BIAS_ENSEMBLE, RID_BIAS_RESTRAINT = 0, 1, 2

# every exported symbol of include/rid.h
EXPORTS = ("rid_version", "rid_status_string", "rid_last_error", "rid_create_system", "rid_destroy_system",
           "rid_set_ensemble", "rid_explore", "rid_label", "rid_eval_forces", "rid_pair_mask", "rid_philox",
           "rid_walkers_load", "rid_walkers_advance", "rid_walkers_read", "rid_profile_enable",
           "rid_profile_read", "rid_launch_count", "rid_ensemble_grad_noalloc", "rid_server_create",
           "rid_server_destroy", "rid_label_batch", "rid_submit", "rid_poll", "rid_cancel", "rid_server_load",
           "rid_trainer_create", "rid_trainer_destroy", "rid_trainer_set_data", "rid_trainer_run",
           "rid_trainer_grad", "rid_trainer_weights", "rid_mcmc", "rid_select",
           "rid_label_constrained", "rid_mcmc_system", "rid_set_mlp_cluster",
           "rid_get_mlp_cluster", "rid_set_ff_threads", "rid_get_ff_threads", "rid_set_fused_steps")
RID_NOT_READY = 6
RID_JOB_LABEL, RID_JOB_EXPLORE = 1, 2


class RidError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"[{code}] {msg}")
        self.code = code


class SystemDesc(C.Structure):
    _fields_ = [("n_beads", C.c_int32), ("n_cv", C.c_int32), ("output_freq", C.c_int32), ("reserved0", C.c_int32),
                ("mass", C.c_double), ("kT", C.c_double), ("dt", C.c_double), ("gamma", C.c_double),
                ("seed", C.c_uint64), ("bond_k", C.c_double), ("bond_r0", C.c_double), ("angle_k", C.c_double),
                ("angle_theta0", C.c_double), ("lj_eps", C.c_double), ("lj_sigma", C.c_double),
                ("lj_rc", C.c_double), ("dihedral_k", C.POINTER(C.c_double)),
                ("dihedral_delta", C.POINTER(C.c_double)), ("cv_atoms", C.POINTER(C.c_int32))]


class EnsembleDesc(C.Structure):
    _fields_ = [("n_models", C.c_int32), ("n_in", C.c_int32), ("n_layers", C.c_int32), ("width", C.c_int32),
                ("resnet", C.c_int32), ("precision", C.c_int32), ("trust_lo", C.c_double),
                ("trust_hi", C.c_double), ("weights", C.POINTER(C.c_float))]


class TrainDesc(C.Structure):
    _fields_ = [("n_models", C.c_int32), ("n_cv", C.c_int32), ("n_layers", C.c_int32), ("width", C.c_int32),
                ("resnet", C.c_int32), ("batch_size", C.c_int32), ("init_lr", C.c_double),
                ("decay_rate", C.c_double), ("decay_steps", C.c_int32), ("beta1", C.c_double),
                ("beta2", C.c_double), ("adam_eps", C.c_double), ("dropout_rate", C.c_double),
                ("dropout_seed", C.c_uint64), ("cv_dist", C.c_void_p)]


class McmcDesc(C.Structure):
    _fields_ = [("n_models", C.c_int32), ("n_cv", C.c_int32), ("n_layers", C.c_int32), ("width", C.c_int32),
                ("resnet", C.c_int32), ("weights", C.c_void_p), ("n_walkers", C.c_int32), ("n_steps", C.c_int64),
                ("n_burn", C.c_int64), ("kT", C.c_double), ("step_size", C.c_double), ("seed", C.c_uint64),
                ("bins", C.c_int32), ("proj_i", C.c_int32), ("proj_j", C.c_int32), ("path_n_nodes", C.c_int32),
                ("path_n_cv", C.c_int32), ("path_cv", C.c_void_p), ("path_nodes", C.c_void_p),
                ("path_lambda", C.c_double), ("path_z_lo", C.c_double), ("path_z_hi", C.c_double),
                ("cv_dist", C.c_void_p), ("cv_lo", C.c_void_p), ("cv_hi", C.c_void_p)]


class McmcPath(C.Structure):
    _fields_ = [("n_nodes", C.c_int32), ("n_cv", C.c_int32), ("cv", C.c_void_p), ("nodes", C.c_void_p),
                ("lam", C.c_double), ("z_lo", C.c_double), ("z_hi", C.c_double)]


def _path_arrays(path):
    """(nodes float32 [P][Cp], cvs int32 [Cp], lambda, z_lo, z_hi) from a path tuple."""
    nodes = np.ascontiguousarray(path[0], dtype=np.float32)
    cvs = np.ascontiguousarray(path[1], dtype=np.int32)
    return nodes, cvs, float(path[2]), float(path[3]), float(path[4])


class SelectDesc(C.Structure):
    _fields_ = [("n_cv", C.c_int32), ("weights", C.POINTER(C.c_float)), ("periodic", C.POINTER(C.c_int32)),
                ("trust_lo", C.c_double), ("trust_hi", C.c_double), ("cluster_threshold", C.c_double),
                ("numb_cluster_lower", C.c_int32), ("numb_cluster_upper", C.c_int32), ("adapt", C.c_int32),
                ("max_selection", C.c_int32)]


class LabelJob(C.Structure):
    _fields_ = [("sys", C.c_void_p), ("n_runs", C.c_int32), ("n_blocks", C.c_int32), ("x0", C.c_void_p),
                ("v0", C.c_void_p), ("s0", C.c_void_p), ("kappa", C.c_void_p), ("step0", C.c_uint64),
                ("n_steps", C.c_int64), ("n_equil", C.c_int64), ("mf_out", C.c_void_p), ("se_out", C.c_void_p),
                ("std_out", C.c_void_p), ("x_out", C.c_void_p), ("v_out", C.c_void_p)]


class Request(C.Structure):
    _fields_ = [("kind", C.c_int32), ("n_walkers", C.c_int32), ("sys", C.c_void_p), ("x0", C.c_void_p),
                ("v0", C.c_void_p), ("step0", C.c_uint64), ("n_steps", C.c_int64), ("s0", C.c_void_p),
                ("kappa", C.c_void_p), ("n_equil", C.c_int64), ("n_blocks", C.c_int32), ("mf_out", C.c_void_p),
                ("se_out", C.c_void_p), ("std_out", C.c_void_p), ("cv_out", C.c_void_p), ("eps_out", C.c_void_p),
                ("x_out", C.c_void_p), ("v_out", C.c_void_p)]


class JobInfo(C.Structure):
    _fields_ = [("status", C.c_int32), ("kind", C.c_int32), ("t_submit_ms", C.c_double),
                ("t_start_ms", C.c_double), ("t_end_ms", C.c_double)]


_lib = None


def lib() -> C.CDLL:
    """Load librid.so; raises if the CUDA library has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"librid.so not found at {LIB_PATH}: run paper_2408_14070_gb300.build.build() first")
    L = C.CDLL(LIB_PATH)
    vp, i32, i64, u64 = C.c_void_p, C.c_int32, C.c_int64, C.c_uint64
    L.rid_version.restype = C.c_int
    L.rid_status_string.restype = C.c_char_p
    L.rid_status_string.argtypes = [C.c_int]
    L.rid_last_error.restype = C.c_char_p
    L.rid_create_system.argtypes = [C.POINTER(SystemDesc), C.POINTER(vp)]
    L.rid_destroy_system.argtypes = [vp]
    L.rid_set_ensemble.argtypes = [vp, C.POINTER(EnsembleDesc)]
    L.rid_explore.argtypes = [vp, i32, vp, vp, u64, i64, vp, vp, vp, vp, vp, i32, vp]
    L.rid_label.argtypes = [vp, i32, vp, vp, vp, vp, u64, i64, i64, i32, vp, vp, vp, vp, vp, i32, vp]
    L.rid_eval_forces.argtypes = [vp, i32, vp, i32, vp, vp, vp, vp, vp, vp, vp, i32, vp]
    L.rid_pair_mask.argtypes = [vp, i32, vp, vp, i32, vp]
    L.rid_philox.argtypes = [i64, vp, u64, vp, vp, i32, vp]
    L.rid_walkers_load.argtypes = [vp, i32, vp, vp, u64, i32, vp]
    L.rid_walkers_advance.argtypes = [vp, i64, vp, vp, vp, i32, vp]
    L.rid_walkers_read.argtypes = [vp, vp, vp, C.POINTER(u64), i32, vp]
    L.rid_profile_enable.argtypes = [vp, i32]
    L.rid_profile_read.argtypes = [vp, i32, C.c_char_p, C.POINTER(C.c_double), C.POINTER(i64), C.POINTER(i32)]
    L.rid_launch_count.argtypes = [vp]
    L.rid_set_mlp_cluster.argtypes = [vp, i32]
    L.rid_get_mlp_cluster.argtypes = [vp, C.POINTER(i32)]
    L.rid_set_ff_threads.argtypes = [vp, i32]
    L.rid_get_ff_threads.argtypes = [vp, C.POINTER(i32)]
    L.rid_set_fused_steps.argtypes = [vp, i32]
    L.rid_ensemble_grad_noalloc.argtypes = [i32, i32, vp, i32, i32, i32, i32, vp, vp, vp, vp]
    L.rid_server_create.argtypes = [u64, C.POINTER(vp)]
    L.rid_server_destroy.argtypes = [vp]
    L.rid_label_batch.argtypes = [vp, C.POINTER(LabelJob), i32, i32, C.POINTER(i32), i32, vp]
    L.rid_submit.argtypes = [vp, C.POINTER(Request), C.POINTER(u64)]
    L.rid_poll.argtypes = [vp, u64, C.POINTER(JobInfo)]
    L.rid_cancel.argtypes = [vp, u64]
    L.rid_server_load.argtypes = [vp, C.POINTER(i32), C.POINTER(i32), C.POINTER(u64)]
    L.rid_launch_count.restype = i64
    L.rid_trainer_create.argtypes = [C.POINTER(TrainDesc), vp, C.POINTER(vp)]
    L.rid_trainer_destroy.argtypes = [vp]
    L.rid_trainer_set_data.argtypes = [vp, i32, vp, vp, i32, vp]
    L.rid_trainer_run.argtypes = [vp, i32, vp, vp, i32, vp]
    L.rid_trainer_grad.argtypes = [vp, vp, vp, vp, i32, vp]
    L.rid_trainer_weights.argtypes = [vp, vp, C.POINTER(i64), i32, vp]
    L.rid_label_constrained.argtypes = [vp, i32, vp, vp, i32, vp, vp, u64, i64, i64, i32, vp, vp, vp, vp, vp,
                                        i32, vp]
    L.rid_mcmc_system.argtypes = [vp, i32, vp, i64, i64, C.c_double, C.c_double, u64, i32, i32, i32, vp, vp,
                                  C.POINTER(McmcPath), vp, vp, vp, vp, vp, vp, vp, C.POINTER(i64), i32, vp]
    L.rid_select.argtypes = [C.POINTER(SelectDesc), i32, vp, vp, vp, C.POINTER(i32), C.POINTER(i32),
                             C.POINTER(C.c_double), i32, vp]
    L.rid_mcmc.argtypes = [C.POINTER(McmcDesc), vp, vp, vp, vp, vp, vp, vp, vp, C.POINTER(i64), i32, vp]
    for name in EXPORTS:
        getattr(L, name).restype = getattr(L, name).restype or C.c_int
    _lib = L
    return L


def _check(code: int):
    if code != RID_OK:
        raise RidError(code, lib().rid_last_error().decode())


# ---------------------------------------------------------------------------
class _Args:
    """Collects array pointers of one call and checks they share a memory side."""

    def __init__(self):
        self.mem = None
        self.keep = []

    def ptr(self, a, dtype, shape=None, writable=False):
        if a is None:
            return None
        if hasattr(a, "data_ptr"):          # torch tensor
            import torch
            want = {np.float32: torch.float32, np.float64: torch.float64, np.uint32: torch.uint32,
                    np.int32: torch.int32, np.uint64: torch.uint64}[dtype]
            if a.dtype != want:
                raise TypeError(f"expected {want}, got {a.dtype}")
            if not a.is_contiguous():
                raise ValueError("tensor must be contiguous")
            side = RID_MEM_DEVICE if a.is_cuda else RID_MEM_HOST
            if shape is not None and a.numel() != int(np.prod(shape)):
                raise ValueError(f"expected {int(np.prod(shape))} elements, got {a.numel()}")
            p = a.data_ptr()
        else:
            if not isinstance(a, np.ndarray) or a.dtype != dtype or not a.flags.c_contiguous:
                raise TypeError(f"expected a C-contiguous numpy array of {np.dtype(dtype)}")
            if writable and not a.flags.writeable:
                raise ValueError("output array is read-only")
            if shape is not None and a.size != int(np.prod(shape)):
                raise ValueError(f"expected {int(np.prod(shape))} elements, got {a.size}")
            side = RID_MEM_HOST
            p = a.ctypes.data
        if self.mem is None:
            self.mem = side
        elif self.mem != side:
            raise ValueError("all arrays of a call must be on the same side (host or device)")
        self.keep.append(a)
        return C.c_void_p(p)


def _stream_ptr(stream):
    if stream is None:
        return None
    return C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


# ---------------------------------------------------------------------------
class System:
    """A bead-chain system on the current CUDA device (wraps rid_system*)."""

    def __init__(self, sp):
        L = lib()
        self.sp = sp
        self.N, self.C = int(sp.n_beads), int(sp.n_cv)
        self._dk = np.ascontiguousarray(sp.dihedral_k, dtype=np.float64)
        self._dd = np.ascontiguousarray(sp.dihedral_delta, dtype=np.float64)
        self._cv = np.ascontiguousarray(sp.cv_atoms, dtype=np.int32)
        d = SystemDesc(self.N, self.C, int(sp.output_freq), 0, sp.mass, sp.kT, sp.dt, sp.gamma, int(sp.seed),
                       sp.bond_k, sp.bond_r0, sp.angle_k, sp.angle_theta0, sp.lj_eps, sp.lj_sigma, sp.lj_rc,
                       self._dk.ctypes.data_as(C.POINTER(C.c_double)),
                       self._dd.ctypes.data_as(C.POINTER(C.c_double)),
                       self._cv.ctypes.data_as(C.POINTER(C.c_int32)))
        h = C.c_void_p()
        _check(L.rid_create_system(C.byref(d), C.byref(h)))
        self.h = h
        self.M = 0

    def close(self):
        if getattr(self, "h", None):
            lib().rid_destroy_system(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_ensemble(self, ens, precision=RID_PREC_FP32):
        w = np.ascontiguousarray(ens.weights, dtype=np.float32)
        d = EnsembleDesc(ens.n_models, ens.n_in, ens.n_layers, ens.width, int(ens.resnet), int(precision),
                         float(ens.trust_lo), float(ens.trust_hi), w.ctypes.data_as(C.POINTER(C.c_float)))
        _check(lib().rid_set_ensemble(self.h, C.byref(d)))
        self.M = ens.n_models

    def explore(self, x0, n_steps, v0=None, step0=0, cv_out=None, eps_out=None, energy_out=None, x_out=None,
                v_out=None, stream=None):
        W = int(x0.shape[0])
        a = _Args()
        px = a.ptr(x0, np.float32, (W, self.N, 3))
        pv = a.ptr(v0, np.float32, (W, self.N, 3))
        T = n_steps // self.sp.output_freq
        pc = a.ptr(cv_out, np.float32, (W, T, self.C), True)
        pe = a.ptr(eps_out, np.float32, (W, T), True)
        pen = a.ptr(energy_out, np.float64, (W, T, 3), True)
        pxo = a.ptr(x_out, np.float32, (W, self.N, 3), True)
        pvo = a.ptr(v_out, np.float32, (W, self.N, 3), True)
        _check(lib().rid_explore(self.h, W, px, pv, C.c_uint64(step0), C.c_int64(n_steps), pc, pe, pen, pxo, pvo,
                                 a.mem, _stream_ptr(stream)))

    def label(self, x0, s0, kappa, n_steps, n_equil, n_blocks, mf_out, se_out, std_out, v0=None, step0=0,
              x_out=None, v_out=None, stream=None):
        R = int(x0.shape[0])
        a = _Args()
        args = [a.ptr(x0, np.float32, (R, self.N, 3)), a.ptr(v0, np.float32, (R, self.N, 3)),
                a.ptr(s0, np.float64, (R, self.C)), a.ptr(kappa, np.float64, (R, self.C))]
        outs = [a.ptr(mf_out, np.float64, (R, self.C), True), a.ptr(se_out, np.float64, (R, self.C), True),
                a.ptr(std_out, np.float64, (R, self.C), True), a.ptr(x_out, np.float32, (R, self.N, 3), True),
                a.ptr(v_out, np.float32, (R, self.N, 3), True)]
        _check(lib().rid_label(self.h, R, *args, C.c_uint64(step0), C.c_int64(n_steps), C.c_int64(n_equil),
                               int(n_blocks), *outs, a.mem, _stream_ptr(stream)))

    def label_constrained(self, x0, pairs, d0, n_steps, n_equil, n_blocks, mf_out, se_out, std_out, v0=None,
                          step0=0, x_out=None, v_out=None, stream=None):
        """Constrained-MD mean forces on the distances of `pairs` [C][2] held
        at d0 [R][C] (rid_label_constrained)."""
        R = int(x0.shape[0])
        pr = np.ascontiguousarray(pairs, dtype=np.int32).reshape(-1, 2)
        Cn = pr.shape[0]
        a = _Args()
        args = [a.ptr(x0, np.float32, (R, self.N, 3)), a.ptr(v0, np.float32, (R, self.N, 3))]
        pd0 = a.ptr(d0, np.float64, (R, Cn))
        outs = [a.ptr(mf_out, np.float64, (R, Cn), True), a.ptr(se_out, np.float64, (R, Cn), True),
                a.ptr(std_out, np.float64, (R, Cn), True), a.ptr(x_out, np.float32, (R, self.N, 3), True),
                a.ptr(v_out, np.float32, (R, self.N, 3), True)]
        _check(lib().rid_label_constrained(self.h, R, *args, Cn, pr.ctypes.data, pd0, C.c_uint64(step0),
                                           C.c_int64(n_steps), C.c_int64(n_equil), int(n_blocks), *outs, a.mem,
                                           _stream_ptr(stream)))

    def mcmc(self, s0, n_steps, n_burn, kT, step_size, seed, bins=101, pair=(0, 1), s_out=None, hist1=None,
             hist2=None, pmf1=None, pmf2=None, path=None, hist_path=None, pmf_path=None, cv_range=None,
             stream=None):
        """MCMC dimension reduction with this system's ensemble at its precision
        (rid_mcmc_system); returns the number of accepted moves.  path = (nodes
        [P][Cp], cvs [Cp], lambda, z_lo, z_hi) adds the (s_path, z_path)
        projection into hist_path / pmf_path [bins][bins].  cv_range = (lo [C],
        hi [C]): the range of each distance CV (systems with distance CVs)."""
        W = int(s0.shape[0])
        a = _Args()
        lo = hi = None
        if cv_range is not None:
            lo = np.ascontiguousarray(cv_range[0], dtype=np.float64)
            hi = np.ascontiguousarray(cv_range[1], dtype=np.float64)
        ps = a.ptr(s0, np.float32, (W, self.C))
        outs = [a.ptr(s_out, np.float32, (W, self.C), True), a.ptr(hist1, np.uint64, (self.C, bins), True),
                a.ptr(hist2, np.uint64, (bins, bins), True), a.ptr(pmf1, np.float64, (self.C, bins), True),
                a.ptr(pmf2, np.float64, (bins, bins), True), a.ptr(hist_path, np.uint64, (bins, bins), True),
                a.ptr(pmf_path, np.float64, (bins, bins), True)]
        pp = None
        if path is not None:
            nodes, cvs, lam, zlo, zhi = _path_arrays(path)
            pp = McmcPath(nodes.shape[0], cvs.size, cvs.ctypes.data, nodes.ctypes.data, lam, zlo, zhi)
        nacc = C.c_int64(0)
        _check(lib().rid_mcmc_system(self.h, W, ps, C.c_int64(n_steps), C.c_int64(n_burn), float(kT),
                                     float(step_size), C.c_uint64(seed), int(bins), int(pair[0]), int(pair[1]),
                                     None if lo is None else lo.ctypes.data, None if hi is None else hi.ctypes.data,
                                     None if pp is None else C.byref(pp), *outs, C.byref(nacc), a.mem,
                                     _stream_ptr(stream)))
        return nacc.value

    def eval_forces(self, x, bias=RID_BIAS_NONE, s0=None, kappa=None, f_out=None, s_out=None, eps_out=None,
                    abar_out=None, grad_out=None, stream=None):
        W = int(x.shape[0])
        a = _Args()
        px = a.ptr(x, np.float32, (W, self.N, 3))
        ps0 = a.ptr(s0, np.float64, (W, self.C))
        pk = a.ptr(kappa, np.float64, (W, self.C))
        outs = [a.ptr(f_out, np.float32, (W, self.N, 3), True), a.ptr(s_out, np.float32, (W, self.C), True),
                a.ptr(eps_out, np.float32, (W,), True), a.ptr(abar_out, np.float32, (W,), True),
                a.ptr(grad_out, np.float32, (max(self.M, 1), W, self.C), True)]
        _check(lib().rid_eval_forces(self.h, W, px, int(bias), ps0, pk, *outs, a.mem, _stream_ptr(stream)))

    # resident walkers -------------------------------------------------------
    def walkers_load(self, x0, v0=None, step0=0, stream=None):
        W = int(x0.shape[0])
        a = _Args()
        px = a.ptr(x0, np.float32, (W, self.N, 3))
        pv = a.ptr(v0, np.float32, (W, self.N, 3))
        _check(lib().rid_walkers_load(self.h, W, px, pv, C.c_uint64(step0), a.mem, _stream_ptr(stream)))
        self.W = W

    def walkers_advance(self, n_steps, cv_out=None, eps_out=None, energy_out=None, stream=None, mem=None):
        a = _Args()
        T = n_steps // self.sp.output_freq
        pc = a.ptr(cv_out, np.float32, (self.W, T, self.C), True)
        pe = a.ptr(eps_out, np.float32, (self.W, T), True)
        pen = a.ptr(energy_out, np.float64, (self.W, T, 3), True)
        m = a.mem if a.mem is not None else (RID_MEM_DEVICE if mem is None else mem)
        _check(lib().rid_walkers_advance(self.h, C.c_int64(n_steps), pc, pe, pen, m, _stream_ptr(stream)))

    def walkers_read(self, x_out=None, v_out=None, stream=None, mem=None):
        a = _Args()
        px = a.ptr(x_out, np.float32, (self.W, self.N, 3), True)
        pv = a.ptr(v_out, np.float32, (self.W, self.N, 3), True)
        nxt = C.c_uint64(0)
        m = a.mem if a.mem is not None else (RID_MEM_HOST if mem is None else mem)
        _check(lib().rid_walkers_read(self.h, px, pv, C.byref(nxt), m, _stream_ptr(stream)))
        return nxt.value

    # kernel timing ------------------------------------------------------------
    def profile_enable(self, on=True):
        _check(lib().rid_profile_enable(self.h, int(bool(on))))

    def profile_read(self, max_kernels=16):
        names = C.create_string_buffer(48 * max_kernels)
        ms = (C.c_double * max_kernels)()
        cnt = (C.c_int64 * max_kernels)()
        nk = C.c_int32(0)
        _check(lib().rid_profile_read(self.h, max_kernels, names, ms, cnt, C.byref(nk)))
        out = {}
        for k in range(min(nk.value, max_kernels)):
            nm = names.raw[48 * k:48 * (k + 1)].split(b"\0", 1)[0].decode()
            out[nm] = (ms[k], int(cnt[k]))
        return out

    def launch_count(self):
        return int(lib().rid_launch_count(self.h))

    def set_mlp_cluster(self, csize):
        """Cluster size of the tensor-core ensemble kernel: 0 tuned, 1, 2 or 4."""
        _check(lib().rid_set_mlp_cluster(self.h, int(csize)))

    def set_ff_threads(self, threads):
        """CTA size of the force-field kernel: 0 tuned, else a multiple of 32."""
        _check(lib().rid_set_ff_threads(self.h, int(threads)))

    def set_fused_steps(self, on):
        """The persistent small-system kernels on or off: exploration calls of small
        FP32 systems, and rid_label below 768 beads, in one launch per call.  The
        results are the same bits either way."""
        _check(lib().rid_set_fused_steps(self.h, 1 if on else 0))

    def ff_threads(self):
        """CTA size of the force-field kernel in use."""
        t = C.c_int32(0)
        _check(lib().rid_get_ff_threads(self.h, C.byref(t)))
        return int(t.value)

    def mlp_cluster(self):
        """Cluster size of the tensor-core ensemble kernel's last launch (0 before any)."""
        cs = C.c_int32(0)
        _check(lib().rid_get_mlp_cluster(self.h, C.byref(cs)))
        return int(cs.value)

    def pair_mask(self, x, mask_out, stream=None):
        W = int(x.shape[0])
        a = _Args()
        px = a.ptr(x, np.float32, (W, self.N, 3))
        pm = a.ptr(mask_out, np.uint32, (W, self.N, (self.N + 31) // 32), True)
        _check(lib().rid_pair_mask(self.h, W, px, pm, a.mem, _stream_ptr(stream)))


def philox(counters, seed, words_out=None, normals_out=None, stream=None):
    n = int(counters.shape[0])
    a = _Args()
    pc = a.ptr(counters, np.uint32, (n, 4))
    pw = a.ptr(words_out, np.uint32, (n, 4), True)
    pn = a.ptr(normals_out, np.float32, (n, 3), True)
    _check(lib().rid_philox(C.c_int64(n), pc, C.c_uint64(int(seed)), pw, pn, a.mem, _stream_ptr(stream)))


class Server:
    """A budgeted device memory pool for batched label runs (wraps rid_server*)."""

    def __init__(self, hbm_budget_bytes):
        h = C.c_void_p()
        _check(lib().rid_server_create(C.c_uint64(int(hbm_budget_bytes)), C.byref(h)))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib().rid_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def label_batch(self, jobs, threads=0, stream=None, raise_nonfinite=True):
        """jobs: list of dicts with keys system, x0, s0, kappa, n_steps, n_equil,
        n_blocks, mf, se, std and optionally v0, step0, x_out, v_out.  Returns
        the per-job status list."""
        a = _Args()
        arr = (LabelJob * max(1, len(jobs)))()
        for k, j in enumerate(jobs):
            sysobj = j["system"]
            R = int(j["x0"].shape[0])
            N, Cn = sysobj.N, sysobj.C
            arr[k] = LabelJob(sysobj.h.value, R, int(j["n_blocks"]),
                              a.ptr(j["x0"], np.float32, (R, N, 3)), a.ptr(j.get("v0"), np.float32, (R, N, 3)),
                              a.ptr(j["s0"], np.float64, (R, Cn)), a.ptr(j["kappa"], np.float64, (R, Cn)),
                              int(j.get("step0", 0)), int(j["n_steps"]), int(j["n_equil"]),
                              a.ptr(j["mf"], np.float64, (R, Cn), True), a.ptr(j["se"], np.float64, (R, Cn), True),
                              a.ptr(j["std"], np.float64, (R, Cn), True),
                              a.ptr(j.get("x_out"), np.float32, (R, N, 3), True),
                              a.ptr(j.get("v_out"), np.float32, (R, N, 3), True))
        status = (C.c_int32 * max(1, len(jobs)))()
        mem = a.mem if a.mem is not None else RID_MEM_HOST
        rc = lib().rid_label_batch(self.h, arr, len(jobs), int(threads), status, mem, _stream_ptr(stream))
        if rc != RID_OK and not (rc == RID_ERR_NONFINITE and not raise_nonfinite):
            _check(rc)
        return [int(status[k]) for k in range(len(jobs))]

    # request loop ------------------------------------------------------------
    def _submit(self, rq, keep):
        jid = C.c_uint64()
        _check(lib().rid_submit(self.h, C.byref(rq), C.byref(jid)))
        if not hasattr(self, "_live"):
            self._live = {}
        self._live[jid.value] = keep          # output arrays stay alive until the job is final
        return jid.value

    def submit_label(self, system, x0, s0, kappa, n_steps, n_equil, n_blocks, mf, se, std, v0=None, step0=0,
                     x_out=None, v_out=None):
        R = int(x0.shape[0])
        N, Cn = system.N, system.C
        a = _Args()
        rq = Request(RID_JOB_LABEL, R, system.h.value, a.ptr(x0, np.float32, (R, N, 3)),
                     a.ptr(v0, np.float32, (R, N, 3)), int(step0), int(n_steps), a.ptr(s0, np.float64, (R, Cn)),
                     a.ptr(kappa, np.float64, (R, Cn)), int(n_equil), int(n_blocks),
                     a.ptr(mf, np.float64, (R, Cn), True), a.ptr(se, np.float64, (R, Cn), True),
                     a.ptr(std, np.float64, (R, Cn), True), None, None,
                     a.ptr(x_out, np.float32, (R, N, 3), True), a.ptr(v_out, np.float32, (R, N, 3), True))
        if a.mem != RID_MEM_HOST:
            raise ValueError("requests take host arrays only")
        return self._submit(rq, a.keep)

    def submit_explore(self, system, x0, n_steps, v0=None, step0=0, cv_out=None, eps_out=None, x_out=None,
                       v_out=None):
        W = int(x0.shape[0])
        N, Cn = system.N, system.C
        T = int(n_steps) // system.sp.output_freq
        a = _Args()
        rq = Request(RID_JOB_EXPLORE, W, system.h.value, a.ptr(x0, np.float32, (W, N, 3)),
                     a.ptr(v0, np.float32, (W, N, 3)), int(step0), int(n_steps), None, None, 0, 0, None, None, None,
                     a.ptr(cv_out, np.float32, (W, T, Cn), True), a.ptr(eps_out, np.float32, (W, T), True),
                     a.ptr(x_out, np.float32, (W, N, 3), True), a.ptr(v_out, np.float32, (W, N, 3), True))
        if a.mem != RID_MEM_HOST:
            raise ValueError("requests take host arrays only")
        return self._submit(rq, a.keep)

    def poll(self, job_id):
        """(status, info dict); status RID_NOT_READY while queued or running."""
        info = JobInfo()
        rc = lib().rid_poll(self.h, C.c_uint64(job_id), C.byref(info))
        if rc == RID_ERR_ARG and info.kind == 0:
            _check(rc)
        d = dict(status=int(info.status), kind=int(info.kind), t_submit_ms=info.t_submit_ms,
                 t_start_ms=info.t_start_ms, t_end_ms=info.t_end_ms)
        if rc != RID_NOT_READY:
            getattr(self, "_live", {}).pop(job_id, None)
        return int(rc), d

    def wait(self, job_ids, timeout=600.0, sleep=0.0005):
        """Poll until every job is final; returns {id: (status, info)}."""
        import time
        left, out = set(job_ids), {}
        t_end = time.time() + timeout
        while left:
            for jid in list(left):
                st, info = self.poll(jid)
                if st != RID_NOT_READY:
                    out[jid] = (st, info)
                    left.discard(jid)
            if left:
                if time.time() > t_end:
                    raise TimeoutError(f"{len(left)} jobs not final after {timeout} s")
                time.sleep(sleep)
        return out

    def cancel(self, job_id):
        """Withdraw a job still queued: True (rid_poll then reports
        RID_ERR_CANCELLED), False if it is running or final (it runs to its end)."""
        rc = lib().rid_cancel(self.h, C.c_uint64(job_id))
        if rc == RID_ERR_STATE:
            return False
        _check(rc)
        return True

    def load(self):
        q, r, b = C.c_int32(), C.c_int32(), C.c_uint64()
        _check(lib().rid_server_load(self.h, C.byref(q), C.byref(r), C.byref(b)))
        return int(q.value), int(r.value), int(b.value)


def ensemble_grad_noalloc(s, weights, n_models, n_layers, width, grad_out, value_out=None, resnet=False,
                          stream=None):
    """Member gradients dA_i/ds [M][P][C] at device points s [P][C] with the
    packed device weights [M][Pw], using only the library's static scratch."""
    P, Cn = int(s.shape[0]), int(s.shape[1])
    M = int(n_models)
    a = _Args()
    ps = a.ptr(s, np.float32, (P, Cn))
    pw = a.ptr(weights, np.float32)
    pg = a.ptr(grad_out, np.float32, (M, P, Cn), True)
    pv = a.ptr(value_out, np.float32, (M, P), True)
    if a.mem != RID_MEM_DEVICE:
        raise ValueError("ensemble_grad_noalloc takes device tensors only")
    _check(lib().rid_ensemble_grad_noalloc(P, Cn, ps, M, int(n_layers), int(width), int(bool(resnet)), pw, pg, pv,
                                           _stream_ptr(stream)))


def version() -> int:
    return lib().rid_version()


# ---------------------------------------------------------------------------
class Trainer:
    """Fits an ensemble to mean-force labels on the current CUDA device (wraps
    rid_trainer*): per member, Adam steps on the mean squared difference
    between dA_i/ds and the labels, learning rate init_lr * decay_rate^(t /
    decay_steps).  Weights use the packed layout of EnsembleParams.weights.
    dropout_rate > 0 thins every hidden layer during training (inverted
    dropout, masks from Philox keyed by dropout_seed).  cv_dist [C] marks
    distance CVs (input (s, 0))."""

    def __init__(self, n_models, n_cv, n_layers, width, weights, batch_size=128, resnet=False, init_lr=8e-4,
                 decay_rate=0.96, decay_steps=120, beta1=0.9, beta2=0.999, adam_eps=1e-8, dropout_rate=0.0,
                 dropout_seed=0, cv_dist=None):
        L = lib()
        self.M, self.C, self.B = int(n_models), int(n_cv), int(batch_size)
        w = np.ascontiguousarray(weights, dtype=np.float32)
        self.P = w.size // self.M
        kd = None if cv_dist is None else np.ascontiguousarray(cv_dist, dtype=np.int32)
        d = TrainDesc(self.M, self.C, int(n_layers), int(width), int(bool(resnet)), self.B, float(init_lr),
                      float(decay_rate), int(decay_steps), float(beta1), float(beta2), float(adam_eps),
                      float(dropout_rate), int(dropout_seed), None if kd is None else kd.ctypes.data)
        h = C.c_void_p()
        _check(L.rid_trainer_create(C.byref(d), w.ctypes.data, C.byref(h)))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib().rid_trainer_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_data(self, s, mf, stream=None):
        a = _Args()
        n = int(s.shape[0])
        ps = a.ptr(s, np.float32, (n, self.C))
        pm = a.ptr(mf, np.float32, (n, self.C))
        _check(lib().rid_trainer_set_data(self.h, n, ps, pm, a.mem, _stream_ptr(stream)))

    def run(self, idx, loss_out=None, stream=None):
        """idx [n_steps][M][B] int32 batch indices; loss_out [n_steps][M] float32."""
        a = _Args()
        n = int(idx.shape[0])
        pi = a.ptr(idx, np.int32, (n, self.M, self.B))
        pl = a.ptr(loss_out, np.float32, (n, self.M), True)
        _check(lib().rid_trainer_run(self.h, n, pi, pl, a.mem, _stream_ptr(stream)))

    def grad(self, idx, loss_out=None, grad_out=None, stream=None):
        a = _Args()
        pi = a.ptr(idx, np.int32, (self.M, self.B))
        pl = a.ptr(loss_out, np.float32, (self.M,), True)
        pg = a.ptr(grad_out, np.float32, (self.M, self.P), True)
        _check(lib().rid_trainer_grad(self.h, pi, pl, pg, a.mem, _stream_ptr(stream)))

    def weights(self, out=None, stream=None):
        """Current weights [M][P] (float32, host unless `out` is a CUDA tensor)
        and the number of steps taken."""
        if out is None:
            out = np.empty((self.M, self.P), dtype=np.float32)
        a = _Args()
        po = a.ptr(out, np.float32, (self.M, self.P), True)
        steps = C.c_int64(0)
        _check(lib().rid_trainer_weights(self.h, po, C.byref(steps), a.mem, _stream_ptr(stream)))
        return out, steps.value


def mcmc(weights, n_models, n_cv, n_layers, width, s0, n_steps, n_burn, kT, step_size, seed, bins=101,
         pair=(0, 1), resnet=False, s_out=None, hist1=None, hist2=None, pmf1=None, pmf2=None, path=None,
         hist_path=None, pmf_path=None, cv_dist=None, cv_range=None, stream=None):
    """MCMC dimension reduction (rid_mcmc): W = len(s0) walkers, Metropolis on
    the ensemble-mean free energy; returns the number of accepted moves.
    Outputs (optional, all on the side of s0): s_out [W][C] float32, hist1
    [C][bins] and hist2 [bins][bins] uint64, pmf1 / pmf2 of the same shapes
    float64.  path = (nodes [P][Cp], cvs [Cp], lambda, z_lo, z_hi) adds the
    (s_path, z_path) projection into hist_path / pmf_path [bins][bins].
    cv_dist [C] (bool) marks distance CVs, moved and binned inside cv_range =
    (lo [C], hi [C])."""
    a = _Args()
    W, Cn = int(s0.shape[0]), int(n_cv)
    pw = a.ptr(weights, np.float32)
    ps = a.ptr(s0, np.float32, (W, Cn))
    po = a.ptr(s_out, np.float32, (W, Cn), True)
    h1 = a.ptr(hist1, np.uint64, (Cn, bins), True)
    h2 = a.ptr(hist2, np.uint64, (bins, bins), True)
    f1 = a.ptr(pmf1, np.float64, (Cn, bins), True)
    f2 = a.ptr(pmf2, np.float64, (bins, bins), True)
    hp = a.ptr(hist_path, np.uint64, (bins, bins), True)
    fp = a.ptr(pmf_path, np.float64, (bins, bins), True)
    nodes = cvs = None
    npn, ncv, lam, zlo, zhi = 0, 0, 1.0, 0.0, 1.0
    if path is not None:
        nodes, cvs, lam, zlo, zhi = _path_arrays(path)
        npn, ncv = nodes.shape[0], cvs.size
    kd = lo = hi = None
    if cv_dist is not None:
        kd = np.ascontiguousarray(cv_dist, dtype=np.int32)
        if cv_range is not None:
            lo = np.ascontiguousarray(cv_range[0], dtype=np.float64)
            hi = np.ascontiguousarray(cv_range[1], dtype=np.float64)
    d = McmcDesc(int(n_models), Cn, int(n_layers), int(width), int(bool(resnet)), pw.value, W, int(n_steps),
                 int(n_burn), float(kT), float(step_size), int(seed), int(bins), int(pair[0]), int(pair[1]),
                 npn, ncv, None if cvs is None else cvs.ctypes.data, None if nodes is None else nodes.ctypes.data,
                 lam, zlo, zhi, None if kd is None else kd.ctypes.data, None if lo is None else lo.ctypes.data,
                 None if hi is None else hi.ctypes.data)
    nacc = C.c_int64(0)
    _check(lib().rid_mcmc(C.byref(d), ps, po, h1, h2, f1, f2, hp, fp, C.byref(nacc), a.mem, _stream_ptr(stream)))
    return nacc.value


def select(cv, eps, trust_lo, trust_hi, threshold, lower=1, upper=1 << 30, adapt=False, max_selection=50,
           weights=None, periodic=None, selected=None, stream=None):
    """Selection phase (rid_select) on frames cv [n][C], eps [n]; returns
    (selected frame indices, n_clusters, threshold).  `selected` may be a
    preallocated int32 array / CUDA tensor of max_selection entries."""
    n, Cn = int(cv.shape[0]), int(cv.shape[1])
    if selected is None:
        selected = np.zeros(max(1, max_selection), dtype=np.int32)
    a = _Args()
    pc = a.ptr(cv, np.float32, (n, Cn))
    pe = a.ptr(eps, np.float32, (n,))
    ps = a.ptr(selected, np.int32, None, True)
    w = None if weights is None else np.ascontiguousarray(weights, dtype=np.float32)
    p = None if periodic is None else np.ascontiguousarray(periodic, dtype=np.int32)
    d = SelectDesc(Cn, None if w is None else w.ctypes.data_as(C.POINTER(C.c_float)),
                   None if p is None else p.ctypes.data_as(C.POINTER(C.c_int32)), float(trust_lo), float(trust_hi),
                   float(threshold), int(lower), int(upper), int(bool(adapt)), int(max_selection))
    ns, nc, thr = C.c_int32(0), C.c_int32(0), C.c_double(0.0)
    _check(lib().rid_select(C.byref(d), n, pc, pe, ps, C.byref(ns), C.byref(nc), C.byref(thr), a.mem,
                            _stream_ptr(stream)))
    return selected[:ns.value], nc.value, thr.value
