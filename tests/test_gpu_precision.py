"""Precision sweep shape (100-bead chain, 32 torsion CVs, 8 x MLP 64 -> 512 x 4
-> 1): bias force and model deviation of the FP32 and BF16 ensemble paths
against the FP64 oracle on sampled walkers: the CV-space bias force (the
ensemble mean force, sigma = 1) and eps, both at the CVs of each walker.

Bounds: FP32 3e-5 normwise (K up to 512 in every GEMM, FP32 accumulation);
BF16 the derived 3e-2 / 5e-2 of the tensor-core tests.  FP8 (e4m3 forward
GEMMs, 3 mantissa bits: up to 2^-4 relative per operand, BF16 input-gradient
GEMMs): 6e-2 on the mean force and 3e-2 on eps -- a host emulation of the same
arithmetic at this shape gives about 2e-2 and 6e-3.  The measured errors are
printed (pytest -s).
"""
import numpy as np
import pytest

from paper_2408_14070_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    from paper_2408_14070_gb300 import build, rid
    build.build()
    return rid


@pytest.mark.parametrize("prec,force_tol,eps_tol", [("fp32", 3e-5, 3e-5), ("bf16", 3e-2, 5e-2),
                                                    ("fp8", 6e-2, 3e-2)])
def test_precision_sweep_errors_against_the_oracle(R, orc, prec, force_tol, eps_tol):
    sp = I.make_system(100, 32, 4)
    W = 256
    x = I.make_chains(W, sp, 4)
    ens = I.make_ensemble(8, 64, 4, 512, 4, trust_lo=1e9, trust_hi=2e9)
    g = np.zeros((8, W, sp.n_cv), np.float32)
    eps = np.zeros(W, np.float32)
    with R.System(sp) as sysobj:
        sysobj.set_ensemble(ens, precision={"fp32": R.RID_PREC_FP32, "bf16": R.RID_PREC_BF16,
                                            "fp8": R.RID_PREC_FP8}[prec])
        sysobj.eval_forces(x, R.RID_BIAS_ENSEMBLE, eps_out=eps, grad_out=g)
    ferr, eerr = [], []
    for w in range(0, W, 16):
        e = orc.ensemble(ens, orc.cvs(sp, x[w].astype(np.float64))[0])
        fbar_ref = e["gradA"].mean(axis=0)          # the CV-space bias force at sigma = 1
        fbar = g[:, w].astype(np.float64).mean(axis=0)
        ferr.append(np.linalg.norm(fbar - fbar_ref) / np.linalg.norm(fbar_ref))
        eerr.append(abs(eps[w] - e["eps"]) / e["eps"])
    print(f"\n[{prec}] bias force rel. error: median {np.median(ferr):.2e} max {np.max(ferr):.2e}; "
          f"eps rel. error: median {np.median(eerr):.2e} max {np.max(eerr):.2e}")
    assert max(ferr) < force_tol
    assert max(eerr) < eps_tol
