"""Pins of the oracle's distance CVs (Sec. "CV selection": a CV may be the
distance between two atoms).  A row (a, b, -1, -1) of cv_atoms is the
distance |x_b - x_a|; it is not periodic, and the ensemble takes it as the
input pair (s, 0) where a torsion gives (cos s, sin s).

Pinned by finite differences of the oracle's own energies, torch.autograd in
FP64, the restraint's special values, and the restrained mean force on the
end-to-end distance of a bonded chain whose distance marginal is known by
quadrature.
"""
import math

import numpy as np
import pytest

from paper_2408_14070_gb300 import inputs as I


def _fd(fun, x, h=1e-6):
    g = np.zeros_like(x)
    for i in range(x.shape[0]):
        for k in range(3):
            xp, xm = x.copy(), x.copy()
            xp[i, k] += h
            xm[i, k] -= h
            g[i, k] = (fun(xp) - fun(xm)) / (2 * h)
    return -g


def test_distance_cv_value_and_jacobian(orc):
    sp = I.make_system(30, 5, 6, n_dist=2)
    assert list(I.cv_is_distance(sp)) == [False, False, False, True, True]
    x = I.make_chains(1, sp, 6)[0].astype(np.float64)
    s, J = orc.cvs(sp, x)
    for j in (3, 4):
        a, b = sp.cv_atoms[j, :2]
        assert s[j] == pytest.approx(np.linalg.norm(x[b] - x[a]), rel=1e-14)
    # the Jacobian of every CV against central differences of its value
    h = 1e-6
    for j in range(5):
        q = [int(v) for v in sp.cv_atoms[j] if v >= 0]
        for slot, at in enumerate(q):
            for k in range(3):
                xp, xm = x.copy(), x.copy()
                xp[at, k] += h
                xm[at, k] -= h
                fd = (orc.cvs(sp, xp)[0][j] - orc.cvs(sp, xm)[0][j]) / (2 * h)
                assert J[j].reshape(4, 3)[slot, k] == pytest.approx(fd, abs=1e-7)
        if len(q) == 2:
            assert not J[j].reshape(4, 3)[2:].any()


def test_ensemble_gradient_on_mixed_cvs_vs_autograd(orc):
    torch = pytest.importorskip("torch")
    sp = I.make_system(30, 4, 7, n_dist=2)
    ens = I.make_ensemble(3, 8, 2, 16, 7, resnet=True)
    s = np.array([0.4, -2.9, 1.7, 3.3])
    r = orc.ensemble(ens, s, sp.cv_atoms)
    dist = torch.tensor(I.cv_is_distance(sp))
    for m in range(3):
        st = torch.tensor(s, requires_grad=True)
        u = torch.stack([torch.where(dist, st, torch.cos(st)), torch.where(dist, torch.zeros_like(st), torch.sin(st))],
                        1).reshape(-1)
        D, L, H = 8, 2, 16
        w = torch.tensor(ens.weights[m].astype(np.float64))
        p, h = 0, u
        for l in range(L):
            fin = D if l == 0 else H
            W = w[p:p + H * fin].reshape(H, fin); p += H * fin
            b = w[p:p + H]; p += H
            t = torch.tanh(W @ h + b)
            h = t + h if l >= 1 else t
        A = w[p:p + H] @ h + w[p + H]
        (g,) = torch.autograd.grad(A, st)
        assert np.allclose(r["gradA"][m], g.numpy(), rtol=1e-11, atol=1e-13)
    # without the kinds every CV is read as a torsion: a different function
    assert not np.allclose(orc.ensemble(ens, s)["gradA"], r["gradA"])


def test_bias_force_with_distance_cvs_is_minus_gradient(orc):
    sp = I.make_system(30, 5, 8, n_dist=2)
    x = I.make_chains(1, sp, 8)[0].astype(np.float64)
    ens = I.make_ensemble(4, 10, 2, 32, 8, trust_lo=1e9, trust_hi=2e9)
    fb = orc.total(sp, x, ens=ens, mode=1)["f"] - orc.total(sp, x, mode=0)["f"]
    fd = _fd(lambda y: -orc.total(sp, y, ens=ens, mode=1)["Abar"], x)
    assert np.abs(fb).max() > 1e-3
    assert np.abs(fd - fb).max() <= 1e-6 * np.abs(fb).max()
    # the distance CVs' beads carry bias force
    for j in (3, 4):
        a, b = sp.cv_atoms[j, :2]
        assert np.abs(fb[[a, b]]).max() > 0


def test_restraint_on_distance_cvs_is_not_wrapped(orc):
    sp = I.make_system(30, 5, 9, n_dist=2)
    x = I.make_chains(1, sp, 9)[0].astype(np.float64)
    s = orc.cvs(sp, x)[0]
    kap = np.array([50.0, 80.0, 120.0, 300.0, 500.0])
    # centres 4 away from the distances: a wrapped offset would be 4 - 2 pi
    s0 = np.concatenate([I.make_label_targets(1, 3, 9)[0], s[3:] - 4.0])
    r = orc.total(sp, x, mode=2, s0=s0, kappa=kap)
    dt = s[:3] - s0[:3]
    dt -= 2 * np.pi * np.floor(dt / (2 * np.pi) + 0.5)
    want = 0.5 * (kap[:3] * dt ** 2).sum() + 0.5 * (kap[3:] * 16.0).sum()
    assert r["U_restraint"] == pytest.approx(want, rel=1e-12)
    fr = r["f"] - orc.total(sp, x)["f"]
    fd = _fd(lambda y: orc.total(sp, y, mode=2, s0=s0, kappa=kap)["U_restraint"], x)
    assert np.abs(fd - fr).max() <= 1e-6 * np.abs(fr).max()


# Restrained labels on the distance R between beads 1 and 3 of a 4-bead chain
# with harmonic bonds only: the two bond vectors are independent and isotropic
# (radial density r^2 exp(-k (r - r0)^2 / 2kT)), so R = |d1 + d2| has the
# density P(R) = R/2 int int g(r1) g(r2) / (r1 r2) [|r1 - r2| <= R <= r1 + r2],
# and the restrained average of R at centre s0 is a 1-D quadrature:
# MF = -kappa (<R>_kappa - s0) with weights P(R) exp(-kappa (R - s0)^2 / 2kT).
KB, R0, KT = 20.0, 1.0, 1.0


def _exact_restrained_mf(s0, kappa):
    r = np.linspace(0.05, 3.0, 20001)
    dr = r[1] - r[0]
    g = r ** 2 * np.exp(-KB * (r - R0) ** 2 / (2 * KT))
    g /= np.trapezoid(g, r)
    h = g / r
    cum = np.concatenate([[0.0], np.cumsum(0.5 * (h[1:] + h[:-1]) * dr)])
    R = np.linspace(0.02, 2.98, 1481)
    P = np.array([0.5 * Ri * np.trapezoid(h * (np.interp(Ri + r, r, cum) - np.interp(np.abs(Ri - r), r, cum)), r)
                  for Ri in R])
    wts = P * np.exp(-kappa * (R - s0) ** 2 / (2 * KT))
    mean = np.trapezoid(R * wts, R) / np.trapezoid(wts, R)
    return -kappa * (mean - s0)


@pytest.mark.parametrize("s0", [1.3, 1.9])
def test_restrained_distance_label_matches_the_exact_marginal(orc, s0):
    sp = I.make_system(4, 1, 3, n_dist=1, dist_span=2, lj_eps=0.0, angle_k=0.0, bond_k=KB, bond_r0=R0, kT=KT)
    sp.dihedral_k[:] = 0.0
    assert list(sp.cv_atoms[0]) == [1, 3, -1, -1]
    R = 8
    x0 = np.zeros((R, 4, 3), np.float32)
    x0[:, :, 0] = np.arange(4)
    x0[:, 2, 1] = 0.5
    kappa = 20.0
    r = orc.label(sp, x0, np.full((R, 1), s0), kappa, 200000, 20000, 20)
    mf = r["mf"][:, 0].mean()
    se = np.sqrt((r["se"][:, 0] ** 2).sum()) / R
    exact = _exact_restrained_mf(s0, kappa)
    assert abs(mf - exact) < 3.5 * se, (mf, se, exact)
    # the label is resolved: the mean force stands well clear of its error
    assert abs(exact) > 5 * se
