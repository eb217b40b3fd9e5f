"""Pins of the constrained-MD labels of the oracle (orc_label_constrained):
the mean force on a constrained distance against the exact derivative of the
free energy along that distance, for a chain whose marginal is known in
closed form, and the constraint and its velocity condition after the run.

The chain: 4 beads joined by harmonic bonds only (no angle, dihedral or LJ
terms); the CV is the distance between beads 0 and 2.  The bond vectors
d1 = x0 - x1 and d2 = x1 - x2 are independent and isotropic with radial
density g(r) ~ r^2 exp(-k (r - r0)^2 / 2kT), so R = |d1 + d2| has the density
P(R) = R/2 int int g(r1) g(r2) / (r1 r2) [|r1 - r2| <= R <= r1 + r2] dr1 dr2
and the mean force is dA/dR = -kT d ln P / dR (the free energy includes the
r^2 of the spherical shell, as the restrained labels do).
"""
import numpy as np
import pytest

from paper_2408_14070_gb300 import inputs as I

KB, R0, KT = 20.0, 1.0, 1.0


def _exact_mean_force(d0):
    r = np.linspace(0.05, 3.0, 200001)
    dr = r[1] - r[0]
    g = r ** 2 * np.exp(-KB * (r - R0) ** 2 / (2 * KT))
    g /= np.trapezoid(g, r)
    h = g / r
    cum = np.concatenate([[0.0], np.cumsum(0.5 * (h[1:] + h[:-1]) * dr)])

    def P(R):
        inner = np.interp(R + r, r, cum) - np.interp(np.abs(R - r), r, cum)
        return 0.5 * R * np.trapezoid(h * inner, r)

    e = 1e-3
    return -KT * (np.log(P(d0 + e)) - np.log(P(d0 - e))) / (2 * e)


def _chain(R):
    sp = I.make_system(4, 1, 3, lj_eps=0.0, angle_k=0.0, bond_k=KB, bond_r0=R0, kT=KT)
    sp.dihedral_k[:] = 0.0
    x0 = np.zeros((R, 4, 3), np.float32)
    x0[:, :, 0] = np.arange(4)
    x0[:, 2, 1] = 0.5
    return sp, x0


@pytest.mark.parametrize("d0", [1.2, 1.5, 1.8])
def test_constrained_mean_force_matches_the_exact_marginal(orc, d0):
    R = 8
    sp, x0 = _chain(R)
    r = orc.label_constrained(sp, x0, [[0, 2]], np.full((R, 1), d0), 200000, 20000, 20)
    mf = r["mf"][:, 0].mean()
    se = np.sqrt((r["se"][:, 0] ** 2).sum()) / R
    exact = _exact_mean_force(d0)
    assert abs(mf - exact) < 3.5 * se, (mf, se, exact)
    # the constraint and its velocity condition hold at the end of the run
    x, v = r["x"], r["v"]
    d = x[:, 0] - x[:, 2]
    rr = np.linalg.norm(d, axis=-1)
    assert np.max(np.abs(rr - d0)) < 1e-12
    assert np.max(np.abs(((v[:, 0] - v[:, 2]) * d).sum(-1) / rr)) < 1e-12
